// Kernel instantiations: D3Q4913 (D1Q17-P1 tensor product), precision f64, N = 5 (see inst_d3q4913_f64.cu).
#include "dispatch.h"

namespace smrt {
const KernelSet *kernels_d3q4913_p0_n5() { return tp_kernel_set<D1Q17P1, 5, 0>(); }
}  // namespace smrt
