// Kernel instantiations: D3Q4913 (D1Q17-P1 tensor product), precision f32, N = 4 (see inst_d3q4913_f32.cu).
#include "dispatch.h"

namespace smrt {
const KernelSet *kernels_d3q4913_p1_n4() { return tp_kernel_set<D1Q17P1, 4, 1>(); }
}  // namespace smrt
