// Kernel instantiations: D3Q729 (D1Q9-P1 tensor product), precision f64, N = 5 (see inst_d3q729_f64.cu).
#include "dispatch.h"

namespace smrt {
const KernelSet *kernels_d3q729_p0_n5() { return tp_kernel_set<D1Q9P1, 5, 0>(); }
}  // namespace smrt
