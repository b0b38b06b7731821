// Kernel instantiations: D3Q729 (D1Q9-P1 tensor product), precision f32, N = 5 (see inst_d3q729_f32.cu).
#include "dispatch.h"

namespace smrt {
const KernelSet *kernels_d3q729_p1_n5() { return tp_kernel_set<D1Q9P1, 5, 1>(); }
}  // namespace smrt
