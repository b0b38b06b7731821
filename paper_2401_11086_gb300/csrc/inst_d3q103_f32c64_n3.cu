// Kernel instantiations: D3Q103, precision f32c64, N = 3 (see inst_d3q103_f32c64.cu).
#include "dispatch.h"

namespace smrt {
const KernelSet *kernels_d3q103_p2_n3() { return kernel_set<D3Q103, 3, 2>(); }
}  // namespace smrt
