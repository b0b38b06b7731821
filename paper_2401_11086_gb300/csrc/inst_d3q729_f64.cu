// Kernel instantiations: D3Q729 (D1Q9-P1 tensor product), precision f64.
#include "dispatch.h"

namespace smrt {
const KernelSet *kernels_d3q729_p0(int N) {
    switch (N) {
        case 4: return tp_kernel_set<D1Q9P1, 4, 0>();
        case 5: return tp_kernel_set<D1Q9P1, 5, 0>();
        default: return nullptr;
    }
}
}  // namespace smrt
