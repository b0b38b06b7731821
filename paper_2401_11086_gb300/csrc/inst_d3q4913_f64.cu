// Kernel instantiations: D3Q4913 (D1Q17-P1 tensor product), precision f64.
#include "dispatch.h"

namespace smrt {
const KernelSet *kernels_d3q4913_p0(int N) {
    switch (N) {
        case 4: return tp_kernel_set<D1Q17P1, 4, 0>();
        case 5: return tp_kernel_set<D1Q17P1, 5, 0>();
        default: return nullptr;
    }
}
}  // namespace smrt
