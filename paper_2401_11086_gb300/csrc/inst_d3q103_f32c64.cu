// Kernel instantiations: D3Q103, precision f32c64 (one translation unit per lattice and
// precision so that the build compiles them in parallel).
#include "dispatch.h"

namespace smrt {
const KernelSet *kernels_d3q103_p2(int N) {
    switch (N) {
        case 3: return kernel_set<D3Q103, 3, 2>();
        case 4: return kernel_set<D3Q103, 4, 2>();
        default: return nullptr;
    }
}
}  // namespace smrt
