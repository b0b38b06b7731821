// Kernel instantiations: D3Q103, precision f32 (one translation unit per lattice and
// precision so that the build compiles them in parallel).
#include "dispatch.h"

namespace smrt {
const KernelSet *kernels_d3q103_p1(int N) {
    switch (N) {
        case 3: return kernel_set<D3Q103, 3, 1>();
        case 4: return kernel_set<D3Q103, 4, 1>();
        default: return nullptr;
    }
}
}  // namespace smrt
