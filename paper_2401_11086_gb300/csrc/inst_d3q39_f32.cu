// Kernel instantiations: D3Q39, precision f32 (one translation unit per lattice and
// precision so that the build compiles them in parallel).
#include "dispatch.h"

namespace smrt {
const KernelSet *kernels_d3q39_p1(int N) {
    switch (N) {
        case 3: return kernel_set<D3Q39, 3, 1>();
        default: return nullptr;
    }
}
}  // namespace smrt
