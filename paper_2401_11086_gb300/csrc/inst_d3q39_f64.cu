// Kernel instantiations: D3Q39, precision f64 (one translation unit per lattice and
// precision so that the build compiles them in parallel).
#include "dispatch.h"

namespace smrt {
const KernelSet *kernels_d3q39_p0(int N) {
    switch (N) {
        case 3: return kernel_set<D3Q39, 3, 0>();
        default: return nullptr;
    }
}
}  // namespace smrt
