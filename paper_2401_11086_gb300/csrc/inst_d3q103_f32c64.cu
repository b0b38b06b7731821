// Kernel instantiations: D3Q103, precision f32c64, N = 4 (one translation unit per lattice,
// precision and, for this the largest set of kernels, order, so that the build compiles them
// in parallel).
#include "dispatch.h"

namespace smrt {
const KernelSet *kernels_d3q103_p2_n3();
const KernelSet *kernels_d3q103_p2(int N) {
    switch (N) {
        case 3: return kernels_d3q103_p2_n3();
        case 4: return kernel_set<D3Q103, 4, 2>();
        default: return nullptr;
    }
}
}  // namespace smrt
