// Kernel instantiations: D3Q4913 (D1Q17-P1 tensor product), precision f32; each order is compiled in a
// translation unit of its own (inst_d3q4913_f32_n*.cu) so that the build compiles them in parallel.
#include "dispatch.h"

namespace smrt {
const KernelSet *kernels_d3q4913_p1_n4();
const KernelSet *kernels_d3q4913_p1_n5();
const KernelSet *kernels_d3q4913_p1(int N) {
    switch (N) {
        case 4: return kernels_d3q4913_p1_n4();
        case 5: return kernels_d3q4913_p1_n5();
        default: return nullptr;
    }
}
}  // namespace smrt
