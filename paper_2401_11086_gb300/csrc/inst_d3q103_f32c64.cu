// Kernel instantiations: D3Q103, precision f32c64. The step and persistent kernels of each
// order are compiled in translation units of their own (inst_d3q103_f32c64_n*_{step,persist}.cu),
// the largest kernels of the library, so that the build compiles them in parallel; this unit
// holds the moments, fill and end-state kernels and assembles the sets.
#include "dispatch.h"

namespace smrt {
cudaError_t d3q103_p2_n3_step(const CtxView &, const void *, void *);
cudaError_t d3q103_p2_n4_step(const CtxView &, const void *, void *);
cudaError_t d3q103_p2_n3_persist(const CtxView &, void *, void *, int, int);
cudaError_t d3q103_p2_n4_persist(const CtxView &, void *, void *, int, int);
int d3q103_p2_n3_occupancy(const CtxView &);
int d3q103_p2_n4_occupancy(const CtxView &);

const KernelSet *kernels_d3q103_p2(int N) {
    static const KernelSet k3 = {&d3q103_p2_n3_step, &launch_moments<D3Q103, 3, float, double>,
                                 &launch_fill<D3Q103, 3, float>, &launch_ghost<D3Q103, 3, float>,
                                 &d3q103_p2_n3_persist, &d3q103_p2_n3_occupancy};
    static const KernelSet k4 = {&d3q103_p2_n4_step, &launch_moments<D3Q103, 4, float, double>,
                                 &launch_fill<D3Q103, 4, float>, &launch_ghost<D3Q103, 4, float>,
                                 &d3q103_p2_n4_persist, &d3q103_p2_n4_occupancy};
    switch (N) {
        case 3: return &k3;
        case 4: return &k4;
        default: return nullptr;
    }
}
}  // namespace smrt
