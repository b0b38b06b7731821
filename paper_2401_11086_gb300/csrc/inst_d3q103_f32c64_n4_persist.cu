// Kernel instantiations: D3Q103, precision f32c64, N = 4, persistent launches (see
// inst_d3q103_f32c64.cu).
#include "dispatch.h"

namespace smrt {
cudaError_t d3q103_p2_n4_persist(const CtxView &v, void *fa, void *fb, int nsteps, int grid) {
    return launch_persistent<D3Q103, 4, float, double, true>(v, fa, fb, nsteps, grid);
}
int d3q103_p2_n4_occupancy(const CtxView &v) { return persistent_occupancy<D3Q103, 4, float, double, true>(v); }
}  // namespace smrt
