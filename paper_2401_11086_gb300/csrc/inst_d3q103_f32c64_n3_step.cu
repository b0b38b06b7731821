// Kernel instantiations: D3Q103, precision f32c64, N = 3, per-step launches (see
// inst_d3q103_f32c64.cu).
#include "dispatch.h"

namespace smrt {
cudaError_t d3q103_p2_n3_step(const CtxView &v, const void *fin, void *fout) {
    return launch_step<D3Q103, 3, float, double, true>(v, fin, fout);
}
}  // namespace smrt
