// Adjoint kernel instantiations for D3Q729, N = 5 (see inst_adj_d3q729.cu).
#include "dispatch.h"

namespace smrt {
const AdjointSet *adjoints_d3q729_n5(int P) {
    return P == 0 ? tp_adjoint_set<D1Q9P1, 5, 0>() : tp_adjoint_set<D1Q9P1, 5, 1>();
}
}  // namespace smrt
