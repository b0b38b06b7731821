// Adjoint kernel instantiations for D3Q4913, N = 4 (see inst_adj_d3q4913.cu).
#include "dispatch.h"

namespace smrt {
const AdjointSet *adjoints_d3q4913_n4(int P) {
    return P == 0 ? tp_adjoint_set<D1Q17P1, 4, 0>() : tp_adjoint_set<D1Q17P1, 4, 1>();
}
}  // namespace smrt
