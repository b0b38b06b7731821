// Adjoint kernel instantiations for D3Q4913, N = 5 (see inst_adj_d3q4913.cu).
#include "dispatch.h"

namespace smrt {
const AdjointSet *adjoints_d3q4913_n5(int P) {
    return P == 0 ? tp_adjoint_set<D1Q17P1, 5, 0>() : tp_adjoint_set<D1Q17P1, 5, 1>();
}
}  // namespace smrt
