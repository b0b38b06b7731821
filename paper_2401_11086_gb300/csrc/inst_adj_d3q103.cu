// Adjoint kernel instantiations for D3Q103 (forward state in double or float; the adjoint
// arithmetic is double in both).
#include "dispatch.h"

namespace smrt {
const AdjointSet *adjoints_d3q103(int N, int precision) {
    const int P = precision == 0 ? 0 : 1;
    switch (N) {
        case 3: return P == 0 ? adjoint_set<D3Q103, 3, 0>() : adjoint_set<D3Q103, 3, 1>();
        case 4: return P == 0 ? adjoint_set<D3Q103, 4, 0>() : adjoint_set<D3Q103, 4, 1>();
        default: return nullptr;
    }
}
}  // namespace smrt
