// Adjoint kernel instantiations for D3Q4913 (forward state in double or float, the adjoint
// arithmetic is double in both); each order is compiled in a translation unit of its own
// (inst_adj_d3q4913_n*.cu) so that the build compiles them in parallel.
#include "dispatch.h"

namespace smrt {
const AdjointSet *adjoints_d3q4913_n4(int P);
const AdjointSet *adjoints_d3q4913_n5(int P);
const AdjointSet *adjoints_d3q4913(int N, int precision) {
    const int P = precision == 0 ? 0 : 1;
    switch (N) {
        case 4: return adjoints_d3q4913_n4(P);
        case 5: return adjoints_d3q4913_n5(P);
        default: return nullptr;
    }
}
}  // namespace smrt
