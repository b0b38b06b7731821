// Host build of the compile-time sign-orbit tables of libsmrt's velocity sets
// (csrc/lattices.cuh) and of the multi-index slot order (csrc/core.cuh), for a CPU test of the
// identity the projection and the rebuild rely on.
#include "../../paper_2401_11086_gb300/csrc/lattices.cuh"

using namespace smrt;

// Per orbit, 15 ints: k, ax[3], a[3], pair[4], flip[4]. Returns the number of orbits.
template <class Lat>
static int dump_orbits(int *out) {
    constexpr SignOrbits<Lat> O{};
    for (int o = 0; o < O.n; ++o) {
        int *r = out + 15 * o;
        r[0] = O.k[o];
        for (int d = 0; d < 3; ++d) r[1 + d] = O.ax[o][d], r[4 + d] = O.a[o][d];
        for (int b = 0; b < 4; ++b) r[7 + b] = O.pair[o][b], r[11 + b] = O.flip[o][b];
    }
    return O.n;
}

// Per (orbit, slot g < nmom(N)): a^gamma and the transform entry of slot g.
template <class Lat>
static void dump_classes(int N, int *mono, int *cls) {
    constexpr SignOrbits<Lat> O{};
    const int M = nmom(N);
    for (int o = 0; o < O.n; ++o)
        for (int g = 0; g < M; ++g) {
            mono[o * M + g] = O.monomial(o, g);
            cls[o * M + g] = O.parity_class(o, g);
        }
}

template <class Lat>
static int dump_vectors(int *e) {
    for (int p = 0; p < Lat::NP; ++p)
        for (int d = 0; d < 3; ++d) e[3 * p + d] = Lat::e(p, d);
    return Lat::NP;
}

extern "C" {
int orbits_d3q39(int *out) { return dump_orbits<D3Q39>(out); }
int orbits_d3q103(int *out) { return dump_orbits<D3Q103>(out); }
void classes_d3q39(int N, int *mono, int *cls) { dump_classes<D3Q39>(N, mono, cls); }
void classes_d3q103(int N, int *mono, int *cls) { dump_classes<D3Q103>(N, mono, cls); }
int vectors_d3q39(int *e) { return dump_vectors<D3Q39>(e); }
int vectors_d3q103(int *e) { return dump_vectors<D3Q103>(e); }
// components of every slot of order <= N, in slot order
void slot_components(int N, int *out) {
    for (int g = 0; g < nmom(N); ++g)
        for (int d = 0; d < 3; ++d) out[3 * g + d] = mi_comp(g, d);
}
}
