// lattices.cuh -- velocity sets this library has kernels for, as compile-time tables.
//
// Each set is a cubic-symmetric degree-Q Gauss-Hermite rule (Sec. 3, Eq. an): abscissae
// xi_i = c e_i with integer e_i, weights constant on each cubic orbit ("shell"). The paper
// uses tensor products of 1D rules (Sec. 4.2); the two sets here are smaller 3D rules of the
// same kind. Only the integer vectors are compile-time: the scale c and the weights are
// solved on the host (lattice.cu) and passed to the kernels at run time.
//
// Library order: population 0 is the rest velocity; population 2p+1 is +e_p and 2p+2 is -e_p
// for pair p. The caller may use any order; lb_init_lattice maps it.
#pragma once

#include "core.cuh"

namespace smrt {

// D3Q39: degree 7, rest + 19 (+e, -e) pairs = 39 velocities.
// Shells (cubic orbits): {0, 0, 0}, {1, 0, 0}, {1, 1, 1}, {2, 0, 0}, {2, 2, 0}, {3, 0, 0}.
struct D3Q39 {
    static constexpr int Q = 39;
    static constexpr int NP = 19;
    static constexpr int DEGREE = 7;
    static constexpr int NMAX = 3;      // highest truncation order with degree >= 2N
    static constexpr int NSHELL = 6;
    static constexpr double C_GUESS = 1.2;  // start of the scale search in the host solver
    static constexpr SMRT_HD int e(int p, int k) {
        constexpr signed char P[NP][3] = {
            {1, 0, 0},
            {0, 1, 0},
            {0, 0, 1},
            {1, 1, 1},
            {1, 1, -1},
            {1, -1, 1},
            {1, -1, -1},
            {2, 0, 0},
            {0, 2, 0},
            {0, 0, 2},
            {2, 2, 0},
            {2, 0, 2},
            {2, 0, -2},
            {2, -2, 0},
            {0, 2, 2},
            {0, 2, -2},
            {3, 0, 0},
            {0, 3, 0},
            {0, 0, 3}};
        return P[p][k];
    }
    static constexpr SMRT_HD int shell(int p) {
        constexpr int S[NP] = {1, 1, 1, 2, 2, 2, 2, 3, 3, 3, 4, 4, 4, 4, 4, 4, 5, 5, 5};
        return S[p];
    }
    static constexpr SMRT_HD int shell_rep(int s, int k) {
        constexpr signed char R[NSHELL][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 1}, {2, 0, 0}, {2, 2, 0}, {3, 0, 0}};
        return R[s][k];
    }
};

// D3Q103: degree 9, rest + 51 (+e, -e) pairs = 103 velocities.
// Shells (cubic orbits): {0, 0, 0}, {1, 1, 1}, {2, 0, 0}, {2, 1, 1}, {2, 2, 0}, {2, 2, 2}, {3, 0, 0}, {4, 0, 0}, {3, 3, 3}, {4, 2, 0}.
struct D3Q103 {
    static constexpr int Q = 103;
    static constexpr int NP = 51;
    static constexpr int DEGREE = 9;
    static constexpr int NMAX = 4;      // highest truncation order with degree >= 2N
    static constexpr int NSHELL = 10;
    static constexpr double C_GUESS = 0.736;  // start of the scale search in the host solver
    static constexpr SMRT_HD int e(int p, int k) {
        constexpr signed char P[NP][3] = {
            {1, 1, 1},
            {1, 1, -1},
            {1, -1, 1},
            {1, -1, -1},
            {2, 0, 0},
            {0, 2, 0},
            {0, 0, 2},
            {2, 1, 1},
            {2, 1, -1},
            {2, -1, 1},
            {2, -1, -1},
            {1, 2, 1},
            {1, 2, -1},
            {1, 1, 2},
            {1, 1, -2},
            {1, -1, 2},
            {1, -1, -2},
            {1, -2, 1},
            {1, -2, -1},
            {2, 2, 0},
            {2, 0, 2},
            {2, 0, -2},
            {2, -2, 0},
            {0, 2, 2},
            {0, 2, -2},
            {2, 2, 2},
            {2, 2, -2},
            {2, -2, 2},
            {2, -2, -2},
            {3, 0, 0},
            {0, 3, 0},
            {0, 0, 3},
            {4, 0, 0},
            {0, 4, 0},
            {0, 0, 4},
            {3, 3, 3},
            {3, 3, -3},
            {3, -3, 3},
            {3, -3, -3},
            {4, 2, 0},
            {4, 0, 2},
            {4, 0, -2},
            {4, -2, 0},
            {2, 4, 0},
            {2, 0, 4},
            {2, 0, -4},
            {2, -4, 0},
            {0, 4, 2},
            {0, 4, -2},
            {0, 2, 4},
            {0, 2, -4}};
        return P[p][k];
    }
    static constexpr SMRT_HD int shell(int p) {
        constexpr int S[NP] = {1, 1, 1, 1, 2, 2, 2, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 4, 4, 4, 4, 4, 4, 5, 5, 5, 5, 6, 6, 6, 7, 7, 7, 8, 8, 8, 8, 9, 9, 9, 9, 9, 9, 9, 9, 9, 9, 9, 9};
        return S[p];
    }
    static constexpr SMRT_HD int shell_rep(int s, int k) {
        constexpr signed char R[NSHELL][3] = {{0, 0, 0}, {1, 1, 1}, {2, 0, 0}, {2, 1, 1}, {2, 2, 0}, {2, 2, 2}, {3, 0, 0}, {4, 0, 0}, {3, 3, 3}, {4, 2, 0}};
        return R[s][k];
    }
};


// Sign orbits. The sets above are closed under a change of sign of any component, so their
// (+e, -e) pairs fall into orbits of vectors with the same absolute components a = |e|: an
// orbit with k nonzero components holds 2^k vectors, i.e. 2^(k-1) pairs. Each member is
// v = s (.) a with signs s; taking v = +e or -e of its pair so that v is positive on the first
// nonzero axis ax[0], the member is labelled by the sign bits b of the other nonzero axes
// (bit t-1 set when v is negative on ax[t]). Then v^gamma = a^gamma (-1)^popcount(b & pi),
// pi = the parities of gamma on ax[1..k-1]: a monomial sum over the orbit is a^gamma times
// one entry of a Walsh-Hadamard transform of the orbit's pair sums (even |gamma|) or pair
// differences (odd |gamma|), and a rebuild is the same transform of per-parity-class sums.
template <class Lat>
struct SignOrbits {
    static constexpr int NP = Lat::NP;
    int n = 0;             // number of orbits
    int k[NP] = {};        // nonzero components of the orbit's vectors
    int ax[NP][3] = {};    // those axes, ascending
    int a[NP][3] = {};     // absolute components
    int pair[NP][4] = {};  // pair of the member with sign bits b
    int flip[NP][4] = {};  // 1 when that member is -e of its pair
    int seen[NP] = {};     // bit b set once the member with sign bits b is found
    int count[NP] = {};
    constexpr SignOrbits() {
        for (int p = 0; p < NP; ++p) {
            int m[3] = {0, 0, 0};
            for (int d = 0; d < 3; ++d) m[d] = Lat::e(p, d) < 0 ? -Lat::e(p, d) : Lat::e(p, d);
            int o = 0;
            while (o < n && !(a[o][0] == m[0] && a[o][1] == m[1] && a[o][2] == m[2])) ++o;
            if (o == n) {
                for (int d = 0; d < 3; ++d) {
                    a[o][d] = m[d];
                    if (m[d] != 0) ax[o][k[o]++] = d;
                }
                ++n;
            }
            const int s0 = Lat::e(p, ax[o][0]) > 0 ? 1 : -1;
            int b = 0;
            for (int t = 1; t < k[o]; ++t)
                if (s0 * Lat::e(p, ax[o][t]) < 0) b |= 1 << (t - 1);
            pair[o][b] = p;
            flip[o][b] = s0 < 0 ? 1 : 0;
            seen[o] |= 1 << b;
            ++count[o];
        }
    }
    // every orbit holds each of its 2^(k-1) sign patterns exactly once (no rest vector here)
    constexpr bool complete() const {
        int pairs = 0;
        for (int o = 0; o < n; ++o) {
            const int np = 1 << (k[o] - 1);
            if (k[o] < 1 || count[o] != np || seen[o] != (1 << np) - 1) return false;
            pairs += np;
        }
        return pairs == NP;
    }
    // a^gamma for the multi-index in slot g (zero when gamma lies off the orbit's axes)
    constexpr int monomial(int o, int g) const {
        int v = 1;
        for (int d = 0; d < 3; ++d)
            for (int j = 0; j < mi_comp(g, d); ++j) v *= a[o][d];
        return v;
    }
    // transform entry of slot g: the parities of gamma on ax[1..k-1]
    constexpr int parity_class(int o, int g) const {
        int c = 0;
        for (int t = 1; t < k[o]; ++t)
            if (mi_comp(g, ax[o][t]) & 1) c |= 1 << (t - 1);
        return c;
    }
};
static_assert(SignOrbits<D3Q39>().complete(), "D3Q39 is closed under sign changes");
static_assert(SignOrbits<D3Q103>().complete(), "D3Q103 is closed under sign changes");

}  // namespace smrt
