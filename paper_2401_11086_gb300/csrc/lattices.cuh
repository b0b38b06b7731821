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

}  // namespace smrt
