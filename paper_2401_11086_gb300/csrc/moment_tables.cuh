// moment_tables.cuh -- compile-time tables for running the moment-space steps of the SMRT
// collision (Sec. 3, Eq. SMRT; Appendix A) with the coefficients spread over the lanes of a warp.
//
// The per-thread code in core.cuh unrolls every step over the multi-index slots at compile
// time. When one cell's coefficients are shared by a warp, a lane holds runtime slots, so the
// constant structure those steps use is tabulated here, in the same divided representation
// (x~ = x / beta!, slots in mi_pos order):
//   hd   ta_alpha = sum_gamma hdiv(alpha, gamma) Rc_gamma          (raw moments -> coefficients)
//   hf   P_gamma  = sum_alpha hfull(alpha, gamma) ta_alpha          (coefficients -> rebuild form)
//   rel  the order-n block of delta^j tr^j for j >= 1 (the lift of the j-fold trace, Appendix A),
//        so that relax_order's  d'_n = sum_j C_j delta^j tr^j d_n  is one small product per slot
//   es   the ordered pairs of order-2 slots adding up to each order-4 slot (ES-BGK target)
#pragma once

#include "core.cuh"

namespace smrt {

// Multi-index components and orders of every slot, computed once (the mi_* helpers loop).
template <int N>
struct SlotIndex {
    static constexpr int M = nmom(N);
    int c[M][3] = {};
    int ord[M] = {};
    constexpr SlotIndex() {
        for (int p = 0; p < M; ++p) {
            for (int k = 0; k < 3; ++k) c[p][k] = mi_comp(p, k);
            ord[p] = c[p][0] + c[p][1] + c[p][2];
        }
    }
    constexpr int with(int p, int k, int v) const {
        int e[3] = {c[p][0], c[p][1], c[p][2]};
        e[k] = v;
        return mi_pos(e[0], e[1], e[2]);
    }
};

constexpr double fact_small(int n) {
    double v = 1.0;
    for (int i = 2; i <= n; ++i) v *= i;
    return v;
}
// coefficient of x^j in He_n(x) (Appendix B), loop form
constexpr double he_coef_l(int n, int j) {
    if (j > n || ((n - j) & 1)) return 0.0;
    const int l = (n - j) / 2;
    return ((l & 1) ? -1.0 : 1.0) * fact_small(n) / (fact_small(l) * fact_small(j) * double(1 << l));
}

// hd and hf: the two Hermite conversions as sparse rows
template <int N>
struct HermiteTables {
    static constexpr int M = nmom(N);
    static constexpr int kNZ = 12;  // largest row for N <= 5
    int hd_n[M] = {};
    int hd_col[M][kNZ] = {};
    double hd_val[M][kNZ] = {};
    int hf_n[M] = {};
    int hf_col[M][kNZ] = {};
    double hf_val[M][kNZ] = {};
    constexpr HermiteTables() {
        const SlotIndex<N> s;
        for (int a = 0; a < M; ++a)
            for (int g = 0; g < M; ++g) {
                double h = 1.0;  // prod_k coefficient of e^gamma_k in He_alpha_k
                for (int k = 0; k < 3; ++k) h *= he_coef_l(s.c[a][k], s.c[g][k]);
                if (h == 0.0) continue;
                const double af = fact_small(s.c[a][0]) * fact_small(s.c[a][1]) * fact_small(s.c[a][2]);
                hd_col[a][hd_n[a]] = g;  // ta_a = sum_g hdiv(a, g) Rc_g
                hd_val[a][hd_n[a]] = h / af;
                ++hd_n[a];
                hf_col[g][hf_n[g]] = a;  // P_g = sum_a hfull(a, g) ta_a
                hf_val[g][hf_n[g]] = h;
                ++hf_n[g];
            }
    }
};

// rel: the order-n block of delta^j tr^j, j >= 1 (dense, local slot indices of order n)
template <int N>
struct RelaxTables {
    static constexpr int M = nmom(N);
    static constexpr int len(int n) { return (n + 1) * (n + 2) / 2; }
    static constexpr int size() {
        int s = 0;
        for (int n = 2; n <= N; ++n) s += (n / 2) * len(n) * len(n);
        return s;
    }
    static constexpr int off(int n, int j) {
        int s = 0;
        for (int m = 2; m < n; ++m) s += (m / 2) * len(m) * len(m);
        return s + (j - 1) * len(n) * len(n);
    }
    double rel[size()] = {};
    // bd[n][j][m] = B(n, m) D(n - 2m, j - m) (Eq. bd): C_j = sum_{m <= j} s_m bd[n][j][m]
    double bd[N + 1][N / 2 + 1][N / 2 + 1] = {};
    constexpr RelaxTables() {
        for (int n = 2; n <= N; ++n)
            for (int j = 0; j <= n / 2; ++j)
                for (int m = 0; m <= j; ++m) bd[n][j][m] = coefB(n, m) * coefD(n - 2 * m, j - m);
        const SlotIndex<N> s;
        for (int n = 2; n <= N; ++n) {
            const int o = ord_off(n);
            for (int j = 1; j <= n / 2; ++j)
                for (int q = 0; q < len(n); ++q) {
                    double x[M] = {};
                    x[o + q] = 1.0;
                    for (int t = 1; t <= j; ++t) {  // trace: order n - 2(t-1) -> n - 2t
                        double y[M] = {};
                        for (int p = ord_off(n - 2 * t); p < ord_off(n - 2 * t + 1); ++p)
                            for (int k = 0; k < 3; ++k)
                                y[p] += double((s.c[p][k] + 2) * (s.c[p][k] + 1)) * x[s.with(p, k, s.c[p][k] + 2)];
                        for (int p = 0; p < M; ++p) x[p] = y[p];
                    }
                    for (int t = j; t >= 1; --t) {  // lift: order r - 2 -> r
                        const int r = n - 2 * t + 2;
                        double y[M] = {};
                        for (int p = ord_off(r); p < ord_off(r + 1); ++p) {
                            double acc = 0.0;
                            for (int k = 0; k < 3; ++k)
                                if (s.c[p][k] >= 2) acc += x[s.with(p, k, s.c[p][k] - 2)];
                            y[p] = acc / double(r * (r - 1));
                        }
                        for (int p = 0; p < M; ++p) x[p] = y[p];
                    }
                    for (int p = 0; p < len(n); ++p) rel[off(n, j) + p * len(n) + q] = x[o + p];
                }
        }
    }
};

// es: the ordered pairs of order-2 slots adding up to each order-4 slot
template <int N>
struct EsTables {
    static constexpr int M = nmom(N);
    int n[M] = {};
    int q1[M][8] = {};
    int q2[M][8] = {};
    constexpr EsTables() {
        const SlotIndex<N> s;
        for (int p = 0; p < M; ++p) {
            if (s.ord[p] != 4) continue;
            for (int a = ord_off(2); a < ord_off(3); ++a)
                for (int b = ord_off(2); b < ord_off(3); ++b)
                    if (s.c[a][0] + s.c[b][0] == s.c[p][0] && s.c[a][1] + s.c[b][1] == s.c[p][1] &&
                        s.c[a][2] + s.c[b][2] == s.c[p][2]) {
                        q1[p][n[p]] = a;
                        q2[p][n[p]] = b;
                        ++n[p];
                    }
        }
    }
};

template <int N>
struct MomentTables {
    SlotIndex<N> si;
    HermiteTables<N> h;
    RelaxTables<N> r;
    EsTables<N> es;
};

// The same tables in compact form for shared memory: slot indices as bytes, values in T.
template <int N, class T>
struct alignas(16) MomentSmem {
    static constexpr int M = nmom(N);
    static constexpr int NZ = HermiteTables<N>::kNZ;
    static constexpr int RS = RelaxTables<N>::size();
    T hd_val[M][NZ] = {};
    T hf_val[M][NZ] = {};
    T rel[RS] = {};
    T bd[N + 1][N / 2 + 1][N / 2 + 1] = {};
    unsigned char c[M][4] = {};  // multi-index components and order
    unsigned char hd_n[M] = {}, hd_col[M][NZ] = {};
    unsigned char hf_n[M] = {}, hf_col[M][NZ] = {};
    unsigned char es_n[M] = {}, es_q1[M][8] = {}, es_q2[M][8] = {};
    constexpr MomentSmem() = default;
    constexpr MomentSmem(const SlotIndex<N> &si, const HermiteTables<N> &h, const RelaxTables<N> &r,
                         const EsTables<N> &es) {
        for (int p = 0; p < M; ++p) {
            for (int k = 0; k < 3; ++k) c[p][k] = (unsigned char)si.c[p][k];
            c[p][3] = (unsigned char)si.ord[p];
            hd_n[p] = (unsigned char)h.hd_n[p];
            hf_n[p] = (unsigned char)h.hf_n[p];
            es_n[p] = (unsigned char)es.n[p];
            for (int q = 0; q < NZ; ++q) {
                hd_col[p][q] = (unsigned char)h.hd_col[p][q];
                hf_col[p][q] = (unsigned char)h.hf_col[p][q];
                hd_val[p][q] = T(h.hd_val[p][q]);
                hf_val[p][q] = T(h.hf_val[p][q]);
            }
            for (int q = 0; q < 8; ++q) {
                es_q1[p][q] = (unsigned char)es.q1[p][q];
                es_q2[p][q] = (unsigned char)es.q2[p][q];
            }
        }
        for (int i = 0; i < RS; ++i) rel[i] = T(r.rel[i]);
        for (int n = 0; n <= N; ++n)
            for (int j = 0; j <= N / 2; ++j)
                for (int m = 0; m <= N / 2; ++m) bd[n][j][m] = T(r.bd[n][j][m]);
    }
};

template <int N>
SMRT_D const MomentTables<N> &moment_tables();

static __device__ const MomentTables<4> kMomentTables4 = {SlotIndex<4>(), HermiteTables<4>(), RelaxTables<4>(), EsTables<4>()};
static __device__ const MomentTables<5> kMomentTables5 = {SlotIndex<5>(), HermiteTables<5>(), RelaxTables<5>(), EsTables<5>()};

template <>
SMRT_D const MomentTables<4> &moment_tables<4>() { return kMomentTables4; }
template <>
SMRT_D const MomentTables<5> &moment_tables<5>() { return kMomentTables5; }

// The shared-memory layout, prebuilt for the double kernels (the only users).
static __device__ const MomentSmem<4, double> kMomentSmem4 = MomentSmem<4, double>(
    SlotIndex<4>(), HermiteTables<4>(), RelaxTables<4>(), EsTables<4>());
static __device__ const MomentSmem<5, double> kMomentSmem5 = MomentSmem<5, double>(
    SlotIndex<5>(), HermiteTables<5>(), RelaxTables<5>(), EsTables<5>());

template <int N>
SMRT_D const MomentSmem<N, double> &moment_smem();
template <>
SMRT_D const MomentSmem<4, double> &moment_smem<4>() { return kMomentSmem4; }
template <>
SMRT_D const MomentSmem<5, double> &moment_smem<5>() { return kMomentSmem5; }

// Copy the prebuilt tables into shared memory with the block's threads, 16 bytes at a time
// (the caller synchronises).
template <int N>
SMRT_D void load_moment_smem(MomentSmem<N, double> &s) {
    const uint4 *src = reinterpret_cast<const uint4 *>(&moment_smem<N>());
    uint4 *dst = reinterpret_cast<uint4 *>(&s);
    constexpr int n16 = int(sizeof(MomentSmem<N, double>) / 16);
    for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = src[i];
}

}  // namespace smrt
