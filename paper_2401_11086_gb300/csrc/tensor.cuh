// tensor.cuh -- LB-SMRT collide-and-stream on three-dimensional tensor-product velocity sets
// (Yan & Shan, arXiv 2401.11086, Sec. 4.2: the 3D products D3Q{d^3} of the 1D rules D1Qd-P1,
// D3Q729 = D1Q9-P1^3 of degree 11 and D3Q4913 = D1Q17-P1^3 of degree 19), batched 1D lines
// along x.
//
// A cell holds d^3 populations: too many for registers, so no pass ever holds them all. The
// projection (Eq. an) and the rebuild (Eq. fi) factor over the three axes because the
// abscissae, the weights and He_alpha(xi) = prod_k He_{alpha_k}(xi_k) all do:
//   a3  raw moments R_(j,k,l) = sum_{a,b,c} df_abc e_a^j e_b^k e_c^l, |(j,k,l)| <= N, summed
//       x first (one x-line of d populations at a time, +-e pairs folded), then y, then z;
//   a7  f'_abc = w_a w_b w_c sum_(j,k,l) P_(j,k,l) e_a^j e_b^k e_c^l, summed z first, then
//       y, then x, each x-line stored as soon as it is formed.
// With d = 9 and N = 5 that is about 4.6k multiply-adds each way instead of 41k for the
// dense d^3 x 56 products. Between the two, the moment-space steps a2, a4-a6 are those of the
// other velocity sets (core.cuh), acting on 56 coefficients in registers.
//
// Library order: population i = a + d b + d^2 c has velocity (e_a, e_b, e_c), where the 1D
// order is a = 0 rest, 2p+1 = +E_p, 2p+2 = -E_p. The caller's order is arbitrary: its plane
// index for every library population sits in a table that each block copies to shared memory.
// Ghost populations (end states beyond a fixed x end) are kept in library order.
#pragma once


#include "kernels.cuh"
#include "moment_tables.cuh"

namespace smrt {

// D1Q9-P1 (Table 3, d = 9, degree 11): abscissae c {0, +-1, +-2, +-3, +-5}.
struct D1Q9P1 {
    static constexpr int Q1 = 9;
    static constexpr int NP1 = 4;
    static constexpr int DEGREE = 11;
    static constexpr double C_GUESS = 0.678;  // start of the scale search in the host solver
    static constexpr SMRT_HD int E(int p) { return p < 3 ? p + 1 : 5; }
};

// D1Q17-P1 (Table 3, d = 17, degree 19): abscissae c {0, +-1, ..., +-7, +-9}.
struct D1Q17P1 {
    static constexpr int Q1 = 17;
    static constexpr int NP1 = 8;
    static constexpr int DEGREE = 19;
    static constexpr double C_GUESS = 0.5639;
    static constexpr SMRT_HD int E(int p) { return p < 7 ? p + 1 : 9; }
};

template <class L1>
constexpr SMRT_HD int e1(int a) {
    return a == 0 ? 0 : ((a & 1) ? L1::E((a - 1) / 2) : -L1::E((a - 1) / 2));
}

constexpr int kMaxQ1 = 17;

template <class T>
struct TPArgs {
    const T *__restrict__ fin;
    T *__restrict__ fout;
    const InstanceInfo *__restrict__ inst;
    const int2 *__restrict__ tiles;    // (instance, first x) per block
    const T *__restrict__ ghosts;      // [instance][2][Q], library order
    const double *__restrict__ ghostsd;
    unsigned *health;
    const int *__restrict__ plane_idx; // caller plane of each library population
    long long stride;                  // elements per population plane
    double w1[kMaxQ1];                 // 1D weights, library order
    double cd;                         // lattice scale c
    unsigned step;
    int tma;                           // 1: the kernel's tensor maps describe fin and fout
};

// Tensor maps of the two states for the block-staged kernels: a 2D view [plane][stride] of a
// state (library order = caller order), box of kSeg elements x d planes (one x-row group).
struct TPMaps {
    CUtensorMap src;  // of TPArgs::fin
    CUtensorMap dst;  // of TPArgs::fout
};

// Shared-memory tables of one block: caller planes (Planes; the block-staged step reads them
// from global memory, and only when the caller's order is not the library's), the 1D abscissae
// (integers, as T) and the 1D weights (as T).
template <class L1, class T, bool Planes = true>
struct TPTables {
    static constexpr int Q = L1::Q1 * L1::Q1 * L1::Q1;
    static constexpr int kPow = 6;  // powers e^0 .. e^5 (N <= 5)
    int plane[Planes ? Q : 1];
    T e[L1::Q1];
    T w[L1::Q1];
    T pw[L1::Q1][kPow];  // e_a^k: the y and z passes read them instead of forming them per cell
};

template <class L1, class T, class U, bool Planes>
SMRT_D void tp_load_tables(const TPArgs<T> &a, TPTables<L1, U, Planes> &s) {
    if constexpr (Planes)
        for (int i = threadIdx.x; i < TPTables<L1, U>::Q; i += blockDim.x) s.plane[i] = a.plane_idx[i];
    if (threadIdx.x < L1::Q1) {
        const U ea = U(e1<L1>(threadIdx.x));
        s.e[threadIdx.x] = ea;
        s.w[threadIdx.x] = U(a.w1[threadIdx.x]);
        U p = U(1);
        for (int k = 0; k < TPTables<L1, U>::kPow; ++k, p *= ea) s.pw[threadIdx.x][k] = p;
    }
    __syncthreads();
}

template <class L1, int N, class T>
struct TPCell {
    static constexpr int Q1 = L1::Q1;
    static constexpr int NP1 = L1::NP1;
    static constexpr int M = nmom(N);

    // g_j = sum_a f_(a, b, c) e_a^j for the x-line starting at library index i0.
    template <class Pop>
    SMRT_D static void xline(Pop &pop, int i0, T (&g)[N + 1]) {
        const T f0 = pop(i0, ic<0>{});
        T S[NP1], D[NP1];
        static_for<NP1>([&](auto P) {
            constexpr int p = decltype(P)::value;
            const T fp = pop(i0 + 2 * p + 1, ic<2 * p + 1>{});
            const T fm = pop(i0 + 2 * p + 2, ic<2 * p + 2>{});
            S[p] = fp + fm;
            D[p] = fp - fm;
        });
        static_for<N + 1>([&](auto J) {
            constexpr int j = decltype(J)::value;
            T acc = (j == 0) ? f0 : T(0);
            static_for<NP1>([&](auto P) {
                constexpr int p = decltype(P)::value;
                constexpr double ej = double(ipow(L1::E(p), j));
                if constexpr (j == 0)
                    acc = acc + S[p];
                else if constexpr (j & 1)
                    acc = fma(T(ej), D[p], acc);
                else
                    acc = fma(T(ej), S[p], acc);
            });
            g[j] = acc;
        });
    }

    // a1 + a3: raw moments of the pulled populations; pop(i, ic<a>) returns population i
    // (library index) whose x-velocity index is a.
    template <class Pop>
    SMRT_D static void project(Pop &&pop, const T *s_e, T (&R)[M]) {
        static_for<M>([&](auto G) { R[decltype(G)::value] = T(0); });
#pragma unroll 1
        for (int cz = 0; cz < Q1; ++cz) {
            T h[N + 1][N + 1];
            static_for<N + 1>([&](auto J) {
                static_for<N + 1 - decltype(J)::value>([&](auto K) { h[decltype(J)::value][decltype(K)::value] = T(0); });
            });
            const int i0 = cz * Q1 * Q1;
            {  // b = rest: only k = 0
                T g[N + 1];
                xline(pop, i0, g);
                static_for<N + 1>([&](auto J) { h[decltype(J)::value][0] += g[decltype(J)::value]; });
            }
            static_for<NP1>([&](auto P) {
                constexpr int p = decltype(P)::value;
                T gp[N + 1], gm[N + 1];
                xline(pop, i0 + Q1 * (2 * p + 1), gp);
                xline(pop, i0 + Q1 * (2 * p + 2), gm);
                static_for<N + 1>([&](auto J) {
                    constexpr int j = decltype(J)::value;
                    const T s = gp[j] + gm[j], d = gp[j] - gm[j];
                    static_for<N + 1 - j>([&](auto K) {
                        constexpr int k = decltype(K)::value;
                        constexpr double ek = double(ipow(L1::E(p), k));
                        if constexpr (k == 0)
                            h[j][0] += s;
                        else if constexpr (k & 1)
                            h[j][k] = fma(T(ek), d, h[j][k]);
                        else
                            h[j][k] = fma(T(ek), s, h[j][k]);
                    });
                });
            });
            const T ec = s_e[cz];
            T pw[N + 1];
            pw[0] = T(1);
            static_for<N>([&](auto L) { pw[decltype(L)::value + 1] = pw[decltype(L)::value] * ec; });
            static_for<M>([&](auto G) {
                constexpr int g = decltype(G)::value;
                constexpr int j = mi_comp(g, 0), k = mi_comp(g, 1), l = mi_comp(g, 2);
                if constexpr (l == 0)
                    R[g] += h[j][k];
                else
                    R[g] = fma(pw[l], h[j][k], R[g]);
            });
        }
    }

    // Pieces of the same sums for a pipeline that sees one +-e_b pair of x-rows at a time.
    // g_j = sum_a f_a e_a^j over one x-row; row(ic<a>) returns the population with x-index a.
    template <class Row>
    SMRT_D static void xrow(const Row &row, T (&g)[N + 1]) {
        const T f0 = row(ic<0>{});
        T S[NP1], D[NP1];
        static_for<NP1>([&](auto P) {
            constexpr int p = decltype(P)::value;
            const T fp = row(ic<2 * p + 1>{});
            const T fm = row(ic<2 * p + 2>{});
            S[p] = fp + fm;
            D[p] = fp - fm;
        });
        static_for<N + 1>([&](auto J) {
            constexpr int j = decltype(J)::value;
            T acc = (j == 0) ? f0 : T(0);
            static_for<NP1>([&](auto P) {
                constexpr int p = decltype(P)::value;
                constexpr double ej = double(ipow(L1::E(p), j));
                if constexpr (j == 0)
                    acc = acc + S[p];
                else if constexpr (j & 1)
                    acc = fma(T(ej), D[p], acc);
                else
                    acc = fma(T(ej), S[p], acc);
            });
            g[j] = acc;
        });
    }
    // h_(j,k) += sum_b g_(b)j e_b^k for the rest row (e_b = 0) ...
    SMRT_D static void yrest(const T (&g)[N + 1], T (&h)[N + 1][N + 1]) {
        static_for<N + 1>([&](auto J) { h[decltype(J)::value][0] += g[decltype(J)::value]; });
    }
    // ... and for the rows +e_b (gp) and -e_b (gm)
    SMRT_D static void ypair(const T (&gp)[N + 1], const T (&gm)[N + 1], T eb, T (&h)[N + 1][N + 1]) {
        T pw[N + 1];
        pw[0] = T(1);
        static_for<N>([&](auto K) { pw[decltype(K)::value + 1] = pw[decltype(K)::value] * eb; });
        ypair_pw(gp, gm, pw, h);
    }
    // ... with the powers e_b^k given (pw[k], k <= N, e.g. a shared-memory table row)
    template <class PW>
    SMRT_D static void ypair_pw(const T (&gp)[N + 1], const T (&gm)[N + 1], const PW &pw, T (&h)[N + 1][N + 1]) {
        static_for<N + 1>([&](auto J) {
            constexpr int j = decltype(J)::value;
            const T s = gp[j] + gm[j], d = gp[j] - gm[j];
            h[j][0] += s;
            static_for<N - j>([&](auto K) {
                constexpr int k = decltype(K)::value + 1;
                h[j][k] = fma(pw[k], (k & 1) ? d : s, h[j][k]);
            });
        });
    }
    // R_(j,k,l) += e_c^l h_(j,k) at the end of z-plane c; h is cleared for the next one
    SMRT_D static void zfold(T (&h)[N + 1][N + 1], T ec, T (&R)[M]) {
        T pw[N + 1];
        pw[0] = T(1);
        static_for<N>([&](auto L) { pw[decltype(L)::value + 1] = pw[decltype(L)::value] * ec; });
        zfold_pw(h, pw, R);
    }
    template <class PW>
    SMRT_D static void zfold_pw(T (&h)[N + 1][N + 1], const PW &pw, T (&R)[M]) {
        static_for<M>([&](auto G) {
            constexpr int g = decltype(G)::value;
            constexpr int j = mi_comp(g, 0), k = mi_comp(g, 1), l = mi_comp(g, 2);
            if constexpr (l == 0)
                R[g] += h[j][k];
            else
                R[g] = fma(pw[l], h[j][k], R[g]);
        });
        static_for<N + 1>([&](auto J) {
            static_for<N + 1 - decltype(J)::value>([&](auto K) { h[decltype(J)::value][decltype(K)::value] = T(0); });
        });
    }
    // Rebuild side: Pc_(j,k) = sum_l P_(j,k,l) e_c^l for z-plane c ...
    template <class U>
    SMRT_D static void zplane(const U (&P)[M], U ec, U (&Pc)[N + 1][N + 1]) {
        U pw[N + 1];
        pw[0] = U(1);
        static_for<N>([&](auto L) { pw[decltype(L)::value + 1] = pw[decltype(L)::value] * ec; });
        zplane_pw(P, pw, Pc);
    }
    template <class U, class PW>
    SMRT_D static void zplane_pw(const U (&P)[M], const PW &pw, U (&Pc)[N + 1][N + 1]) {
        static_for<N + 1>([&](auto J) {
            constexpr int j = decltype(J)::value;
            static_for<N + 1 - j>([&](auto K) {
                constexpr int k = decltype(K)::value;
                U acc = P[mi_pos(j, k, 0)];
                static_for<N - j - k>([&](auto L) {
                    constexpr int l = decltype(L)::value + 1;
                    acc = fma(pw[l], P[mi_pos(j, k, l)], acc);
                });
                Pc[j][k] = acc;
            });
        });
    }
    // ... and the x-row coefficients Pb_j = sum_k Pc_(j,k) (+-e_b)^k of the rows +e_b, -e_b
    template <class U>
    SMRT_D static void yrows(const U (&Pc)[N + 1][N + 1], U eb, U (&Pp)[N + 1], U (&Pm)[N + 1]) {
        U pw[N + 1];
        pw[0] = U(1);
        static_for<N>([&](auto K) { pw[decltype(K)::value + 1] = pw[decltype(K)::value] * eb; });
        yrows_pw(Pc, pw, Pp, Pm);
    }
    template <class U, class PW>
    SMRT_D static void yrows_pw(const U (&Pc)[N + 1][N + 1], const PW &pw, U (&Pp)[N + 1], U (&Pm)[N + 1]) {
        static_for<N + 1>([&](auto J) {
            constexpr int j = decltype(J)::value;
            U ev = Pc[j][0], od = U(0);
            static_for<N - j>([&](auto K) {
                constexpr int k = decltype(K)::value + 1;
                if constexpr (k & 1)
                    od = fma(pw[k], Pc[j][k], od);
                else
                    ev = fma(pw[k], Pc[j][k], ev);
            });
            Pp[j] = ev + od;
            Pm[j] = ev - od;
        });
    }

    SMRT_D static void relax_es(T (&v)[M], T rho, T A, T B, T b) { relax_es_divided<N, T>(v, rho, A, B, b); }

    // a2, a4-a6 on the raw moments: R (in) -> rebuild coefficients P (out, same slots) with
    // f'_i = w_i sum_gamma P_gamma e_i^gamma. model 1: ES-BGK with parameter es_b, else SMRT.
    // Returns false when rho or theta is not positive.
    SMRT_D static bool collide_moments(T (&R)[M], T c, const T *tauA, const T *tauB, int model = 0,
                                       T es_b = T(0)) {
        T cp[N + 1];
        cp[0] = T(1);
        static_for<N>([&](auto J) { cp[decltype(J)::value + 1] = cp[decltype(J)::value] * c; });
        T Rc[M];
        static_for<M>([&](auto G) {
            constexpr int g = decltype(G)::value;
            Rc[g] = R[g] * cp[mi_order(g)];
        });
        // a2: rho - 1 = Rc_0, rho u = Rc_1, E - 3 = tr Rc_2 (deviations from w_i)
        const T rhom1 = Rc[0];
        const T rho = T(1) + rhom1;
        const T ir = rcp(rho);
        const T u[3] = {Rc[mi_pos(1, 0, 0)] * ir, Rc[mi_pos(0, 1, 0)] * ir, Rc[mi_pos(0, 0, 1)] * ir};
        const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const T em3 = Rc[mi_pos(2, 0, 0)] + Rc[mi_pos(0, 2, 0)] + Rc[mi_pos(0, 0, 2)];
        const T thm1 = (em3 - T(3) * rhom1 - rho * uu) * ir * T(1.0 / 3.0);
        const T theta = T(1) + thm1;
        const bool ok = (rho > T(0)) && (theta > T(0));
        // a3 (end): ta_alpha = a_alpha / alpha! = sum_gamma hdiv(alpha, gamma) Rc_gamma
        T v[M];
        static_for<M>([&](auto A) {
            constexpr int al = decltype(A)::value;
            T acc = T(0);
            static_for<M>([&](auto G) {
                constexpr int g = decltype(G)::value;
                constexpr double h = hdiv(al, g);
                if constexpr (h != 0.0) acc = fma(T(h), Rc[g], acc);
            });
            v[al] = acc;
        });
        v[0] = rho;
        to_local_divided<N, T>(v, u, theta, thm1);
        // a5
        if (model == 1) {
            relax_es(v, rho, tauA[0], tauB[0], es_b);
        } else {
            T s[ntau(N)];
            static_for<ntau(N)>([&](auto K) {
                constexpr int k = decltype(K)::value;
                s[k] = T(1) - rcp_tau<T>(tauA[k], tauB[k], rho);
            });
            static_for<N - 1>([&](auto Nn) { relax_order<N, decltype(Nn)::value + 2, T>(v, s); });
        }
        // a6
        const T sq = theta * rsq(theta);
        T sp[N + 1];
        sp[0] = T(1);
        static_for<N>([&](auto J) { sp[decltype(J)::value + 1] = sp[decltype(J)::value] * sq; });
        static_for<M>([&](auto A) {
            constexpr int p = decltype(A)::value;
            if constexpr (mi_order(p) == 0)
                v[p] = rho;
            else if constexpr (mi_order(p) == 1)
                v[p] = T(0);
            else
                v[p] *= sp[mi_order(p)];
        });
        T G[3][N + 1];
        static_for<3>([&](auto K) {
            constexpr int k = decltype(K)::value;
            maxwell_divided<N, T>(G[k], u[k], thm1);
        });
        binomial_divided<N, T>(v, G);
        v[0] = rhom1;  // deviation from the coefficients of w_i
        to_rebuild(v, c, R);
        return ok;
    }

    // The steps of collide_moments (a2, a4-a6) with one cell's coefficients spread over the 32
    // lanes of a warp: lane l owns slots l and l + 32, each step reads the whole vector from
    // shared memory and writes its own slots (the per-slot constants come from MomentTables).
    // Executing the single-thread version on every lane would spend a full warp's FP64 issue
    // on each scalar operation. R (shared, M values): raw moments in, rebuild coefficients out;
    // w (shared, M values) and gs (shared, 3 (N + 1) values): scratch. Every lane calls it.
    SMRT_D static bool collide_moments_lanes(const MomentSmem<N, double> &tb, T *R, T *w, T *gs, T c, const T *tauA,
                                             const T *tauB, int model, T es_b) {
        const int lane = threadIdx.x & 31;
        const int pa = lane, pb = lane + 32;
        const bool two = pb < M;
        // the lane's slots: components and orders in registers
        const int ca[3] = {tb.c[pa][0], tb.c[pa][1], tb.c[pa][2]};
        const int cb[3] = {two ? tb.c[pb][0] : 0, two ? tb.c[pb][1] : 0, two ? tb.c[pb][2] : 0};
        const int oa = tb.c[pa][3], ob = two ? tb.c[pb][3] : 0;
        auto ipow_t = [](T x, int e) {
            T r = T(1);
            for (int i = 0; i < e; ++i) r *= x;
            return r;
        };
        auto axis_pass = [&](const T *src, T *dst, int k) {  // dst = T_k src (one binomial axis)
            auto one = [&](int p, const int (&cc)[3]) {
                const int ak = cc[k];
                T acc = src[p];
                for (int b = 0; b < ak; ++b) {
                    const int q = k == 0 ? mi_pos(b, cc[1], cc[2]) : (k == 1 ? mi_pos(cc[0], b, cc[2]) : mi_pos(cc[0], cc[1], b));
                    acc = fma(gs[k * (N + 1) + ak - b], src[q], acc);
                }
                dst[p] = acc;
            };
            one(pa, ca);
            if (two) one(pb, cb);
            __syncwarp();
        };
        // Rc = c^|gamma| R
        w[pa] = R[pa] * ipow_t(c, oa);
        if (two) w[pb] = R[pb] * ipow_t(c, ob);
        __syncwarp();
        // a2 (every lane): rho - 1 = Rc_0, rho u = Rc_1, E - 3 = tr Rc_2
        const T rhom1 = w[0];
        const T rho = T(1) + rhom1;
        const T ir = rcp(rho);
        const T u0 = w[mi_pos(1, 0, 0)] * ir, u1 = w[mi_pos(0, 1, 0)] * ir, u2 = w[mi_pos(0, 0, 1)] * ir;
        const T uu = u0 * u0 + u1 * u1 + u2 * u2;
        const T thm1 = (w[mi_pos(2, 0, 0)] + w[mi_pos(0, 2, 0)] + w[mi_pos(0, 0, 2)] - T(3) * rhom1 - rho * uu) * ir *
                       T(1.0 / 3.0);
        const T theta = T(1) + thm1;
        const bool ok = (rho > T(0)) && (theta > T(0));
        // ta = hdiv Rc (into R), full a_0 = rho
        auto hd_row = [&](int p) {
            T acc = T(0);
            for (int i = 0; i < tb.hd_n[p]; ++i) acc = fma(tb.hd_val[p][i], w[tb.hd_col[p][i]], acc);
            R[p] = p == 0 ? rho : acc;
        };
        hd_row(pa);
        if (two) hd_row(pb);
        // a4: T(-u, 2 - theta) then theta^(-|beta|/2)
        if (lane < 3) {
            T G[N + 1];
            maxwell_divided<N, T>(G, lane == 0 ? -u0 : (lane == 1 ? -u1 : -u2), -thm1);
            for (int j = 0; j <= N; ++j) gs[lane * (N + 1) + j] = G[j];
        }
        __syncwarp();
        axis_pass(R, w, 0);
        axis_pass(w, R, 1);
        axis_pass(R, w, 2);
        const T is = rsq(theta);
        w[pa] *= ipow_t(is, oa);
        if (two) w[pb] *= ipow_t(is, ob);
        __syncwarp();
        // a5: w -> R
        if (model == 1) {
            const T tau = fma(tauB[0], rho, tauA[0]) * ir;
            const T om = rcp(tau);
            const T bp = T(1) - (T(1) - es_b) * tau * rcp(fma(T(-0.5), es_b, tau));
            const T sr = T(1) - om, s2 = fma(om, bp, sr), k4 = om * bp * bp * T(0.5) * ir;
            auto es_slot = [&](int p, int n) {
                T v = w[p];
                if (n == 2) {
                    v *= s2;
                } else if (n == 4) {
                    T t4 = T(0);
                    for (int i = 0; i < tb.es_n[p]; ++i) t4 = fma(w[tb.es_q1[p][i]], w[tb.es_q2[p][i]], t4);
                    v = fma(k4, t4, sr * v);
                } else if (n >= 3) {
                    v *= sr;
                }
                R[p] = v;
            };
            es_slot(pa, oa);
            if (two) es_slot(pb, ob);
        } else {
            auto smrt_slot = [&](int p, int n) {
                if (n < 2) {
                    R[p] = w[p];
                    return;
                }
                const int k0 = tau_slot(n, 0);  // s_m for m = 0, 1, 2 (n <= 5)
                const T s0 = T(1) - rcp_tau<T>(tauA[k0], tauB[k0], rho);
                const T s1 = T(1) - rcp_tau<T>(tauA[k0 + 1], tauB[k0 + 1], rho);
                const T s2 = n >= 4 ? T(1) - rcp_tau<T>(tauA[k0 + 2], tauB[k0 + 2], rho) : T(0);
                const int len = (n + 1) * (n + 2) / 2, o = ord_off(n), lp = p - o;
                T acc = s0 * w[p];  // C_0 = s_0 B(n,0) D(n,0) = s_0
                for (int j = 1; j <= n / 2; ++j) {
                    T Cj = s0 * T(tb.bd[n][j][0]);
                    Cj = fma(s1, T(tb.bd[n][j][1]), Cj);
                    if (j >= 2) Cj = fma(s2, T(tb.bd[n][j][2]), Cj);
                    const T *row = tb.rel + RelaxTables<N>::off(n, j) + lp * len;
                    T dot = T(0);
                    for (int q = 0; q < len; ++q) dot = fma(row[q], w[o + q], dot);
                    acc = fma(Cj, dot, acc);
                }
                R[p] = acc;
            };
            smrt_slot(pa, oa);
            if (two) smrt_slot(pb, ob);
        }
        // a6: theta^(|beta|/2), order 0 = rho, order 1 = 0, then T(u, theta)
        const T sq = theta * is;
        auto back_scale = [&](int p, int n) { R[p] = n == 0 ? rho : (n == 1 ? T(0) : R[p] * ipow_t(sq, n)); };
        back_scale(pa, oa);
        if (two) back_scale(pb, ob);
        if (lane < 3) {
            T G[N + 1];
            maxwell_divided<N, T>(G, lane == 0 ? u0 : (lane == 1 ? u1 : u2), thm1);
            for (int j = 0; j <= N; ++j) gs[lane * (N + 1) + j] = G[j];
        }
        __syncwarp();
        axis_pass(R, w, 0);
        axis_pass(w, R, 1);
        axis_pass(R, w, 2);
        if (lane == 0) w[0] = rhom1;  // deviation from the coefficients of w_i
        __syncwarp();
        // P_gamma = c^|gamma| sum_alpha hfull(alpha, gamma) ta_alpha (into R)
        auto hf_row = [&](int p, int n) {
            T acc = T(0);
            for (int i = 0; i < tb.hf_n[p]; ++i) acc = fma(tb.hf_val[p][i], w[tb.hf_col[p][i]], acc);
            R[p] = acc * ipow_t(c, n);
        };
        hf_row(pa, oa);
        if (two) hf_row(pb, ob);
        __syncwarp();
        return ok;
    }

    // P_gamma = c^|gamma| sum_alpha hfull(alpha, gamma) ta_alpha (the monomial form of Eq. fi)
    template <class U>
    SMRT_D static void to_rebuild(const U (&ta)[M], U c, U (&P)[M]) {
        U cp[N + 1];
        cp[0] = U(1);
        static_for<N>([&](auto J) { cp[decltype(J)::value + 1] = cp[decltype(J)::value] * c; });
        static_for<M>([&](auto G) {
            constexpr int g = decltype(G)::value;
            U acc = U(0);
            static_for<M>([&](auto A) {
                constexpr int al = decltype(A)::value;
                constexpr double h = hfull(al, g);
                if constexpr (h != 0.0) acc = fma(U(h), ta[al], acc);
            });
            P[g] = acc * cp[mi_order(g)];
        });
    }

    // One x-line of the rebuild: f'_(a,b,c) = wbc w_a sum_j Pb_j e_a^j, pairs folded.
    template <class U, class Put>
    SMRT_D static void emit_x(const U (&Pb)[N + 1], U wbc, const U *s_w, int i0, Put &put) {
        put(i0, wbc * s_w[0] * Pb[0]);
        static_for<NP1>([&](auto Q) {
            constexpr int q = decltype(Q)::value;
            U ev = Pb[0], od = U(0);
            static_for<N>([&](auto J) {
                constexpr int j = decltype(J)::value + 1;
                constexpr double ej = double(ipow(L1::E(q), j));
                if constexpr (j & 1)
                    od = fma(U(ej), Pb[j], od);
                else
                    ev = fma(U(ej), Pb[j], ev);
            });
            const U w = wbc * s_w[2 * q + 1];
            put(i0 + 2 * q + 1, w * (ev + od));
            put(i0 + 2 * q + 2, w * (ev - od));
        });
    }

    // a7: every population from the rebuild coefficients P; put(i, value) receives population
    // i (library index). s_e, s_w: 1D abscissae and weights in U.
    template <class U, class Put>
    SMRT_D static void rebuild(const U (&P)[M], const U *s_e, const U *s_w, Put &&put) {
#pragma unroll 1
        for (int cz = 0; cz < Q1; ++cz) {
            const U ec = s_e[cz], wc = s_w[cz];
            U pw[N + 1];
            pw[0] = U(1);
            static_for<N>([&](auto L) { pw[decltype(L)::value + 1] = pw[decltype(L)::value] * ec; });
            U Pc[N + 1][N + 1];
            static_for<N + 1>([&](auto J) {
                constexpr int j = decltype(J)::value;
                static_for<N + 1 - j>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    U acc = P[mi_pos(j, k, 0)];
                    static_for<N - j - k>([&](auto L) {
                        constexpr int l = decltype(L)::value + 1;
                        acc = fma(pw[l], P[mi_pos(j, k, l)], acc);
                    });
                    Pc[j][k] = acc;
                });
            });
            const int i0 = cz * Q1 * Q1;
            {  // b = rest
                U Pb[N + 1];
                static_for<N + 1>([&](auto J) { Pb[decltype(J)::value] = Pc[decltype(J)::value][0]; });
                emit_x<U>(Pb, wc * s_w[0], s_w, i0, put);
            }
            static_for<NP1>([&](auto Pp) {
                constexpr int p = decltype(Pp)::value;
                U ev[N + 1], od[N + 1];
                static_for<N + 1>([&](auto J) {
                    constexpr int j = decltype(J)::value;
                    U e0 = Pc[j][0], o0 = U(0);
                    static_for<N - j>([&](auto K) {
                        constexpr int k = decltype(K)::value + 1;
                        constexpr double ek = double(ipow(L1::E(p), k));
                        if constexpr (k & 1)
                            o0 = fma(U(ek), Pc[j][k], o0);
                        else
                            e0 = fma(U(ek), Pc[j][k], e0);
                    });
                    ev[j] = e0;
                    od[j] = o0;
                });
                const U wbc = wc * s_w[2 * p + 1];
                U Pb[N + 1];
                static_for<N + 1>([&](auto J) { Pb[decltype(J)::value] = ev[decltype(J)::value] + od[decltype(J)::value]; });
                emit_x<U>(Pb, wbc, s_w, i0 + Q1 * (2 * p + 1), put);
                static_for<N + 1>([&](auto J) { Pb[decltype(J)::value] = ev[decltype(J)::value] - od[decltype(J)::value]; });
                emit_x<U>(Pb, wbc, s_w, i0 + Q1 * (2 * p + 2), put);
            });
        }
    }

    // Order-N equilibrium of (rho, u, theta) as deviations from w_i: rebuild coefficients in U.
    template <class U>
    SMRT_D static void equilibrium(U rho, const U (&u)[3], U theta, U c, U (&P)[M]) {
        U G[3][N + 1];
        static_for<3>([&](auto K) {
            constexpr int k = decltype(K)::value;
            maxwell_divided<N, U>(G[k], u[k], theta - U(1));
        });
        U ta[M];
        static_for<M>([&](auto A) {
            constexpr int p = decltype(A)::value;
            ta[p] = rho * G[0][mi_comp(p, 0)] * G[1][mi_comp(p, 1)] * G[2][mi_comp(p, 2)];
        });
        ta[0] = rho - U(1);
        to_rebuild<U>(ta, c, P);
    }
};

// One plain arrival on mbarrier b (a warp's release of a stage buffer).
SMRT_D void mbar_arrive(unsigned long long *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
// One element global -> shared by an asynchronous copy (4 or 8 bytes, element-aligned) ...
template <class T>
SMRT_D void cp_async_elem(T *dst, const T *src) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src), "n"(int(sizeof(T)))
                 : "memory");
}
// ... and the phase of mbarrier b waits for every such copy this thread has issued (the
// barrier's pending count is raised now and lowered when they complete).
SMRT_D void cp_async_mbar_arrive(unsigned long long *b) {
    asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(smem_addr(b)) : "memory");
}

// ------------------------------------------------------------------ block-staged line tile
// A block of W warps owns a tile of 32 W consecutive cells of one line (warp w takes cells
// 32 w .. 32 w + 31, one per lane) and one copy pipeline. The step's d^3 pulls per cell reach
// shared memory by stage: stage st covers z-plane c = st / (NP1 + 1) and, within it, either the
// rest x-row (e_b = 0, d planes) or the pair of x-rows +e_b, -e_b (2 d planes). Each plane
// arrives as one contiguous x-segment [x0 - k - E_max, x0 + 32 W - 1 - k + E_max] (every pull of
// the tile, rounded out to 16 bytes) that all the block's warps read, so a halo of 2 E_max is
// loaded once per 32 W cells and each copied row is 32 W cells long. kStages fills are in
// flight: each buffer has a "full" mbarrier (the copy's bytes) and an "empty" one (one arrival
// per warp that is done with the buffer), which warp 0 waits on before refilling it. No
// block-wide barrier is taken inside a tile; the warps drift up to kStages stages apart.
// (Measured on 512 Table 3 shocks, D3Q729 float, 128-cell tiles: 0.248 ms per step; five
// stages 0.271 ms; refills issued by whichever warp releases a buffer last, counted by shared
// atomics, 0.259 ms; one warp per tile, 0.287 ms.)
template <class L1, class T, int W>
struct TPBlockStage {
    static constexpr int kW = 32 * W;                   // cells per block tile
    static constexpr int kStages = 3;                   // fills in flight per block
    static constexpr int kAlign = 16 / int(sizeof(T));  // elements per 16 bytes
    static constexpr int kEmax = L1::E(L1::NP1 - 1);    // largest |e| of the 1D rule
    static constexpr int kSeg = kW + ((2 * kEmax + kAlign - 1) + kAlign - 1) / kAlign * kAlign;
    static_assert(kSeg <= 256, "a tensor-map box spans at most 256 elements");
    // a stage buffer holds two groups of d rows (the +e_b and -e_b x-rows), each group
    // starting 128-byte aligned so that one tensor-map box fills it
    static constexpr int kGrp = int((L1::Q1 * kSeg * sizeof(T) + 127) / 128 * 128 / sizeof(T));
    // then the end-state populations of the stage's planes, [left, right][2 d], for the pulls
    // from beyond a line's fixed ends
    static constexpr int kGhost = int((4 * L1::Q1 * sizeof(T) + 127) / 128 * 128 / sizeof(T));
    static constexpr int kStage = 2 * kGrp + kGhost;    // elements per stage buffer
    static constexpr int kPerZ = L1::NP1 + 1;           // stages per z-plane
    static constexpr int kTotal = L1::Q1 * kPerZ;       // stages per step
    static_assert(kTotal % kStages == 0, "each tile starts the buffers' cycle at buffer 0");
    static_assert(kStages * 16 <= 128, "the full and empty mbarriers fit the 128-byte head");
    static constexpr size_t kBytes = 128 + size_t(kStages) * kStage * sizeof(T);  // mbarriers, buffers
};

// ------------------------------------------------------------------ x-row sums on tensor cores
// The x-row sums of one stage, g_j = sum_a f_a e_a^j for each of the warp's 32 cells and the
// stage's one or two x-rows, as one warp-wide matrix product: rows (x-row, cell), columns
// j = 0..7 (those above N are zero), inner index a = 1 .. d - 1 in k-steps of 8; the rest
// velocity (e_0 = 0) adds to g_0 only and seeds the accumulator. mma.sync m16n8k8 with TF32
// operands and FP32 accumulation; single-precision accuracy from the operand split of Ootomo &
// Yokota (2022, "Recovering single precision accuracy from Tensor Cores while surpassing the
// FP32 theoretical peak performance"): f = f_hi + f_lo with f_hi = f rounded to TF32 and f_lo
// the remainder rounded to TF32 (each rounding within 2^-11 relative), e^j = E_hi + E_lo
// likewise and exactly (e^j <= 9^5 has at most 16 significant bits, E_lo at most 5), and
// g = f_lo E_hi + f_hi E_lo + f_hi E_hi; the dropped f_lo E_lo and the rounding of f_lo are
// each below 2^-22 of |f| e^j.
// m16n8k8 TF32 fragments, lane = 4 r + q: A rows r and r + 8, columns q and q + 4; B rows
// (inner index) q and q + 4, column r; C rows r and r + 8, columns 2q and 2q + 1.
template <class L1, int N>
struct TPTensorRows {
    static constexpr int KS = (L1::Q1 - 1) / 8;  // k-steps over a = 1 .. d - 1
    static_assert((L1::Q1 - 1) % 8 == 0 && N + 1 <= 8, "k-steps of 8 velocities, j <= 7");
    static constexpr int kPitch = 10;            // floats per (x-row, cell) row of the scratch
    unsigned bhi[KS][2], blo[KS][2];             // B fragments, e_a^j split in two
    int off[KS][2];                              // a SEG - e_a for the lane's two columns
    int r, q;

    SMRT_D static unsigned tf32(float x) {
        unsigned u;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
        return u;
    }
    SMRT_D static void mma(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
        asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
            "{%8, %9}, {%0, %1, %2, %3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }

    // seg: elements per staged row
    SMRT_D void init(int lane, int seg) {
        r = lane >> 2;
        q = lane & 3;
#pragma unroll
        for (int ks = 0; ks < KS; ++ks)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int av = 8 * ks + q + 4 * h + 1;
                int e = 0;
                static_for<L1::Q1>([&](auto A) {
                    if (decltype(A)::value == av) e = e1<L1>(decltype(A)::value);
                });
                off[ks][h] = av * seg - e;
                float pw = r <= N ? 1.f : 0.f;  // e^r, exact in float
                for (int j = 0; j < r; ++j) pw *= float(e);
                const unsigned hi = tf32(pw);
                bhi[ks][h] = hi;
                blo[ks][h] = tf32(pw - __uint_as_float(hi));
            }
    }

    // g[x][j], x < NR, for the lane's cell: the pull of x-row x by velocity a of cell c sits at
    // bs[x grp + a SEG + tb0 + c - e_a]. Every lane calls it. The first NR 32 kPitch floats of bs
    // serve as scratch to hand each cell its row sums, so bs is overwritten.
    template <int NR>
    SMRT_D void rows(float *bs, int grp, int tb0, int lane, float (&g)[NR][N + 1]) const {
        float acc[NR][2][4];
#pragma unroll
        for (int x = 0; x < NR; ++x)
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const float *p = bs + x * grp + tb0 + 16 * mt + r;
                float(&d)[4] = acc[x][mt];
                d[0] = q == 0 ? p[0] : 0.f;  // the rest velocity: column j = 0
                d[1] = 0.f;
                d[2] = q == 0 ? p[8] : 0.f;
                d[3] = 0.f;
#pragma unroll
                for (int ks = 0; ks < KS; ++ks) {
                    const float v[4] = {p[off[ks][0]], p[off[ks][0] + 8], p[off[ks][1]], p[off[ks][1] + 8]};
                    unsigned ahi[4], alo[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        ahi[i] = tf32(v[i]);
                        alo[i] = tf32(v[i] - __uint_as_float(ahi[i]));
                    }
                    mma(d, alo, bhi[ks][0], bhi[ks][1]);
                    mma(d, ahi, blo[ks][0], blo[ks][1]);
                    mma(d, ahi, bhi[ks][0], bhi[ks][1]);
                }
            }
        __syncwarp();  // every lane holds its operands: the buffer is free
        if (2 * q <= N) {
#pragma unroll
            for (int x = 0; x < NR; ++x)
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    float *o = bs + (x * 32 + 16 * mt + r) * kPitch + 2 * q;
                    *reinterpret_cast<float2 *>(o) = make_float2(acc[x][mt][0], acc[x][mt][1]);
                    *reinterpret_cast<float2 *>(o + 8 * kPitch) = make_float2(acc[x][mt][2], acc[x][mt][3]);
                }
        }
        __syncwarp();
#pragma unroll
        for (int x = 0; x < NR; ++x)
            static_for<N + 1>([&](auto J) { g[x][decltype(J)::value] = bs[(x * 32 + lane) * kPitch + decltype(J)::value]; });
    }
};

// One block tile of the step; every thread of the block calls it. buf, full, empty: the block's
// stage buffers and their mbarriers; nt: tiles this block has stepped before (the buffers'
// phases follow from it: each tile makes kTotal / kStages uses of every buffer). Returns false,
// with LB_HEALTH_TIMEOUT in the health word, when a wait did not end within its bound (warp 0
// then lets the fills it has in flight land before it leaves).
// tm: tensor map of fin (one box per x-row group), or null to copy plane by plane.
// TC (float, one warp per block): the x-row sums of every stage on the tensor cores.
// Ident: the caller's plane order is the library's (no plane table lookups on the stores).
template <class L1, int N, class T, int W, bool FixedX, bool Coherent, bool TC = false, bool Ident = false>
SMRT_D bool tp_block_tile(const TPArgs<T> &a, const TPTables<L1, T, false> &s, const T *__restrict__ fin,
                          T *__restrict__ fout, int tile_index, T *buf, unsigned long long *full,
                          unsigned long long *empty, unsigned nt, const CUtensorMap *tm) {
    using C = TPCell<L1, N, T>;
    using S = TPBlockStage<L1, T, W>;
    static_assert(N + 1 <= TPTables<L1, T>::kPow, "the powers table holds e^0 .. e^5");
    static_assert(!TC || (W == 1 && std::is_same<T, float>::value),
                  "tensor-core x-rows: float states, one warp per block (its stage buffer is its scratch)");
    constexpr int Q1 = L1::Q1;
    constexpr int NP1 = L1::NP1;
    constexpr int P2 = Q1 * Q1;
    constexpr int Q = P2 * Q1;
    constexpr int EM = S::kEmax;
    constexpr int SEG = S::kSeg;
    constexpr int NS = S::kStages;
    const int warp = int(threadIdx.x >> 5), lane = int(threadIdx.x & 31);
    const int2 tile = a.tiles[tile_index];
    const InstanceInfo &in = a.inst[tile.x];
    const int x0 = tile.y, x = x0 + 32 * warp + lane, L = in.nx, kx = in.kx;
    const bool active = x < L;
    const long long base = in.cell_off;
    const T *gl = a.ghosts + (long long)tile.x * 2 * Q;
    const T *gr = gl + Q;
    // every plane contributes elements [g_al, g_al + SEG) of itself, clipped to [0, stride)
    const long long g_al = (base + x0 - kx - EM) & ~(long long)(S::kAlign - 1);
    const long long cs = g_al < 0 ? 0 : g_al;
    const long long ce = (g_al + SEG < a.stride) ? g_al + SEG : a.stride;
    const unsigned nbytes = unsigned((ce - cs) * (long long)sizeof(T));
    const int dst_off = int(cs - g_al);
    const unsigned long long u0 = (unsigned long long)nt * (S::kTotal / NS);  // earlier uses of each buffer
    // does any pull of the tile come from beyond the left / right fixed end (block-uniform)?
    const int xmax = (x0 + 32 * W < L ? x0 + 32 * W : L) - 1;
    const bool needL = FixedX && x0 - EM - kx < 0;
    const bool needR = FixedX && xmax + EM - kx >= L;
    // caller plane of library population i
    auto plane = [&](int i) -> long long {
        if constexpr (Ident)
            return i;
        else
            return __ldg(a.plane_idx + i);
    };
    // warp 0: bit b of pending says buffer b has a fill issued and not yet waited for, bit b of
    // fpar is that fill's phase parity
    unsigned pending = 0u, fpar = 0u;
    // warp 0 only: refill the buffer of stage st once every warp has released its previous fill
    auto issue = [&](int st) -> bool {
        const int sb = st % NS;
        const unsigned long long u = u0 + (unsigned long long)(st / NS);  // this fill is use u of buffer sb
        if (u > 0 && !__all_sync(0xffffffffu, mbar_wait(empty + sb, unsigned((u - 1) & 1ull)))) return false;
        pending |= 1u << sb;
        fpar = (fpar & ~(1u << sb)) | (unsigned(u & 1ull) << sb);
        const int cz = st / S::kPerZ, p = st % S::kPerZ;
        const int nplanes = p ? 2 * Q1 : Q1;
        const int k0 = p ? (2 * p - 1) * Q1 : 0;  // in-plane index of the stage's first population
        unsigned long long *b = full + sb;
        T *sbuf = buf + size_t(sb) * S::kStage;
        if constexpr (Coherent) fence_async_global();
        fence_async_shared();
        if (needL || needR) {  // the stage's end-state populations ride along with its fill
            T *gs = sbuf + 2 * S::kGrp;
            const int i0 = cz * P2 + k0;
            for (int k = lane; k < nplanes; k += 32) {
                if (needL) cp_async_elem(gs + k, gl + i0 + k);
                if (needR) cp_async_elem(gs + 2 * Q1 + k, gr + i0 + k);
            }
            cp_async_mbar_arrive(b);
            __syncwarp();  // before lane 0's arrival below can complete the phase
        }
        if (tm) {  // one box per row group: d planes (library order) x SEG elements from g_al
            if (lane == 0) {
                mbar_arrive_expect_tx(b, unsigned(nplanes) * unsigned(SEG * sizeof(T)));
                tma_load_2d(sbuf, tm, int(g_al), cz * P2 + k0, b);
                if (p) tma_load_2d(sbuf + S::kGrp, tm, int(g_al), cz * P2 + k0 + Q1, b);
            }
        } else {
            if (lane == 0) mbar_arrive_expect_tx(b, unsigned(nplanes) * nbytes);
            __syncwarp();
            for (int k = lane; k < nplanes; k += 32)  // a pair stage of D1Q17 has 34 planes
                bulk_copy_g2s(sbuf + (k / Q1) * S::kGrp + (k % Q1) * SEG + dst_off,
                              fin + plane(cz * P2 + k0 + k) * a.stride + cs, nbytes, b);
        }
        return true;
    };
    auto fail = [&]() -> bool {
        if (lane == 0) atomicOr(a.health, 2u);
        // warp 0: let the fills still in flight land before the block can leave (each wait bounded)
        for (int q = 0; q < NS; ++q)
            if ((pending >> q) & 1u) mbar_wait(full + q, (fpar >> q) & 1u);
        return false;
    };
    // the lane's pull by x-velocity a of a staged row sits at row + a SEG + tb - e_a; each
    // (plane, slot) is read by this lane only, so the lane may overwrite its own slots
    const int tb = int(base + x - kx - g_al);
    // pulls from beyond the line's ends: their slots get what the pull must see (the end
    // state's population, or the wrapped population of a periodic line) once the fill lands
    unsigned beyond = 0u;
    if (active)
        static_for<Q1>([&](auto A) {
            constexpr int av = decltype(A)::value;
            const int t = x - e1<L1>(av) - kx;
            if (t < 0 || t >= L) beyond |= 1u << av;
        });
    if (warp == 0)
        for (int st = 0; st < NS; ++st)
            if (!issue(st)) return fail();
    TPTensorRows<L1, N> tc;
    if constexpr (TC) {
        static_assert(2 * 32 * TPTensorRows<L1, N>::kPitch <= S::kStage, "scratch fits a stage buffer");
        tc.init(lane, SEG);
    }
    T R[C::M];
    static_for<C::M>([&](auto G) { R[decltype(G)::value] = T(0); });
    T h[N + 1][N + 1];
    static_for<N + 1>([&](auto J) {
        static_for<N + 1 - decltype(J)::value>([&](auto K) { h[decltype(J)::value][decltype(K)::value] = T(0); });
    });
#pragma unroll 1
    for (int st = 0; st < S::kTotal; ++st) {
        const int sb = st % NS;
        const unsigned long long u = u0 + (unsigned long long)(st / NS);
        if (!__all_sync(0xffffffffu, mbar_wait(full + sb, unsigned(u & 1ull)))) return fail();
        pending &= ~(1u << sb);
        const int cz = st / S::kPerZ, p = st % S::kPerZ;
        T *bs = buf + size_t(sb) * S::kStage;
        if (active && beyond) {
            const int nrows = p ? 2 : 1;
            const int k0 = p ? (2 * p - 1) * Q1 : 0;
            static_for<Q1>([&](auto A) {
                constexpr int av = decltype(A)::value;
                if ((beyond >> av) & 1u) {
                    const int t = x - e1<L1>(av) - kx;
                    for (int r = 0; r < nrows; ++r) {
                        T v;
                        if constexpr (FixedX)  // the end state's population, staged with the fill
                            v = bs[2 * S::kGrp + (t < 0 ? 0 : 2 * Q1) + r * Q1 + av];
                        else
                            v = load_pop<Coherent>(fin + plane(cz * P2 + k0 + r * Q1 + av) * a.stride + base +
                                                   wrap(t, L));
                        bs[r * S::kGrp + av * SEG + tb - e1<L1>(av)] = v;
                    }
                }
            });
            fence_async_shared();  // own slots rewritten: before the buffer's next fill
        }
        if constexpr (TC) {
            __syncwarp();  // the rewritten slots are operands of other lanes
            if (p == 0) {
                float g[1][N + 1];
                tc.template rows<1>(bs, S::kGrp, tb - lane, lane, g);
                if (active) C::yrest(g[0], h);
            } else {
                float g[2][N + 1];
                tc.template rows<2>(bs, S::kGrp, tb - lane, lane, g);
                if (active) C::ypair_pw(g[0], g[1], s.pw[2 * p - 1], h);
            }
            if (active && p == NP1) C::zfold_pw(h, s.pw[cz], R);
            fence_async_shared();  // scratch written and read: before the buffer's next fill
        } else if (active) {
            const T *r0 = bs + tb;
            auto rowp = [&](auto A) -> T {
                constexpr int av = decltype(A)::value;
                return r0[av * SEG - e1<L1>(av)];
            };
            if (p == 0) {
                T g[N + 1];
                C::xrow(rowp, g);
                C::yrest(g, h);
            } else {
                const T *r1 = r0 + S::kGrp;
                auto rowm = [&](auto A) -> T {
                    constexpr int av = decltype(A)::value;
                    return r1[av * SEG - e1<L1>(av)];
                };
                T gp[N + 1], gm[N + 1];
                C::xrow(rowp, gp);
                C::xrow(rowm, gm);
                C::ypair_pw(gp, gm, s.pw[2 * p - 1], h);
            }
            if (p == NP1) C::zfold_pw(h, s.pw[cz], R);
        }
        __syncwarp();  // every lane of this warp is done with buffer sb
        if (lane == 0) mbar_arrive(empty + sb);
        if (warp == 0 && st + NS < S::kTotal && !issue(st + NS)) return fail();
    }
    if (active) {
        const bool ok = C::collide_moments(R, T(a.cd), tau_a<T>(in), tau_b<T>(in), in.model, T(in.es_b));
        if (!ok) atomicOr(a.health, 1u);
        T *dst = fout + base + x;
        auto put = [&](int i, T v) { dst[plane(i) * a.stride] = v; };
#pragma unroll 1
        for (int cz = 0; cz < Q1; ++cz) {
            T Pc[N + 1][N + 1];
            C::template zplane_pw<T>(R, s.pw[cz], Pc);
            const T wc = s.w[cz];
            {
                T Pb[N + 1];
                static_for<N + 1>([&](auto J) { Pb[decltype(J)::value] = Pc[decltype(J)::value][0]; });
                C::template emit_x<T>(Pb, wc * s.w[0], s.w, cz * P2, put);
            }
#pragma unroll 1
            for (int p = 1; p <= NP1; ++p) {
                T Pp[N + 1], Pm[N + 1];
                C::template yrows_pw<T>(Pc, s.pw[2 * p - 1], Pp, Pm);
                const T wbc = wc * s.w[2 * p - 1];
                C::template emit_x<T>(Pp, wbc, s.w, cz * P2 + (2 * p - 1) * Q1, put);
                C::template emit_x<T>(Pm, wbc, s.w, cz * P2 + 2 * p * Q1, put);
            }
        }
    }
    return true;
}

// The block's mbarriers (full[kStages], then empty[kStages]) and stage buffers in dynamic
// shared memory; thread 0 initialises the barriers (published by the block barrier that
// follows in the kernel).
template <class L1, class T, int W>
SMRT_D void tp_block_setup(unsigned char *dyn, unsigned long long *&full, unsigned long long *&empty, T *&buf) {
    using S = TPBlockStage<L1, T, W>;
    full = reinterpret_cast<unsigned long long *>(dyn);
    empty = full + S::kStages;
    buf = reinterpret_cast<T *>(dyn + 128);
    if (threadIdx.x == 0) {
        for (int q = 0; q < S::kStages; ++q) {
            mbar_init(full + q, 1);
            mbar_init(empty + q, W);
        }
        fence_mbar_init();
    }
}

// One step: block b (W warps) takes the block tile b.
// maps: tensor maps of the two states, used when a.tma is set (and the dynamic shared memory
// is 128-byte aligned, as the boxes need).
template <class L1, int N, class T, int W, bool FixedX, bool TC = false, bool Ident = false>
__global__ void __launch_bounds__(128) tp_step_line_block(TPArgs<T> a, int ntiles, const __grid_constant__ TPMaps maps) {
    __shared__ TPTables<L1, T, false> s;
    extern __shared__ __align__(128) unsigned char dyn[];
    unsigned long long *full, *empty;
    T *buf;
    tp_block_setup<L1, T, W>(dyn, full, empty, buf);
    tp_load_tables<L1>(a, s);  // ends with __syncthreads
    const int t = blockIdx.x;
    if (t >= ntiles) return;
    const CUtensorMap *tm = (a.tma && (smem_addr(dyn) & 127u) == 0u) ? &maps.src : nullptr;
    tp_block_tile<L1, N, T, W, FixedX, false, TC, Ident>(a, s, a.fin, a.fout, t, buf, full, empty, 0u, tm);
}

// All nsteps steps in one cooperative launch (see step_line_persistent in kernels.cuh); the
// blocks stride over the block tiles.
template <class L1, int N, class T, int W, bool FixedX, bool TC = false, bool Ident = false>
__global__ void __launch_bounds__(128) tp_step_line_persistent_block(TPArgs<T> a, int nsteps, int ntiles,
                                                                     unsigned *barg, const __grid_constant__ TPMaps maps) {
    __shared__ TPTables<L1, T, false> s;
    __shared__ int failed;
    extern __shared__ __align__(128) unsigned char dyn[];
    unsigned long long *full, *empty;
    T *buf;
    tp_block_setup<L1, T, W>(dyn, full, empty, buf);
    if (threadIdx.x == 0) failed = 0;
    tp_load_tables<L1>(a, s);
    unsigned gen = 0;
    if (threadIdx.x == 0) gen = atomicAdd(&barg[1], 0u);
    const unsigned step0 = __ldcg(&barg[2]);
    const T *src = a.fin;
    T *dst = a.fout;
    const bool use_tma = a.tma && (smem_addr(dyn) & 127u) == 0u;
    unsigned nt = 0;  // tiles this block has stepped
    for (int st = 0; st < nsteps; ++st) {
        const CUtensorMap *tm = use_tma ? (src == a.fin ? &maps.src : &maps.dst) : nullptr;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            if (*static_cast<volatile int *>(&failed)) break;  // another warp gave up
            if (!tp_block_tile<L1, N, T, W, FixedX, true, TC, Ident>(a, s, src, dst, t, buf, full, empty, nt, tm)) {
                failed = 1;
                break;
            }
            ++nt;
        }
        __syncthreads();
        if (failed) return;
        if (st + 1 < nsteps) {
            if (!grid_barrier(barg, gen, a.health)) return;
            const T *nsrc = dst;
            dst = (dst == a.fout) ? const_cast<T *>(a.fin) : a.fout;
            src = nsrc;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) barg[2] = step0 + unsigned(nsteps);
}

// ------------------------------------------------------------------------------ kernels
// ------------------------------------------------------------------ one cell per block
// For problems too small to fill the GPU with one thread per cell (the paper's own runs are
// single shocks of 100 cells), each block takes one cell: its d^3 pulled populations go to
// shared memory, the x-rows and the raw moments are summed by the block's threads, the
// moment-space steps run in warp 0 with the coefficients spread over its lanes, and the
// rebuild is spread over the x-rows again. Block b takes cell x0 + b % 32 of the 32-cell tile b / 32.
template <class L1, int N, class T>
struct TPCellShared {
    static constexpr int Q1 = L1::Q1, P2 = Q1 * Q1, Q = P2 * Q1, M = nmom(N);
    T f[Q];             // pulled populations, library order
    T g[P2][N + 1];     // x-row sums g_j of row (b, c) = b + d c
    T ep[Q1][N + 1];    // e_a^j
    T R[M];             // raw moments, then the rebuild coefficients
    T h[Q1][N + 1][N + 1];  // per z-plane c: sum over y of the x-row sums (then of the rebuild)
    T w[M];             // moment-space scratch
    T gs[3 * (N + 1)];  // per-axis Maxwellian coefficients of the frame transforms
};

template <class L1, int N, class T, bool FixedX>
__global__ void __launch_bounds__(128) tp_step_cell_kernel(TPArgs<T> a) {
    using C = TPCell<L1, N, T>;
    using SH = TPCellShared<L1, N, T>;
    constexpr int Q1 = SH::Q1, P2 = SH::P2, Q = SH::Q, M = SH::M;
    __shared__ TPTables<L1, T> s;
    __shared__ SH sh;
    // double: the moment-space steps spread over warp 0's lanes need their tables in shared
    // memory (a redundant full-warp FP64 instruction costs a full warp of the FP64 pipe); float
    // keeps the one-thread form, whose compile-time constants beat the tables' latency
    constexpr bool kLanes = std::is_same<T, double>::value;
    struct NoTables {};
    __shared__ typename std::conditional<kLanes, MomentSmem<N, double>, NoTables>::type ms;
    if constexpr (kLanes) load_moment_smem<N>(ms);
    tp_load_tables<L1>(a, s);  // ends with __syncthreads
    const int tid = threadIdx.x;
    const int2 tile = a.tiles[blockIdx.x >> 5];
    const InstanceInfo &in = a.inst[tile.x];
    const int x = tile.y + int(blockIdx.x & 31u), L = in.nx, kx = in.kx;
    if (x >= L) return;  // the whole block: no barrier follows for it
    const long long base = in.cell_off;
    const T *gl = a.ghosts + (long long)tile.x * 2 * Q;
    const T *gr = gl + Q;
    for (int q = tid; q < Q1 * (N + 1); q += blockDim.x) {
        const int av = q / (N + 1), j = q % (N + 1);
        T p = T(1);
        for (int r = 0; r < j; ++r) p *= s.e[av];
        sh.ep[av][j] = p;
    }
    // a1: pull every population of the cell
    for (int i = tid; i < Q; i += blockDim.x) {
        const int t = x - e1<L1>(i % Q1) - kx;
        T v;
        if (FixedX && t < 0)
            v = gl[i];
        else if (FixedX && t >= L)
            v = gr[i];
        else
            v = a.fin[(long long)s.plane[i] * a.stride + base + (FixedX ? t : wrap(t, L))];
        sh.f[i] = v;
    }
    __syncthreads();
    // a3, x first: one x-row per thread
    for (int row = tid; row < P2; row += blockDim.x) {
        const T *fr = sh.f + row * Q1;
        T g[N + 1];
        C::xrow([&](auto A) -> T { return fr[decltype(A)::value]; }, g);
        static_for<N + 1>([&](auto J) { sh.g[row][decltype(J)::value] = g[decltype(J)::value]; });
    }
    __syncthreads();
    // ... then y: h_c(j,k) = sum_b g_(b,c)j e_b^k ...
    constexpr int JK = (N + 1) * (N + 1);
    for (int q = tid; q < Q1 * JK; q += blockDim.x) {
        const int c = q / JK, j = (q % JK) / (N + 1), k = q % (N + 1);
        if (j + k > N) continue;
        T acc = T(0);
        for (int b = 0; b < Q1; ++b) acc = fma(sh.g[b + Q1 * c][j], sh.ep[b][k], acc);
        sh.h[c][j][k] = acc;
    }
    __syncthreads();
    // ... then z: R_(j,k,l) = sum_c h_c(j,k) e_c^l, one moment per thread
    for (int m = tid; m < M; m += blockDim.x) {
        const int j = mi_comp(m, 0), k = mi_comp(m, 1), l = mi_comp(m, 2);
        T acc = T(0);
        for (int c = 0; c < Q1; ++c) acc = fma(sh.h[c][j][k], sh.ep[c][l], acc);
        sh.R[m] = acc;
    }
    __syncthreads();
    // a2, a4-a6 in warp 0
    if (tid < 32) {
        if constexpr (kLanes) {
            const bool ok = C::collide_moments_lanes(ms, sh.R, sh.w, sh.gs, T(a.cd), tau_a<T>(in),
                                                     tau_b<T>(in), in.model, T(in.es_b));
            if (tid == 0 && !ok) atomicOr(a.health, 1u);
        } else {
            T R[M];
            static_for<M>([&](auto G) { R[decltype(G)::value] = sh.R[decltype(G)::value]; });
            const bool ok = C::collide_moments(R, T(a.cd), tau_a<T>(in), tau_b<T>(in), in.model, T(in.es_b));
            __syncwarp();
            if (tid == 0) {
                if (!ok) atomicOr(a.health, 1u);
                static_for<M>([&](auto G) { sh.R[decltype(G)::value] = R[decltype(G)::value]; });
            }
        }
    }
    __syncthreads();
    // a7 + a8: z first, Pc_c(j,k) = sum_l P_(j,k,l) e_c^l ...
    for (int q = tid; q < Q1 * JK; q += blockDim.x) {
        const int c = q / JK, j = (q % JK) / (N + 1), k = q % (N + 1);
        if (j + k > N) continue;
        T acc = T(0);
        for (int l = 0; l + j + k <= N; ++l) acc = fma(sh.R[mi_pos(j, k, l)], sh.ep[c][l], acc);
        sh.h[c][j][k] = acc;
    }
    __syncthreads();
    // ... then one x-row per thread, Pb_j = sum_k Pc_c(j,k) e_b^k, stored as it is formed
    T *dst = a.fout + base + x;
    auto put = [&](int i, T v) { dst[(long long)s.plane[i] * a.stride] = v; };
    for (int row = tid; row < P2; row += blockDim.x) {
        const int b = row % Q1, c = row / Q1;
        T Pb[N + 1];
        static_for<N + 1>([&](auto J) {
            constexpr int j = decltype(J)::value;
            T acc = T(0);
            static_for<N + 1 - j>([&](auto K) {
                constexpr int k = decltype(K)::value;
                acc = fma(sh.h[c][j][k], sh.ep[b][k], acc);
            });
            Pb[j] = acc;
        });
        C::template emit_x<T>(Pb, s.w[b] * s.w[c], s.w, row * Q1, put);
    }
}

// lb_moments of the pulled (pre-collision) populations.
template <class L1, int N, class T>
__global__ void __launch_bounds__(128) tp_moments_kernel(TPArgs<T> a, double *out, long long ncells,
                                                         unsigned mask, int fixedx) {
    __shared__ TPTables<L1, T> s;
    tp_load_tables<L1>(a, s);
    using C = TPCell<L1, N, T>;
    constexpr int Q1 = L1::Q1;
    constexpr int Q = Q1 * Q1 * Q1;
    const int2 tile = a.tiles[blockIdx.x];
    const InstanceInfo &in = a.inst[tile.x];
    const int x = tile.y + threadIdx.x;
    const int L = in.nx;
    if (x >= L) return;
    const long long base = in.cell_off;
    const T *gl = a.ghosts + (long long)tile.x * 2 * Q;
    const T *gr = gl + Q;
    int xs[Q1];
    static_for<Q1>([&](auto A) {
        constexpr int av = decltype(A)::value;
        xs[av] = x - (e1<L1>(av) + in.kx);
    });
    auto pop = [&](int i, auto A) -> T {
        const int t = xs[decltype(A)::value];
        if (fixedx && t < 0) return gl[i];
        if (fixedx && t >= L) return gr[i];
        return a.fin[(long long)s.plane[i] * a.stride + base + wrap(t, L)];
    };
    T R[C::M];
    C::project(pop, s.e, R);
    const T c = T(a.cd);
    T cp[N + 1];
    cp[0] = T(1);
    static_for<N>([&](auto J) { cp[decltype(J)::value + 1] = cp[decltype(J)::value] * c; });
    static_for<C::M>([&](auto G) { R[decltype(G)::value] *= cp[mi_order(decltype(G)::value)]; });
    const T rhom1 = R[0], rho = T(1) + rhom1, ir = rcp(rho);
    const T u[3] = {R[mi_pos(1, 0, 0)] * ir, R[mi_pos(0, 1, 0)] * ir, R[mi_pos(0, 0, 1)] * ir};
    const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const T thm1 = (R[mi_pos(2, 0, 0)] + R[mi_pos(0, 2, 0)] + R[mi_pos(0, 0, 2)] - T(3) * rhom1 - rho * uu) *
                   ir * T(1.0 / 3.0);
    const T theta = T(1) + thm1;
    T v[C::M];
    static_for<C::M>([&](auto A) {
        constexpr int al = decltype(A)::value;
        T acc = T(0);
        static_for<C::M>([&](auto G) {
            constexpr int g = decltype(G)::value;
            constexpr double h = hdiv(al, g);
            if constexpr (h != 0.0) acc = fma(T(h), R[g], acc);
        });
        v[al] = acc;
    });
    v[0] = rho;
    to_local_divided<N, T>(v, u, theta, thm1);
    const double up[3] = {double(u[0]) + a.cd * in.kx, double(u[1]), double(u[2])};
    store_moments<N, T>(out, ncells, base + x, mask, double(rho), up, double(theta), v);
}

// Equilibrium fill: df = order-N equilibrium of (rho, u_phys - u_bar, theta) minus w_i,
// formed in double and stored as T.
template <class L1, int N, class T>
__global__ void __launch_bounds__(128) tp_fill_kernel(TPArgs<T> a, const double *rho, const double *u,
                                                      const double *theta, long long ncells) {
    __shared__ TPTables<L1, double> s;
    tp_load_tables<L1>(a, s);
    using C = TPCell<L1, N, double>;
    const int2 tile = a.tiles[blockIdx.x];
    const InstanceInfo &in = a.inst[tile.x];
    const int x = tile.y + threadIdx.x;
    if (x >= in.nx) return;
    const long long cell = in.cell_off + x;
    const double uu[3] = {u[cell] - a.cd * in.kx, u[ncells + cell], u[2 * ncells + cell]};
    double P[C::M];
    C::template equilibrium<double>(rho[cell], uu, theta[cell], a.cd, P);
    T *dst = a.fout + cell;
    C::template rebuild<double>(P, s.e, s.w, [&](int i, double v) { dst[(long long)s.plane[i] * a.stride] = T(v); });
}

// End-state populations of every instance, library order: thread t = 2 j + side.
template <class L1, int N, class T>
__global__ void __launch_bounds__(64) tp_ghost_kernel(TPArgs<T> a, const double *states, int ninst, T *ghosts,
                                                      double *ghostsd) {
    __shared__ TPTables<L1, double> s;
    tp_load_tables<L1>(a, s);
    using C = TPCell<L1, N, double>;
    constexpr int Q = L1::Q1 * L1::Q1 * L1::Q1;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * ninst) return;
    const int j = t / 2;
    const double *st = states + 5 * t;
    const double uu[3] = {st[1] - a.cd * a.inst[j].kx, st[2], st[3]};
    double P[C::M];
    C::template equilibrium<double>(st[0], uu, st[4], a.cd, P);
    T *g = ghosts + (long long)t * Q;
    double *gd = ghostsd + (long long)t * Q;
    C::template rebuild<double>(P, s.e, s.w, [&](int i, double v) {
        g[i] = T(v);
        gd[i] = v;
    });
}

}  // namespace smrt
