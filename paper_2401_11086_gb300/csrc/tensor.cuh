// tensor.cuh -- LB-SMRT collide-and-stream on three-dimensional tensor-product velocity sets
// (Yan & Shan, arXiv 2401.11086, Sec. 4.2: the 3D products D3Q{d^3} of the 1D rules D1Qd-P1,
// D3Q729 = D1Q9-P1 x D1Q9-P1 x D1Q9-P1 of degree 11), batched 1D lines along x.
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
};

// Shared-memory tables of one block: caller planes, the 1D abscissae (integers, as T) and the
// 1D weights (as T).
template <class L1, class T>
struct TPTables {
    static constexpr int Q = L1::Q1 * L1::Q1 * L1::Q1;
    int plane[Q];
    T e[L1::Q1];
    T w[L1::Q1];
};

template <class L1, class T, class U>
SMRT_D void tp_load_tables(const TPArgs<T> &a, TPTables<L1, U> &s) {
    for (int i = threadIdx.x; i < TPTables<L1, U>::Q; i += blockDim.x) s.plane[i] = a.plane_idx[i];
    if (threadIdx.x < L1::Q1) {
        s.e[threadIdx.x] = U(e1<L1>(threadIdx.x));
        s.w[threadIdx.x] = U(a.w1[threadIdx.x]);
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

    // a2, a4-a6 on the raw moments: R (in) -> rebuild coefficients P (out, same slots) with
    // f'_i = w_i sum_gamma P_gamma e_i^gamma. Returns false when rho or theta is not positive.
    SMRT_D static bool collide_moments(T (&R)[M], T c, const T *tauA, const T *tauB) {
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
        T s[ntau(N)];
        static_for<ntau(N)>([&](auto K) {
            constexpr int k = decltype(K)::value;
            s[k] = T(1) - rcp_tau<T>(tauA[k], tauB[k], rho);
        });
        static_for<N - 1>([&](auto Nn) { relax_order<N, decltype(Nn)::value + 2, T>(v, s); });
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

// ------------------------------------------------------------------------------ kernels
// One thread per cell of tile tile_index (instance j, cells x0 .. x0 + blockDim - 1).
template <class L1, int N, class T, bool FixedX, bool Coherent>
SMRT_D void tp_line_tile(const TPArgs<T> &a, const TPTables<L1, T> &s, const T *__restrict__ fin,
                         T *__restrict__ fout, int tile_index) {
    using C = TPCell<L1, N, T>;
    constexpr int Q1 = L1::Q1;
    constexpr int Q = Q1 * Q1 * Q1;
    const int2 tile = a.tiles[tile_index];
    const InstanceInfo &in = a.inst[tile.x];
    const int x = tile.y + threadIdx.x;
    const int L = in.nx;
    if (x >= L) return;
    const long long base = in.cell_off;
    const T *gl = a.ghosts + (long long)tile.x * 2 * Q;
    const T *gr = gl + Q;
    // a1: the x-velocity e_a of a population fixes where it is pulled from: x - e_a - k
    // (periodic lines wrap once: the reach plus |k| never exceeds the length)
    int xs[Q1];
    static_for<Q1>([&](auto A) {
        constexpr int av = decltype(A)::value;
        const int t = x - (e1<L1>(av) + in.kx);
        xs[av] = FixedX ? t : wrap(t, L);
    });
    auto pop = [&](int i, auto A) -> T {
        const int t = xs[decltype(A)::value];
        if constexpr (FixedX) {
            if (t < 0) return gl[i];
            if (t >= L) return gr[i];
        }
        return load_pop<Coherent>(fin + (long long)s.plane[i] * a.stride + base + t);
    };
    T R[C::M];
    C::project(pop, s.e, R);
    const bool ok = C::collide_moments(R, T(a.cd), tau_a<T>(in), tau_b<T>(in));
    if (!ok) atomicOr(a.health, 1u);
    T *dst = fout + base + x;
    C::template rebuild<T>(R, s.e, s.w, [&](int i, T v) { dst[(long long)s.plane[i] * a.stride] = v; });
}

template <class L1, int N, class T, bool FixedX>
__global__ void __launch_bounds__(128) tp_step_line_kernel(TPArgs<T> a) {
    __shared__ TPTables<L1, T> s;
    tp_load_tables<L1>(a, s);
    tp_line_tile<L1, N, T, FixedX, false>(a, s, a.fin, a.fout, blockIdx.x);
}

// All nsteps steps in one cooperative launch (see step_line_persistent in kernels.cuh).
template <class L1, int N, class T, bool FixedX>
__global__ void __launch_bounds__(128) tp_step_line_persistent(TPArgs<T> a, int nsteps, int ntiles, unsigned *bar) {
    __shared__ TPTables<L1, T> s;
    tp_load_tables<L1>(a, s);
    unsigned gen = 0;
    if (threadIdx.x == 0) gen = atomicAdd(&bar[1], 0u);
    const unsigned step0 = __ldcg(&bar[2]);
    const T *src = a.fin;
    T *dst = a.fout;
    for (int st = 0; st < nsteps; ++st) {
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x)
            tp_line_tile<L1, N, T, FixedX, true>(a, s, src, dst, t);
        if (st + 1 < nsteps) {
            if (!grid_barrier(bar, gen, a.health)) return;
            const T *nsrc = dst;
            dst = (dst == a.fout) ? const_cast<T *>(a.fin) : a.fout;
            src = nsrc;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) bar[2] = step0 + unsigned(nsteps);
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
