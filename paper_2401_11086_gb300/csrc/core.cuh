// core.cuh -- per-cell arithmetic of the LB-SMRT collision (Yan & Shan, arXiv 2401.11086),
// written for compile-time velocity sets so that every zero coefficient disappears at compile
// time and the remaining constants fold into the instruction stream.
//
// Notation. A multi-index beta = (b0, b1, b2) labels one distinct component of a symmetric
// tensor of order |beta| (Sec. 2.2: H^(n)_{i1..in} = prod_k He_{beta_k}(xi_k), beta_k = number
// of indices equal to k). All multi-indices with |beta| <= N are stored in one array ordered
// by order, then descending lexicographically; mi_pos() maps beta to its slot.
//
// Divided representation. Coefficient vectors are kept divided by beta! = prod_k beta_k!:
//   ta_alpha = a_alpha / alpha!,  td_beta = d_beta / beta!.
// In that form (derivations in the comments of each routine)
//   * the binomial frame transform (Sec. 3, Shan's binomial transform between the absolute
//     expansion of Eq. hermite1 and the local expansion that defines SMRT) is, per axis,
//     out_alpha = sum_{b <= alpha_k} G[alpha_k - b] in_{alpha with alpha_k -> b},
//     with G[j] = g_j / j!, g_j the 1D absolute coefficient of a unit Maxwellian
//     (Appendix B closed form), so it costs one FMA per term and no constants;
//   * the rebuild of Eq. fi, f_i = w_i sum_alpha a_alpha He_alpha(xi_i) / alpha!, reads ta
//     directly;
//   * the trace and the delta-product of Appendix A become sums with folded constants.
#pragma once

#include <cstdint>
#include <type_traits>
#include <utility>

namespace smrt {

#define SMRT_HD __host__ __device__ __forceinline__
#define SMRT_D __device__ __forceinline__

// Reciprocal and reciprocal square root: correctly rounded reciprocal and the hardware
// reciprocal square root for float (within 2 ulp), exact division for double.
SMRT_D float rcp(float x) { return __frcp_rn(x); }
SMRT_D double rcp(double x) { return 1.0 / x; }
SMRT_D float rsq(float x) { return rsqrtf(x); }
SMRT_D double rsq(double x) { return 1.0 / sqrt(x); }

// ------------------------------------------------------------------ compile-time loops
template <int V>
using ic = std::integral_constant<int, V>;

template <class F, int... I>
SMRT_HD void static_for_impl(F &&f, std::integer_sequence<int, I...>) {
    (f(ic<I>{}), ...);
}
template <int Count, class F>
SMRT_HD void static_for(F &&f) {
    static_for_impl(f, std::make_integer_sequence<int, Count>{});
}

// ------------------------------------------------------------------ constexpr arithmetic
constexpr int nmom(int N) { return (N + 1) * (N + 2) * (N + 3) / 6; }
constexpr int ord_off(int n) { return n * (n + 1) * (n + 2) / 6; }
constexpr int mi_pos(int a, int b, int c) {
    return ord_off(a + b + c) + (b + c) * (b + c + 1) / 2 + c;
}
constexpr int mi_order(int p) {
    int n = 0;
    while (ord_off(n + 1) <= p) ++n;
    return n;
}
// within order n the slot r = T(j) + (j - b), j = n - a, T(j) = j (j + 1) / 2
constexpr int mi_j(int p) {
    const int r = p - ord_off(mi_order(p));
    int j = 0;
    while ((j + 1) * (j + 2) / 2 <= r) ++j;
    return j;
}
constexpr int mi_comp(int p, int k) {
    const int n = mi_order(p), j = mi_j(p), r = p - ord_off(n);
    const int a = n - j, b = j - (r - j * (j + 1) / 2);
    return k == 0 ? a : (k == 1 ? b : n - a - b);
}
constexpr int mi_with(int p, int k, int v) {  // slot of p with component k replaced by v
    const int a = mi_comp(p, 0), b = mi_comp(p, 1), c = mi_comp(p, 2);
    return k == 0 ? mi_pos(v, b, c) : (k == 1 ? mi_pos(a, v, c) : mi_pos(a, b, v));
}
constexpr int mi_plus2(int p, int k) {  // slot of p + 2 e_k
    return mi_with(p, k, mi_comp(p, k) + 2);
}
constexpr int mi_minus2(int p, int k) {  // slot of p - 2 e_k (caller checks comp >= 2)
    return mi_with(p, k, mi_comp(p, k) - 2);
}
constexpr double cfact(int n) { return n <= 1 ? 1.0 : n * cfact(n - 1); }
constexpr double cdfact(int n) { return n <= 1 ? 1.0 : n * cdfact(n - 2); }
constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }
constexpr double mi_fact(int p) {
    return cfact(mi_comp(p, 0)) * cfact(mi_comp(p, 1)) * cfact(mi_comp(p, 2));
}

// Coefficient of x^j in He_n(x): (-1)^l n! / (2^l l! j!) with n - j = 2l (Appendix B).
constexpr double he_coef(int n, int j) {
    if (j > n || ((n - j) & 1)) return 0.0;
    const int l = (n - j) / 2;
    return ((l & 1) ? -1.0 : 1.0) * cfact(n) / (cfact(l) * cfact(j) * double(1 << l));
}
// Coefficient of e^gamma (with c^{|gamma|} factored out) in He_alpha(c e) / alpha!.
constexpr double hdiv(int alpha, int gamma) {
    double v = 1.0;
    for (int k = 0; k < 3; ++k) v *= he_coef(mi_comp(alpha, k), mi_comp(gamma, k));
    return v / mi_fact(alpha);
}
// Coefficient of e^gamma in He_alpha(c e), undivided.
constexpr double hfull(int alpha, int gamma) { return hdiv(alpha, gamma) * mi_fact(alpha); }

// Eq. bd (Appendix A).
constexpr double coefB(int n, int m) {
    return cfact(n) * cdfact(2 * n - 4 * m + 1) /
           (cfact(m) * double(1 << m) * cfact(n - 2 * m) * cdfact(2 * n - 2 * m + 1));
}
constexpr double coefD(int n, int m) {
    return ((m & 1) ? -1.0 : 1.0) * cfact(n) * cdfact(2 * n - 2 * m - 1) /
           (cfact(m) * double(1 << m) * cfact(n - 2 * m) * cdfact(2 * n - 1));
}
// Number of (n, m) relaxation times for orders 2..N and the slot of (n, m).
constexpr int ntau(int N) {
    int k = 0;
    for (int n = 2; n <= N; ++n) k += n / 2 + 1;
    return k;
}
constexpr int tau_slot(int n, int m) { return ntau(n - 1) + m; }

// ------------------------------------------------------------------ separable transforms
// v_alpha <- sum_{beta <= alpha} prod_k G[k][alpha_k - beta_k] v_beta   (divided form)
// Applied axis by axis; each pass leaves every slot |alpha| <= N defined.
template <int N, class T>
SMRT_HD void binomial_divided(T (&v)[nmom(N)], const T (&G)[3][N + 1]) {
    constexpr int M = nmom(N);
    static_for<3>([&](auto K) {
        constexpr int k = decltype(K)::value;
        T out[M];
        static_for<M>([&](auto A) {
            constexpr int p = decltype(A)::value;
            constexpr int ak = mi_comp(p, k);
            T acc = v[p];  // b = alpha_k term, G[k][0] = 1
            static_for<ak>([&](auto B) {
                constexpr int b = decltype(B)::value;
                acc = fma(G[k][ak - b], v[mi_with(p, k, b)], acc);
            });
            out[p] = acc;
        });
        static_for<M>([&](auto A) { v[decltype(A)::value] = out[decltype(A)::value]; });
    });
}

// G[j] = g_j(u, th) / j!, with g_{j+1} = u g_j + j (th - 1) g_{j-1}, g_0 = 1, g_1 = u: the
// recurrence of the generating function exp(u t + (th - 1) t^2 / 2) of the 1D Maxwellian's
// absolute Hermite coefficients (Appendix B closed form). In divided form:
// G[j+1] = (u G[j] + (th - 1) G[j-1]) / (j + 1).
template <int N, class T>
SMRT_HD void maxwell_divided(T (&G)[N + 1], T u, T thm1) {
    G[0] = T(1);
    if constexpr (N >= 1) G[1] = u;
    static_for<(N >= 1 ? N - 1 : 0)>([&](auto J) {
        constexpr int j = decltype(J)::value + 1;
        G[j + 1] = (u * G[j] + thm1 * G[j - 1]) * T(1.0 / (j + 1));
    });
}

// a4 in divided form: td_beta = d_beta / beta! = theta^(-|beta|/2) [T(-u, 2 - theta) ta]_beta,
// v holding ta on entry (with the full a_0 = rho in slot 0) and td on exit.
template <int Nm, class T>
SMRT_D void to_local_divided(T (&v)[nmom(Nm)], const T (&u)[3], T theta, T thm1) {
    T G[3][Nm + 1];
    static_for<3>([&](auto K) {
        constexpr int k = decltype(K)::value;
        maxwell_divided<Nm, T>(G[k], -u[k], -thm1);
    });
    binomial_divided<Nm, T>(v, G);
    const T is = rsq(theta);
    T sp[Nm + 1];
    sp[0] = T(1);
    static_for<Nm>([&](auto J) { sp[decltype(J)::value + 1] = sp[decltype(J)::value] * is; });
    static_for<nmom(Nm)>([&](auto A) {
        constexpr int p = decltype(A)::value;
        if constexpr (mi_order(p) >= 1) v[p] *= sp[mi_order(p)];
    });
}

// ------------------------------------------------------------------ irreducible relaxation
// Appendix A: the part of order n with m traces is P_m d = B(n,m) Q^(n-2m)_0 tr^m d delta^m,
// Q^(r)_0 = sum_k D(r,k) delta^k tr^k. Collecting terms with j = m + k traces gives
//   sum_m s_m P_m d = sum_j C_j delta^j tr^j d,  C_j = sum_{m<=j} s_m B(n,m) D(n-2m, j-m),
// with s_m = 1 - 1/tau_{n,m} (Eq. SMRT). In divided form (x~ = x / beta!):
//   (tr X)~_beta = sum_k (beta_k + 2)(beta_k + 1) X~_{beta + 2e_k}
//   (delta Y)~_alpha = 1/(n(n-1)) sum_{k: alpha_k >= 2} Y~_{alpha - 2e_k}    (rank n result)
// where the symmetric product delta Y of Eq. symm has the multi-index form
// (delta Y)_alpha = sum_k alpha_k(alpha_k - 1)/(n(n-1)) Y_{alpha - 2e_k}.
template <int N, int n, class T>
SMRT_HD void relax_order(T (&d)[nmom(N)], const T (&s)[ntau(N)]) {
    constexpr int J = n / 2;
    constexpr int M = nmom(N);
    // t[j] holds tr^j d (order n - 2j) in slots of the full array layout
    T t[J + 1][M];
    static_for<M>([&](auto A) {
        constexpr int p = decltype(A)::value;
        if constexpr (mi_order(p) == n) t[0][p] = d[p];
    });
    static_for<J>([&](auto Jm) {
        constexpr int j = decltype(Jm)::value + 1;
        static_for<M>([&](auto A) {
            constexpr int p = decltype(A)::value;
            if constexpr (mi_order(p) == n - 2 * j) {
                T acc = T(0);
                static_for<3>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    constexpr double f = double((mi_comp(p, k) + 2) * (mi_comp(p, k) + 1));
                    acc = fma(T(f), t[j - 1][mi_plus2(p, k)], acc);
                });
                t[j][p] = acc;
            }
        });
    });
    // C_j from the per-part factors s_m
    T C[J + 1];
    static_for<J + 1>([&](auto Jm) {
        constexpr int j = decltype(Jm)::value;
        T acc = T(0);
        static_for<j + 1>([&](auto Mm) {
            constexpr int m = decltype(Mm)::value;
            constexpr double k = coefB(n, m) * coefD(n - 2 * m, j - m);
            acc = fma(T(k), s[tau_slot(n, m)], acc);
        });
        C[j] = acc;
    });
    // lift: L_j = delta^j tr^j d, built from order n - 2j up to n; then d' = sum_j C_j L_j
    static_for<M>([&](auto A) {
        constexpr int p = decltype(A)::value;
        if constexpr (mi_order(p) == n) d[p] = C[0] * t[0][p];
    });
    static_for<J>([&](auto Jm) {
        constexpr int j = decltype(Jm)::value + 1;
        T y[M];
        static_for<M>([&](auto A) {
            constexpr int p = decltype(A)::value;
            if constexpr (mi_order(p) == n - 2 * j) y[p] = t[j][p];
        });
        static_for<j>([&](auto Lm) {  // raise order n-2j -> n, one delta at a time
            constexpr int r = n - 2 * j + 2 * (decltype(Lm)::value + 1);  // order after step
            T z[M];
            static_for<M>([&](auto A) {
                constexpr int p = decltype(A)::value;
                if constexpr (mi_order(p) == r) {
                    T acc = T(0);
                    static_for<3>([&](auto K) {
                        constexpr int k = decltype(K)::value;
                        if constexpr (mi_comp(p, k) >= 2) acc = acc + y[mi_minus2(p, k)];
                    });
                    z[p] = acc * T(1.0 / double(r * (r - 1)));
                }
            });
            static_for<M>([&](auto A) {
                constexpr int p = decltype(A)::value;
                if constexpr (mi_order(p) == r) y[p] = z[p];
            });
        });
        static_for<M>([&](auto A) {
            constexpr int p = decltype(A)::value;
            if constexpr (mi_order(p) == n) d[p] = fma(C[j], y[p], d[p]);
        });
    });
}

// ------------------------------------------------------------------ ES-BGK relaxation
// a5 for the ES-BGK model (Sec. 3, Eq. ES-BGK): every order n >= 2 relaxes at the one
// discrete rate 1/tau_20 toward the local-frame coefficients of Holway's Gaussian of
// covariance theta delta + b' sigma / rho. In divided form they are the monomial
// coefficients of rho exp(t.B.t / 2), B = (b'/rho) D2: order 2 is b' v2, order 4 is
// (b'^2 / (2 rho)) times the sum over ordered pairs of order-2 slots adding up to the slot,
// odd orders are zero. b' = 1 - (1 - b) tau_20 / (tau_20 - b/2) keeps the continuous stress
// rate (1 - b)/tau_c under the second-order scheme (tau -> tau + 1/2 per mode), so
// Pr = 1/(1 - b).
template <int N, class T>
SMRT_D void relax_es_divided(T (&v)[nmom(N)], T rho, T A, T B, T b) {
    constexpr int M = nmom(N);
    const T tau = fma(B, rho, A) * rcp(rho);
    const T om = rcp(tau);
    const T bp = T(1) - (T(1) - b) * tau * rcp(fma(T(-0.5), b, tau));
    const T s = T(1) - om;
    T t4[M];
    static_for<M>([&](auto P) {
        constexpr int p = decltype(P)::value;
        if constexpr (mi_order(p) == 4) {
            T acc = T(0);
            static_for<M>([&](auto Q1s) {
                constexpr int q1 = decltype(Q1s)::value;
                if constexpr (mi_order(q1) == 2) {
                    static_for<M>([&](auto Q2s) {
                        constexpr int q2 = decltype(Q2s)::value;
                        if constexpr (mi_order(q2) == 2 && mi_comp(q1, 0) + mi_comp(q2, 0) == mi_comp(p, 0) &&
                                      mi_comp(q1, 1) + mi_comp(q2, 1) == mi_comp(p, 1))
                            acc = fma(v[q1], v[q2], acc);
                    });
                }
            });
            t4[p] = acc;
        }
    });
    const T k4 = om * bp * bp * T(0.5) * rcp(rho);
    const T s2 = fma(om, bp, s);
    static_for<M>([&](auto P) {
        constexpr int p = decltype(P)::value;
        constexpr int n = mi_order(p);
        if constexpr (n == 2)
            v[p] *= s2;
        else if constexpr (n == 4)
            v[p] = fma(k4, t4[p], s * v[p]);
        else if constexpr (n >= 3)
            v[p] *= s;
    });
}

}  // namespace smrt
