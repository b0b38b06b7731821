// adjoint.cuh -- reverse-mode (vector-Jacobian) products of the per-cell SMRT collision and of
// the reported moments, in double precision, written by hand stage by stage.
//
// Forward stages of the collision (the same as Collide<> in kernels.cuh, deviations
// df_i = f_i - w_i, divided coefficients x~ = x / beta!):
//   F1 raw moments      Rc_g = c^|g| sum_i df_i e_i^g
//   F2 conserved        rho = 1 + Rc_0, u_k = Rc_{e_k} / rho,
//                       th - 1 = (tr Rc_2 - 3 Rc_0 - rho |u|^2) / (3 rho)
//   F3 absolute         ta_a = sum_g hdiv(a, g) Rc_g, then ta_0 := rho
//   F4 local frame      p3 = X_z X_y X_x ta (binomial passes with G- = g(-u, 2 - th)),
//                       td_b = p3_b th^(-|b|/2)
//   F5 relaxation       td'_n = sum_j C_j(s) delta^j tr^j td_n, n = 2..N, s_k = 1 - rho/(A_k + B_k rho)
//   F6 back             y_b = td'_b th^(|b|/2) (|b| >= 2), y_0 = rho, y_1 = 0;
//                       ta' = X_z X_y X_x y (G+ = g(u, th)), then ta'_0 := rho - 1
//   F7 rebuild          out_i = w_i sum_g P_g e_i^g, P_g = c^|g| sum_a hfull(a, g) ta'_a
// Each stage below has its transpose; the chain runs F7' ... F1'. Relaxation-time derivatives:
// with R = 1/(A + B rho), ds/drho = -A R^2, ds/dA = rho R^2, ds/dB = rho^2 R^2, and
// A = tau_c rho_ref (Maxwell molecules) or B = tau_c + 1/2 (constant times).
#pragma once

#include "core.cuh"
#include "lattices.cuh"

namespace smrt {

// The moment-space stages (independent of the velocity set).
template <int Nm>
struct AdjMoments {
    static constexpr int M = nmom(Nm);

    // F3 (hdiv) / F7 (hfull) coefficient maps and their transposes
    template <bool Full>
    SMRT_HD static void hmap(const double (&in)[M], double (&out)[M]) {
        static_for<M>([&](auto A) {
            constexpr int a = decltype(A)::value;
            double acc = 0.0;
            static_for<M>([&](auto G) {
                constexpr int g = decltype(G)::value;
                constexpr double h = Full ? hfull(a, g) : hdiv(a, g);
                if constexpr (h != 0.0) acc += h * in[g];
            });
            out[a] = acc;
        });
    }
    template <bool Full>
    SMRT_HD static void hmap_T(const double (&outb)[M], double (&inb)[M]) {
        static_for<M>([&](auto G) {
            constexpr int g = decltype(G)::value;
            double acc = 0.0;
            static_for<M>([&](auto A) {
                constexpr int a = decltype(A)::value;
                constexpr double h = Full ? hfull(a, g) : hdiv(a, g);
                if constexpr (h != 0.0) acc += h * outb[a];
            });
            inb[g] += acc;
        });
    }

    // one binomial pass along axis k: out_p = sum_{b <= p_k} G[p_k - b] in_{p with p_k -> b}
    template <int k>
    SMRT_HD static void pass(const double (&in)[M], const double (&G)[Nm + 1], double (&out)[M]) {
        static_for<M>([&](auto A) {
            constexpr int p = decltype(A)::value;
            constexpr int pk = mi_comp(p, k);
            double acc = in[p];
            static_for<pk>([&](auto B) {
                constexpr int b = decltype(B)::value;
                acc += G[pk - b] * in[mi_with(p, k, b)];
            });
            out[p] = acc;
        });
    }
    // transpose of pass<k>: inb += d out/d in^T outb, Gb += d out/d G^T outb
    template <int k>
    SMRT_HD static void pass_T(const double (&outb)[M], const double (&G)[Nm + 1], const double (&in)[M],
                               double (&inb)[M], double (&Gb)[Nm + 1]) {
        static_for<M>([&](auto A) {
            constexpr int p = decltype(A)::value;
            constexpr int pk = mi_comp(p, k);
            inb[p] += outb[p];
            static_for<pk>([&](auto B) {
                constexpr int b = decltype(B)::value;
                constexpr int q = mi_with(p, k, b);
                inb[q] += G[pk - b] * outb[p];
                Gb[pk - b] += in[q] * outb[p];
            });
        });
    }

    // G[0] = 1, G[1] = u, G[j+1] = (u G[j] + t G[j-1]) / (j + 1)
    SMRT_HD static void maxwell(double u, double t, double (&G)[Nm + 1]) {
        G[0] = 1.0;
        G[1] = u;
        for (int j = 1; j < Nm; ++j) G[j + 1] = (u * G[j] + t * G[j - 1]) / (j + 1);
    }
    // transpose of maxwell: consumes Gb, accumulates ub and tb
    SMRT_HD static void maxwell_T(double u, double t, const double (&G)[Nm + 1], double (&Gb)[Nm + 1],
                                  double &ub, double &tb) {
        for (int j = Nm - 1; j >= 1; --j) {
            const double g = Gb[j + 1] / (j + 1);
            ub += g * G[j];
            Gb[j] += g * u;
            tb += g * G[j - 1];
            Gb[j - 1] += g * t;
        }
        ub += Gb[1];
    }

    // divided-form trace of the order-r block (result order r - 2) and the delta-product
    // (order r - 2 -> r), plus their transposes; arrays use full-slot layout
    template <int r>
    SMRT_HD static void tr(const double (&X)[M], double (&Z)[M]) {
        static_for<M>([&](auto A) {
            constexpr int p = decltype(A)::value;
            if constexpr (mi_order(p) == r - 2) {
                double acc = 0.0;
                static_for<3>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    acc += double((mi_comp(p, k) + 2) * (mi_comp(p, k) + 1)) * X[mi_plus2(p, k)];
                });
                Z[p] = acc;
            }
        });
    }
    template <int r>
    SMRT_HD static void tr_T(const double (&Zb)[M], double (&Xb)[M]) {
        static_for<M>([&](auto A) {
            constexpr int p = decltype(A)::value;
            if constexpr (mi_order(p) == r - 2) {
                static_for<3>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    Xb[mi_plus2(p, k)] += double((mi_comp(p, k) + 2) * (mi_comp(p, k) + 1)) * Zb[p];
                });
            }
        });
    }
    template <int r>
    SMRT_HD static void delta(const double (&Y)[M], double (&W)[M]) {
        static_for<M>([&](auto A) {
            constexpr int p = decltype(A)::value;
            if constexpr (mi_order(p) == r) {
                double acc = 0.0;
                static_for<3>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    if constexpr (mi_comp(p, k) >= 2) acc += Y[mi_minus2(p, k)];
                });
                W[p] = acc / double(r * (r - 1));
            }
        });
    }
    template <int r>
    SMRT_HD static void delta_T(const double (&Wb)[M], double (&Yb)[M]) {
        static_for<M>([&](auto A) {
            constexpr int p = decltype(A)::value;
            if constexpr (mi_order(p) == r) {
                static_for<3>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    if constexpr (mi_comp(p, k) >= 2) Yb[mi_minus2(p, k)] += Wb[p] / double(r * (r - 1));
                });
            }
        });
    }

    // L_j td = delta^j tr^j td restricted to order n (full-slot arrays, other orders untouched)
    template <int n, int j>
    SMRT_HD static void lift(const double (&td)[M], double (&out)[M]) {
        double cur[M];
        static_for<M>([&](auto A) { cur[decltype(A)::value] = td[decltype(A)::value]; });
        static_for<j>([&](auto I) {
            constexpr int r = n - 2 * decltype(I)::value;
            double nxt[M];
            tr<r>(cur, nxt);
            static_for<M>([&](auto A) {
                constexpr int p = decltype(A)::value;
                if constexpr (mi_order(p) == r - 2) cur[p] = nxt[p];
            });
        });
        static_for<j>([&](auto I) {
            constexpr int r = n - 2 * j + 2 * (decltype(I)::value + 1);
            double nxt[M];
            delta<r>(cur, nxt);
            static_for<M>([&](auto A) {
                constexpr int p = decltype(A)::value;
                if constexpr (mi_order(p) == r) cur[p] = nxt[p];
            });
        });
        static_for<M>([&](auto A) {
            constexpr int p = decltype(A)::value;
            if constexpr (mi_order(p) == n) out[p] = cur[p];
        });
    }
    // L_j^T wb (order n) accumulated into tdb (order n)
    template <int n, int j>
    SMRT_HD static void lift_T(const double (&wb)[M], double (&tdb)[M]) {
        double cur[M];
        static_for<M>([&](auto A) { cur[decltype(A)::value] = 0.0; });
        static_for<M>([&](auto A) {
            constexpr int p = decltype(A)::value;
            if constexpr (mi_order(p) == n) cur[p] = wb[p];
        });
        static_for<j>([&](auto I) {  // delta^T from order n down to n - 2j
            constexpr int r = n - 2 * decltype(I)::value;
            double nxt[M];
            static_for<M>([&](auto A) { nxt[decltype(A)::value] = 0.0; });
            delta_T<r>(cur, nxt);
            static_for<M>([&](auto A) {
                constexpr int p = decltype(A)::value;
                if constexpr (mi_order(p) == r - 2) cur[p] = nxt[p];
            });
        });
        static_for<j>([&](auto I) {  // tr^T from order n - 2j up to n
            constexpr int r = n - 2 * j + 2 * (decltype(I)::value + 1);
            double nxt[M];
            static_for<M>([&](auto A) { nxt[decltype(A)::value] = 0.0; });
            tr_T<r>(cur, nxt);
            static_for<M>([&](auto A) {
                constexpr int p = decltype(A)::value;
                if constexpr (mi_order(p) == r) cur[p] = nxt[p];
            });
        });
        static_for<M>([&](auto A) {
            constexpr int p = decltype(A)::value;
            if constexpr (mi_order(p) == n) tdb[p] += cur[p];
        });
    }
};

// ... and the sums over the populations of a velocity set with compile-time vectors.
template <class Lat, int Nm>
struct AdjMath : AdjMoments<Nm> {
    static constexpr int Q = Lat::Q;
    static constexpr int NP = Lat::NP;
    static constexpr int M = nmom(Nm);

    // The contractions run per sign orbit of the velocity set (lattices.cuh): a monomial sum over
    // an orbit is a^gamma times one entry of a Walsh-Hadamard transform of its pair sums (even
    // |gamma|) or differences (odd |gamma|), and the transposed contraction is the same
    // transform of per-parity-class sums; a quarter of the multiply-adds of a pair-by-pair sum
    // on the 8-member orbits.
    static constexpr SignOrbits<Lat> kOrb = SignOrbits<Lat>();

    // unnormalised Walsh-Hadamard transform of NB = 1, 2 or 4 values in place:
    // x_out[c] = sum_b (-1)^popcount(b & c) x_in[b]
    template <int NB>
    SMRT_HD static void wht_d(double (&x)[NB]) {
        static_for<(NB >= 4 ? 2 : (NB >= 2 ? 1 : 0))>([&](auto Tt) {
            constexpr int bit = 1 << decltype(Tt)::value;
            static_for<NB>([&](auto Bb) {
                constexpr int bb = decltype(Bb)::value;
                if constexpr ((bb & bit) == 0) {
                    const double lo = x[bb], hi = x[bb | bit];
                    x[bb] = lo + hi;
                    x[bb | bit] = lo - hi;
                }
            });
        });
    }

    // F1: Rc_g = c^|g| sum_i x_i e_i^g  (x in library order)
    SMRT_HD static void raw(const double (&x)[Q], double c, double (&Rc)[M]) {
        double cpow[Nm + 1];
        double cp = 1.0;
        static_for<Nm + 1>([&](auto J) {
            cpow[decltype(J)::value] = cp;
            cp *= c;
        });
        static_for<M>([&](auto G) { Rc[decltype(G)::value] = 0.0; });
        Rc[0] = x[0];
        static_for<kOrb.n>([&](auto O) {
            constexpr int o = decltype(O)::value;
            constexpr int np = 1 << (kOrb.k[o] - 1);
            double S[np], D[np];
            static_for<np>([&](auto B) {
                constexpr int bb = decltype(B)::value, p = kOrb.pair[o][bb];
                constexpr bool fl = kOrb.flip[o][bb] != 0;
                const double fp = x[2 * p + 1], fm = x[2 * p + 2];
                S[bb] = fp + fm;
                D[bb] = fl ? fm - fp : fp - fm;
            });
            wht_d<np>(S);
            wht_d<np>(D);
            static_for<M>([&](auto G) {
                constexpr int g = decltype(G)::value;
                constexpr int m = kOrb.monomial(o, g);
                if constexpr (m != 0) {
                    constexpr int cl = kOrb.parity_class(o, g);
                    if constexpr ((mi_order(g) & 1) == 0)
                        Rc[g] += double(m) * S[cl];
                    else
                        Rc[g] += double(m) * D[cl];
                }
            });
        });
        static_for<M>([&](auto G) {
            constexpr int g = decltype(G)::value;
            if constexpr (mi_order(g) > 0) Rc[g] *= cpow[mi_order(g)];
        });
    }

    // F1': xb_i += sum_g c^|g| e_i^g Rcb_g
    SMRT_HD static void raw_T(const double (&Rcb)[M], double c, double (&xb)[Q]) {
        double cp = 1.0;
        double sc[M];
        double cpow[Nm + 1];
        static_for<Nm + 1>([&](auto J) {
            cpow[decltype(J)::value] = cp;
            cp *= c;
        });
        static_for<M>([&](auto G) { sc[decltype(G)::value] = Rcb[decltype(G)::value] * cpow[mi_order(decltype(G)::value)]; });
        xb[0] += sc[0];
        static_for<kOrb.n>([&](auto O) {
            constexpr int o = decltype(O)::value;
            constexpr int np = 1 << (kOrb.k[o] - 1);
            double E[np], Od[np];
            static_for<np>([&](auto B) {
                E[decltype(B)::value] = 0.0;
                Od[decltype(B)::value] = 0.0;
            });
            static_for<M>([&](auto G) {
                constexpr int g = decltype(G)::value;
                constexpr int m = kOrb.monomial(o, g);
                if constexpr (m != 0) {
                    constexpr int cl = kOrb.parity_class(o, g);
                    if constexpr ((mi_order(g) & 1) == 0)
                        E[cl] += double(m) * sc[g];
                    else
                        Od[cl] += double(m) * sc[g];
                }
            });
            wht_d<np>(E);  // the even and odd parts of the sum at each member of the orbit
            wht_d<np>(Od);
            static_for<np>([&](auto B) {
                constexpr int bb = decltype(B)::value, p = kOrb.pair[o][bb];
                constexpr bool fl = kOrb.flip[o][bb] != 0;
                const double vplus = E[bb] + Od[bb], vminus = E[bb] - Od[bb];
                xb[2 * p + 1] += fl ? vminus : vplus;
                xb[2 * p + 2] += fl ? vplus : vminus;
            });
        });
    }
};

// Conserved moments from the raw moments (F2) and the transpose of F2 (onto Rcb).
template <int M>
struct Conserved {
    double rho, rhom1, u[3], thm1, th;
    SMRT_HD void from_raw(const double (&Rc)[M]) {
        rhom1 = Rc[0];
        rho = 1.0 + rhom1;
        u[0] = Rc[mi_pos(1, 0, 0)] / rho;
        u[1] = Rc[mi_pos(0, 1, 0)] / rho;
        u[2] = Rc[mi_pos(0, 0, 1)] / rho;
        const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const double em3 = Rc[mi_pos(2, 0, 0)] + Rc[mi_pos(0, 2, 0)] + Rc[mi_pos(0, 0, 2)];
        thm1 = (em3 - 3.0 * rhom1 - rho * uu) / (3.0 * rho);
        th = 1.0 + thm1;
    }
    // rhob collects every adjoint of rho (and of rho - 1); ub, tb those of u and theta - 1
    SMRT_HD void transpose(double rhob, const double (&ub)[3], double tb, double (&Rcb)[M]) const {
        const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        Rcb[0] += rhob - (ub[0] * u[0] + ub[1] * u[1] + ub[2] * u[2]) / rho +
                  tb * ((uu - 3.0) / (3.0 * rho) - thm1 / rho);
        Rcb[mi_pos(1, 0, 0)] += ub[0] / rho - tb * 2.0 * u[0] / (3.0 * rho);
        Rcb[mi_pos(0, 1, 0)] += ub[1] / rho - tb * 2.0 * u[1] / (3.0 * rho);
        Rcb[mi_pos(0, 0, 1)] += ub[2] / rho - tb * 2.0 * u[2] / (3.0 * rho);
        Rcb[mi_pos(2, 0, 0)] += tb / (3.0 * rho);
        Rcb[mi_pos(0, 2, 0)] += tb / (3.0 * rho);
        Rcb[mi_pos(0, 0, 2)] += tb / (3.0 * rho);
    }
};

// Moment-space part of the collision's VJP, common to every velocity set: Rc_g = c^|g| sum_i
// df_i e_i^g (the pre-collision raw moments) and Lc_g = c^|g| sum_i w_i lam_i e_i^g (the
// projection of the weighted adjoint of the rebuilt populations) in; Rcb (out, overwritten) =
// the adjoint of Rc, so that fb_i = sum_g c^|g| e_i^g Rcb_g; taub_k += sum over the cell of
// lam . d out / d tau_c,k. dAdt / dBdt: derivatives of the per-slot A, B with respect to tau_c
// (see top).
template <int N>
SMRT_HD void moment_vjp(const double (&Rc)[nmom(N)], const double (&Lc)[nmom(N)], const double *tauA,
                        const double *tauB, double dAdt, double dBdt, double (&Rcb)[nmom(N)],
                        double (&taub)[ntau(N)]) {
    using AM = AdjMoments<N>;
    constexpr int M = nmom(N);
    constexpr int KT = ntau(N);
    // ---- forward recompute
    Conserved<M> cs;
    cs.from_raw(Rc);
    const double rho = cs.rho, th = cs.th, t1 = cs.thm1;
    double ta[M];
    AM::template hmap<false>(Rc, ta);
    ta[0] = rho;
    double Gm[3][N + 1], Gp[3][N + 1];
    for (int k = 0; k < 3; ++k) {
        AM::maxwell(-cs.u[k], -t1, Gm[k]);
        AM::maxwell(cs.u[k], t1, Gp[k]);
    }
    double p1[M], p2[M], p3[M];
    AM::template pass<0>(ta, Gm[0], p1);
    AM::template pass<1>(p1, Gm[1], p2);
    AM::template pass<2>(p2, Gm[2], p3);
    const double sq = sqrt(th), is = 1.0 / sq;
    double isp[N + 1], sqp[N + 1];
    isp[0] = sqp[0] = 1.0;
    for (int j = 1; j <= N; ++j) {
        isp[j] = isp[j - 1] * is;
        sqp[j] = sqp[j - 1] * sq;
    }
    double td[M];
    static_for<M>([&](auto A) {
        constexpr int p = decltype(A)::value;
        td[p] = p3[p] * isp[mi_order(p)];
    });
    double s[KT], R[KT];
    for (int k = 0; k < KT; ++k) {
        R[k] = 1.0 / (tauA[k] + tauB[k] * rho);
        s[k] = 1.0 - rho * R[k];
    }
    // relaxation: td'_n = sum_j C_j L_j td_n; keep L_j td_n for the C_j adjoints
    double tdp[M];
    static_for<M>([&](auto A) { tdp[decltype(A)::value] = 0.0; });
    double Lj[N + 1][N / 2 + 1][M];
    static_for<N - 1>([&](auto Nn) {
        constexpr int n = decltype(Nn)::value + 2;
        static_for<n / 2 + 1>([&](auto Jj) {
            constexpr int j = decltype(Jj)::value;
            AM::template lift<n, j>(td, Lj[n][j]);
            double Cj = 0.0;
            static_for<j + 1>([&](auto Mm) {
                constexpr int m = decltype(Mm)::value;
                Cj += coefB(n, m) * coefD(n - 2 * m, j - m) * s[tau_slot(n, m)];
            });
            static_for<M>([&](auto A) {
                constexpr int p = decltype(A)::value;
                if constexpr (mi_order(p) == n) tdp[p] += Cj * Lj[n][j][p];
            });
        });
    });
    double y[M];
    static_for<M>([&](auto A) {
        constexpr int p = decltype(A)::value;
        if constexpr (mi_order(p) == 0)
            y[p] = rho;
        else if constexpr (mi_order(p) == 1)
            y[p] = 0.0;
        else
            y[p] = tdp[p] * sqp[mi_order(p)];
    });
    double q1[M], q2[M];
    AM::template pass<0>(y, Gp[0], q1);
    AM::template pass<1>(q1, Gp[1], q2);

    // ---- reverse
    double tapb[M];
    static_for<M>([&](auto A) { tapb[decltype(A)::value] = 0.0; });
    AM::template hmap<true>(Lc, tapb);  // F7': tapb_a = sum_g hfull(a, g) Lc_g
    double rhob = tapb[0];               // ta'_0 := rho - 1 after the transform
    tapb[0] = 0.0;
    double ub[3] = {0.0, 0.0, 0.0}, tb = 0.0;
    double q2b[M], q1b[M], yb[M];
    double Gb[3][N + 1];
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j <= N; ++j) Gb[k][j] = 0.0;
    static_for<M>([&](auto A) {
        constexpr int p = decltype(A)::value;
        q2b[p] = q1b[p] = yb[p] = 0.0;
    });
    AM::template pass_T<2>(tapb, Gp[2], q2, q2b, Gb[2]);
    AM::template pass_T<1>(q2b, Gp[1], q1, q1b, Gb[1]);
    AM::template pass_T<0>(q1b, Gp[0], y, yb, Gb[0]);
    for (int k = 0; k < 3; ++k) AM::maxwell_T(cs.u[k], t1, Gp[k], Gb[k], ub[k], tb);
    // F6'
    rhob += yb[0];
    double tdpb[M];
    static_for<M>([&](auto A) {
        constexpr int p = decltype(A)::value;
        constexpr int o = mi_order(p);
        if constexpr (o >= 2) {
            tdpb[p] = yb[p] * sqp[o];
            tb += yb[p] * tdp[p] * (0.5 * o) * sqp[o] / th;
        } else {
            tdpb[p] = 0.0;
        }
    });
    // F5'
    double tdb[M], sb[KT];
    static_for<M>([&](auto A) { tdb[decltype(A)::value] = 0.0; });
    for (int k = 0; k < KT; ++k) sb[k] = 0.0;
    static_for<N - 1>([&](auto Nn) {
        constexpr int n = decltype(Nn)::value + 2;
        static_for<n / 2 + 1>([&](auto Jj) {
            constexpr int j = decltype(Jj)::value;
            double Cj = 0.0, Cjb = 0.0;
            static_for<j + 1>([&](auto Mm) {
                constexpr int m = decltype(Mm)::value;
                Cj += coefB(n, m) * coefD(n - 2 * m, j - m) * s[tau_slot(n, m)];
            });
            double scaled[M];
            static_for<M>([&](auto A) {
                constexpr int p = decltype(A)::value;
                if constexpr (mi_order(p) == n) {
                    Cjb += tdpb[p] * Lj[n][j][p];
                    scaled[p] = Cj * tdpb[p];
                } else {
                    scaled[p] = 0.0;
                }
            });
            AM::template lift_T<n, j>(scaled, tdb);
            static_for<j + 1>([&](auto Mm) {
                constexpr int m = decltype(Mm)::value;
                sb[tau_slot(n, m)] += coefB(n, m) * coefD(n - 2 * m, j - m) * Cjb;
            });
        });
    });
    for (int k = 0; k < KT; ++k) {
        rhob += sb[k] * (-tauA[k] * R[k] * R[k]);
        taub[k] += sb[k] * (rho * R[k] * R[k] * dAdt + rho * rho * R[k] * R[k] * dBdt);
    }
    // F4'
    double p3b[M], p2b[M], p1b[M], tab[M];
    static_for<M>([&](auto A) {
        constexpr int p = decltype(A)::value;
        constexpr int o = mi_order(p);
        p2b[p] = p1b[p] = tab[p] = 0.0;
        if constexpr (o >= 2) {
            p3b[p] = tdb[p] * isp[o];
            tb -= tdb[p] * p3[p] * (0.5 * o) * isp[o] / th;
        } else {
            p3b[p] = 0.0;
        }
    });
    double Gmb[3][N + 1];
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j <= N; ++j) Gmb[k][j] = 0.0;
    AM::template pass_T<2>(p3b, Gm[2], p2, p2b, Gmb[2]);
    AM::template pass_T<1>(p2b, Gm[1], p1, p1b, Gmb[1]);
    AM::template pass_T<0>(p1b, Gm[0], ta, tab, Gmb[0]);
    for (int k = 0; k < 3; ++k) {
        double umb = 0.0, tmb = 0.0;
        AM::maxwell_T(-cs.u[k], -t1, Gm[k], Gmb[k], umb, tmb);
        ub[k] -= umb;
        tb -= tmb;
    }
    // F3'
    rhob += tab[0];
    tab[0] = 0.0;
    static_for<M>([&](auto A) { Rcb[decltype(A)::value] = 0.0; });
    AM::template hmap_T<false>(tab, Rcb);
    // F2', F1'
    cs.transpose(rhob, ub, tb, Rcb);
}

// Per-cell VJP of the collision: given pre-collision deviations f and lam = dL/d out,
// fb = (d out / d f)^T lam and taub_k = sum over the cell of lam . d out / d tau_c,k.
template <class Lat, int N>
SMRT_HD void collide_vjp(const double (&f)[Lat::Q], const double (&lam)[Lat::Q], double c,
                         const double (&wp)[Lat::NP + 1], const double *tauA, const double *tauB,
                         double dAdt, double dBdt, double (&fb)[Lat::Q], double (&taub)[ntau(N)]) {
    using AM = AdjMath<Lat, N>;
    constexpr int M = nmom(N);
    constexpr int Q = Lat::Q;
    constexpr int NP = Lat::NP;
    double Rc[M], Lc[M], Rcb[M];
    AM::raw(f, c, Rc);
    double wl[Q];
    wl[0] = wp[0] * lam[0];
    static_for<NP>([&](auto Pp) {
        constexpr int p = decltype(Pp)::value;
        wl[2 * p + 1] = wp[p + 1] * lam[2 * p + 1];
        wl[2 * p + 2] = wp[p + 1] * lam[2 * p + 2];
    });
    AM::raw(wl, c, Lc);
    moment_vjp<N>(Rc, Lc, tauA, tauB, dAdt, dBdt, Rcb, taub);
    static_for<Q>([&](auto I) { fb[decltype(I)::value] = 0.0; });
    AM::raw_T(Rcb, c, fb);
}

// Moment-space part of the VJP of the moments rho, u (physical), theta, q of lb_moments: Rc (the
// raw moments, c-scaled, |g| <= max(N, 3)) in; Rcb (out, overwritten) their adjoint given the
// moments' adjoints, so that fb_i = sum_g c^|g| e_i^g Rcb_g. Uses the order-3 local
// coefficients.
template <int Nm>
SMRT_HD void moments_vjp_m(const double (&Rc)[nmom(Nm)], double rhob_out, const double (&ub_out)[3],
                           double thb_out, const double (&qb)[3], double (&Rcb)[nmom(Nm)]) {
    using AM = AdjMoments<Nm>;
    constexpr int M = nmom(Nm);
    Conserved<M> cs;
    cs.from_raw(Rc);
    const double th = cs.th, t1 = cs.thm1;
    double ta[M];
    AM::template hmap<false>(Rc, ta);
    ta[0] = cs.rho;
    double Gm[3][Nm + 1];
    for (int k = 0; k < 3; ++k) AM::maxwell(-cs.u[k], -t1, Gm[k]);
    double p1[M], p2[M], p3[M];
    AM::template pass<0>(ta, Gm[0], p1);
    AM::template pass<1>(p1, Gm[1], p2);
    AM::template pass<2>(p2, Gm[2], p3);
    const double sq = sqrt(th), is = 1.0 / sq;
    const double is3 = is * is * is;
    // q_k = 1/2 th^(3/2) sum_l d_{e_k + 2 e_l}, d = beta! td, td = p3 th^(-3/2) (order 3)
    // so q_k = 1/2 sum_l beta! p3_{e_k + 2 e_l}: the theta factors cancel.
    double p3b[M];
    static_for<M>([&](auto A) { p3b[decltype(A)::value] = 0.0; });
    static_for<3>([&](auto K) {
        constexpr int k = decltype(K)::value;
        static_for<3>([&](auto Ll) {
            constexpr int l = decltype(Ll)::value;
            constexpr int a0 = (k == 0) + 2 * (l == 0), a1 = (k == 1) + 2 * (l == 1), a2 = (k == 2) + 2 * (l == 2);
            constexpr int p = mi_pos(a0, a1, a2);
            p3b[p] += 0.5 * mi_fact(p) * qb[k];
        });
    });
    (void)is3;
    double p2b[M], p1b[M], tab[M];
    static_for<M>([&](auto A) {
        constexpr int p = decltype(A)::value;
        p2b[p] = p1b[p] = tab[p] = 0.0;
    });
    double Gmb[3][Nm + 1];
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j <= Nm; ++j) Gmb[k][j] = 0.0;
    AM::template pass_T<2>(p3b, Gm[2], p2, p2b, Gmb[2]);
    AM::template pass_T<1>(p2b, Gm[1], p1, p1b, Gmb[1]);
    AM::template pass_T<0>(p1b, Gm[0], ta, tab, Gmb[0]);
    double ub[3] = {ub_out[0], ub_out[1], ub_out[2]}, tb = thb_out;
    for (int k = 0; k < 3; ++k) {
        double umb = 0.0, tmb = 0.0;
        AM::maxwell_T(-cs.u[k], -t1, Gm[k], Gmb[k], umb, tmb);
        ub[k] -= umb;
        tb -= tmb;
    }
    double rhob = rhob_out + tab[0];
    tab[0] = 0.0;
    static_for<M>([&](auto A) { Rcb[decltype(A)::value] = 0.0; });
    AM::template hmap_T<false>(tab, Rcb);
    cs.transpose(rhob, ub, tb, Rcb);
}

// Per-cell VJP of the moments rho, u (physical), theta, q of lb_moments: given their adjoints
// (qb[3], ub_out[3]), fb = (d moments / d f)^T (.).
template <class Lat, int N>
SMRT_HD void moments_vjp(const double (&f)[Lat::Q], double c, double rhob_out, const double (&ub_out)[3],
                         double thb_out, const double (&qb)[3], double (&fb)[Lat::Q]) {
    constexpr int Nm = N < 3 ? 3 : N;
    using AM = AdjMath<Lat, Nm>;
    constexpr int M = nmom(Nm);
    double Rc[M], Rcb[M];
    AM::raw(f, c, Rc);
    moments_vjp_m<Nm>(Rc, rhob_out, ub_out, thb_out, qb, Rcb);
    static_for<Lat::Q>([&](auto I) { fb[decltype(I)::value] = 0.0; });
    AM::raw_T(Rcb, c, fb);
}

}  // namespace smrt
