// kernels.cuh -- the fused collide-and-stream kernel of LB-SMRT and its helpers
// (Yan & Shan, arXiv 2401.11086), templated on the velocity set, the truncation order N,
// the storage/arithmetic type T and the type Acc of the conserved sums.
//
// Per cell and step (one thread per cell, pull scheme, structure-of-arrays populations):
//   a1  pull f_i from x - e_i - k of the previous state (Sec. 3 streaming with the shifted
//       stencil of Sec. 4.1); cells beyond a fixed x end read the end state's equilibrium
//       (Sec. 4.2);
//   a2  conserved sums rho, rho u, rho(|u|^2 + 3 theta) in Acc (Eq. hermite1 moments);
//   a3  raw lattice moments R_gamma = sum_i f_i e_i^gamma, |gamma| <= N, with +-e pairs folded,
//       then the absolute Hermite coefficients a_alpha = sum_i f_i He_alpha(xi_i) (Eq. an);
//   a4  binomial transform to the local frame, d = T(u, theta)^-1 a (Sec. 3);
//   a5  irreducible split and relaxation of each order n >= 2 with its own times (Eq. SMRT,
//       Appendix A), orders 0 and 1 untouched;
//   a6  back to the absolute frame, truncated at N;
//   a7  rebuild f_i' = w_i sum_alpha a'_alpha He_alpha(xi_i)/alpha! (Eq. fi) as a polynomial in
//       the integer e_i, evaluated once per +-e pair (even and odd parts);
//   a8  store f_i' at x (aligned, coalesced).
// Relaxation times: 1/tau_nm(x) = rho / (A_nm + B_nm rho), which covers both the
// Maxwell-molecule law tau_nm = tau_c,nm rho_ref / rho + 1/2 (A = tau_c rho_ref, B = 1/2) and
// constant times (A = 0, B = tau_c + 1/2).
#pragma once

#include <cuda.h>  // CUtensorMap (the type only; maps are encoded by the host)
#include <cuda_runtime.h>

#include "core.cuh"
#include "lattices.cuh"

namespace smrt {

constexpr int kMaxTau = 10;

struct InstanceInfo {
    long long cell_off;  // first cell of the instance in the concatenated cell index
    int nx;              // cells along x
    int kx;              // frame shift along x (u_bar_x = c kx)
    double tauA[kMaxTau];
    double tauB[kMaxTau];
    float tauAf[kMaxTau];  // the same in float, read by the float kernels
    float tauBf[kMaxTau];
    double dAdt, dBdt;     // d tauA / d tau_c and d tauB / d tau_c (adjoint)
    int model;             // collision model: 0 SMRT, 1 ES-BGK (tensor-product sets)
    double es_b;           // ES-BGK parameter b of the continuous model
};

template <class T>
SMRT_D const T *tau_a(const InstanceInfo &in);
template <>
SMRT_D const double *tau_a<double>(const InstanceInfo &in) { return in.tauA; }
template <>
SMRT_D const float *tau_a<float>(const InstanceInfo &in) { return in.tauAf; }
template <class T>
SMRT_D const T *tau_b(const InstanceInfo &in);
template <>
SMRT_D const double *tau_b<double>(const InstanceInfo &in) { return in.tauB; }
template <>
SMRT_D const float *tau_b<float>(const InstanceInfo &in) { return in.tauBf; }

template <class Lat, class T>
struct StepArgs {
    const T *__restrict__ fin;
    T *__restrict__ fout;
    const InstanceInfo *__restrict__ inst;
    const int2 *__restrict__ tiles;  // line kernel: (instance, first x) per block
    const T *__restrict__ ghosts;    // [instance][2][Q], library order
    const double *__restrict__ ghostsd;  // the same end-state deviations in double
    unsigned *health;
    long long plane[Lat::Q];  // element offset of each population plane, library order
    T wp[Lat::NP + 1];        // weight of the rest velocity, then of each pair
    double wpd[Lat::NP + 1];  // the same weights in double, for every double-precision rebuild
    float wlo[Lat::NP + 1];   // w - float(w): the weights as two-float numbers (split precision)
    T c;
    double cd;                // c in double
    float clo;                // c - float(c)
    int nx, ny, nz;           // box kernel geometry
    int kx, ky, kz;           // box kernel frame shift
    unsigned step;            // step counter (stochastic rounding of the split precision)
};

// Conversions between float and double on the IEEE 754 bit patterns, in integer instructions:
// the split-precision step converts every population twice, and on this GPU the double
// conversion instructions share the slow double-precision pipe with the arithmetic.
// widen: binary32 -> binary64, exponent rebiased by 1023 - 127 = 896, fraction moved up 29 bits.
// Zeros and subnormals (|x| < 2^-126) give signed zero; infinities and NaNs keep their class.
template <class To, class From>
SMRT_D To widen(From x) {
    return To(x);
}
template <>
SMRT_D double widen<double, float>(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned s = b & 0x80000000u, m = b ^ s;
    unsigned hi = s | ((m >> 3) + (896u << 20)), lo = b << 29;
    if (m < 0x00800000u) hi = s, lo = 0u;
    if (m >= 0x7f800000u) hi = s | 0x7ff00000u | ((m >> 3) & 0x000fffffu);
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}

// Stochastic rounding of a double to float: the result is the float neighbour above or below
// x with probabilities proportional to the closeness of x to each, drawn from a counter-based
// hash of (cell, population, step), so that storing a steady state leaves no systematic bias.
// On the bit pattern: a uniform 29-bit integer is added to the magnitude below the 24 bits a
// float keeps (a carry rounds the magnitude up, with probability equal to the dropped fraction
// of a float spacing; a carry into the exponent gives the next binade's first float), the
// dropped bits are discarded and the exponent rebiased. Magnitudes below 2^-126 give signed
// zero, at or above 2^128 infinity; NaNs stay NaN.
SMRT_D unsigned mix32(unsigned h) {  // the 32-bit finaliser of MurmurHash3
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}
SMRT_D float round_stochastic(double x, unsigned key) {
    const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned s = static_cast<unsigned>(bits >> 32) & 0x80000000u;
    const unsigned long long mag = bits & 0x7fffffffffffffffull;
    const unsigned long long t = mag + static_cast<unsigned long long>(mix32(key) >> 3);  // 29 bits
    unsigned y = s | (static_cast<unsigned>(t >> 29) - (896u << 23));
    if (mag < 0x3810000000000000ull) y = s;                               // below 2^-126
    if (t >= 0x47f0000000000000ull) y = s | 0x7f800000u;                  // 2^128 and above
    if (mag > 0x7ff0000000000000ull) y = s | 0x7fc00000u;                 // NaN
    return __uint_as_float(y);
}

// ------------------------------------------------------------------------------ two-float
// Unevaluated sums hi + lo of two floats (about 48 significant bits) built from error-free
// transformations: Knuth's two-sum (a + b and its rounding error in six additions) and the
// product with its rounding error from one fused multiply-add. The split-precision step uses
// them, on the single-precision pipe, wherever it needs more than a float's 24 bits. The
// __f*_rn intrinsics are never contracted into fused operations by the compiler, which these
// transformations rely on.
struct ff {
    float hi, lo;
};
SMRT_D ff ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
SMRT_D ff ff_quick(float a, float b) {  // two-sum when |a| >= |b| or a = 0
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
SMRT_D ff operator+(ff a, ff b) {
    const ff s = ff_two_sum(a.hi, b.hi);
    return ff_quick(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
SMRT_D ff operator-(ff a) { return {-a.hi, -a.lo}; }
SMRT_D ff operator-(ff a, ff b) { return a + (-b); }
SMRT_D ff operator+(ff a, float b) {
    const ff s = ff_two_sum(a.hi, b);
    return ff_quick(s.hi, __fadd_rn(s.lo, a.lo));
}
SMRT_D ff operator*(ff a, float b) {
    const float p = __fmul_rn(a.hi, b);
    return ff_quick(p, __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p)));
}
SMRT_D ff operator*(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return ff_quick(p, e);
}
SMRT_D ff ff_div(ff a, ff b) {  // one correction step after the float quotient
    const float r = __frcp_rn(b.hi);
    const float q1 = __fmul_rn(a.hi, r);
    const ff rem = a - b * q1;
    return ff_quick(q1, __fmul_rn(rem.hi, r));
}

// 1/n as a two-float number (the double quotient split in two floats, about 2^-50)
template <int n>
SMRT_D ff ff_inv() {
    constexpr float hi = float(1.0 / n);
    constexpr float lo = float(1.0 / n - double(hi));
    return ff{hi, lo};
}

// Fixed point: x 2^S rounded to the nearest integer (the hardware conversion of the exactly
// scaled float). Sums of such integers are exact and independent of their order. Valid for
// |x| < 2^(62 - S); magnitudes below 2^-(S + 1) give 0. The split-precision step keeps
// populations and raw moments at S = kFix (2^-44 resolution, range 2^18) and the equilibrium's
// monomial coefficients at S = kFixP (2^-48, range 2^14).
constexpr int kFix = 44;
constexpr int kFixP = 48;
constexpr float pow2f(int e) { return e >= 0 ? float(1ull << e) : 1.0f / float(1ull << -e); }
template <int S = kFix>
SMRT_D long long to_fixed(float x) {
    return __float2ll_rn(x * pow2f(S));
}
template <int S = kFix>
SMRT_D long long to_fixed(double x) {
    return __double2ll_rn(x * static_cast<double>(1ull << S));
}
// Exact sum of products m x (m a small positive constant, x a 64-bit integer) in one 64-bit
// accumulator, each product formed as m lo32(x) (a 32 x 32 -> 64-bit multiply-add) plus
// m hi32(x) added to the upper word. Arithmetic is modulo 2^64, so the sum is exact whenever it
// fits in 64 bits.
struct SplitAcc {
    unsigned long long v = 0;
    template <int m>
    SMRT_D void madd(long long x) {
        static_assert(m > 0, "positive multiplier");
        const unsigned long long ux = static_cast<unsigned long long>(x);
        v += static_cast<unsigned long long>(static_cast<unsigned>(ux)) * static_cast<unsigned>(m);
        v += static_cast<unsigned long long>(static_cast<unsigned>(ux >> 32) * static_cast<unsigned>(m)) << 32;
    }
    SMRT_D void add(long long x) { v += static_cast<unsigned long long>(x); }
    SMRT_D long long value() const { return static_cast<long long>(v); }
};

// q 2^-S as a two-float number: q = a 2^48 + b 2^24 + c with 0 <= b, c < 2^24, each piece
// exact as a float
template <int S = kFix>
SMRT_D ff fixed_to_ff(long long q) {
    const float a = float(int(q >> 48)) * pow2f(48 - S);
    const float b = float(int((q >> 24) & 0xffffff)) * pow2f(24 - S);
    const float c = float(int(q & 0xffffff)) * pow2f(-S);
    const ff s = ff_two_sum(a, b);
    return ff_quick(s.hi, __fadd_rn(s.lo, c));
}

// Stochastic rounding of a two-float value hi + lo (|lo| at most half a float spacing of hi) to
// a float: hi's neighbour on lo's side with probability |lo| / (distance to that neighbour),
// else hi, drawn from the same counter-based hash as above.
SMRT_D float round_stochastic(ff x, unsigned key) {
    const unsigned hb = __float_as_uint(x.hi);
    const bool away = (x.lo > 0.f) == (x.hi > 0.f);  // the neighbour of larger magnitude
    const float nb = __uint_as_float(away ? hb + 1u : hb - 1u);
    const float gap = fabsf(__fsub_rn(nb, x.hi));
    const float u = __fmul_rn(__uint2float_rn(mix32(key) >> 8), 0x1p-24f);  // uniform in [0, 1)
    return fabsf(x.lo) > __fmul_rn(u, gap) ? nb : x.hi;
}

template <class T>
SMRT_D T rcp_tau(T A, T B, T rho) {
    return rho * rcp(fma(B, rho, A));
}

// Moments of the unit Maxwellian (rho = 1, u = 0, theta = 1), which the weights reproduce up to
// the set's degree: sum_i w_i xi_i^g = prod_k (g_k - 1)!! for even g_k, 0 otherwise.
constexpr double unit_moment3(int a, int b, int c) {
    return ((a & 1) || (b & 1) || (c & 1)) ? 0.0 : cdfact(a - 1) * cdfact(b - 1) * cdfact(c - 1);
}
constexpr double unit_moment(int g) { return unit_moment3(mi_comp(g, 0), mi_comp(g, 1), mi_comp(g, 2)); }

// Unnormalised Walsh-Hadamard transform of NB = 1, 2 or 4 values in place:
// x_out[c] = sum_b (-1)^popcount(b & c) x_in[b].
template <int NB, class U>
SMRT_D void wht(U (&x)[NB]) {
    static_for<(NB >= 4 ? 2 : (NB >= 2 ? 1 : 0))>([&](auto Tt) {
        constexpr int bit = 1 << decltype(Tt)::value;
        static_for<NB>([&](auto Bb) {
            constexpr int b = decltype(Bb)::value;
            if constexpr ((b & bit) == 0) {
                const U lo = x[b], hi = x[b | bit];
                x[b] = lo + hi;
                x[b | bit] = lo - hi;
            }
        });
    });
}

// ------------------------------------------------------------------------------ collision
template <class Lat, int N, class T, class Acc, bool Split>
struct Collide {
    static constexpr int Q = Lat::Q;
    static constexpr int NP = Lat::NP;
    static constexpr int M = nmom(N);
    static constexpr int KT = ntau(N);
    static constexpr SignOrbits<Lat> kOrb = SignOrbits<Lat>();

    // a2: conserved sums, in Acc. The state holds deviations df_i = f_i - w_i; the quadrature
    // gives sum w_i = 1, sum w_i xi_i = 0, sum w_i |xi_i|^2 = 3, so
    //   rho - 1 = sum df_i,  rho u = c sum e_i df_i,  E - 3 = c^2 sum |e_i|^2 df_i,
    //   theta - 1 = (E - 3 - 3 (rho - 1) - rho |u|^2) / (3 rho),
    // which keeps rho - 1 and theta - 1 free of cancellation.
    SMRT_D static void conserved(const T (&f)[Q], Acc c, Acc &rho, Acc &rhom1, Acc (&u)[3],
                                 Acc &theta, Acc &thm1) {
        Acc raw[5];
        conserved(f, c, rho, rhom1, u, theta, thm1, raw);
    }
    // ... also returning the raw sums (sum df, sum e df, sum |e|^2 df) in raw[0..4]
    SMRT_D static void conserved(const T (&f)[Q], Acc c, Acc &rho, Acc &rhom1, Acc (&u)[3],
                                 Acc &theta, Acc &thm1, Acc (&raw)[5]) {
        conserved_sums(f, raw);
        from_raw_sums(raw, c, rho, rhom1, u, theta, thm1);
    }
    // sum x_i, sum e_i x_i, sum |e_i|^2 x_i in Acc, per sign orbit: the orbit's pair sums
    // added up once (|e|^2 is constant on it) and its pair differences transformed, so that
    // each total takes one term per orbit (short dependency chains) instead of one per pair
    template <class U>
    SMRT_D static void conserved_sums(const U (&x)[Q], Acc (&raw)[5]) {
        Acc j[3] = {Acc(0), Acc(0), Acc(0)};
        Acc r = widen<Acc>(x[0]), en = Acc(0);
        static_for<kOrb.n>([&](auto O) {
            constexpr int o = decltype(O)::value;
            constexpr int k = kOrb.k[o], np = 1 << (k - 1);
            Acc S[np], D[np];
            static_for<np>([&](auto B) {
                constexpr int b = decltype(B)::value, p = kOrb.pair[o][b];
                constexpr bool fl = kOrb.flip[o][b] != 0;
                const Acc xp = widen<Acc>(x[2 * p + 1]), xm = widen<Acc>(x[2 * p + 2]);
                S[b] = xp + xm;
                D[b] = fl ? xm - xp : xp - xm;
            });
            wht<np>(S);
            wht<np>(D);
            constexpr int aa = kOrb.a[o][0] * kOrb.a[o][0] + kOrb.a[o][1] * kOrb.a[o][1] + kOrb.a[o][2] * kOrb.a[o][2];
            r += S[0];
            en = fma(Acc(aa), S[0], en);
            // sum over the orbit of e_d x = a_d times transform entry 0 (d = ax[0]) or the entry
            // with the single bit of ax[t]
            static_for<k>([&](auto Tt) {
                constexpr int t = decltype(Tt)::value, d = kOrb.ax[o][t];
                constexpr int cl = t == 0 ? 0 : 1 << (t - 1), ad = kOrb.a[o][d];
                j[d] = fma(Acc(ad), D[cl], j[d]);
            });
        });
        raw[0] = r;
        raw[1] = j[0];
        raw[2] = j[1];
        raw[3] = j[2];
        raw[4] = en;
    }
    // rho, u, theta from the raw sums (sum df, sum e df, sum |e|^2 df)
    SMRT_D static void from_raw_sums(const Acc (&raw)[5], Acc c, Acc &rho, Acc &rhom1, Acc (&u)[3],
                                     Acc &theta, Acc &thm1) {
        rhom1 = raw[0];
        rho = Acc(1) + raw[0];
        const Acc ir = rcp(rho);
        u[0] = c * raw[1] * ir;
        u[1] = c * raw[2] * ir;
        u[2] = c * raw[3] * ir;
        const Acc uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        thm1 = (c * c * raw[4] - Acc(3) * raw[0] - rho * uu) * ir * Acc(1.0 / 3.0);
        theta = Acc(1) + thm1;
    }

    // Raw moments R_gamma = sum_i f_i e_i^gamma, |gamma| <= Nm, summed per sign orbit: pair sums
    // and differences, their Walsh-Hadamard transform over the orbit, then one multiply-add by
    // the constant a^gamma per monomial that does not vanish on the orbit.
    template <int Nm, class U>
    SMRT_D static void raw_moments(const U (&f)[Q], U (&R)[nmom(Nm)]) {
        raw_moments_of<Nm>([&](auto I) { return f[decltype(I)::value]; }, R);
    }
    // ... with population i read as get(ic<i>) where it is needed (a pull, for the split step)
    template <int Nm, class U, class Get>
    SMRT_D static void raw_moments_of(Get &&get, U (&R)[nmom(Nm)]) {
        constexpr int Mm = nmom(Nm);
        static_for<Mm>([&](auto G) { R[decltype(G)::value] = U(0); });
        R[0] = get(ic<0>{});
        static_for<kOrb.n>([&](auto O) {
            constexpr int o = decltype(O)::value;
            constexpr int np = 1 << (kOrb.k[o] - 1);
            U S[np], D[np];
            static_for<np>([&](auto B) {
                constexpr int b = decltype(B)::value, p = kOrb.pair[o][b];
                constexpr bool fl = kOrb.flip[o][b] != 0;
                const U fp = get(ic<2 * p + 1>{}), fm = get(ic<2 * p + 2>{});
                S[b] = fp + fm;
                D[b] = fl ? fm - fp : fp - fm;
            });
            wht<np>(S);
            wht<np>(D);
            static_for<Mm>([&](auto G) {
                constexpr int g = decltype(G)::value;
                constexpr int m = kOrb.monomial(o, g);
                if constexpr (m != 0) {
                    constexpr int cl = kOrb.parity_class(o, g);
                    if constexpr ((mi_order(g) & 1) == 0)
                        R[g] = fma(U(m), S[cl], R[g]);
                    else
                        R[g] = fma(U(m), D[cl], R[g]);
                }
            });
        });
    }

    // Split precision, a2 + a3: the raw moments R_gamma = sum_i df_i e_i^gamma, |gamma| <= Nm,
    // exactly, in fixed point (get(ic<i>) gives population i in fixed point), per sign orbit as
    // raw_moments_of does, with the pair sums and transforms taken on 64-bit integers and the
    // products by a^gamma accumulated in two parts (SplitAcc).
    template <int Nm, class Get>
    SMRT_D static void fixed_moments(Get &&get, long long (&R)[nmom(Nm)]) {
        constexpr int Mm = nmom(Nm);
        SplitAcc acc[Mm];
        acc[0].add(get(ic<0>{}));
        static_for<kOrb.n>([&](auto O) {
            constexpr int o = decltype(O)::value;
            constexpr int np = 1 << (kOrb.k[o] - 1);
            long long S[np], D[np];
            static_for<np>([&](auto B) {
                constexpr int b = decltype(B)::value, p = kOrb.pair[o][b];
                constexpr bool fl = kOrb.flip[o][b] != 0;
                const long long fp = get(ic<2 * p + 1>{}), fm = get(ic<2 * p + 2>{});
                S[b] = fp + fm;
                D[b] = fl ? fm - fp : fp - fm;
            });
            wht<np>(S);
            wht<np>(D);
            static_for<Mm>([&](auto G) {
                constexpr int g = decltype(G)::value;
                constexpr int m = kOrb.monomial(o, g);
                if constexpr (m != 0) {
                    constexpr int cl = kOrb.parity_class(o, g);
                    if constexpr ((mi_order(g) & 1) == 0)
                        acc[g].template madd<m>(S[cl]);
                    else
                        acc[g].template madd<m>(D[cl]);
                }
            });
        });
        static_for<Mm>([&](auto G) { R[decltype(G)::value] = acc[decltype(G)::value].value(); });
    }

    // a3: ta_alpha = a_alpha / alpha! = sum_gamma hdiv(alpha, gamma) c^|gamma| R_gamma.
    template <int Nm>
    SMRT_D static void absolute(const T (&f)[Q], T c, T (&ta)[nmom(Nm)]) {
        T Rc[nmom(Nm)];
        absolute<Nm>(f, c, ta, Rc);
    }
    // ... and the scaled raw moments Rc_gamma = c^|gamma| sum_i df_i e_i^gamma themselves
    template <int Nm>
    SMRT_D static void absolute(const T (&f)[Q], T c, T (&ta)[nmom(Nm)], T (&Rc)[nmom(Nm)]) {
        raw_moments<Nm>(f, Rc);
        scaled_to_absolute<Nm>(c, ta, Rc);
    }
    // Rc: raw moments in, scaled by c^|gamma| out; ta: the divided absolute coefficients
    template <int Nm, class U>
    SMRT_D static void scaled_to_absolute(U c, U (&ta)[nmom(Nm)], U (&Rc)[nmom(Nm)]) {
        constexpr int Mm = nmom(Nm);
        U cp[Nm + 1];
        cp[0] = U(1);
        static_for<Nm>([&](auto J) { cp[decltype(J)::value + 1] = cp[decltype(J)::value] * c; });
        static_for<Mm>([&](auto G) {
            constexpr int g = decltype(G)::value;
            if constexpr (mi_order(g) > 0) Rc[g] *= cp[mi_order(g)];
        });
        static_for<Mm>([&](auto A) {
            constexpr int al = decltype(A)::value;
            U acc = U(0);
            static_for<Mm>([&](auto G) {
                constexpr int g = decltype(G)::value;
                constexpr double h = hdiv(al, g);
                if constexpr (h != 0.0) acc = fma(U(h), Rc[g], acc);
            });
            ta[al] = acc;
        });
    }

    // a4: td_beta = d_beta / beta! = theta^(-|beta|/2) [T(-u, 2 - theta) ta]_beta
    template <int Nm>
    SMRT_D static void to_local(T (&v)[nmom(Nm)], const T (&u)[3], T theta, T thm1) {
        to_local_divided<Nm, T>(v, u, theta, thm1);
    }

    // a7 + a8 helper: values f'_i = w_i sum_gamma P_gamma e_i^gamma with
    // P_gamma = c^|gamma| sum_alpha hfull(alpha, gamma) ta'_alpha; U is the arithmetic type.
    // corr (optional): (base, B_0, B_1, B_2, C) added to the monomial coefficients P of orders
    // 0, 1 and the diagonal of 2, i.e. w_i (base + B.e_i + C |e_i|^2) added to every out_i.
    template <class U, class W>
    SMRT_D static void rebuild(const U (&ta)[M], U c, const W (&wp)[NP + 1], U (&out)[Q],
                               const U *corr = nullptr) {
        rebuild_emit(ta, c, wp, [&](int i, U v) { out[i] = v; }, corr);
    }
    // ... handing each value to put(i, value) as soon as it is formed
    template <class U, class W, class Put>
    SMRT_D static void rebuild_emit(const U (&ta)[M], U c, const W (&wp)[NP + 1], Put &&put,
                                    const U *corr = nullptr) {
        U cp[N + 1];
        cp[0] = U(1);
        static_for<N>([&](auto J) { cp[decltype(J)::value + 1] = cp[decltype(J)::value] * c; });
        U P[M];
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
        if (corr) {
            P[0] += corr[0];
            P[mi_pos(1, 0, 0)] += corr[1];
            P[mi_pos(0, 1, 0)] += corr[2];
            P[mi_pos(0, 0, 1)] += corr[3];
            P[mi_pos(2, 0, 0)] += corr[4];
            P[mi_pos(0, 2, 0)] += corr[4];
            P[mi_pos(0, 0, 2)] += corr[4];
        }
        put(0, U(wp[0]) * P[0]);
        // per sign orbit: sums of a^gamma P_gamma per parity class, their Walsh-Hadamard
        // transform (the even and odd parts of the polynomial at each member), then the pair
        static_for<kOrb.n>([&](auto O) {
            constexpr int o = decltype(O)::value;
            constexpr int np = 1 << (kOrb.k[o] - 1);
            U E[np], Od[np];
            static_for<np>([&](auto B) {
                E[decltype(B)::value] = U(0);
                Od[decltype(B)::value] = U(0);
            });
            static_for<M>([&](auto G) {
                constexpr int g = decltype(G)::value;
                constexpr int m = kOrb.monomial(o, g);
                if constexpr (m != 0) {
                    constexpr int cl = kOrb.parity_class(o, g);
                    if constexpr ((mi_order(g) & 1) == 0)
                        E[cl] = fma(U(m), P[g], E[cl]);
                    else
                        Od[cl] = fma(U(m), P[g], Od[cl]);
                }
            });
            wht<np>(E);
            wht<np>(Od);
            static_for<np>([&](auto B) {
                constexpr int b = decltype(B)::value, p = kOrb.pair[o][b];
                constexpr bool fl = kOrb.flip[o][b] != 0;
                const U w = U(wp[p + 1]);
                const U vplus = w * (E[b] + Od[b]), vminus = w * (E[b] - Od[b]);
                put(2 * p + 1, fl ? vminus : vplus);
                put(2 * p + 2, fl ? vplus : vminus);
            });
        });
    }

    // ta^eq_alpha = rho prod_k g_{alpha_k}(u_k, theta) / alpha_k!  (3D product of the
    // Appendix B closed form), minus the coefficients of f = w_i (1 in slot 0), in U.
    template <class U>
    SMRT_D static void equilibrium(U rho, U rhom1, const U (&u)[3], U thm1, U (&ta)[M]) {
        U G[3][N + 1];
        static_for<3>([&](auto K) {
            constexpr int k = decltype(K)::value;
            maxwell_divided<N, U>(G[k], u[k], thm1);
        });
        static_for<M>([&](auto A) {
            constexpr int p = decltype(A)::value;
            ta[p] = rho * G[0][mi_comp(p, 0)] * G[1][mi_comp(p, 1)] * G[2][mi_comp(p, 2)];
        });
        ta[0] = rhom1;
    }

    // a4-a6 on divided absolute coefficients v: to the local frame, relaxation of orders 2..N
    // with their own times, back to the absolute frame (truncated at N); the slot of order 0
    // leaves as o0 and those of order 1 as zero (u is the frame velocity).
    // model 1: the ES-BGK relaxation (Sec. 3, Eq. ES-BGK) with parameter es_b, at the rate of
    // the first time (tau_20); else SMRT.
    SMRT_D static void relax_coefficients(T (&v)[M], const T (&u)[3], T rho, T theta, T thm1, T o0,
                                          const T *tauA, const T *tauB, int model = 0, T es_b = T(0)) {
        to_local<N>(v, u, theta, thm1);
        // a5: relax orders 2..N; order 0 is rho, order 1 is zero by definition of u
        if (model == 1) {
            relax_es_divided<N, T>(v, rho, tauA[0], tauB[0], es_b);
        } else {
            T s[KT];
            static_for<KT>([&](auto K) {
                constexpr int k = decltype(K)::value;
                s[k] = T(1) - rcp_tau<T>(tauA[k], tauB[k], rho);
            });
            static_for<N - 1>([&](auto Nn) { relax_order<N, decltype(Nn)::value + 2, T>(v, s); });
        }
        // a6: back to the absolute frame: scale by theta^(|beta|/2), transform with T(u, theta)
        const T sq = theta * rsq(theta);
        T sp[N + 1];
        sp[0] = T(1);
        static_for<N>([&](auto J) { sp[decltype(J)::value + 1] = sp[decltype(J)::value] * sq; });
        static_for<M>([&](auto A) {
            constexpr int p = decltype(A)::value;
            if constexpr (mi_order(p) == 0)
                v[p] = o0;
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
    }

    // The whole collision: df (pre-collision deviations, library order) -> df (post-collision).
    // Returns false when rho or theta is not positive (or NaN).
    SMRT_D static bool collide(T (&f)[Q], const T (&wp)[NP + 1], const float (&wlo)[NP + 1], T c,
                               float clo, const T *tauA, const T *tauB, unsigned key = 0u, int model = 0,
                               T es_b = T(0)) {
        if constexpr (Split) {
            bool finite = true;
            const bool ok = collide_split(
                [&](auto I) {
                    finite &= (__float_as_uint(f[decltype(I)::value]) & 0x7f800000u) != 0x7f800000u;
                    return to_fixed(f[decltype(I)::value]);
                },
                [&](int i, T v) { f[i] = v; }, wp, wlo, c, clo, tauA, tauB, key, model, es_b);
            return ok && finite;
        } else {
            // a3: coefficients of the deviations; the full a has 1 more in slot 0, i.e. a_0 = rho
            T v[M], Rc[M];
            absolute<N>(f, c, v, Rc);
            // a2 from the raw moments already formed: rho - 1 = Rc_0, rho u = Rc_1,
            // E - 3 = tr Rc_2
            const T rhom1 = Rc[0];
            const T rho = T(1) + rhom1;
            const T ir = rcp(rho);
            const T u[3] = {Rc[mi_pos(1, 0, 0)] * ir, Rc[mi_pos(0, 1, 0)] * ir, Rc[mi_pos(0, 0, 1)] * ir};
            const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            const T em3 = Rc[mi_pos(2, 0, 0)] + Rc[mi_pos(0, 2, 0)] + Rc[mi_pos(0, 0, 2)];
            const T thm1 = (em3 - T(3) * rhom1 - rho * uu) * ir * T(1.0 / 3.0);
            const T theta = T(1) + thm1;
            const bool ok = (rho > T(0)) && (theta > T(0));
            v[0] = rho;
            relax_coefficients(v, u, rho, theta, thm1, rho, tauA, tauB, model, es_b);
            v[0] = rhom1;  // deviation from the coefficients of w_i
            T out[Q];
            rebuild<T>(v, c, wp, out);
            static_for<Q>([&](auto I) { f[decltype(I)::value] = out[decltype(I)::value]; });
            return ok;
        }
    }

    // Split precision (T float): pullq(ic<i>) gives pulled population i in fixed point (the stored
    // float exactly, or the exact double end-state value beyond a fixed end), read once;
    // store(i, value) receives post-collision population i as soon as it is formed.
    //
    // Precision design. Float arithmetic is used only for the non-equilibrium part, whose own
    // size then bounds its rounding errors; whatever the equilibrium carries is formed to about
    // 2^-44 of its size, so that an equilibrium state is reproduced with no float rounding that
    // would freeze (a steady bias in the stress or heat flux of an equilibrium far field shifts
    // its state through the flux balance and lets a shock drift):
    //  * raw moments R_gamma, |gamma| <= N, exactly in 64-bit fixed point;
    //  * in two-float arithmetic: rho, u, theta from them; the equilibrium's raw moments
    //    (Maxwellian moments, which the order-N equilibrium matches for |gamma| <= N); the
    //    non-equilibrium raw moments R - R^eq, then rounded to float;
    //  * in float: absolute coefficients of the non-equilibrium part and a4-a6 (to the local
    //    frame, relaxation, back);
    //  * in two-float: the order-N equilibrium's coefficients plus the relaxed non-equilibrium
    //    ones, their monomial coefficients Q_g (f'_i = w_i sum_g Q_g xi_i^g), and an exact
    //    restoration of mass, momentum and energy on them;
    //  * the polynomial at each population in fixed point (per sign orbit), times w_i in
    //    two-float, rounded to float stochastically.
    // Conservation: with the quadrature moments M_g = sum_i w_i xi_i^g (the unit Maxwellian's,
    // prod_k (g_k - 1)!! for even g, exact to the set's degree), the rebuilt populations carry
    // mass sum_g Q_g M_g, momentum sum_g Q_g M_(g+e_k) and energy sum_g Q_g sum_k M_(g+2e_k).
    // Whatever float rounding left in them is removed along w_i (A + B.xi_i + C (|xi_i|^2 - 3))
    // (sum w = 1, sum w xi xi = delta, sum w |xi|^4 = 15), i.e. added to Q_0, Q_k and Q_kk, so
    // that they equal the pre-collision sums. The stored values then conserve rho, rho u and
    // energy in expectation, stochastic rounding being the only remaining error.
    template <class Pull, class Store>
    SMRT_D static bool collide_split(Pull &&pullq, Store &&store, const T (&wp)[NP + 1],
                                     const float (&wlo)[NP + 1], T c, float clo, const T *tauA,
                                     const T *tauB, unsigned key, int model = 0, T es_b = T(0)) {
        static_assert(std::is_same<T, float>::value, "the split precision stores floats");
        constexpr int px = mi_pos(1, 0, 0), py = mi_pos(0, 1, 0), pz = mi_pos(0, 0, 1);
        constexpr int pxx = mi_pos(2, 0, 0), pyy = mi_pos(0, 2, 0), pzz = mi_pos(0, 0, 2);
        // a2 + a3: exact raw moments; rho, u, theta in two-float
        long long Rq[M];
        fixed_moments<N>(pullq, Rq);
        const ff cc = {c, clo};
        ff cp[N + 1];  // c^j
        cp[0] = ff{1.f, 0.f};
        static_for<N>([&](auto J) { cp[decltype(J)::value + 1] = cp[decltype(J)::value] * cc; });
        const ff r = fixed_to_ff(Rq[0]);  // rho - 1
        const ff rho = r + 1.f;
        const ff irho = ff_div(ff{1.f, 0.f}, rho);
        const ff mom[3] = {cc * fixed_to_ff(Rq[px]), cc * fixed_to_ff(Rq[py]), cc * fixed_to_ff(Rq[pz])};
        const ff uf[3] = {mom[0] * irho, mom[1] * irho, mom[2] * irho};
        const ff en = cp[2] * fixed_to_ff(Rq[pxx] + Rq[pyy] + Rq[pzz]);  // E - 3
        // theta - 1 = (E - 3 - 3 (rho - 1) - rho |u|^2) / (3 rho)
        const ff thm1 = (en - r * 3.f - (mom[0] * uf[0] + mom[1] * uf[1] + mom[2] * uf[2])) *
                        (ff_inv<3>() * irho);
        const ff theta = thm1 + 1.f;
        // non-equilibrium raw moments in xi-units, c^|g| R_g - (rho prod_k mu_{g_k}(u_k, theta)
        // - prod_k mu_{g_k}(0, 1)), mu_j the raw moments of a 1D Gaussian of mean u and variance
        // theta (mu_{j+1} = u mu_j + j theta mu_{j-1}); orders 0 and 1 vanish by definition of
        // rho and u
        T v[M];
        {
            ff mu[3][N + 1];
            static_for<3>([&](auto K) {
                constexpr int k = decltype(K)::value;
                mu[k][0] = ff{1.f, 0.f};
                mu[k][1] = uf[k];
                static_for<N - 1>([&](auto J) {
                    constexpr int j = decltype(J)::value + 1;
                    mu[k][j + 1] = uf[k] * mu[k][j] + theta * mu[k][j - 1] * float(j);
                });
            });
            T Rx[M];
            static_for<M>([&](auto G) {
                constexpr int g = decltype(G)::value;
                if constexpr (mi_order(g) <= 1) {
                    Rx[g] = T(0);
                } else {
                    constexpr int g0 = mi_comp(g, 0), g1 = mi_comp(g, 1), g2 = mi_comp(g, 2);
                    ff eq = rho;
                    if constexpr (g0 > 0) eq = eq * mu[0][g0];
                    if constexpr (g1 > 0) eq = eq * mu[1][g1];
                    if constexpr (g2 > 0) eq = eq * mu[2][g2];
                    Rx[g] = (fixed_to_ff(Rq[g]) * cp[mi_order(g)] - (eq + float(-unit_moment(g)))).hi;
                }
            });
            // a3 on the non-equilibrium part: divided absolute coefficients (float)
            static_for<M>([&](auto A) {
                constexpr int al = decltype(A)::value;
                T acc = T(0);
                static_for<M>([&](auto G) {
                    constexpr int g = decltype(G)::value;
                    constexpr double h = hdiv(al, g);
                    if constexpr (h != 0.0 && mi_order(g) >= 2) acc = fma(T(h), Rx[g], acc);
                });
                v[al] = acc;
            });
        }
        const T rhof = rho.hi, thm1f = thm1.hi, thetaf = theta.hi;
        const T u[3] = {uf[0].hi, uf[1].hi, uf[2].hi};
        const bool ok = (rhof > T(0)) && (thetaf > T(0));
        // a4-a6 on the non-equilibrium part; orders 0 and 1 leave as zero
        relax_coefficients(v, u, rhof, thetaf, thm1f, T(0), tauA, tauB, model, es_b);
        // the post-collision coefficients: order-N equilibrium ta^eq_alpha = rho prod_k
        // G_k[alpha_k] (slot 0: rho - 1; G_k[j+1] = (u_k G_k[j] + (theta - 1) G_k[j-1]) / (j + 1))
        // plus the relaxed non-equilibrium part, then the monomial coefficients in xi,
        // Q_g = sum_alpha hfull(alpha, g) ta_alpha (integers hfull)
        ff Qx[M];
        {
            ff G[3][N + 1];
            static_for<3>([&](auto K) {
                constexpr int k = decltype(K)::value;
                G[k][0] = ff{1.f, 0.f};
                G[k][1] = uf[k];
                static_for<N - 1>([&](auto J) {
                    constexpr int j = decltype(J)::value + 1;
                    G[k][j + 1] = (uf[k] * G[k][j] + thm1 * G[k][j - 1]) * ff_inv<j + 1>();
                });
            });
            ff ta[M];
            static_for<M>([&](auto A) {
                constexpr int al = decltype(A)::value;
                constexpr int a0 = mi_comp(al, 0), a1 = mi_comp(al, 1), a2 = mi_comp(al, 2);
                if constexpr (al == 0) {
                    ta[al] = r;
                } else {
                    ff t = rho;
                    if constexpr (a0 > 0) t = t * G[0][a0];
                    if constexpr (a1 > 0) t = t * G[1][a1];
                    if constexpr (a2 > 0) t = t * G[2][a2];
                    ta[al] = mi_order(al) >= 2 ? t + v[al] : t;
                }
            });
            static_for<M>([&](auto G_) {
                constexpr int g = decltype(G_)::value;
                ff acc = ff{0.f, 0.f};
                static_for<M>([&](auto A) {
                    constexpr int al = decltype(A)::value;
                    constexpr double h = hfull(al, g);
                    if constexpr (h == 1.0)
                        acc = acc + ta[al];
                    else if constexpr (h != 0.0)
                        acc = acc + ta[al] * float(h);
                });
                Qx[g] = acc;
            });
        }
        // exact restoration of mass, momentum and energy (targets: rho - 1, rho u, E - 3)
        {
            ff ms = ff{0.f, 0.f}, es = ff{0.f, 0.f}, js[3] = {ff{0.f, 0.f}, ff{0.f, 0.f}, ff{0.f, 0.f}};
            static_for<M>([&](auto G_) {
                constexpr int g = decltype(G_)::value;
                constexpr int g0 = mi_comp(g, 0), g1 = mi_comp(g, 1), g2 = mi_comp(g, 2);
                constexpr double m0 = unit_moment(g);
                constexpr double e0 = unit_moment3(g0 + 2, g1, g2) + unit_moment3(g0, g1 + 2, g2) +
                                      unit_moment3(g0, g1, g2 + 2);
                if constexpr (m0 != 0.0) ms = ms + (m0 == 1.0 ? Qx[g] : Qx[g] * float(m0));
                if constexpr (e0 != 0.0) es = es + Qx[g] * float(e0);
                static_for<3>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    constexpr double j0 = unit_moment3(g0 + (k == 0), g1 + (k == 1), g2 + (k == 2));
                    if constexpr (j0 != 0.0) js[k] = js[k] + (j0 == 1.0 ? Qx[g] : Qx[g] * float(j0));
                });
            });
            const ff A = r - ms;
            const ff Cc = (en - es - A * 3.f) * ff_inv<6>();
            Qx[0] = Qx[0] + (A - Cc * 3.f);
            Qx[px] = Qx[px] + (mom[0] - js[0]);
            Qx[py] = Qx[py] + (mom[1] - js[1]);
            Qx[pz] = Qx[pz] + (mom[2] - js[2]);
            Qx[pxx] = Qx[pxx] + Cc;
            Qx[pyy] = Qx[pyy] + Cc;
            Qx[pzz] = Qx[pzz] + Cc;
        }
        // monomial coefficients in e (xi = c e), in fixed point
        long long Pq[M];
        static_for<M>([&](auto G_) {
            constexpr int g = decltype(G_)::value;
            const ff P = mi_order(g) > 0 ? Qx[g] * cp[mi_order(g)] : Qx[g];
            Pq[g] = to_fixed<kFixP>(P.hi) + to_fixed<kFixP>(P.lo);
        });
        // a7 + a8: f'_i = w_i P(e_i), P(e_i) per sign orbit in fixed point (sums per parity
        // class, Walsh-Hadamard transform), then times w_i in two-float, rounded stochastically
        auto out = [&](int i, int wi, long long poly) {
            const ff w = {wp[wi], wlo[wi]};
            store(i, round_stochastic(w * fixed_to_ff<kFixP>(poly), key ^ (0x9e3779b9u * unsigned(i + 1))));
        };
        out(0, 0, Pq[0]);
        static_for<kOrb.n>([&](auto O) {
            constexpr int o = decltype(O)::value;
            constexpr int np = 1 << (kOrb.k[o] - 1);
            SplitAcc Ea[np], Oa[np];
            static_for<M>([&](auto G_) {
                constexpr int g = decltype(G_)::value;
                constexpr int m = kOrb.monomial(o, g);
                if constexpr (m != 0) {
                    constexpr int cl = kOrb.parity_class(o, g);
                    if constexpr ((mi_order(g) & 1) == 0)
                        Ea[cl].template madd<m>(Pq[g]);
                    else
                        Oa[cl].template madd<m>(Pq[g]);
                }
            });
            long long E[np], Od[np];
            static_for<np>([&](auto B) {
                E[decltype(B)::value] = Ea[decltype(B)::value].value();
                Od[decltype(B)::value] = Oa[decltype(B)::value].value();
            });
            wht<np>(E);
            wht<np>(Od);
            static_for<np>([&](auto B) {
                constexpr int b = decltype(B)::value, p = kOrb.pair[o][b];
                constexpr bool fl = kOrb.flip[o][b] != 0;
                out(fl ? 2 * p + 2 : 2 * p + 1, p + 1, E[b] + Od[b]);
                out(fl ? 2 * p + 1 : 2 * p + 2, p + 1, E[b] - Od[b]);
            });
        });
        return ok;
    }
};

// ------------------------------------------------------------------------------ async copies (sm_90+)
SMRT_D unsigned smem_addr(const void *p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }

SMRT_D void mbar_init(unsigned long long *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
SMRT_D void mbar_arrive_expect_tx(unsigned long long *b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes)
                 : "memory");
}
// One contiguous global -> shared copy by the bulk-copy engine; its bytes count against the
// transaction count of mbarrier b. Addresses and size must be multiples of 16 bytes.
SMRT_D void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(b))
                 : "memory");
}
// One box of a 2D tensor map (coordinates: element within the plane, plane) -> shared memory,
// bytes counted against mbarrier b. The x coordinate must be a multiple of 16 bytes; the
// destination is 128-byte aligned. Elements outside the tensor read as zero.
SMRT_D void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1, unsigned long long *b) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(smem_addr(b))
        : "memory");
}
// Order this thread's earlier generic-proxy accesses of shared (global) memory before its
// later async-proxy ones: a buffer read or written by the threads, then refilled by the copy
// engine; data written by other blocks, then copied.
SMRT_D void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
SMRT_D void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
// Make mbarrier initialisations visible to the async proxy (the copy engine).
SMRT_D void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
SMRT_D unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait until the phase of parity `parity` of mbarrier b has completed. Gives up after about a
// second (or 2^26 polls) and returns false.
SMRT_D bool mbar_wait(unsigned long long *b, unsigned parity) {
    const unsigned addr = smem_addr(b);
    const unsigned long long t0 = global_ns();
    for (unsigned spin = 0; spin < (1u << 26); ++spin) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if ((spin & 63u) == 63u && global_ns() - t0 > 1000000000ull) return false;
    }
    return false;
}

// ------------------------------------------------------------------------------ loaders
// Blocks of 128 threads per SM that the step kernels leave room for (0: no minimum, the
// compiler's own register choice). The split-precision collision would take all 255 registers
// at two blocks per SM; capped at 168 (three blocks) it spills a few hundred bytes to L1 and runs
// the batched D3Q103 shocks 1.4x faster (0.60 -> 0.44 ms per step; 128 registers gives the
// same). An explicit minimum of 1 would instead let the float box kernel grow from 64 to 128
// registers and halve its occupancy.
template <bool Split>
constexpr int kStepMinBlocks = Split ? 3 : 0;

SMRT_HD int wrap(int t, int n) { return t < 0 ? t + n : (t >= n ? t - n : t); }

// Periodic 3D box: one thread per cell, block covers a run of x, grid (x-blocks, ny, nz).
template <class Lat, int N, class T, class Acc, bool Split>
__global__ void __launch_bounds__(128, kStepMinBlocks<Split>) step_box_kernel(StepArgs<Lat, T> a) {
    using C = Collide<Lat, N, T, Acc, Split>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= a.nx) return;
    const long long row = (long long)a.nx;
    const long long slab = row * a.ny;
    T f[Lat::Q];
    f[0] = a.fin[a.plane[0] + wrap(z - a.kz, a.nz) * slab + wrap(y - a.ky, a.ny) * row + wrap(x - a.kx, a.nx)];
    static_for<Lat::NP>([&](auto P) {
        constexpr int p = decltype(P)::value;
        static_for<2>([&](auto Sg) {
            constexpr int sg = decltype(Sg)::value == 0 ? 1 : -1;
            constexpr int i = 2 * p + 1 + decltype(Sg)::value;
            const int xs = wrap(x - (sg * Lat::e(p, 0) + a.kx), a.nx);
            const int ys = wrap(y - (sg * Lat::e(p, 1) + a.ky), a.ny);
            const int zs = wrap(z - (sg * Lat::e(p, 2) + a.kz), a.nz);
            f[i] = a.fin[a.plane[i] + zs * slab + ys * row + xs];
        });
    });
    const bool ok = C::collide(f, a.wp, a.wlo, a.c, a.clo, tau_a<T>(a.inst[0]), tau_b<T>(a.inst[0]),
                               mix32(unsigned(z * slab + y * row + x) ^ mix32(a.step)), a.inst[0].model,
                               T(a.inst[0].es_b));
    if (!ok) atomicOr(a.health, 1u);
    const long long cell = z * slab + y * row + x;
    static_for<Lat::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        a.fout[a.plane[i] + cell] = f[i];
    });
}

// Batched 1D lines (ny = nz = 1): block b handles cells x0 .. x0+blockDim-1 of instance j,
// (j, x0) = tiles[b]. FixedX: pulls from beyond either end read the end-state populations.
// Coherent: read the previous state through L2 only (__ldcg). Inside a persistent launch a
// buffer is rewritten between two reads by the same SM, and L1 is not kept coherent.
template <bool Coherent, class T>
SMRT_D T load_pop(const T *p) {
    if constexpr (Coherent)
        return __ldcg(p);
    else
        return *p;
}

template <class Lat, int N, class T, class Acc, bool Split, bool FixedX, bool Coherent = false>
SMRT_D void line_tile(const StepArgs<Lat, T> &a, const T *__restrict__ fin, T *__restrict__ fout,
                      int tile_index, unsigned step) {
    using C = Collide<Lat, N, T, Acc, Split>;
    const int2 tile = a.tiles[tile_index];
    const InstanceInfo &in = a.inst[tile.x];
    const int x = tile.y + threadIdx.x;
    const int L = in.nx;
    if (x >= L) return;
    const long long base = in.cell_off;
    const T *gl = a.ghosts + (long long)tile.x * 2 * Lat::Q;
    const T *gr = gl + Lat::Q;
    const double *gld = a.ghostsd + (long long)tile.x * 2 * Lat::Q;
    const double *grd = gld + Lat::Q;
    // pull of population i from cell xs of the instance: the stored state inside, the end
    // states beyond a fixed end
    auto pull = [&](int i, int xs) -> T {
        if constexpr (FixedX) {
            if (xs < 0) return gl[i];
            if (xs >= L) return gr[i];
            return load_pop<Coherent>(fin + a.plane[i] + base + xs);
        } else {
            return load_pop<Coherent>(fin + a.plane[i] + base + wrap(xs, L));
        }
    };
    // ... for the split precision, in fixed point (the exact double end state beyond a fixed
    // end); a non-finite stored value is recorded
    bool finite = true;
    auto pull_split = [&](int i, int xs) -> long long {
        if constexpr (FixedX) {
            if (xs < 0) return to_fixed(gld[i]);
            if (xs >= L) return to_fixed(grd[i]);
        }
        const float v = float(pull(i, xs));
        finite &= (__float_as_uint(v) & 0x7f800000u) != 0x7f800000u;
        return to_fixed(v);
    };
    // x-distance of population i's pull: the rest population streams by k as well
    auto src_x = [&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int ex = i == 0 ? 0 : ((i & 1) ? Lat::e((i - 1) / 2, 0) : -Lat::e((i - 1) / 2, 0));
        return x - (ex + in.kx);
    };
    bool ok;
    if constexpr (Split) {
        ok = C::collide_split([&](auto I) { return pull_split(decltype(I)::value, src_x(I)); },
                              [&](int i, T v) { fout[a.plane[i] + base + x] = v; }, a.wp, a.wlo, a.c,
                              a.clo, tau_a<T>(in), tau_b<T>(in), mix32(unsigned(base + x) ^ mix32(step)),
                              in.model, T(in.es_b));
        ok = ok && finite;
    } else {
        T f[Lat::Q];
        static_for<Lat::Q>([&](auto I) { f[decltype(I)::value] = pull(decltype(I)::value, src_x(I)); });
        ok = C::collide(f, a.wp, a.wlo, a.c, a.clo, tau_a<T>(in), tau_b<T>(in),
                        mix32(unsigned(base + x) ^ mix32(step)), in.model, T(in.es_b));
        static_for<Lat::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            fout[a.plane[i] + base + x] = f[i];
        });
    }
    if (!ok) atomicOr(a.health, 1u);
}

template <class Lat, int N, class T, class Acc, bool Split, bool FixedX>
__global__ void __launch_bounds__(128, kStepMinBlocks<Split>) step_line_kernel(StepArgs<Lat, T> a) {
    line_tile<Lat, N, T, Acc, Split, FixedX>(a, a.fin, a.fout, blockIdx.x, a.step);
}

// Grid-wide barrier of a cooperative launch (all blocks resident). bar[0] counts arrivals,
// bar[1] is the generation. The spin gives up after about a second: it then records
// LB_HEALTH_TIMEOUT and returns false, and the caller leaves the kernel.
SMRT_D bool grid_barrier(unsigned *bar, unsigned &gen, unsigned *health) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        __threadfence();
        const unsigned target = gen + 1u;
        if (atomicAdd(&bar[0], 1u) + 1u == gridDim.x) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            atomicExch(&bar[1], target);
        } else {
            unsigned spins = 0;
            while (atomicAdd(&bar[1], 0u) != target) {
                if (++spins > (1u << 22)) {  // ~1 s at 256 ns per spin
                    atomicOr(health, 2u);
                    ok = 0;
                    break;
                }
                __nanosleep(256);
            }
        }
        __threadfence();
        gen = target;
    }
    __syncthreads();
    return ok != 0;
}

// Persistent batched step: one cooperative launch runs nsteps steps of every tile of a batch
// of 1D lines, tiles distributed over the blocks (grid-stride), a grid barrier between steps.
// bar[2] holds the running step counter (seeds the stochastic rounding across launches).
template <class Lat, int N, class T, class Acc, bool Split, bool FixedX>
__global__ void __launch_bounds__(128, kStepMinBlocks<Split>) step_line_persistent(StepArgs<Lat, T> a, int nsteps, int ntiles,
                                                            unsigned *bar) {
    unsigned gen = 0;
    if (threadIdx.x == 0) gen = atomicAdd(&bar[1], 0u);
    const unsigned step0 = __ldcg(&bar[2]);
    const T *src = a.fin;
    T *dst = a.fout;
    for (int s = 0; s < nsteps; ++s) {
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x)
            line_tile<Lat, N, T, Acc, Split, FixedX, true>(a, src, dst, t, step0 + unsigned(s));
        if (s + 1 < nsteps) {
            if (!grid_barrier(bar, gen, a.health)) return;
            // next step reads what this one wrote; swap buffers (f_a -> f_b -> f_a ...)
            const T *nsrc = dst;
            dst = (dst == a.fout) ? const_cast<T *>(a.fin) : a.fout;
            src = nsrc;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) bar[2] = step0 + unsigned(nsteps);
}

// ------------------------------------------------------------------------------ staged lines
// Split-precision batched lines with the pulls staged in shared memory. Each warp owns 32
// consecutive cells of a tile; every pull of those cells from the previous state lies in the
// x-segment [base + x0 - k - E, base + x0 + 31 - k + E] of each population plane (E the largest
// |e_x|), so one box of a 2D tensor map of the state ([Q planes][stride cells], library plane
// order), rounded out to 16 bytes, brings all Q rows in by one copy, completion counted in
// bytes on the warp's mbarrier. The lanes then read their pulls from shared memory instead of
// issuing Q dependent loads each. Pulls from beyond a fixed end read the end states (in
// double, exactly) and wrapped pulls of a periodic line read the state directly.
template <class Lat>
struct LineStage {
    static constexpr int kEmax = [] {
        int m = 0;
        for (int p = 0; p < Lat::NP; ++p) m = Lat::e(p, 0) > m ? Lat::e(p, 0) : (-Lat::e(p, 0) > m ? -Lat::e(p, 0) : m);
        return m;
    }();
    static constexpr int kSeg = (32 + 2 * kEmax + 3 + 3) / 4 * 4;  // elements per staged row
    static constexpr size_t kRows = size_t(kSeg) * Lat::Q * sizeof(float);
    static constexpr size_t kWarpBytes = 128 + (kRows + 127) / 128 * 128;  // mbarrier, then rows
    SMRT_HD static size_t bytes(int threads) { return size_t(threads / 32) * kWarpBytes; }
    // the persistent kernel keeps a block-wide failure flag after the warps' areas
    SMRT_HD static size_t persistent_bytes(int threads) { return bytes(threads) + 16; }
};

// One warp's 32 cells of tile tile_index. All lanes call it. Returns false (LB_HEALTH_TIMEOUT
// recorded) when the copy did not land within the bounded wait.
template <class Lat, int N, class Acc, bool FixedX, bool Coherent>
SMRT_D bool line_warp_staged(const StepArgs<Lat, float> &a, const float *__restrict__ fin, float *__restrict__ fout,
                             int tile_index, unsigned step, unsigned long long *bar, float *buf, unsigned &parity,
                             const CUtensorMap *tm) {
    using C = Collide<Lat, N, float, Acc, true>;
    using S = LineStage<Lat>;
    const int lane = threadIdx.x & 31;
    const int2 tile = a.tiles[tile_index];
    const InstanceInfo &in = a.inst[tile.x];
    const int xw = tile.y + int(threadIdx.x & ~31u);  // the warp's first cell
    const int L = in.nx;
    if (xw >= L) return true;  // the whole warp lies beyond the line's end
    const long long base = in.cell_off;
    const long long g_al = (base + xw - in.kx - S::kEmax) & ~3ll;  // first staged element, 16-byte aligned
    // the previous tile's reads of buf (generic proxy) and, in a persistent launch, other
    // blocks' writes of the state come before the copy engine's accesses
    __syncwarp();
    if (lane == 0) {
        if constexpr (Coherent) fence_async_global();
        fence_async_shared();
        mbar_arrive_expect_tx(bar, unsigned(S::kRows));
        tma_load_2d(buf, tm, int(g_al), 0, bar);
    }
    const bool landed = __all_sync(0xffffffffu, mbar_wait(bar, parity));
    if (!landed) {
        if (lane == 0) atomicOr(a.health, 2u);
        mbar_wait(bar, parity);  // let the copy in flight land before leaving (bounded)
        return false;
    }
    parity ^= 1u;
    const int x = xw + lane;
    if (x >= L) return true;
    const double *gld = a.ghostsd + (long long)tile.x * 2 * Lat::Q;
    const double *grd = gld + Lat::Q;
    const int tb = int(base + x - in.kx - g_al);  // staged offset of this lane's pull with e_x = 0
    bool finite = true;
    auto pullq = [&](auto I) -> long long {
        constexpr int i = decltype(I)::value;
        constexpr int ex = i == 0 ? 0 : ((i & 1) ? Lat::e((i - 1) / 2, 0) : -Lat::e((i - 1) / 2, 0));
        const int xs = x - ex - in.kx;
        float v;
        if (xs < 0 || xs >= L) {
            if constexpr (FixedX) return to_fixed(xs < 0 ? gld[i] : grd[i]);
            v = load_pop<Coherent>(fin + a.plane[i] + base + wrap(xs, L));
        } else {
            v = buf[i * S::kSeg + tb - ex];
        }
        finite &= (__float_as_uint(v) & 0x7f800000u) != 0x7f800000u;
        return to_fixed(v);
    };
    const bool ok = C::collide_split(pullq, [&](int i, float v) { fout[a.plane[i] + base + x] = v; }, a.wp, a.wlo,
                                     a.c, a.clo, tau_a<float>(in), tau_b<float>(in),
                                     mix32(unsigned(base + x) ^ mix32(step)), in.model, float(in.es_b));
    if (!(ok && finite)) atomicOr(a.health, 1u);
    return true;
}

// Warp w of a block takes the warp part w of tile blockIdx.x (tile width = block size).
template <class Lat, int N, class Acc, bool FixedX>
__global__ void __launch_bounds__(128, kStepMinBlocks<true>) step_line_staged(StepArgs<Lat, float> a,
                                                                               const __grid_constant__ CUtensorMap map) {
    extern __shared__ __align__(128) unsigned char dyn[];
    unsigned char *w = dyn + size_t(threadIdx.x >> 5) * LineStage<Lat>::kWarpBytes;
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(w);
    float *buf = reinterpret_cast<float *>(w + 128);
    if ((threadIdx.x & 31) == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    unsigned parity = 0u;
    line_warp_staged<Lat, N, Acc, FixedX, false>(a, a.fin, a.fout, blockIdx.x, a.step, bar, buf, parity, &map);
}

// All nsteps steps in one cooperative launch (as step_line_persistent), the pulls staged.
template <class Lat, int N, class Acc, bool FixedX>
__global__ void __launch_bounds__(128, kStepMinBlocks<true>) step_line_persistent_staged(
    StepArgs<Lat, float> a, int nsteps, int ntiles, unsigned *barg, const __grid_constant__ CUtensorMap map_a,
    const __grid_constant__ CUtensorMap map_b) {
    extern __shared__ __align__(128) unsigned char dyn[];
    int &failed = *reinterpret_cast<int *>(dyn + LineStage<Lat>::bytes(blockDim.x));
    unsigned char *w = dyn + size_t(threadIdx.x >> 5) * LineStage<Lat>::kWarpBytes;
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(w);
    float *buf = reinterpret_cast<float *>(w + 128);
    if ((threadIdx.x & 31) == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    if (threadIdx.x == 0) failed = 0;
    __syncthreads();
    unsigned parity = 0u;
    unsigned gen = 0;
    if (threadIdx.x == 0) gen = atomicAdd(&barg[1], 0u);
    const unsigned step0 = __ldcg(&barg[2]);
    const float *src = a.fin;
    float *dst = a.fout;
    for (int s = 0; s < nsteps; ++s) {
        const CUtensorMap *tm = src == a.fin ? &map_a : &map_b;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x)
            if (!line_warp_staged<Lat, N, Acc, FixedX, true>(a, src, dst, t, step0 + unsigned(s), bar, buf, parity, tm)) {
                failed = 1;  // the warp stops (its lanes agree); the block leaves after this step
                break;
            }
        __syncthreads();
        if (failed) return;
        if (s + 1 < nsteps) {
            if (!grid_barrier(barg, gen, a.health)) return;
            const float *nsrc = dst;
            dst = (dst == a.fout) ? const_cast<float *>(a.fin) : a.fout;
            src = nsrc;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) barg[2] = step0 + unsigned(nsteps);
}

// ------------------------------------------------------------------------------ moments
// The rows of lb_moments selected by mask, for one cell: rho, the physical velocity up,
// theta, and the local-frame coefficients in divided form v (td_beta = d_beta / beta!,
// |beta| <= Nm) of the pulled (pre-collision) populations.
template <int Nm, class T>
SMRT_D void store_moments(double *o, long long nc, long long cell, unsigned mask, double rho,
                          const double (&up)[3], double thd, const T (&v)[nmom(Nm)]) {
    constexpr int Mm = nmom(Nm);
    // undivide: d_beta = beta! td_beta
    double d[Mm];
    static_for<Mm>([&](auto A) {
        constexpr int p = decltype(A)::value;
        d[p] = double(v[p]) * mi_fact(p);
    });
    d[0] = rho;
    long long r = 0;
    if (mask & 0x1u) o[(r++) * nc + cell] = rho;
    if (mask & 0x2u) {
        o[(r++) * nc + cell] = up[0];
        o[(r++) * nc + cell] = up[1];
        o[(r++) * nc + cell] = up[2];
    }
    if (mask & 0x4u) o[(r++) * nc + cell] = thd;
    if (mask & 0x8u) {
        o[(r++) * nc + cell] = thd * d[mi_pos(2, 0, 0)];
        o[(r++) * nc + cell] = thd * d[mi_pos(0, 2, 0)];
        o[(r++) * nc + cell] = thd * d[mi_pos(0, 0, 2)];
        o[(r++) * nc + cell] = thd * d[mi_pos(1, 1, 0)];
        o[(r++) * nc + cell] = thd * d[mi_pos(1, 0, 1)];
        o[(r++) * nc + cell] = thd * d[mi_pos(0, 1, 1)];
    }
    if (mask & 0x10u) {
        const double s = 0.5 * thd * sqrt(thd);
        o[(r++) * nc + cell] = s * (d[mi_pos(3, 0, 0)] + d[mi_pos(1, 2, 0)] + d[mi_pos(1, 0, 2)]);
        o[(r++) * nc + cell] = s * (d[mi_pos(2, 1, 0)] + d[mi_pos(0, 3, 0)] + d[mi_pos(0, 1, 2)]);
        o[(r++) * nc + cell] = s * (d[mi_pos(2, 0, 1)] + d[mi_pos(0, 2, 1)] + d[mi_pos(0, 0, 3)]);
    }
    if (mask & 0x20u) {
        static_for<Mm>([&](auto A) {
            constexpr int p = decltype(A)::value;
            o[(r + p) * nc + cell] = d[p];
        });
    }
}

// Moments of the pulled (pre-collision) populations; see lb_moments in smrt.h.
template <class Lat, int N, class T, class Acc>
struct MomentArgs {
    StepArgs<Lat, T> s;
    double *out;
    long long ncells;
    unsigned mask;
    int line;    // 1: batched-line geometry (tiles), 0: box
    int fixedx;
};

template <class Lat, int N, class T, class Acc>
__global__ void __launch_bounds__(128) moments_kernel(MomentArgs<Lat, N, T, Acc> m) {
    constexpr int Nm = N < 3 ? 3 : N;
    constexpr int Mm = nmom(Nm);
    using C = Collide<Lat, N, T, Acc, false>;
    using Cm = Collide<Lat, Nm, T, Acc, false>;
    const StepArgs<Lat, T> &a = m.s;
    T f[Lat::Q];
    long long cell;
    double ubar_x;
    if (m.line) {
        const int2 tile = a.tiles[blockIdx.x];
        const InstanceInfo &in = a.inst[tile.x];
        const int x = tile.y + threadIdx.x;
        const int L = in.nx;
        if (x >= L) return;
        cell = in.cell_off + x;
        ubar_x = a.cd * in.kx;
        const T *gl = a.ghosts + (long long)tile.x * 2 * Lat::Q;
        const T *gr = gl + Lat::Q;
        {
            const int xs = x - in.kx;
            if (m.fixedx && xs < 0)
                f[0] = gl[0];
            else if (m.fixedx && xs >= L)
                f[0] = gr[0];
            else
                f[0] = a.fin[a.plane[0] + in.cell_off + wrap(xs, L)];
        }
        static_for<Lat::NP>([&](auto P) {
            constexpr int p = decltype(P)::value;
            static_for<2>([&](auto Sg) {
                constexpr int sg = decltype(Sg)::value == 0 ? 1 : -1;
                constexpr int i = 2 * p + 1 + decltype(Sg)::value;
                const int xs = x - (sg * Lat::e(p, 0) + in.kx);
                if (m.fixedx && xs < 0)
                    f[i] = gl[i];
                else if (m.fixedx && xs >= L)
                    f[i] = gr[i];
                else
                    f[i] = a.fin[a.plane[i] + in.cell_off + wrap(xs, L)];
            });
        });
    } else {
        const int x = blockIdx.x * blockDim.x + threadIdx.x;
        const int y = blockIdx.y, z = blockIdx.z;
        if (x >= a.nx) return;
        const long long row = a.nx, slab = row * a.ny;
        cell = z * slab + y * row + x;
        ubar_x = a.cd * a.kx;
        f[0] = a.fin[a.plane[0] + wrap(z - a.kz, a.nz) * slab + wrap(y - a.ky, a.ny) * row + wrap(x - a.kx, a.nx)];
        static_for<Lat::NP>([&](auto P) {
            constexpr int p = decltype(P)::value;
            static_for<2>([&](auto Sg) {
                constexpr int sg = decltype(Sg)::value == 0 ? 1 : -1;
                constexpr int i = 2 * p + 1 + decltype(Sg)::value;
                const int xs = wrap(x - (sg * Lat::e(p, 0) + a.kx), a.nx);
                const int ys = wrap(y - (sg * Lat::e(p, 1) + a.ky), a.ny);
                const int zs = wrap(z - (sg * Lat::e(p, 2) + a.kz), a.nz);
                f[i] = a.fin[a.plane[i] + zs * slab + ys * row + xs];
            });
        });
    }
    Acc rho, rhom1, u[3], th, thm1;
    C::conserved(f, Acc(a.cd), rho, rhom1, u, th, thm1);
    T v[Mm];
    Cm::template absolute<Nm>(f, a.c, v);
    v[0] = T(rho);
    const T ut[3] = {T(u[0]), T(u[1]), T(u[2])};
    Cm::template to_local<Nm>(v, ut, T(th), T(thm1));
    const double up[3] = {double(u[0]) + ubar_x, double(u[1]) + a.cd * a.ky, double(u[2]) + a.cd * a.kz};
    store_moments<Nm, T>(m.out, m.ncells, cell, m.mask, double(rho), up, double(th), v);
}

// ------------------------------------------------------------------------------ equilibrium
// df = order-N equilibrium of (rho, u_phys - u_bar, theta) minus w_i, in double, stored as T.
template <class Lat, int N, class T>
SMRT_D void equilibrium_cell(double rho, const double (&u)[3], double theta, double c,
                             const double (&wp)[Lat::NP + 1], double (&out)[Lat::Q]) {
    using C = Collide<Lat, N, T, double, false>;
    double ta[nmom(N)];
    C::template equilibrium<double>(rho, rho - 1.0, u, theta - 1.0, ta);
    C::template rebuild<double>(ta, c, wp, out);
}

template <class Lat, int N, class T>
__global__ void __launch_bounds__(128) fill_kernel(StepArgs<Lat, T> a, const double *rho,
                                                   const double *u, const double *theta,
                                                   long long ncells, int line) {
    long long cell;
    int kx;
    if (line) {
        const int2 tile = a.tiles[blockIdx.x];
        const InstanceInfo &in = a.inst[tile.x];
        const int x = tile.y + threadIdx.x;
        if (x >= in.nx) return;
        cell = in.cell_off + x;
        kx = in.kx;
    } else {
        cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        if (cell >= ncells) return;
        kx = a.kx;
    }
    const double uu[3] = {u[cell] - a.cd * kx, u[ncells + cell] - a.cd * a.ky,
                          u[2 * ncells + cell] - a.cd * a.kz};
    double out[Lat::Q];
    equilibrium_cell<Lat, N, T>(rho[cell], uu, theta[cell], a.cd, a.wpd, out);
    static_for<Lat::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        a.fout[a.plane[i] + cell] = T(out[i]);
    });
}

// End-state populations of instance j: states[j] = (rho, u_phys, theta) left then right.
template <class Lat, int N, class T>
__global__ void ghost_kernel(StepArgs<Lat, T> a, const double *states, int ninst, T *ghosts,
                             double *ghostsd) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * ninst) return;
    const int j = t / 2;
    const double *s = states + 5 * t;
    const double ub = a.cd * a.inst[j].kx;
    const double uu[3] = {s[1] - ub, s[2] - a.cd * a.ky, s[3] - a.cd * a.kz};
    double out[Lat::Q];
    equilibrium_cell<Lat, N, T>(s[0], uu, s[4], a.cd, a.wpd, out);
    static_for<Lat::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        ghosts[(long long)t * Lat::Q + i] = T(out[i]);
        ghostsd[(long long)t * Lat::Q + i] = out[i];
    });
}

}  // namespace smrt
