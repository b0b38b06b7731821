// lattice.cu -- host-side velocity-set support for libsmrt:
//   * solve the scale c and shell weights of the library's cubic velocity sets from the
//     even-moment conditions of a degree-Q Gauss-Hermite rule (Sec. 3, Eq. an: the rule must
//     integrate every polynomial of degree <= Q against the unit Gaussian exactly);
//   * check any caller-supplied set by brute force against the Gaussian moments;
//   * the Rankine-Hugoniot end states of a normal shock (Sec. 4.2, Eq. rankine).
//
// Solver. Every member of a cubic orbit ("shell") carries the shell's weight, so odd moments
// vanish and each even pattern xi_x^a xi_y^b xi_z^c (a >= b >= c, all even) gives one
// condition that is linear in the weights for fixed c. With S shells there are S + 1 patterns
// up to degree Q - 1 (Q odd). For fixed c the first S patterns (by ascending degree) fix the
// weights through an S x S linear solve; the last pattern's residual r(c) is then a scalar
// function of c whose root is found by bracketing and bisection.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/smrt.h"
#include "lattices.cuh"
#include "tensor.cuh"

namespace smrt {

static long double gauss_moment(int a) {  // E[x^a], x ~ N(0,1): (a-1)!! or 0
    if (a & 1) return 0.0L;
    long double v = 1.0L;
    for (int k = a - 1; k > 1; k -= 2) v *= k;
    return v;
}

struct Pattern {
    int a, b, c;
};

static std::vector<Pattern> even_patterns(int max_total) {
    std::vector<Pattern> out;
    for (int t = 0; t <= max_total; t += 2)
        for (int a = t; a >= 0; a -= 2)
            for (int b = a; b >= 0; b -= 2) {
                const int c = t - a - b;
                if (c < 0 || c > b || (c & 1)) continue;
                out.push_back({a, b, c});
            }
    return out;
}

template <class Lat>
static void shell_members(std::vector<std::vector<int>> &members) {
    members.assign(Lat::NSHELL, {});
    members[0].push_back(-1);  // rest velocity: the zero vector
    for (int p = 0; p < Lat::NP; ++p) members[Lat::shell(p)].push_back(p);
}

// sum over the members of shell s of (c e)^pattern, counting both +e and -e of a pair.
template <class Lat>
static long double shell_moment(const std::vector<int> &mem, const Pattern &pt, long double c) {
    long double acc = 0.0L;
    for (int p : mem) {
        if (p < 0) {
            acc += (pt.a == 0 && pt.b == 0 && pt.c == 0) ? 1.0L : 0.0L;
            continue;
        }
        const long double x = c * Lat::e(p, 0), y = c * Lat::e(p, 1), z = c * Lat::e(p, 2);
        acc += 2.0L * powl(x, pt.a) * powl(y, pt.b) * powl(z, pt.c);
    }
    return acc;
}

static bool solve_linear(std::vector<long double> A, std::vector<long double> b, int n,
                         std::vector<long double> &x) {
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabsl(A[r * n + col]) > fabsl(A[piv * n + col])) piv = r;
        if (fabsl(A[piv * n + col]) < 1e-300L) return false;
        if (piv != col) {
            for (int k = 0; k < n; ++k) std::swap(A[col * n + k], A[piv * n + k]);
            std::swap(b[col], b[piv]);
        }
        for (int r = col + 1; r < n; ++r) {
            const long double f = A[r * n + col] / A[col * n + col];
            for (int k = col; k < n; ++k) A[r * n + k] -= f * A[col * n + k];
            b[r] -= f * b[col];
        }
    }
    x.assign(n, 0.0L);
    for (int r = n - 1; r >= 0; --r) {
        long double s = b[r];
        for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * x[k];
        x[r] = s / A[r * n + r];
    }
    return true;
}

template <class Lat>
static bool weights_for(long double c, std::vector<long double> &W, long double &resid) {
    std::vector<std::vector<int>> mem;
    shell_members<Lat>(mem);
    const std::vector<Pattern> pts = even_patterns(Lat::DEGREE - 1);
    const int S = Lat::NSHELL;
    if ((int)pts.size() != S + 1) return false;
    std::vector<long double> A(S * S), b(S);
    for (int r = 0; r < S; ++r) {
        for (int s = 0; s < S; ++s) A[r * S + s] = shell_moment<Lat>(mem[s], pts[r], c);
        b[r] = gauss_moment(pts[r].a) * gauss_moment(pts[r].b) * gauss_moment(pts[r].c);
    }
    if (!solve_linear(A, b, S, W)) return false;
    const Pattern &last = pts[S];
    long double v = 0.0L;
    for (int s = 0; s < S; ++s) v += W[s] * shell_moment<Lat>(mem[s], last, c);
    resid = v - gauss_moment(last.a) * gauss_moment(last.b) * gauss_moment(last.c);
    return true;
}

template <class Lat>
static bool solve_lattice(double &c_out, std::vector<double> &w_pair, double &w_rest) {
    // scan [0.9, 1.1] x guess for sign changes of r(c); bisect each; keep the root closest to
    // the guess whose residual vanishes (a pole of the linear solve also flips the sign) and
    // whose weights are all positive
    const long double c0 = Lat::C_GUESS;
    const int steps = 400;
    std::vector<long double> W;
    long double prev_c = c0 * 0.9L, prev_r;
    if (!weights_for<Lat>(prev_c, W, prev_r)) return false;
    bool have = false;
    long double best_c = 0.0L;
    std::vector<long double> best_W;
    for (int k = 1; k <= steps; ++k) {
        const long double cc = c0 * (0.9L + 0.2L * k / steps);
        long double r;
        if (!weights_for<Lat>(cc, W, r)) return false;
        if ((r < 0) != (prev_r < 0)) {
            long double lo = prev_c, hi = cc, rlo = prev_r, rm = 0.0L;
            for (int it = 0; it < 200; ++it) {
                const long double mid = 0.5L * (lo + hi);
                weights_for<Lat>(mid, W, rm);
                if ((rm < 0) == (rlo < 0))
                    lo = mid, rlo = rm;
                else
                    hi = mid;
            }
            const long double cm = 0.5L * (lo + hi);
            weights_for<Lat>(cm, W, rm);
            bool positive = true;
            for (long double wv : W) positive = positive && (wv > 0.0L);
            if (fabsl(rm) < 1e-9L && positive && (!have || fabsl(cm - c0) < fabsl(best_c - c0))) {
                have = true;
                best_c = cm;
                best_W = W;
            }
        }
        prev_c = cc, prev_r = r;
    }
    if (!have) return false;
    c_out = (double)best_c;
    w_rest = (double)best_W[0];
    w_pair.assign(Lat::NP, 0.0);
    for (int p = 0; p < Lat::NP; ++p) w_pair[p] = (double)best_W[Lat::shell(p)];
    return true;
}

template <class Lat>
static lb_status named(int8_t *e_out, double *w_out, double *c_out, int *q_out, int *deg_out,
                       int capacity) {
    if (capacity < Lat::Q) return LB_ERR_INVALID;
    double c, w0;
    std::vector<double> wp;
    if (!solve_lattice<Lat>(c, wp, w0)) return LB_ERR_INVALID;
    e_out[0] = e_out[1] = e_out[2] = 0;
    w_out[0] = w0;
    for (int p = 0; p < Lat::NP; ++p) {
        for (int k = 0; k < 3; ++k) {
            e_out[3 * (2 * p + 1) + k] = (int8_t)Lat::e(p, k);
            e_out[3 * (2 * p + 2) + k] = (int8_t)(-Lat::e(p, k));
        }
        w_out[2 * p + 1] = w_out[2 * p + 2] = wp[p];
    }
    *c_out = c;
    *q_out = Lat::Q;
    *deg_out = Lat::DEGREE;
    return LB_OK;
}

// Largest |sum_i w_i xi_i^alpha - E[xi^alpha]| / max(1, E) over all |alpha| <= degree.
double quadrature_defect(int q, const int8_t *e, const double *w, double c, int degree) {
    double worst = 0.0;
    for (int a = 0; a <= degree; ++a)
        for (int b = 0; a + b <= degree; ++b)
            for (int d = 0; a + b + d <= degree; ++d) {
                long double s = 0.0L;
                for (int i = 0; i < q; ++i)
                    s += (long double)w[i] * powl(c * e[3 * i], a) * powl(c * e[3 * i + 1], b) *
                         powl(c * e[3 * i + 2], d);
                const long double g = gauss_moment(a) * gauss_moment(b) * gauss_moment(d);
                const double err = (double)(fabsl(s - g) / (g > 1.0L ? g : 1.0L));
                if (err > worst) worst = err;
            }
    return worst;
}

// 1D rule on c {0, +-E_0, .., +-E_{NP1-1}} (Sec. 4.2, D1Qd-P1): rest weight W_0 and pair
// weights W_1..W_NP1 from the even-moment conditions sum_i w_i (c e_i)^(2m) = (2m - 1)!!,
// m = 0..NP1, at fixed c (NP1 + 1 linear equations); the remaining condition, m = NP1 + 1,
// fixes c by bracketing and bisection, as for the cubic sets.
template <class L1>
static bool weights_1d(long double c, std::vector<long double> &W, long double &resid) {
    const int S = L1::NP1 + 1;
    auto mom = [&](int s, int a) -> long double {
        if (s == 0) return a == 0 ? 1.0L : 0.0L;
        return 2.0L * powl(c * L1::E(s - 1), a);
    };
    std::vector<long double> A(S * S), b(S);
    for (int r = 0; r < S; ++r) {
        for (int s = 0; s < S; ++s) A[r * S + s] = mom(s, 2 * r);
        b[r] = gauss_moment(2 * r);
    }
    if (!solve_linear(A, b, S, W)) return false;
    long double v = 0.0L;
    for (int s = 0; s < S; ++s) v += W[s] * mom(s, 2 * S);
    resid = v - gauss_moment(2 * S);
    return 2 * S + 1 == L1::DEGREE;
}

template <class L1>
static bool solve_rule_1d(double &c_out, std::vector<double> &w_out) {
    const long double c0 = L1::C_GUESS;
    const int steps = 400;
    std::vector<long double> W;
    long double prev_c = c0 * 0.9L, prev_r;
    if (!weights_1d<L1>(prev_c, W, prev_r)) return false;
    bool have = false;
    long double best_c = 0.0L;
    std::vector<long double> best_W;
    for (int k = 1; k <= steps; ++k) {
        const long double cc = c0 * (0.9L + 0.2L * k / steps);
        long double r;
        if (!weights_1d<L1>(cc, W, r)) return false;
        if ((r < 0) != (prev_r < 0)) {
            long double lo = prev_c, hi = cc, rlo = prev_r, rm = 0.0L;
            for (int it = 0; it < 200; ++it) {
                const long double mid = 0.5L * (lo + hi);
                weights_1d<L1>(mid, W, rm);
                if ((rm < 0) == (rlo < 0))
                    lo = mid, rlo = rm;
                else
                    hi = mid;
            }
            const long double cm = 0.5L * (lo + hi);
            weights_1d<L1>(cm, W, rm);
            bool positive = true;
            for (long double wv : W) positive = positive && (wv > 0.0L);
            if (fabsl(rm) < 1e-9L * gauss_moment(2 * (L1::NP1 + 1)) && positive && (!have || fabsl(cm - c0) < fabsl(best_c - c0))) {
                have = true;
                best_c = cm;
                best_W = W;
            }
        }
        prev_c = cc, prev_r = r;
    }
    if (!have) return false;
    c_out = (double)best_c;
    w_out.assign(L1::Q1, 0.0);  // library order: rest, then +E_p, -E_p
    w_out[0] = (double)best_W[0];
    for (int p = 0; p < L1::NP1; ++p) w_out[2 * p + 1] = w_out[2 * p + 2] = (double)best_W[p + 1];
    return true;
}

// The 3D tensor product of a 1D rule in library order i = a + d b + d^2 c.
template <class L1>
static lb_status named_tensor(int8_t *e_out, double *w_out, double *c_out, int *q_out, int *deg_out,
                              int capacity) {
    constexpr int Q1 = L1::Q1, Q = Q1 * Q1 * Q1;
    if (capacity < Q) return LB_ERR_INVALID;
    double c;
    std::vector<double> w1;
    if (!solve_rule_1d<L1>(c, w1)) return LB_ERR_INVALID;
    for (int i = 0; i < Q; ++i) {
        const int a = i % Q1, b = (i / Q1) % Q1, cc = i / (Q1 * Q1);
        e_out[3 * i] = (int8_t)e1<L1>(a);
        e_out[3 * i + 1] = (int8_t)e1<L1>(b);
        e_out[3 * i + 2] = (int8_t)e1<L1>(cc);
        w_out[i] = w1[a] * w1[b] * w1[cc];
    }
    *c_out = c;
    *q_out = Q;
    *deg_out = L1::DEGREE;
    return LB_OK;
}

}  // namespace smrt

extern "C" lb_status lb_lattice_named(const char *name, int8_t *e_out, double *w_out, double *c_out,
                                      int *q_out, int *degree_out, int capacity) {
    if (!name || !e_out || !w_out || !c_out || !q_out || !degree_out) return LB_ERR_INVALID;
    if (std::strcmp(name, "D3Q39") == 0)
        return smrt::named<smrt::D3Q39>(e_out, w_out, c_out, q_out, degree_out, capacity);
    if (std::strcmp(name, "D3Q103") == 0)
        return smrt::named<smrt::D3Q103>(e_out, w_out, c_out, q_out, degree_out, capacity);
    if (std::strcmp(name, "D3Q729") == 0)
        return smrt::named_tensor<smrt::D1Q9P1>(e_out, w_out, c_out, q_out, degree_out, capacity);
    if (std::strcmp(name, "D3Q4913") == 0)
        return smrt::named_tensor<smrt::D1Q17P1>(e_out, w_out, c_out, q_out, degree_out, capacity);
    return LB_ERR_INVALID;
}

extern "C" lb_status lb_rankine_hugoniot(double Ma, double gamma, double rho1, double theta1,
                                         lb_state *left, lb_state *right) {
    if (!left || !right || !(Ma >= 1.0) || !(gamma > 1.0) || !(rho1 > 0.0) || !(theta1 > 0.0))
        return LB_ERR_INVALID;
    const double M2 = Ma * Ma;
    const double r = (gamma + 1.0) * M2 / ((gamma - 1.0) * M2 + 2.0);
    const double t = (2.0 * gamma * M2 - gamma + 1.0) * ((gamma - 1.0) * M2 + 2.0) /
                     ((gamma + 1.0) * (gamma + 1.0) * M2);
    const double u1 = Ma * std::sqrt(gamma * theta1);
    *left = lb_state{rho1, {u1, 0.0, 0.0}, theta1};
    *right = lb_state{rho1 * r, {u1 / r, 0.0, 0.0}, theta1 * t};
    return LB_OK;
}

extern "C" lb_status lb_shock_frame(double Ma, double gamma, double c, double theta2_max, double *theta1,
                                    int *kx) {
    if (!theta1 || !kx || !(Ma >= 1.0) || !(gamma > 1.0) || !(c > 0.0) || !(theta2_max > 0.0))
        return LB_ERR_INVALID;
    lb_state l, r;
    lb_rankine_hugoniot(Ma, gamma, 1.0, 1.0, &l, &r);
    const double ratio = r.theta;  // theta2 / theta1
    // the hottest state must stay well below the convergence bound theta < 2 (Sec. 4.1)
    const double t1 = std::min(1.0, theta2_max / ratio);
    *theta1 = t1;
    return lb_shock_shift(Ma, gamma, c, t1, kx);
}

extern "C" lb_status lb_shock_shift(double Ma, double gamma, double c, double theta1, int *kx) {
    if (!kx || !(Ma >= 1.0) || !(gamma > 1.0) || !(c > 0.0) || !(theta1 > 0.0)) return LB_ERR_INVALID;
    const double c1 = std::sqrt(gamma * theta1);
    const double mean = (gamma * Ma * Ma + 1.0) / ((gamma + 1.0) * Ma) * c1;  // (u1 + u2) / 2
    *kx = (int)std::lround(mean / c);
    return LB_OK;
}
