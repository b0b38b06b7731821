// tensor_adjoint.cuh -- lb_step_adjoint and lb_moments_adjoint on the tensor-product sets
// (D3Q729 = D1Q9-P1^3, D3Q4913 = D1Q17-P1^3; Sec. 4.2, Table 3), in double whatever the
// precision of the forward state.
//
// The collision maps the pulled deviations f of a cell to f'_i = w_i sum_g P_g e_i^g, with the
// rebuild coefficients P a function of the raw moments R_g = sum_i f_i e_i^g. Its VJP therefore
// needs only sums over the populations of the same two shapes as the forward step: the
// projection of the weighted adjoint, Lc_g = c^|g| sum_i w_i lam_i e_i^g, and the evaluation
// fb_i = sum_g c^|g| e_i^g Rcb_g of the raw moments' adjoint Rcb; both factor over the axes
// exactly as the forward projection and rebuild do (TPCell::project / TPCell::rebuild with unit
// weights). Between them sits the moment-space VJP shared with the other sets (moment_vjp in
// adjoint.cuh). One thread per cell, 32-cell tiles; the streaming transpose is the push of
// adjoint_kernels.cuh (every lam^t_i(y) written once, zero where nothing pulls from y); the
// relaxation-time gradients are reduced per tile by a warp shuffle in a fixed order, then over
// tiles in tile order.
#pragma once

#include "adjoint.cuh"
#include "tensor.cuh"

namespace smrt {

template <class L1, int N, class T, bool FixedX>
struct TPAdjCell {
    static constexpr int Q1 = L1::Q1;
    static constexpr int P2 = Q1 * Q1;
    static constexpr int Q = P2 * Q1;

    const TPArgs<T> &a;
    const TPTables<L1, double> &s;
    int x, L, kx;
    long long base;
    const T *gl, *gr;

    SMRT_D TPAdjCell(const TPArgs<T> &a_, const TPTables<L1, double> &s_, const int2 tile) : a(a_), s(s_) {
        const InstanceInfo &in = a.inst[tile.x];
        x = tile.y + int(threadIdx.x);
        L = in.nx;
        kx = in.kx;
        base = in.cell_off;
        gl = a.ghosts + (long long)tile.x * 2 * Q;
        gr = gl + Q;
    }
    // the pulled (pre-collision) deviation of population i, x-velocity index av
    template <int av>
    SMRT_D double pulled(int i) const {
        const int xs = x - e1<L1>(av) - kx;
        if constexpr (FixedX) {
            if (xs < 0) return double(gl[i]);
            if (xs >= L) return double(gr[i]);
        }
        return double(a.fin[(long long)s.plane[i] * a.stride + base + wrap(xs, L)]);
    }
    // lam^t_i at the cell population i was pulled from = v; zero at (i, x) when no cell pulls
    // population i from x (beyond a fixed end)
    SMRT_D void push(double *lam_t, int i, double v) const {
        const int ex = int(s.e[i % Q1]);
        const long long pl = (long long)s.plane[i] * a.stride + base;
        const int xs = x - ex - kx;
        if constexpr (FixedX) {
            if (xs >= 0 && xs < L) lam_t[pl + xs] = v;
            const int xd = x + ex + kx;
            if (xd < 0 || xd >= L) lam_t[pl + x] = 0.0;
        } else {
            lam_t[pl + wrap(xs, L)] = v;
        }
    }
};

template <int M, int N>
SMRT_D void scale_by_c_powers(double c, double (&v)[M]) {
    double cp[N + 1];
    cp[0] = 1.0;
    for (int j = 1; j <= N; ++j) cp[j] = cp[j - 1] * c;
    static_for<M>([&](auto G) {
        constexpr int g = decltype(G)::value;
        v[g] *= cp[mi_order(g)];
    });
}

template <class L1, int N, class T, bool FixedX>
__global__ void __launch_bounds__(32) tp_adjoint_step_kernel(TPArgs<T> a, const double *lam_next, double *lam_t,
                                                             double *partials) {
    constexpr int M = nmom(N);
    constexpr int KT = ntau(N);
    constexpr int Q1 = L1::Q1;
    using C = TPCell<L1, N, double>;
    __shared__ TPTables<L1, double> s;
    tp_load_tables<L1>(a, s);
    const int2 tile = a.tiles[blockIdx.x];
    const TPAdjCell<L1, N, T, FixedX> cell(a, s, tile);
    double tb[KT];
    for (int k = 0; k < KT; ++k) tb[k] = 0.0;
    if (cell.x < cell.L) {
        const InstanceInfo &in = a.inst[tile.x];
        double Rc[M], Lc[M], Rcb[M];
        C::project([&](int i, auto A) { return cell.template pulled<decltype(A)::value>(i); }, s.e, Rc);
        C::project(
            [&](int i, auto A) {
                constexpr int av = decltype(A)::value;
                const int bc = i / Q1;
                return s.w[av] * s.w[bc % Q1] * s.w[bc / Q1] *
                       lam_next[(long long)s.plane[i] * a.stride + cell.base + cell.x];
            },
            s.e, Lc);
        scale_by_c_powers<M, N>(a.cd, Rc);
        scale_by_c_powers<M, N>(a.cd, Lc);
        moment_vjp<N>(Rc, Lc, in.tauA, in.tauB, in.dAdt, in.dBdt, Rcb, tb);
        scale_by_c_powers<M, N>(a.cd, Rcb);
        double ones[Q1];
        for (int k = 0; k < Q1; ++k) ones[k] = 1.0;
        C::template rebuild<double>(Rcb, s.e, ones, [&](int i, double v) { cell.push(lam_t, i, v); });
    }
    // tile sum of the relaxation-time gradients, fixed order
    for (int k = 0; k < KT; ++k) {
        double v = tb[k];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (threadIdx.x == 0) partials[(long long)blockIdx.x * KT + k] = v;
    }
}

template <class L1, int N, class T, bool FixedX>
__global__ void __launch_bounds__(32) tp_adjoint_moments_kernel(TPArgs<T> a, const double *gbar, unsigned mask,
                                                                double *lam, long long ncells) {
    constexpr int M = nmom(N);  // N >= 4 on these sets: the order-3 coefficients are inside
    constexpr int Q1 = L1::Q1;
    using C = TPCell<L1, N, double>;
    __shared__ TPTables<L1, double> s;
    tp_load_tables<L1>(a, s);
    const int2 tile = a.tiles[blockIdx.x];
    const TPAdjCell<L1, N, T, FixedX> cell(a, s, tile);
    if (cell.x >= cell.L) return;
    const long long cidx = cell.base + cell.x;
    long long r = 0;
    double rb = 0.0, ub[3] = {0.0, 0.0, 0.0}, thb = 0.0, qb[3] = {0.0, 0.0, 0.0};
    if (mask & 0x1u) rb = gbar[(r++) * ncells + cidx];
    if (mask & 0x2u)
        for (int k = 0; k < 3; ++k) ub[k] = gbar[(r++) * ncells + cidx];
    if (mask & 0x4u) thb = gbar[(r++) * ncells + cidx];
    if (mask & 0x10u)
        for (int k = 0; k < 3; ++k) qb[k] = gbar[(r++) * ncells + cidx];
    double Rc[M], Rcb[M];
    C::project([&](int i, auto A) { return cell.template pulled<decltype(A)::value>(i); }, s.e, Rc);
    scale_by_c_powers<M, N>(a.cd, Rc);
    moments_vjp_m<N>(Rc, rb, ub, thb, qb, Rcb);
    scale_by_c_powers<M, N>(a.cd, Rcb);
    double ones[Q1];
    for (int k = 0; k < Q1; ++k) ones[k] = 1.0;
    C::template rebuild<double>(Rcb, s.e, ones, [&](int i, double v) { cell.push(lam, i, v); });
}

}  // namespace smrt
