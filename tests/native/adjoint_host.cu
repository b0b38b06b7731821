// Host build of the per-cell adjoint arithmetic of libsmrt (csrc/adjoint.cuh), for CPU tests
// against the oracle's complex-step vector-Jacobian products. Arrays are in library order.
#include "../../paper_2401_11086_gb300/csrc/adjoint.cuh"

using namespace smrt;

template <class Lat, int N>
static void cvjp(const double *f, const double *lam, double c, const double *wp, const double *tauA,
                 const double *tauB, double dAdt, double dBdt, double *fb, double *taub) {
    double ff[Lat::Q], ll[Lat::Q], ww[Lat::NP + 1], out[Lat::Q], tb[ntau(N)];
    for (int i = 0; i < Lat::Q; ++i) ff[i] = f[i], ll[i] = lam[i];
    for (int p = 0; p <= Lat::NP; ++p) ww[p] = wp[p];
    for (int k = 0; k < ntau(N); ++k) tb[k] = 0.0;
    collide_vjp<Lat, N>(ff, ll, c, ww, tauA, tauB, dAdt, dBdt, out, tb);
    for (int i = 0; i < Lat::Q; ++i) fb[i] = out[i];
    for (int k = 0; k < ntau(N); ++k) taub[k] = tb[k];
}

template <class Lat, int N>
static void mvjp(const double *f, double c, const double *bar /* rho, ux, uy, uz, theta, qx, qy, qz */,
                 double *fb) {
    double ff[Lat::Q], out[Lat::Q];
    for (int i = 0; i < Lat::Q; ++i) ff[i] = f[i];
    const double ub[3] = {bar[1], bar[2], bar[3]}, qb[3] = {bar[5], bar[6], bar[7]};
    moments_vjp<Lat, N>(ff, c, bar[0], ub, bar[4], qb, out);
    for (int i = 0; i < Lat::Q; ++i) fb[i] = out[i];
}

extern "C" {
void collide_vjp_d3q39_n3(const double *f, const double *lam, double c, const double *wp, const double *tauA,
                          const double *tauB, double dAdt, double dBdt, double *fb, double *taub) {
    cvjp<D3Q39, 3>(f, lam, c, wp, tauA, tauB, dAdt, dBdt, fb, taub);
}
void collide_vjp_d3q103_n4(const double *f, const double *lam, double c, const double *wp, const double *tauA,
                           const double *tauB, double dAdt, double dBdt, double *fb, double *taub) {
    cvjp<D3Q103, 4>(f, lam, c, wp, tauA, tauB, dAdt, dBdt, fb, taub);
}
void moments_vjp_d3q39_n3(const double *f, double c, const double *bar, double *fb) { mvjp<D3Q39, 3>(f, c, bar, fb); }
void moments_vjp_d3q103_n4(const double *f, double c, const double *bar, double *fb) { mvjp<D3Q103, 4>(f, c, bar, fb); }
}
