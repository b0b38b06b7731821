// convergence.cu -- the Appendix B study of Yan & Shan (arXiv 2401.11086): how many Hermite
// orders the expansion of a 1D Maxwellian needs (Appendix B, Eq. fexp).
//
// For each (theta, u) the expansion f_N = omega(xi) sum_{n<=N} a^(n) He_n(xi)/n! of
// f = exp(-(xi - u)^2 / (2 theta)) / sqrt(2 pi theta) is built order by order and its L1 error
// int |f - f_N| dxi is taken after every order; the first N below the tolerance is reported.
// a^(n) follows its recurrence a^(n+1) = u a^(n) + n (theta - 1) a^(n-1) (the generating
// function of the Appendix B closed form), He_n its three-term recurrence, both normalised by
// sqrt(n!) so that the terms stay bounded:
//   omega a^(n) He_n / n! = [a^(n)/sqrt(n!)] [omega(xi) He_n(xi)/sqrt(n!)].
// The integral is composite Simpson on NXI points of [-L, L],
// L = max(|u| + 12 sqrt(theta), 2 sqrt(nmax + 1) + 10).
//
// One block per (theta, u) point (grid-stride), 1024 threads over the xi points, a fixed-order
// block reduction per order (deterministic), and an early exit once the error is below tol.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/smrt.h"

namespace {

constexpr int kNxi = 4097;
constexpr int kThreads = 1024;
constexpr int kSlots = (kNxi + kThreads - 1) / kThreads;  // xi points per thread

__global__ void __launch_bounds__(kThreads) hermite_convergence_kernel(const double *__restrict__ theta,
                                                                       const double *__restrict__ u, int npts,
                                                                       double tol, int nmax, int *order,
                                                                       double *err) {
    __shared__ double warp_sum[kThreads / 32];
    __shared__ int stop;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int p = blockIdx.x; p < npts; p += gridDim.x) {
        const double th = theta[p], up = u[p];
        if (!(th > 0.0) || !isfinite(th) || !isfinite(up)) {
            if (tid == 0) {
                order[p] = -1;
                err[p] = NAN;
            }
            continue;
        }
        const double L = fmax(fabs(up) + 12.0 * sqrt(th), 2.0 * sqrt(nmax + 1.0) + 10.0);
        const double h = 2.0 * L / (kNxi - 1);
        // per xi point: the Simpson weight w is folded into f and f_N (w |f - f_N| = |w f - w f_N|),
        // and w exp(-xi^2/4)/sqrt(2 pi) into the Hermite function, which keeps its recurrence
        // (psi_n = w omega(xi) He_n(xi)/sqrt(n!))
        auto xi_of = [&](int s) { return -L + h * (tid + s * kThreads); };
        double f[kSlots], psi[kSlots], psim[kSlots], fN[kSlots];
#pragma unroll
        for (int s = 0; s < kSlots; ++s) {
            const int k = tid + s * kThreads;
            const double w = k < kNxi ? (h / 3.0) * ((k == 0 || k == kNxi - 1) ? 1.0 : ((k & 1) ? 4.0 : 2.0)) : 0.0;
            const double x = xi_of(s), d = x - up;
            f[s] = w * (exp(-d * d / (2.0 * th)) / sqrt(2.0 * M_PI * th));
            psi[s] = w * (exp(-x * x / 2.0) / sqrt(2.0 * M_PI));  // psi_0
            psim[s] = 0.0;
            fN[s] = 0.0;
        }
        double a_prev = 0.0, a = 1.0;  // a^(n-1)/sqrt((n-1)!), a^(n)/sqrt(n!)
        int found = nmax + 1;
        double e_last = 0.0;
        for (int n = 0; n <= nmax; ++n) {
            double part = 0.0;
#pragma unroll
            for (int s = 0; s < kSlots; ++s) {
                fN[s] = fma(a, psi[s], fN[s]);
                part += fabs(f[s] - fN[s]);
            }
            for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
            if (lane == 0) warp_sum[warp] = part;
            __syncthreads();
            if (tid == 0) {
                double e = 0.0;
                for (int q = 0; q < kThreads / 32; ++q) e += warp_sum[q];
                e_last = e;
                stop = e < tol;
                if (stop) {
                    order[p] = n;
                    err[p] = e;
                }
            }
            __syncthreads();
            if (stop) {
                found = n;
                break;
            }
            // next order: He_{n+1} = xi He_n - n He_{n-1}; a^(n+1) = u a^(n) + n (theta - 1) a^(n-1)
            const double rn = sqrt(double(n)), rn1 = 1.0 / sqrt(n + 1.0);
#pragma unroll
            for (int s = 0; s < kSlots; ++s) {
                const double nx = (xi_of(s) * psi[s] - rn * psim[s]) * rn1;
                psim[s] = psi[s];
                psi[s] = nx;
            }
            const double an = (up * a + rn * (th - 1.0) * a_prev) * rn1;
            a_prev = a;
            a = an;
        }
        if (found > nmax && tid == 0) {
            order[p] = nmax + 1;
            err[p] = e_last;
        }
        __syncthreads();  // warp_sum and stop are reused by the next point
    }
}

}  // namespace

extern "C" lb_status lb_hermite_convergence(const double *theta, const double *u, int npts, double tol, int nmax,
                                            int *order, double *err, void *stream) {
    if (npts < 0 || nmax < 0 || nmax > LB_HERMITE_MAX_ORDER || !(tol > 0.0)) return LB_ERR_INVALID;
    if (npts == 0) return LB_OK;
    if (!theta || !u || !order || !err) return LB_ERR_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LB_ERR_CUDA;
    const int grid = npts < 4 * sms ? npts : 4 * sms;
    hermite_convergence_kernel<<<grid, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(theta, u, npts, tol, nmax,
                                                                                        order, err);
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}
