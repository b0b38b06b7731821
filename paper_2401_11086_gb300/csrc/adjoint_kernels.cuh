// adjoint_kernels.cuh -- kernels of lb_step_adjoint and lb_moments_adjoint.
//
// One step maps h^t to h^{t+1} = C(S h^t): S pulls population i at cell x from x - e_i - k
// (cells beyond a fixed x end hold constant end-state populations), C collides each cell. The
// adjoint, per cell x, recomputes the pulled f(x), forms mu(x) = J_C(f(x))^T lam^{t+1}(x) with
// the hand-written VJP of adjoint.cuh, and pushes mu_i(x) back to the cell it was pulled from,
// lam^t_i(x - e_i - k) (S^T). Every (i, y) of lam^t is written exactly once: by the cell
// x = y + e_i + k when that cell exists, otherwise (beyond a fixed end) by cell y itself with 0.
// Relaxation-time gradients are summed per block in a fixed tree order into a per-block slot
// of a scratch array, then over blocks in block order by reduce_kernel: the result does not
// depend on scheduling.
#pragma once

#include "adjoint.cuh"
#include "kernels.cuh"

namespace smrt {

template <class Lat, class T>
struct AdjArgs {
    StepArgs<Lat, T> s;
    const double *lam_in;  // step: lam^{t+1}; moments: the moments' adjoints (rows x cells)
    double *lam_out;       // lam^t (state layout, double)
    double *partials;      // [block][ntau] (step only)
    double wpd[Lat::NP + 1];
    double c;
    int line, fixedx;
    unsigned mask;         // moments: which row groups lam_in holds
    long long ncells;
};

// Pull the populations of cell (x, y, z) or (instance, x); sets cell index and shifts.
template <class Lat, class T>
struct CellPull {
    long long cell;
    int L;      // line length (line mode)
    int sx[Lat::Q];  // x shift of each population (including k)
    bool valid;
    SMRT_D void load(const AdjArgs<Lat, T> &A, double (&f)[Lat::Q]) {
        const StepArgs<Lat, T> &a = A.s;
        if (A.line) {
            const int2 tile = a.tiles[blockIdx.x];
            const InstanceInfo &in = a.inst[tile.x];
            const int x = tile.y + threadIdx.x;
            L = in.nx;
            valid = x < L;
            if (!valid) return;
            cell = in.cell_off + x;
            const T *gl = a.ghosts + (long long)tile.x * 2 * Lat::Q;
            const T *gr = gl + Lat::Q;
            static_for<Lat::Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int ex = i == 0 ? 0 : ((i & 1) ? Lat::e((i - 1) / 2, 0) : -Lat::e((i - 1) / 2, 0));
                sx[i] = ex + in.kx;
                const int xs = x - sx[i];
                if (A.fixedx && xs < 0)
                    f[i] = double(gl[i]);
                else if (A.fixedx && xs >= L)
                    f[i] = double(gr[i]);
                else
                    f[i] = double(a.fin[a.plane[i] + in.cell_off + wrap(xs, L)]);
            });
        } else {
            const int x = blockIdx.x * blockDim.x + threadIdx.x;
            const int y = blockIdx.y, z = blockIdx.z;
            valid = x < a.nx;
            if (!valid) return;
            const long long row = a.nx, slab = row * a.ny;
            cell = z * slab + y * row + x;
            static_for<Lat::Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int ex = i == 0 ? 0 : ((i & 1) ? Lat::e((i - 1) / 2, 0) : -Lat::e((i - 1) / 2, 0));
                constexpr int ey = i == 0 ? 0 : ((i & 1) ? Lat::e((i - 1) / 2, 1) : -Lat::e((i - 1) / 2, 1));
                constexpr int ez = i == 0 ? 0 : ((i & 1) ? Lat::e((i - 1) / 2, 2) : -Lat::e((i - 1) / 2, 2));
                const int xs = wrap(x - (ex + a.kx), a.nx);
                const int ys = wrap(y - (ey + a.ky), a.ny);
                const int zs = wrap(z - (ez + a.kz), a.nz);
                f[i] = double(a.fin[a.plane[i] + zs * slab + ys * row + xs]);
            });
        }
    }
    // lam^t_i(source of i at this cell) = mu_i; zero where no cell pulls from this one
    SMRT_D void push(const AdjArgs<Lat, T> &A, const double (&mu)[Lat::Q]) {
        const StepArgs<Lat, T> &a = A.s;
        if (A.line) {
            const int2 tile = a.tiles[blockIdx.x];
            const InstanceInfo &in = a.inst[tile.x];
            const int x = tile.y + threadIdx.x;
            static_for<Lat::Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                const int xs = x - sx[i];
                if (!A.fixedx)
                    A.lam_out[a.plane[i] + in.cell_off + wrap(xs, L)] = mu[i];
                else if (xs >= 0 && xs < L)
                    A.lam_out[a.plane[i] + in.cell_off + xs] = mu[i];
                const int xd = x + sx[i];  // the cell that pulls population i from here
                if (A.fixedx && (xd < 0 || xd >= L)) A.lam_out[a.plane[i] + cell] = 0.0;
            });
        } else {
            const int x = blockIdx.x * blockDim.x + threadIdx.x;
            const int y = blockIdx.y, z = blockIdx.z;
            const long long row = a.nx, slab = row * a.ny;
            static_for<Lat::Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int ex = i == 0 ? 0 : ((i & 1) ? Lat::e((i - 1) / 2, 0) : -Lat::e((i - 1) / 2, 0));
                constexpr int ey = i == 0 ? 0 : ((i & 1) ? Lat::e((i - 1) / 2, 1) : -Lat::e((i - 1) / 2, 1));
                constexpr int ez = i == 0 ? 0 : ((i & 1) ? Lat::e((i - 1) / 2, 2) : -Lat::e((i - 1) / 2, 2));
                const int xs = wrap(x - (ex + a.kx), a.nx);
                const int ys = wrap(y - (ey + a.ky), a.ny);
                const int zs = wrap(z - (ez + a.kz), a.nz);
                A.lam_out[a.plane[i] + zs * slab + ys * row + xs] = mu[i];
            });
        }
    }
};

template <class Lat, int N, class T>
__global__ void __launch_bounds__(128) adjoint_step_kernel(AdjArgs<Lat, T> A) {
    constexpr int KT = ntau(N);
    __shared__ double red[KT][128];
    CellPull<Lat, T> cp;
    double f[Lat::Q];
    cp.load(A, f);
    double tb[KT];
    for (int k = 0; k < KT; ++k) tb[k] = 0.0;
    if (cp.valid) {
        const InstanceInfo &in = A.line ? A.s.inst[A.s.tiles[blockIdx.x].x] : A.s.inst[0];
        double lam[Lat::Q], mu[Lat::Q];
        static_for<Lat::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            lam[i] = A.lam_in[A.s.plane[i] + cp.cell];
        });
        collide_vjp<Lat, N>(f, lam, A.c, A.wpd, in.tauA, in.tauB, in.dAdt, in.dBdt, mu, tb);
        cp.push(A, mu);
    }
    for (int k = 0; k < KT; ++k) red[k][threadIdx.x] = tb[k];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {  // blockDim.x: 32, 64 or 128
        if ((int)threadIdx.x < w)
            for (int k = 0; k < KT; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long long blk = (long long)blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
        for (int k = 0; k < KT; ++k) A.partials[blk * KT + k] = red[k][0];
    }
}

// dtau[k] += sum over blocks (block order) of partials[b][k]
static __global__ void reduce_partials_kernel(const double *partials, long long nblocks, int kt, double *dtau) {
    const int k = threadIdx.x;
    if (k >= kt) return;
    double acc = 0.0;
    for (long long b = 0; b < nblocks; ++b) acc += partials[b * kt + k];
    dtau[k] += acc;
}

template <class Lat, int N, class T>
__global__ void __launch_bounds__(128) adjoint_moments_kernel(AdjArgs<Lat, T> A) {
    CellPull<Lat, T> cp;
    double f[Lat::Q];
    cp.load(A, f);
    if (!cp.valid) return;
    const long long nc = A.ncells;
    long long r = 0;
    double rb = 0.0, ub[3] = {0.0, 0.0, 0.0}, thb = 0.0, qb[3] = {0.0, 0.0, 0.0};
    if (A.mask & 0x1u) rb = A.lam_in[(r++) * nc + cp.cell];
    if (A.mask & 0x2u)
        for (int k = 0; k < 3; ++k) ub[k] = A.lam_in[(r++) * nc + cp.cell];
    if (A.mask & 0x4u) thb = A.lam_in[(r++) * nc + cp.cell];
    if (A.mask & 0x10u)
        for (int k = 0; k < 3; ++k) qb[k] = A.lam_in[(r++) * nc + cp.cell];
    double mu[Lat::Q];
    moments_vjp<Lat, N>(f, A.c, rb, ub, thb, qb, mu);
    cp.push(A, mu);
}

}  // namespace smrt
