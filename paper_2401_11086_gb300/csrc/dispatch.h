// dispatch.h -- what the C-ABI layer (api.cu) needs to launch the templated kernels that the
// per-lattice, per-precision translation units instantiate.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstring>

#include "kernels.cuh"
#include "tensor.cuh"

namespace smrt {

constexpr int kMaxQ = 103;   // largest set with a per-population plane table in the launch
constexpr int kMaxQTP = 4913; // largest tensor-product set (plane table in device memory)
constexpr int kMaxNP = 51;
constexpr int kTile = 128;  // cells per block (threads per block) for every kernel

// Everything a launch needs, in library population order.
struct CtxView {
    cudaStream_t stream;
    long long plane[kMaxQ];
    double wp[kMaxNP + 1];
    double c;
    int nx, ny, nz;
    int kx, ky, kz;
    int line;    // 1: batched 1D lines (tiles), 0: periodic box
    int fixedx;  // line mode: fixed end states in x
    const InstanceInfo *inst;
    const int2 *tiles;
    int ntiles;
    const void *ghosts;
    const double *ghostsd;  // end-state deviations in double
    unsigned *health;
    long long ncells;
    unsigned step;   // launch counter of lb_step (seeds the stochastic rounding)
    int tile_width;  // cells (threads) per block of the line kernels: 32, 64 or 128
    unsigned *bar;   // persistent launch: arrival count, generation, step counter
    // tensor-product sets (D3Q729, D3Q4913): caller plane of each library population (device table),
    // the plane stride, and the 1D weights in library order
    const int *plane_idx;
    long long stride;
    double w1[kMaxQ1];
    int plane_identity;  // 1: library population i is caller plane i (tensor-map staging applies)
    int tensor_cores;    // 1: float tensor-product lines with fixed ends sum their x-rows on the
                         // tensor cores (lb_schedule::tensor_cores)
    // tensor-product lines: the step kernels' block tiles (instance, first x) of tile_width cells
    const int2 *btiles;
    int nbtiles;
};

using StepFn = cudaError_t (*)(const CtxView &, const void *fin, void *fout);
using MomentsFn = cudaError_t (*)(const CtxView &, const void *f, double *out, unsigned mask);
using FillFn = cudaError_t (*)(const CtxView &, void *f, const double *rho, const double *u,
                               const double *theta);
using GhostFn = cudaError_t (*)(const CtxView &, const double *states, int ninst, void *ghosts,
                                double *ghostsd);

using PersistFn = cudaError_t (*)(const CtxView &, void *fa, void *fb, int nsteps, int grid);
using OccupancyFn = int (*)(const CtxView &);

struct KernelSet {
    StepFn step;
    MomentsFn moments;
    FillFn fill;
    GhostFn ghost;
    PersistFn persist;      // line geometry: all steps in one cooperative launch
    OccupancyFn occupancy;  // resident blocks per SM of the persistent kernel
};

// precision: 0 double, 1 float, 2 float with double conserved sums and equilibrium rebuild

template <class Lat, class T>
StepArgs<Lat, T> make_args(const CtxView &v, const void *fin, void *fout) {
    StepArgs<Lat, T> a;
    a.fin = static_cast<const T *>(fin);
    a.fout = static_cast<T *>(fout);
    a.inst = v.inst;
    a.tiles = v.tiles;
    a.ghosts = static_cast<const T *>(v.ghosts);
    a.ghostsd = v.ghostsd;
    a.health = v.health;
    for (int i = 0; i < Lat::Q; ++i) a.plane[i] = v.plane[i];
    for (int p = 0; p <= Lat::NP; ++p) {
        a.wp[p] = T(v.wp[p]);
        a.wpd[p] = v.wp[p];
        a.wlo[p] = float(v.wp[p] - double(float(v.wp[p])));
    }
    a.c = T(v.c);
    a.cd = v.c;
    a.clo = float(v.c - double(float(v.c)));
    a.nx = v.nx;
    a.ny = v.ny;
    a.nz = v.nz;
    a.kx = v.kx;
    a.ky = v.ky;
    a.kz = v.kz;
    a.step = v.step;
    return a;
}

// cuTensorMapEncodeTiled, looked up through the runtime (no link-time dependence on the
// driver library).
using TensorMapEncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                       const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                       CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                       CUtensorMapFloatOOBfill);
inline TensorMapEncodeFn tensor_map_encoder() {
    static const TensorMapEncodeFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return TensorMapEncodeFn(nullptr);
        return reinterpret_cast<TensorMapEncodeFn>(p);
    }();
    return fn;
}

// Tensor map of a float state for the staged split-precision lines: [Q planes][stride cells],
// box of kSeg cells x Q planes (every row a warp's pulls can reach). False when staging does not
// apply (caller plane order differs from the library order, base or plane stride not on 16
// bytes, coordinates beyond int32) or the driver refuses the map; the plain kernels run then.
template <class Lat>
bool line_staging_applies(const CtxView &v) {
    return tensor_map_encoder() && v.plane_identity && (v.stride * 4ll) % 16 == 0 &&
           v.stride + 2 * LineStage<Lat>::kSeg < (1ll << 31);
}
template <class Lat>
bool line_encode_map(const CtxView &v, const void *state, CUtensorMap *m) {
    const TensorMapEncodeFn enc = tensor_map_encoder();
    if (!line_staging_applies<Lat>(v) || !state || (reinterpret_cast<unsigned long long>(state) & 15ull) != 0ull)
        return false;
    const cuuint64_t dims[2] = {cuuint64_t(v.stride), cuuint64_t(Lat::Q)};
    const cuuint64_t strides[1] = {cuuint64_t(v.stride) * 4u};
    const cuuint32_t box[2] = {cuuint32_t(LineStage<Lat>::kSeg), cuuint32_t(Lat::Q)};
    const cuuint32_t estr[2] = {1u, 1u};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(state), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The staged kernels may take more than the default 48 KB of dynamic shared memory: raise the
// limit of each instantiation to what a 128-thread block needs, once per device.
template <auto Kernel, class Lat>
cudaError_t line_smem_limit() {
    constexpr int kDevices = 64;
    static std::atomic<int> state[kDevices];  // 0 not set, 1 set, 2 failed
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kDevices) return cudaErrorInvalidDevice;
    if (state[dev].load(std::memory_order_acquire) == 1) return cudaSuccess;
    e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(LineStage<Lat>::persistent_bytes(128)));
    state[dev].store(e == cudaSuccess ? 1 : 2, std::memory_order_release);
    return e;
}

template <class Lat, int N, class T, class Acc, bool Split>
cudaError_t launch_step(const CtxView &v, const void *fin, void *fout) {
    const StepArgs<Lat, T> a = make_args<Lat, T>(v, fin, fout);
    if constexpr (Split) {
        CUtensorMap map;
        if (v.line && line_encode_map<Lat>(v, fin, &map)) {
            const size_t smem = LineStage<Lat>::bytes(v.tile_width);
            if (v.fixedx) {
                const cudaError_t e = line_smem_limit<step_line_staged<Lat, N, Acc, true>, Lat>();
                if (e != cudaSuccess) return e;
                step_line_staged<Lat, N, Acc, true><<<v.ntiles, v.tile_width, smem, v.stream>>>(a, map);
            } else {
                const cudaError_t e = line_smem_limit<step_line_staged<Lat, N, Acc, false>, Lat>();
                if (e != cudaSuccess) return e;
                step_line_staged<Lat, N, Acc, false><<<v.ntiles, v.tile_width, smem, v.stream>>>(a, map);
            }
            return cudaGetLastError();
        }
    }
    if (v.line) {
        if (v.fixedx)
            step_line_kernel<Lat, N, T, Acc, Split, true><<<v.ntiles, v.tile_width, 0, v.stream>>>(a);
        else
            step_line_kernel<Lat, N, T, Acc, Split, false><<<v.ntiles, v.tile_width, 0, v.stream>>>(a);
    } else {
        const dim3 grid((v.nx + kTile - 1) / kTile, v.ny, v.nz);
        step_box_kernel<Lat, N, T, Acc, Split><<<grid, kTile, 0, v.stream>>>(a);
    }
    return cudaGetLastError();
}

template <class Lat, int N, class T, class Acc>
cudaError_t launch_moments(const CtxView &v, const void *f, double *out, unsigned mask) {
    MomentArgs<Lat, N, T, Acc> m;
    m.s = make_args<Lat, T>(v, f, nullptr);
    m.out = out;
    m.ncells = v.ncells;
    m.mask = mask;
    m.line = v.line;
    m.fixedx = v.fixedx;
    if (v.line) {
        moments_kernel<Lat, N, T, Acc><<<v.ntiles, v.tile_width, 0, v.stream>>>(m);
    } else {
        const dim3 grid((v.nx + kTile - 1) / kTile, v.ny, v.nz);
        moments_kernel<Lat, N, T, Acc><<<grid, kTile, 0, v.stream>>>(m);
    }
    return cudaGetLastError();
}

template <class Lat, int N, class T>
cudaError_t launch_fill(const CtxView &v, void *f, const double *rho, const double *u,
                        const double *theta) {
    const StepArgs<Lat, T> a = make_args<Lat, T>(v, nullptr, f);
    if (v.line) {
        fill_kernel<Lat, N, T><<<v.ntiles, v.tile_width, 0, v.stream>>>(a, rho, u, theta, v.ncells, 1);
    } else {
        const long long nb = (v.ncells + kTile - 1) / kTile;
        fill_kernel<Lat, N, T><<<(unsigned)nb, kTile, 0, v.stream>>>(a, rho, u, theta, v.ncells, 0);
    }
    return cudaGetLastError();
}

template <class Lat, int N, class T>
cudaError_t launch_ghost(const CtxView &v, const double *states, int ninst, void *ghosts, double *ghostsd) {
    const StepArgs<Lat, T> a = make_args<Lat, T>(v, nullptr, nullptr);
    const int n = 2 * ninst;
    ghost_kernel<Lat, N, T><<<(n + 63) / 64, 64, 0, v.stream>>>(a, states, ninst, static_cast<T *>(ghosts),
                                                                 ghostsd);
    return cudaGetLastError();
}

// One cooperative launch (all blocks resident; the launch fails rather than waits when they
// do not fit) running nsteps steps of every tile; the state ends in fb for odd nsteps.
template <class Lat, int N, class T, class Acc, bool Split>
cudaError_t launch_persistent(const CtxView &v, void *fa, void *fb, int nsteps, int grid) {
    const StepArgs<Lat, T> a = make_args<Lat, T>(v, fa, fb);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(v.tile_width);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = v.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int ntiles = v.ntiles;
    unsigned *bar = v.bar;
    if constexpr (Split) {
        CUtensorMap ma, mb;
        if (line_encode_map<Lat>(v, fa, &ma) && line_encode_map<Lat>(v, fb, &mb)) {
            cfg.dynamicSmemBytes = LineStage<Lat>::persistent_bytes(v.tile_width);
            if (v.fixedx) {
                const cudaError_t e = line_smem_limit<step_line_persistent_staged<Lat, N, Acc, true>, Lat>();
                if (e != cudaSuccess) return e;
                return cudaLaunchKernelEx(&cfg, step_line_persistent_staged<Lat, N, Acc, true>, a, nsteps, ntiles, bar,
                                          ma, mb);
            }
            const cudaError_t e = line_smem_limit<step_line_persistent_staged<Lat, N, Acc, false>, Lat>();
            if (e != cudaSuccess) return e;
            return cudaLaunchKernelEx(&cfg, step_line_persistent_staged<Lat, N, Acc, false>, a, nsteps, ntiles, bar, ma,
                                      mb);
        }
    }
    if (v.fixedx)
        return cudaLaunchKernelEx(&cfg, step_line_persistent<Lat, N, T, Acc, Split, true>, a, nsteps, ntiles, bar);
    return cudaLaunchKernelEx(&cfg, step_line_persistent<Lat, N, T, Acc, Split, false>, a, nsteps, ntiles, bar);
}

template <class Lat, int N, class T, class Acc, bool Split>
int persistent_occupancy(const CtxView &v) {
    int n = 0;
    if constexpr (Split) {
        if (line_staging_applies<Lat>(v)) {
            const size_t smem = LineStage<Lat>::persistent_bytes(v.tile_width);
            cudaError_t e;
            if (v.fixedx) {
                e = line_smem_limit<step_line_persistent_staged<Lat, N, Acc, true>, Lat>();
                if (e == cudaSuccess)
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_line_persistent_staged<Lat, N, Acc, true>,
                                                                      v.tile_width, smem);
            } else {
                e = line_smem_limit<step_line_persistent_staged<Lat, N, Acc, false>, Lat>();
                if (e == cudaSuccess)
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_line_persistent_staged<Lat, N, Acc, false>,
                                                                      v.tile_width, smem);
            }
            return e == cudaSuccess ? n : 0;
        }
    }
    const cudaError_t e =
        v.fixedx ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_line_persistent<Lat, N, T, Acc, Split, true>,
                                                                 v.tile_width, 0)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_line_persistent<Lat, N, T, Acc, Split, false>,
                                                                 v.tile_width, 0);
    return e == cudaSuccess ? n : 0;
}

template <class Lat, int N, int P>
const KernelSet *kernel_set() {
    using T = typename std::conditional<P == 0, double, float>::type;
    using Acc = typename std::conditional<P == 1, float, double>::type;
    constexpr bool Split = (P == 2);
    static const KernelSet ks = {&launch_step<Lat, N, T, Acc, Split>, &launch_moments<Lat, N, T, Acc>,
                                 &launch_fill<Lat, N, T>, &launch_ghost<Lat, N, T>,
                                 &launch_persistent<Lat, N, T, Acc, Split>,
                                 &persistent_occupancy<Lat, N, T, Acc, Split>};
    return &ks;
}

// ------------------------------------------------------------------ tensor-product sets
template <class T>
TPArgs<T> make_tp_args(const CtxView &v, const void *fin, void *fout) {
    TPArgs<T> a;
    a.fin = static_cast<const T *>(fin);
    a.fout = static_cast<T *>(fout);
    a.inst = v.inst;
    a.tiles = v.tiles;
    a.ghosts = static_cast<const T *>(v.ghosts);
    a.ghostsd = v.ghostsd;
    a.health = v.health;
    a.plane_idx = v.plane_idx;
    a.stride = v.stride;
    for (int k = 0; k < kMaxQ1; ++k) a.w1[k] = v.w1[k];
    a.cd = v.c;
    a.step = v.step;
    a.tma = 0;
    return a;
}

// Tensor map of a state for the block-staged kernels: [Q planes][stride elements], box of
// kSeg x d (one x-row group of a W-warp block tile). False when the staging cannot use it
// (caller order differs from the library order, a plane stride or base address not on 16 bytes,
// coordinates beyond int32) or the driver refuses it; the kernels then copy plane by plane.
template <class L1, class T, int W>
bool tp_encode_map(const CtxView &v, const void *state, CUtensorMap *m) {
    constexpr int Q = L1::Q1 * L1::Q1 * L1::Q1;
    constexpr int kSeg = TPBlockStage<L1, T, W>::kSeg;
    const TensorMapEncodeFn enc = tensor_map_encoder();
    if (!enc || !v.plane_identity || !state) return false;
    if ((reinterpret_cast<unsigned long long>(state) & 15ull) != 0ull || (v.stride * (long long)sizeof(T)) % 16 != 0 ||
        v.stride + 2 * kSeg >= (1ll << 31))
        return false;
    const cuuint64_t dims[2] = {cuuint64_t(v.stride), cuuint64_t(Q)};
    const cuuint64_t strides[1] = {cuuint64_t(v.stride) * sizeof(T)};
    const cuuint32_t box[2] = {cuuint32_t(kSeg), cuuint32_t(L1::Q1)};
    const cuuint32_t estr[2] = {1u, 1u};
    return enc(m, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
               const_cast<void *>(state), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The block-staged kernels may take more than the default 48 KB of dynamic shared memory:
// raise the limit of each instantiation to what its block needs, once per device (the
// attribute belongs to the device the call is made on).
template <auto Kernel>
cudaError_t tp_smem_limit(size_t bytes) {
    constexpr int kDevices = 64;
    static std::atomic<int> state[kDevices];  // 0 not set, 1 set, 2 failed
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kDevices) return cudaErrorInvalidDevice;
    const int s = state[dev].load(std::memory_order_acquire);
    if (s == 1) return cudaSuccess;
    e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    state[dev].store(e == cudaSuccess ? 1 : 2, std::memory_order_release);
    return e;
}

// Tensor-product lines step in block tiles of tile_width cells (tile_width / 32 warps, one
// 32-cell row of the tile each); the other tensor-product kernels keep 32-cell tiles.
template <class L1, int N, class T, int W, bool FixedX, bool TC, bool Ident>
cudaError_t tp_launch_block(const CtxView &v, TPArgs<T> a, const void *fin) {
    constexpr size_t smem = TPBlockStage<L1, T, W>::kBytes;
    TPMaps maps;
    std::memset(&maps, 0, sizeof(maps));
    a.tma = tp_encode_map<L1, T, W>(v, fin, &maps.src) ? 1 : 0;
    a.tiles = v.btiles;
    const cudaError_t e = tp_smem_limit<tp_step_line_block<L1, N, T, W, FixedX, TC, Ident>>(smem);
    if (e != cudaSuccess) return e;
    tp_step_line_block<L1, N, T, W, FixedX, TC, Ident><<<v.nbtiles, 32 * W, smem, v.stream>>>(a, v.nbtiles, maps);
    return cudaGetLastError();
}

template <class L1, int N, class T, bool FixedX, bool TC, bool Ident>
cudaError_t tp_launch_block_w(const CtxView &v, const TPArgs<T> &a, const void *fin) {
    switch (v.tile_width) {
        case 32: return tp_launch_block<L1, N, T, 1, FixedX, TC, Ident>(v, a, fin);
        case 64:
            if constexpr (!TC) return tp_launch_block<L1, N, T, 2, FixedX, false, Ident>(v, a, fin);
            return cudaErrorInvalidConfiguration;
        case 128:
            if constexpr (!TC) return tp_launch_block<L1, N, T, 4, FixedX, false, Ident>(v, a, fin);
            return cudaErrorInvalidConfiguration;
        default: return cudaErrorInvalidConfiguration;
    }
}

template <class L1, int N, class T>
cudaError_t tp_launch_step(const CtxView &v, const void *fin, void *fout) {
    TPArgs<T> a = make_tp_args<T>(v, fin, fout);
    if (v.tile_width == 1) {  // one cell per block (D1Q9-P1 sets only: its tables fit in 48 KB)
        if constexpr (L1::Q1 == 9) {
            if (v.fixedx)
                tp_step_cell_kernel<L1, N, T, true><<<v.ntiles * 32, 128, 0, v.stream>>>(a);
            else
                tp_step_cell_kernel<L1, N, T, false><<<v.ntiles * 32, 128, 0, v.stream>>>(a);
            return cudaGetLastError();
        } else {
            return cudaErrorInvalidConfiguration;
        }
    }
    // the lines with fixed ends in the library's plane order (the shock runs) take a form that
    // stores without the plane table
    if constexpr (std::is_same<T, float>::value)
        if (v.fixedx && v.tensor_cores)
            return v.plane_identity ? tp_launch_block_w<L1, N, T, true, true, true>(v, a, fin)
                                    : tp_launch_block_w<L1, N, T, true, true, false>(v, a, fin);
    if (v.fixedx && v.plane_identity) return tp_launch_block_w<L1, N, T, true, false, true>(v, a, fin);
    if (v.fixedx) return tp_launch_block_w<L1, N, T, true, false, false>(v, a, fin);
    return tp_launch_block_w<L1, N, T, false, false, false>(v, a, fin);
}

template <class L1, int N, class T>
cudaError_t tp_launch_moments(const CtxView &v, const void *f, double *out, unsigned mask) {
    const TPArgs<T> a = make_tp_args<T>(v, f, nullptr);
    tp_moments_kernel<L1, N, T><<<v.ntiles, 32, 0, v.stream>>>(a, out, v.ncells, mask, v.fixedx);
    return cudaGetLastError();
}

template <class L1, int N, class T>
cudaError_t tp_launch_fill(const CtxView &v, void *f, const double *rho, const double *u, const double *theta) {
    const TPArgs<T> a = make_tp_args<T>(v, nullptr, f);
    tp_fill_kernel<L1, N, T><<<v.ntiles, 32, 0, v.stream>>>(a, rho, u, theta, v.ncells);
    return cudaGetLastError();
}

template <class L1, int N, class T>
cudaError_t tp_launch_ghost(const CtxView &v, const double *states, int ninst, void *ghosts, double *ghostsd) {
    const TPArgs<T> a = make_tp_args<T>(v, nullptr, nullptr);
    const int n = 2 * ninst;
    tp_ghost_kernel<L1, N, T><<<(n + 63) / 64, 64, 0, v.stream>>>(a, states, ninst, static_cast<T *>(ghosts), ghostsd);
    return cudaGetLastError();
}

// The persistent launch of the block-staged kernel (cooperative; grid given) and its number
// of resident blocks per SM.
template <class L1, int N, class T, int W, bool FixedX, bool TC, bool Ident>
cudaError_t tp_persist_block(const CtxView &v, TPArgs<T> a, void *fa, void *fb, int nsteps, int grid, int *occ) {
    constexpr size_t smem = TPBlockStage<L1, T, W>::kBytes;
    constexpr auto kernel = tp_step_line_persistent_block<L1, N, T, W, FixedX, TC, Ident>;
    cudaError_t e = tp_smem_limit<kernel>(smem);
    if (e != cudaSuccess) return e;
    if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kernel, 32 * W, smem);
    TPMaps maps;
    std::memset(&maps, 0, sizeof(maps));
    a.tma = (tp_encode_map<L1, T, W>(v, fa, &maps.src) && tp_encode_map<L1, T, W>(v, fb, &maps.dst)) ? 1 : 0;
    a.tiles = v.btiles;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32 * W);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = v.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int ntiles = v.nbtiles;
    unsigned *bar = v.bar;
    return cudaLaunchKernelEx(&cfg, kernel, a, nsteps, ntiles, bar, maps);
}

template <class L1, int N, class T, bool FixedX, bool TC, bool Ident>
cudaError_t tp_persist_block_w(const CtxView &v, const TPArgs<T> &a, void *fa, void *fb, int nsteps, int grid,
                               int *occ) {
    switch (v.tile_width) {
        case 32: return tp_persist_block<L1, N, T, 1, FixedX, TC, Ident>(v, a, fa, fb, nsteps, grid, occ);
        case 64:
            if constexpr (!TC)
                return tp_persist_block<L1, N, T, 2, FixedX, false, Ident>(v, a, fa, fb, nsteps, grid, occ);
            return cudaErrorInvalidConfiguration;
        case 128:
            if constexpr (!TC)
                return tp_persist_block<L1, N, T, 4, FixedX, false, Ident>(v, a, fa, fb, nsteps, grid, occ);
            return cudaErrorInvalidConfiguration;
        default: return cudaErrorInvalidConfiguration;
    }
}

// occ non-null: report the resident blocks per SM instead of launching
template <class L1, int N, class T>
cudaError_t tp_persist_dispatch(const CtxView &v, void *fa, void *fb, int nsteps, int grid, int *occ) {
    const TPArgs<T> a = make_tp_args<T>(v, fa, fb);
    if constexpr (std::is_same<T, float>::value)
        if (v.fixedx && v.tensor_cores)
            return v.plane_identity ? tp_persist_block_w<L1, N, T, true, true, true>(v, a, fa, fb, nsteps, grid, occ)
                                    : tp_persist_block_w<L1, N, T, true, true, false>(v, a, fa, fb, nsteps, grid, occ);
    if (v.fixedx && v.plane_identity)
        return tp_persist_block_w<L1, N, T, true, false, true>(v, a, fa, fb, nsteps, grid, occ);
    if (v.fixedx) return tp_persist_block_w<L1, N, T, true, false, false>(v, a, fa, fb, nsteps, grid, occ);
    return tp_persist_block_w<L1, N, T, false, false, false>(v, a, fa, fb, nsteps, grid, occ);
}

template <class L1, int N, class T>
cudaError_t tp_launch_persistent(const CtxView &v, void *fa, void *fb, int nsteps, int grid) {
    return tp_persist_dispatch<L1, N, T>(v, fa, fb, nsteps, grid, nullptr);
}

template <class L1, int N, class T>
int tp_persistent_occupancy(const CtxView &v) {
    int n = 0;
    const cudaError_t e = tp_persist_dispatch<L1, N, T>(v, nullptr, nullptr, 1, 1, &n);
    return e == cudaSuccess ? n : 0;
}

// P: 0 double, 1 float (the split precision has no tensor-product kernel)
template <class L1, int N, int P>
const KernelSet *tp_kernel_set() {
    using T = typename std::conditional<P == 0, double, float>::type;
    static const KernelSet ks = {&tp_launch_step<L1, N, T>,       &tp_launch_moments<L1, N, T>,
                                 &tp_launch_fill<L1, N, T>,       &tp_launch_ghost<L1, N, T>,
                                 &tp_launch_persistent<L1, N, T>, &tp_persistent_occupancy<L1, N, T>};
    return &ks;
}

}  // namespace smrt

#include "adjoint_kernels.cuh"

namespace smrt {

using AdjStepFn = cudaError_t (*)(const CtxView &, const void *f, const double *lam_next, double *lam_t,
                                  double *partials, double *dtau);
using AdjMomentsFn = cudaError_t (*)(const CtxView &, const void *f, const double *gbar, unsigned mask,
                                     double *lam);
struct AdjointSet {
    AdjStepFn step;
    AdjMomentsFn moments;
};
const AdjointSet *adjoints_d3q39(int N, int precision);
const AdjointSet *adjoints_d3q103(int N, int precision);
const AdjointSet *adjoints_d3q729(int N, int precision);
const AdjointSet *adjoints_d3q4913(int N, int precision);

template <class Lat, class T>
AdjArgs<Lat, T> make_adj_args(const CtxView &v, const void *f) {
    AdjArgs<Lat, T> A;
    A.s = make_args<Lat, T>(v, f, nullptr);
    for (int p = 0; p <= Lat::NP; ++p) A.wpd[p] = v.wp[p];
    A.c = v.c;
    A.line = v.line;
    A.fixedx = v.fixedx;
    A.ncells = v.ncells;
    A.mask = 0;
    A.lam_in = nullptr;
    A.lam_out = nullptr;
    A.partials = nullptr;
    return A;
}

inline long long adj_blocks(const CtxView &v) {
    return v.line ? (long long)v.ntiles : (long long)((v.nx + kTile - 1) / kTile) * v.ny * v.nz;
}

template <class Lat, int N, class T>
cudaError_t launch_adj_step(const CtxView &v, const void *f, const double *lam_next, double *lam_t,
                            double *partials, double *dtau) {
    AdjArgs<Lat, T> A = make_adj_args<Lat, T>(v, f);
    A.lam_in = lam_next;
    A.lam_out = lam_t;
    A.partials = partials;
    if (v.line) {
        adjoint_step_kernel<Lat, N, T><<<v.ntiles, v.tile_width, 0, v.stream>>>(A);
    } else {
        const dim3 grid((v.nx + kTile - 1) / kTile, v.ny, v.nz);
        adjoint_step_kernel<Lat, N, T><<<grid, kTile, 0, v.stream>>>(A);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_partials_kernel<<<1, 32, 0, v.stream>>>(partials, adj_blocks(v), ntau(N), dtau);
    return cudaGetLastError();
}

template <class Lat, int N, class T>
cudaError_t launch_adj_moments(const CtxView &v, const void *f, const double *gbar, unsigned mask, double *lam) {
    AdjArgs<Lat, T> A = make_adj_args<Lat, T>(v, f);
    A.lam_in = gbar;
    A.lam_out = lam;
    A.mask = mask;
    if (v.line) {
        adjoint_moments_kernel<Lat, N, T><<<v.ntiles, v.tile_width, 0, v.stream>>>(A);
    } else {
        const dim3 grid((v.nx + kTile - 1) / kTile, v.ny, v.nz);
        adjoint_moments_kernel<Lat, N, T><<<grid, kTile, 0, v.stream>>>(A);
    }
    return cudaGetLastError();
}

template <class Lat, int N, int P>
const AdjointSet *adjoint_set() {
    using T = typename std::conditional<P == 0, double, float>::type;
    static const AdjointSet as = {&launch_adj_step<Lat, N, T>, &launch_adj_moments<Lat, N, T>};
    return &as;
}

}  // namespace smrt

#include "tensor_adjoint.cuh"

namespace smrt {

// Tensor-product sets: 32-cell tiles, one thread per cell (tensor_adjoint.cuh).
template <class L1, int N, class T>
cudaError_t tp_launch_adj_step(const CtxView &v, const void *f, const double *lam_next, double *lam_t,
                               double *partials, double *dtau) {
    const TPArgs<T> a = make_tp_args<T>(v, f, nullptr);
    if (v.fixedx)
        tp_adjoint_step_kernel<L1, N, T, true><<<v.ntiles, 32, 0, v.stream>>>(a, lam_next, lam_t, partials);
    else
        tp_adjoint_step_kernel<L1, N, T, false><<<v.ntiles, 32, 0, v.stream>>>(a, lam_next, lam_t, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_partials_kernel<<<1, 32, 0, v.stream>>>(partials, (long long)v.ntiles, ntau(N), dtau);
    return cudaGetLastError();
}

template <class L1, int N, class T>
cudaError_t tp_launch_adj_moments(const CtxView &v, const void *f, const double *gbar, unsigned mask, double *lam) {
    const TPArgs<T> a = make_tp_args<T>(v, f, nullptr);
    if (v.fixedx)
        tp_adjoint_moments_kernel<L1, N, T, true><<<v.ntiles, 32, 0, v.stream>>>(a, gbar, mask, lam, v.ncells);
    else
        tp_adjoint_moments_kernel<L1, N, T, false><<<v.ntiles, 32, 0, v.stream>>>(a, gbar, mask, lam, v.ncells);
    return cudaGetLastError();
}

template <class L1, int N, int P>
const AdjointSet *tp_adjoint_set() {
    using T = typename std::conditional<P == 0, double, float>::type;
    static const AdjointSet as = {&tp_launch_adj_step<L1, N, T>, &tp_launch_adj_moments<L1, N, T>};
    return &as;
}

}  // namespace smrt
