// api.cu -- the extern "C" entry points of libsmrt (declared and documented in smrt.h).
// Host-side validation, the context's small device tables, and dispatch to the kernels
// instantiated per velocity set and precision.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/smrt.h"
#include "dispatch.h"

namespace smrt {
double quadrature_defect(int q, const int8_t *e, const double *w, double c, int degree);
const KernelSet *kernels_d3q39_p0(int N);
const KernelSet *kernels_d3q39_p1(int N);
const KernelSet *kernels_d3q39_p2(int N);
const KernelSet *kernels_d3q103_p0(int N);
const KernelSet *kernels_d3q103_p1(int N);
const KernelSet *kernels_d3q103_p2(int N);
const KernelSet *kernels_d3q729_p0(int N);
const KernelSet *kernels_d3q729_p1(int N);
const KernelSet *kernels_d3q4913_p0(int N);
const KernelSet *kernels_d3q4913_p1(int N);
}  // namespace smrt

using namespace smrt;

struct lb_ctx {
    int kind;  // 0 D3Q39, 1 D3Q103, 2 D3Q729 (D1Q9-P1 cubed), 3 D3Q4913 (D1Q17-P1 cubed)
    int q, np, N, degree;
    lb_precision prec;
    size_t elem;  // bytes per population value
    const KernelSet *ks;
    const AdjointSet *as;
    CtxView view;
    std::vector<int> perm;  // library index -> caller index
    std::vector<int> nx_inst;
    int batch;
    size_t ncells, stride;
    std::vector<InstanceInfo> h_inst;
    std::vector<double> h_states;  // [instance][side][rho, ux, uy, uz, theta]
    bool relax_set;
    // settings not yet on the device: the instance table, and the end states of instances
    // [ghost_lo, ghost_hi) (flush_tables uploads them before the next launch)
    bool tables_dirty;
    int ghost_lo, ghost_hi;
    // device tables owned by the context
    InstanceInfo *d_inst;
    int2 *d_tiles;
    int2 *d_btiles;      // tensor-product lines: block tiles of the step kernels (tile_width cells)
    int *d_plane;        // tensor-product sets: caller plane of each library population
    void *d_ghosts;
    double *d_ghostsd;
    double *d_states;
    unsigned *d_health;  // [0] health flags, [1..3] grid barrier and step counter
    double *d_partials;  // per-block relaxation-time gradients of lb_step_adjoint
    long long max_tiles; // tile capacity (32-cell tiles) of d_tiles, d_btiles and d_partials
    int btile_width;     // cells per block tile in d_btiles
    lb_schedule sched;
    int num_sms;
    // cached graph of the persistent launch (lb_step_graph)
    cudaGraphExec_t graph;
    cudaStream_t capture_stream;
    const void *graph_fa, *graph_fb;
    int graph_steps;
    lb_schedule graph_sched;
};

namespace {

std::vector<int2> make_tiles(const std::vector<int> &nx_inst, int width) {
    std::vector<int2> tiles;
    for (int j = 0; j < (int)nx_inst.size(); ++j)
        for (int x0 = 0; x0 < nx_inst[j]; x0 += width) tiles.push_back(make_int2(j, x0));
    return tiles;
}

template <class Lat>
bool match_set(const lb_lattice_desc *d, std::vector<int> &perm) {
    if (d->q != Lat::Q) return false;
    perm.assign(Lat::Q, -1);
    std::vector<char> used(d->q, 0);
    auto find = [&](int x, int y, int z) {
        for (int i = 0; i < d->q; ++i)
            if (!used[i] && d->e[3 * i] == x && d->e[3 * i + 1] == y && d->e[3 * i + 2] == z) return i;
        return -1;
    };
    int r = find(0, 0, 0);
    if (r < 0) return false;
    used[r] = 1;
    perm[0] = r;
    for (int p = 0; p < Lat::NP; ++p) {
        for (int s = 0; s < 2; ++s) {
            const int sg = s == 0 ? 1 : -1;
            const int i = find(sg * Lat::e(p, 0), sg * Lat::e(p, 1), sg * Lat::e(p, 2));
            if (i < 0) return false;
            used[i] = 1;
            perm[2 * p + 1 + s] = i;
        }
    }
    return true;
}

// A tensor-product set (Sec. 4.2): every velocity (e_a, e_b, e_c) of the 1D rule's abscissae
// present once, with weight w_a w_b w_c. The 1D weights are read off the axis velocities:
// w(0,0,0) = w_0^3 and w(e_a,0,0) = w_a w_0^2.
template <class L1>
bool match_tensor(const lb_lattice_desc *d, std::vector<int> &perm, double (&w1)[kMaxQ1]) {
    constexpr int Q1 = L1::Q1;
    if (d->q != Q1 * Q1 * Q1) return false;
    perm.assign(d->q, -1);
    std::map<long long, int> where;  // velocity -> caller index
    auto key = [](int x, int y, int z) { return ((long long)(x + 128) << 16) | ((y + 128) << 8) | (z + 128); };
    for (int k = 0; k < d->q; ++k)
        if (!where.emplace(key(d->e[3 * k], d->e[3 * k + 1], d->e[3 * k + 2]), k).second) return false;
    for (int i = 0; i < d->q; ++i) {
        const int a = i % Q1, b = (i / Q1) % Q1, cc = i / (Q1 * Q1);
        const auto it = where.find(key(e1<L1>(a), e1<L1>(b), e1<L1>(cc)));
        if (it == where.end()) return false;
        perm[i] = it->second;
    }
    const double w0 = std::cbrt(d->w[perm[0]]);
    for (int a = 0; a < Q1; ++a) w1[a] = d->w[perm[a]] / (w0 * w0);
    for (int a = Q1; a < kMaxQ1; ++a) w1[a] = 0.0;
    for (int p = 0; p < L1::NP1; ++p)  // the rebuild folds +e and -e: they share a weight
        if (std::fabs(w1[2 * p + 1] - w1[2 * p + 2]) > 1e-14 * w1[2 * p + 1]) return false;
    for (int i = 0; i < d->q; ++i) {
        const double want = w1[i % Q1] * w1[(i / Q1) % Q1] * w1[i / (Q1 * Q1)];
        if (std::fabs(d->w[perm[i]] - want) > 1e-12 * want) return false;
    }
    return true;
}

template <class Lat>
int max_reach(int axis) {
    int m = 0;
    for (int p = 0; p < Lat::NP; ++p) m = std::max(m, std::abs(Lat::e(p, axis)));
    return m;
}

lb_status cuda_status(cudaError_t e) { return e == cudaSuccess ? LB_OK : LB_ERR_CUDA; }

void free_tables(lb_ctx *c) {
    if (!c) return;
    cudaFree(c->d_inst);
    cudaFree(c->d_tiles);
    cudaFree(c->d_btiles);
    cudaFree(c->d_plane);
    cudaFree(c->d_ghosts);
    cudaFree(c->d_ghostsd);
    cudaFree(c->d_states);
    cudaFree(c->d_health);
    cudaFree(c->d_partials);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
}

}  // namespace

extern "C" lb_status lb_init_lattice(lb_ctx **out, const lb_lattice_desc *lat, const lb_grid_desc *grid,
                                     int N, lb_precision prec, void *stream) {
    if (!out || !lat || !grid || !lat->e || !lat->w) return LB_ERR_INVALID;
    *out = nullptr;
    if (prec != LB_F64 && prec != LB_F32 && prec != LB_F32_CONS64) return LB_ERR_INVALID;
    if (!(lat->c > 0.0) || lat->q <= 0 || lat->q > kMaxQTP) return LB_ERR_INVALID;
    if (N < 2 || lat->degree < 2 * N) return LB_ERR_INVALID;
    if (grid->batch < 1 || grid->nx < 0 || grid->ny < 1 || grid->nz < 1) return LB_ERR_INVALID;
    if (grid->bc_x != 0 && grid->bc_x != 1) return LB_ERR_INVALID;
    for (int i = 0; i < lat->q; ++i)
        if (!(lat->w[i] > 0.0)) return LB_ERR_INVALID;
    // the set must integrate every monomial of degree <= 2N exactly (Sec. 3, Eq. an)
    if (quadrature_defect(lat->q, lat->e, lat->w, lat->c, 2 * N) > 1e-9) return LB_ERR_INVALID;

    lb_ctx *c = new (std::nothrow) lb_ctx();
    if (!c) return LB_ERR_NOMEM;
    c->q = lat->q;
    c->N = N;
    c->degree = lat->degree;
    c->prec = prec;
    c->elem = prec == LB_F64 ? sizeof(double) : sizeof(float);
    int reach[3] = {0, 0, 0};
    double w1[kMaxQ1] = {0.0};
    const bool t729 = match_tensor<D1Q9P1>(lat, c->perm, w1);
    const bool t4913 = !t729 && match_tensor<D1Q17P1>(lat, c->perm, w1);
    const bool tensor = t729 || t4913;
    if (tensor) {
        c->kind = t729 ? 2 : 3;
        c->np = 0;
        for (int k = 0; k < 3; ++k) reach[k] = t729 ? D1Q9P1::E(D1Q9P1::NP1 - 1) : D1Q17P1::E(D1Q17P1::NP1 - 1);
        if (t729)
            c->ks = prec == LB_F64 ? kernels_d3q729_p0(N) : (prec == LB_F32 ? kernels_d3q729_p1(N) : nullptr);
        else
            c->ks = prec == LB_F64 ? kernels_d3q4913_p0(N) : (prec == LB_F32 ? kernels_d3q4913_p1(N) : nullptr);
        c->as = t729 ? adjoints_d3q729(N, prec) : adjoints_d3q4913(N, prec);
        // batched 1D lines only, shifted along x only
        if (grid->ny != 1 || grid->nz != 1 || lat->shift[1] != 0 || lat->shift[2] != 0) c->ks = nullptr;
    } else if (match_set<D3Q39>(lat, c->perm)) {
        c->kind = 0;
        c->np = D3Q39::NP;
        for (int k = 0; k < 3; ++k) reach[k] = max_reach<D3Q39>(k);
        c->ks = prec == LB_F64 ? kernels_d3q39_p0(N) : (prec == LB_F32 ? kernels_d3q39_p1(N) : kernels_d3q39_p2(N));
        c->as = adjoints_d3q39(N, prec);
    } else if (match_set<D3Q103>(lat, c->perm)) {
        c->kind = 1;
        c->np = D3Q103::NP;
        for (int k = 0; k < 3; ++k) reach[k] = max_reach<D3Q103>(k);
        c->ks = prec == LB_F64 ? kernels_d3q103_p0(N) : (prec == LB_F32 ? kernels_d3q103_p1(N) : kernels_d3q103_p2(N));
        c->as = adjoints_d3q103(N, prec);
    } else {
        delete c;
        return LB_ERR_UNSUPPORTED;
    }
    if (!c->ks) {
        delete c;
        return LB_ERR_UNSUPPORTED;
    }
    // pair members must share a weight (the rebuild folds +e and -e)
    for (int p = 0; p < c->np; ++p) {
        const double wa = lat->w[c->perm[2 * p + 1]], wb = lat->w[c->perm[2 * p + 2]];
        if (std::fabs(wa - wb) > 1e-14 * wa) {
            delete c;
            return LB_ERR_INVALID;
        }
    }

    // geometry
    const bool line = (grid->ny == 1 && grid->nz == 1);
    c->batch = grid->batch;
    if (grid->batch > 1 && !line) {
        delete c;
        return LB_ERR_INVALID;
    }
    if (grid->bc_x == 1 && !line) {
        delete c;
        return LB_ERR_UNSUPPORTED;
    }
    if (grid->batch > 1 && !grid->nx_per_instance) {
        delete c;
        return LB_ERR_INVALID;
    }
    c->nx_inst.resize(grid->batch);
    for (int j = 0; j < grid->batch; ++j) {
        c->nx_inst[j] = grid->nx_per_instance ? grid->nx_per_instance[j] : grid->nx;
        if (c->nx_inst[j] < 1) {
            delete c;
            return LB_ERR_INVALID;
        }
    }
    const int k0 = lat->shift[0], k1 = lat->shift[1], k2 = lat->shift[2];
    // periodic axes wrap at most once: reach + |shift| <= extent
    if (!line) {
        if (reach[0] + std::abs(k0) > grid->nx || reach[1] + std::abs(k1) > grid->ny ||
            reach[2] + std::abs(k2) > grid->nz) {
            delete c;
            return LB_ERR_INVALID;
        }
    } else if (grid->bc_x == 0) {
        for (int j = 0; j < grid->batch; ++j)
            if (reach[0] + std::abs(k0) > c->nx_inst[j]) {
                delete c;
                return LB_ERR_INVALID;
            }
    }
    size_t ncells = 0;
    c->h_inst.resize(grid->batch);
    std::vector<int2> tiles;
    for (int j = 0; j < grid->batch; ++j) {
        InstanceInfo &in = c->h_inst[j];
        std::memset(&in, 0, sizeof(in));
        in.cell_off = (long long)ncells;
        in.nx = c->nx_inst[j];
        in.kx = k0;
        ncells += line ? (size_t)in.nx : (size_t)grid->nx * grid->ny * grid->nz;
    }
    // tensor-product contexts keep a table of 32-cell tiles (the moments, fill and adjoint
    // kernels) and step in block tiles of the schedule's width. Default widths, as measured:
    // float states stage best in 128-cell tiles; double ones, bound by the FP64 pipe, in one-warp
    // blocks on D3Q729 and two-warp ones on D3Q4913 (whose stage buffers are twice the size)
    const int width0 = tensor ? (prec != LB_F64 ? 128 : (c->kind == 3 ? 64 : 32)) : kTile;
    if (line) tiles = make_tiles(c->nx_inst, tensor ? 32 : width0);
    c->max_tiles = line ? (long long)make_tiles(c->nx_inst, 32).size() : 0;
    c->sched.tile_width = line ? width0 : kTile;
    c->sched.blocks_per_sm = 0;
    c->sched.persistent = 0;
    c->sched.tensor_cores = 0;
    c->sched.ms_per_step = 0.0;
    c->ncells = ncells;
    c->stride = (ncells + 63) / 64 * 64;  // planes start on 256-byte boundaries (float)
    c->h_states.assign((size_t)grid->batch * 10, 0.0);

    CtxView &v = c->view;
    std::memset(&v, 0, sizeof(v));
    v.stream = static_cast<cudaStream_t>(stream);
    if (!tensor) {
        for (int i = 0; i < c->q; ++i) v.plane[i] = (long long)c->perm[i] * (long long)c->stride;
        v.wp[0] = lat->w[c->perm[0]];
        for (int p = 0; p < c->np; ++p) v.wp[p + 1] = lat->w[c->perm[2 * p + 1]];
    }
    for (int k = 0; k < kMaxQ1; ++k) v.w1[k] = w1[k];
    v.plane_identity = 1;
    for (int i = 0; i < c->q; ++i)
        if (c->perm[i] != i) v.plane_identity = 0;
    v.stride = (long long)c->stride;
    v.c = lat->c;
    v.nx = line ? c->nx_inst[0] : grid->nx;
    v.ny = grid->ny;
    v.nz = grid->nz;
    v.kx = k0;
    v.ky = k1;
    v.kz = k2;
    v.line = line ? 1 : 0;
    v.fixedx = grid->bc_x;
    v.ntiles = (int)tiles.size();
    v.ncells = (long long)ncells;
    v.tile_width = line ? width0 : kTile;

    cudaError_t e = cudaSuccess;
    e = cudaMalloc(&c->d_inst, sizeof(InstanceInfo) * grid->batch);
    if (e == cudaSuccess && line) e = cudaMalloc(&c->d_tiles, sizeof(int2) * c->max_tiles);
    if (e == cudaSuccess && line && tensor) e = cudaMalloc(&c->d_btiles, sizeof(int2) * c->max_tiles);
    if (e == cudaSuccess && tensor) e = cudaMalloc(&c->d_plane, sizeof(int) * c->q);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_ghosts, c->elem * c->q * 2 * grid->batch);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_ghostsd, sizeof(double) * c->q * 2 * grid->batch);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_states, sizeof(double) * 10 * grid->batch);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_health, 16);
    if (e == cudaSuccess)
        e = cudaMalloc(&c->d_partials, sizeof(double) * kMaxTau * std::max(1LL, line ? c->max_tiles : adj_blocks(v)));
    if (e == cudaSuccess) {
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    // D3Q729 problems of at most 48 (double) or 32 (float) cells per SM take one block per cell
    // (measured crossovers with the tiled kernel)
    if (e == cudaSuccess && c->kind == 2 && (long long)ncells <= (prec == LB_F64 ? 48LL : 32LL) * c->num_sms) {
        c->sched.tile_width = 1;
        v.tile_width = 1;
    }
    if (e != cudaSuccess) {
        free_tables(c);
        delete c;
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? LB_ERR_NOMEM : LB_ERR_CUDA;
    }
    if (!tiles.empty())
        e = cudaMemcpyAsync(c->d_tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, v.stream);
    // block tiles of the default width (a one-cell-per-block schedule leaves them unused until a
    // tiled width is set)
    const std::vector<int2> btiles = line && tensor ? make_tiles(c->nx_inst, width0) : std::vector<int2>();
    if (e == cudaSuccess && !btiles.empty())
        e = cudaMemcpyAsync(c->d_btiles, btiles.data(), sizeof(int2) * btiles.size(), cudaMemcpyHostToDevice,
                            v.stream);
    v.nbtiles = (int)btiles.size();
    c->btile_width = width0;
    if (e == cudaSuccess && tensor)
        e = cudaMemcpyAsync(c->d_plane, c->perm.data(), sizeof(int) * c->q, cudaMemcpyHostToDevice, v.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_health, 0, 16, v.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_ghosts, 0, c->elem * c->q * 2 * grid->batch, v.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_ghostsd, 0, sizeof(double) * c->q * 2 * grid->batch, v.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_inst, c->h_inst.data(), sizeof(InstanceInfo) * grid->batch,
                            cudaMemcpyHostToDevice, v.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(v.stream);
    if (e != cudaSuccess) {
        free_tables(c);
        delete c;
        return LB_ERR_CUDA;
    }
    v.inst = c->d_inst;
    v.tiles = c->d_tiles;
    v.btiles = c->d_btiles;
    v.plane_idx = c->d_plane;
    v.ghosts = c->d_ghosts;
    v.ghostsd = c->d_ghostsd;
    v.health = c->d_health;
    v.bar = c->d_health + 1;
    c->relax_set = false;
    c->tables_dirty = false;
    c->ghost_lo = grid->batch;
    c->ghost_hi = 0;
    *out = c;
    return LB_OK;
}

namespace {

// Upload what lb_set_relaxation, lb_set_frame_shift and lb_set_collision_model changed since the
// last launch: the instance table, then the end-state populations of the instances whose end
// states or frame changed, in one launch over their range; synchronises once (the host tables
// are reused by the next setting).
lb_status flush_tables(lb_ctx *c) {
    if (!c->tables_dirty) return LB_OK;
    cudaStream_t st = c->view.stream;
    cudaError_t e = cudaMemcpyAsync(c->d_inst, c->h_inst.data(), sizeof(InstanceInfo) * c->batch,
                                    cudaMemcpyHostToDevice, st);
    const int j0 = c->ghost_lo, j1 = c->ghost_hi;
    if (e == cudaSuccess && c->view.fixedx && j0 < j1) {
        e = cudaMemcpyAsync(c->d_states, c->h_states.data(), sizeof(double) * 10 * c->batch, cudaMemcpyHostToDevice,
                            st);
        if (e == cudaSuccess) {
            // a view whose instance table starts at j0
            CtxView gv = c->view;
            gv.inst = c->d_inst + j0;
            e = c->ks->ghost(gv, c->d_states + 10 * (size_t)j0, j1 - j0,
                             static_cast<char *>(c->d_ghosts) + c->elem * c->q * 2 * (size_t)j0,
                             c->d_ghostsd + (size_t)c->q * 2 * j0);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return LB_ERR_CUDA;
    c->tables_dirty = false;
    c->ghost_lo = c->batch;
    c->ghost_hi = 0;
    return LB_OK;
}

// The adjoint kernels differentiate the SMRT collision only.
bool any_es_bgk(const lb_ctx *c) {
    for (const InstanceInfo &in : c->h_inst)
        if (in.model != LB_MODEL_SMRT) return true;
    return false;
}

void mark_ghosts(lb_ctx *c, int j0, int j1) {
    c->tables_dirty = true;
    if (!c->view.fixedx) return;
    c->ghost_lo = std::min(c->ghost_lo, j0);
    c->ghost_hi = std::max(c->ghost_hi, j1);
}

}  // namespace

extern "C" lb_status lb_set_relaxation(lb_ctx *c, const double *tau, int maxwell, double rho_ref,
                                       const lb_state *left, const lb_state *right, int instance) {
    if (!c || !tau) return LB_ERR_INVALID;
    if (maxwell != 0 && maxwell != 1) return LB_ERR_INVALID;
    if (maxwell && !(rho_ref > 0.0)) return LB_ERR_INVALID;
    if (instance < -1 || instance >= c->batch) return LB_ERR_INVALID;
    const int nt = ntau(c->N);
    for (int k = 0; k < nt; ++k)
        if (!(tau[k] > 0.0) || !std::isfinite(tau[k])) return LB_ERR_INVALID;
    if (c->view.fixedx) {
        if (!left || !right) return LB_ERR_INVALID;
        for (const lb_state *s : {left, right})
            if (!(s->rho > 0.0) || !(s->theta > 0.0) || !std::isfinite(s->u[0]) ||
                !std::isfinite(s->u[1]) || !std::isfinite(s->u[2]))
                return LB_ERR_INVALID;
    }
    const int j0 = instance < 0 ? 0 : instance, j1 = instance < 0 ? c->batch : instance + 1;
    for (int j = j0; j < j1; ++j) {
        InstanceInfo &in = c->h_inst[j];
        for (int k = 0; k < nt; ++k) {
            in.tauA[k] = maxwell ? tau[k] * rho_ref : 0.0;
            in.tauB[k] = maxwell ? 0.5 : tau[k] + 0.5;
            in.tauAf[k] = (float)in.tauA[k];
            in.tauBf[k] = (float)in.tauB[k];
        }
        in.dAdt = maxwell ? rho_ref : 0.0;
        in.dBdt = maxwell ? 0.0 : 1.0;
        if (c->view.fixedx) {
            double *s = &c->h_states[(size_t)j * 10];
            const lb_state *st[2] = {left, right};
            for (int side = 0; side < 2; ++side) {
                s[5 * side + 0] = st[side]->rho;
                s[5 * side + 1] = st[side]->u[0];
                s[5 * side + 2] = st[side]->u[1];
                s[5 * side + 3] = st[side]->u[2];
                s[5 * side + 4] = st[side]->theta;
            }
        }
    }
    mark_ghosts(c, j0, j1);
    c->relax_set = true;
    return LB_OK;
}

extern "C" lb_status lb_set_frame_shift(lb_ctx *c, int instance, int kx) {
    if (!c || instance < -1 || instance >= c->batch) return LB_ERR_INVALID;
    if (!c->view.line && instance != -1) return LB_ERR_INVALID;
    const int j0 = instance < 0 ? 0 : instance, j1 = instance < 0 ? c->batch : instance + 1;
    for (int j = j0; j < j1; ++j) c->h_inst[j].kx = kx;
    if (!c->view.line) c->view.kx = kx;
    if (c->relax_set)
        mark_ghosts(c, j0, j1);  // end states already set are rebuilt in the new frame
    else
        c->tables_dirty = true;
    return LB_OK;
}

extern "C" lb_status lb_set_collision_model(lb_ctx *c, int instance, int model, double b) {
    if (!c || instance < -1 || instance >= c->batch) return LB_ERR_INVALID;
    if (model != LB_MODEL_SMRT && model != LB_MODEL_ES_BGK) return LB_ERR_INVALID;
    if (model == LB_MODEL_ES_BGK && !(b >= -0.5 && b < 1.0)) return LB_ERR_INVALID;
    const int j0 = instance < 0 ? 0 : instance, j1 = instance < 0 ? c->batch : instance + 1;
    for (int j = j0; j < j1; ++j) {
        c->h_inst[j].model = model;
        c->h_inst[j].es_b = model == LB_MODEL_ES_BGK ? b : 0.0;
    }
    c->tables_dirty = true;
    return LB_OK;
}

extern "C" lb_status lb_fill_equilibrium(lb_ctx *c, void *f, const double *rho, const double *u,
                                         const double *theta) {
    if (!c || !f || !rho || !u || !theta) return LB_ERR_INVALID;
    const lb_status fs = flush_tables(c);
    if (fs != LB_OK) return fs;
    return cuda_status(c->ks->fill(c->view, f, rho, u, theta));
}

namespace {

lb_status check_pair(const lb_ctx *c, const void *fa, const void *fb, int nsteps) {
    if (!c || !fa || !fb || fa == fb || nsteps < 1) return LB_ERR_INVALID;
    if (!c->relax_set) return LB_ERR_INVALID;
    const size_t bytes = c->elem * lb_state_elems(c);
    const char *a0 = static_cast<const char *>(fa), *b0 = static_cast<const char *>(fb);
    if (a0 < b0 + bytes && b0 < a0 + bytes) return LB_ERR_INVALID;  // overlap
    // the tensor-product kernels copy population segments with the bulk-copy engine, which
    // needs 16-byte aligned addresses
    if (c->kind >= 2 && ((reinterpret_cast<uintptr_t>(fa) | reinterpret_cast<uintptr_t>(fb)) & 15u))
        return LB_ERR_INVALID;
    return LB_OK;
}

// grid of the persistent launch: blocks_per_sm (0 = as many as fit) on every SM, at most one
// block per tile
long long persistent_grid(const lb_ctx *c) {
    // blocks with work: one per tile (block tiles on tensor-product sets, whose
    // one-cell-per-block schedule, tile width 1, has no persistent form)
    if (c->kind >= 2 && c->view.tile_width < 32) return 0;
    const int occ = c->ks->occupancy(c->view);
    if (occ < 1) return 0;
    const int bps = c->sched.blocks_per_sm > 0 ? std::min(c->sched.blocks_per_sm, occ) : occ;
    const long long needed = c->kind >= 2 ? c->view.nbtiles : c->view.ntiles;
    return std::max(1LL, std::min((long long)bps * c->num_sms, needed));
}

cudaError_t launch_persistent(lb_ctx *c, const CtxView &v, void *fa, void *fb, int nsteps) {
    const long long grid = persistent_grid(c);
    if (grid < 1) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaMemsetAsync(c->d_health + 1, 0, sizeof(unsigned), v.stream);  // arrivals
    if (e == cudaSuccess) e = c->ks->persist(v, fa, fb, nsteps, (int)grid);
    return e;
}

}  // namespace

extern "C" lb_status lb_step(lb_ctx *c, void *fa, void *fb, int nsteps) {
    lb_status st = check_pair(c, fa, fb, nsteps);
    if (st == LB_OK) st = flush_tables(c);
    if (st != LB_OK) return st;
    if (c->view.line && c->sched.persistent) return cuda_status(launch_persistent(c, c->view, fa, fb, nsteps));
    void *src = fa, *dst = fb;
    for (int s = 0; s < nsteps; ++s) {
        c->view.step++;
        const cudaError_t e = c->ks->step(c->view, src, dst);
        if (e != cudaSuccess) return LB_ERR_CUDA;
        std::swap(src, dst);
    }
    return LB_OK;
}

extern "C" lb_status lb_set_schedule(lb_ctx *c, const lb_schedule *s) {
    if (!c || !s) return LB_ERR_INVALID;
    const bool cell_blocks = s->tile_width == 1;  // D3Q729: one cell per block, one launch per step
    if (s->tile_width != 32 && s->tile_width != 64 && s->tile_width != 128 && !cell_blocks) return LB_ERR_INVALID;
    if (cell_blocks && (c->kind != 2 || s->persistent)) return LB_ERR_UNSUPPORTED;
    if (s->blocks_per_sm < 0 || (s->persistent != 0 && s->persistent != 1)) return LB_ERR_INVALID;
    if (s->tensor_cores != 0 && s->tensor_cores != 1) return LB_ERR_INVALID;
    // tensor-core x-rows: the block-staged kernels of float tensor-product lines with fixed ends
    if (s->tensor_cores && (c->kind < 2 || c->prec != LB_F32 || !c->view.line || !c->view.fixedx || s->tile_width != 32))
        return LB_ERR_UNSUPPORTED;
    if (!c->view.line) {  // the box kernel has one fixed launch shape
        if (s->persistent || s->tile_width != kTile) return LB_ERR_UNSUPPORTED;
        c->sched = *s;
        return LB_OK;
    }
    if (c->kind >= 2) {
        // the 32-cell tiles stay; the step kernels' block tiles follow the width
        if (!cell_blocks && s->tile_width != c->btile_width) {
            const std::vector<int2> bt = make_tiles(c->nx_inst, s->tile_width);
            if ((long long)bt.size() > c->max_tiles) return LB_ERR_INVALID;
            cudaError_t e = cudaMemcpyAsync(c->d_btiles, bt.data(), sizeof(int2) * bt.size(), cudaMemcpyHostToDevice,
                                            c->view.stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->view.stream);
            if (e != cudaSuccess) return LB_ERR_CUDA;
            c->view.nbtiles = (int)bt.size();
            c->btile_width = s->tile_width;
        }
        c->view.tile_width = s->tile_width;
    } else if (s->tile_width != c->view.tile_width) {
        const std::vector<int2> tiles = make_tiles(c->nx_inst, s->tile_width);
        if ((long long)tiles.size() > c->max_tiles) return LB_ERR_INVALID;
        cudaError_t e = cudaMemcpyAsync(c->d_tiles, tiles.data(), sizeof(int2) * tiles.size(),
                                        cudaMemcpyHostToDevice, c->view.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->view.stream);
        if (e != cudaSuccess) return LB_ERR_CUDA;
        c->view.ntiles = (int)tiles.size();
        c->view.tile_width = s->tile_width;
    }
    c->sched = *s;
    c->view.tensor_cores = s->tensor_cores;
    if (c->sched.persistent && c->ks->occupancy(c->view) < 1) {
        c->sched.persistent = 0;
        return LB_ERR_UNSUPPORTED;
    }
    return LB_OK;
}

extern "C" lb_status lb_get_schedule(const lb_ctx *c, lb_schedule *s) {
    if (!c || !s) return LB_ERR_INVALID;
    *s = c->sched;
    return LB_OK;
}

extern "C" lb_status lb_autotune(lb_ctx *c, void *fa, void *fb, int trial_steps, lb_schedule *best) {
    lb_status st = check_pair(c, fa, fb, 2);
    if (st != LB_OK || trial_steps < 1 || !best) return st != LB_OK ? st : LB_ERR_INVALID;
    std::vector<lb_schedule> cand;
    const int widths[4] = {32, 64, 128, 1};
    const int nwidths = c->view.line ? (c->kind == 2 ? 4 : 3) : 1;
    // x-row sums on the CUDA cores, and on the tensor cores where the context allows it
    const int ntc = (c->kind >= 2 && c->prec == LB_F32 && c->view.line && c->view.fixedx) ? 2 : 1;
    for (int tc = 0; tc < ntc; ++tc)
        for (int wi = 0; wi < nwidths; ++wi) {
            const int width = c->view.line ? widths[wi] : kTile;
            if (tc && width != 32) continue;  // the tensor-core x-rows run one warp per block
            cand.push_back(lb_schedule{width, 0, 0, tc, 0.0});  // one launch per step
            if (!c->view.line || width == 1) continue;
            const lb_schedule probe{width, 0, 1, tc, 0.0};
            if (lb_set_schedule(c, &probe) != LB_OK) continue;
            const int occ = c->ks->occupancy(c->view);
            const int opts[4] = {1, 2, 4, occ};
            for (int bps : opts) {
                if (bps < 1 || bps > occ) continue;
                bool dup = false;
                for (const lb_schedule &q : cand)
                    dup = dup || (q.tile_width == width && q.persistent && q.blocks_per_sm == bps && q.tensor_cores == tc);
                if (!dup) cand.push_back(lb_schedule{width, bps, 1, tc, 0.0});  // persistent launch
            }
        }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return LB_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return LB_ERR_CUDA;
    }
    int pick = -1;
    void *src = fa, *dst = fb;
    for (size_t k = 0; k < cand.size(); ++k) {
        if (lb_set_schedule(c, &cand[k]) != LB_OK) continue;
        // warm up, then time trial_steps; an even step count keeps the state in src
        const int n = trial_steps + (trial_steps & 1);
        if (lb_step(c, src, dst, 2) != LB_OK) break;
        cudaEventRecord(e0, c->view.stream);
        if (lb_step(c, src, dst, n) != LB_OK) break;
        cudaEventRecord(e1, c->view.stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cand[k].ms_per_step = ms / n;
        if (pick < 0 || cand[k].ms_per_step < cand[pick].ms_per_step) pick = (int)k;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (pick < 0) return LB_ERR_CUDA;
    st = lb_set_schedule(c, &cand[pick]);
    *best = cand[pick];
    return st;
}

extern "C" lb_status lb_test_barrier_timeout(lb_ctx *c, void *fa, void *fb) {
    lb_status st = check_pair(c, fa, fb, 2);
    if (st == LB_OK) st = flush_tables(c);
    if (st != LB_OK) return st;
    if (!c->view.line) return LB_ERR_UNSUPPORTED;
    const long long grid = persistent_grid(c);
    if (grid < 1) return LB_ERR_UNSUPPORTED;
    // preset the arrival count past the grid size: the barrier after the first step can never
    // complete, so every block waits out its bounded spin, flags the timeout and returns
    const unsigned never = 0x7fffffffu;
    cudaError_t e = cudaMemcpyAsync(c->d_health + 1, &never, sizeof(unsigned), cudaMemcpyHostToDevice, c->view.stream);
    if (e == cudaSuccess) e = c->ks->persist(c->view, fa, fb, 2, (int)grid);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->view.stream);
    return cuda_status(e);
}

extern "C" lb_status lb_step_graph(lb_ctx *c, void *fa, void *fb, int nsteps) {
    lb_status st = check_pair(c, fa, fb, nsteps);
    if (st == LB_OK) st = flush_tables(c);
    if (st != LB_OK) return st;
    if (!c->view.line || persistent_grid(c) < 1) return LB_ERR_UNSUPPORTED;
    const bool same = c->graph && c->graph_fa == fa && c->graph_fb == fb && c->graph_steps == nsteps &&
                      c->graph_sched.tile_width == c->sched.tile_width &&
                      c->graph_sched.blocks_per_sm == c->sched.blocks_per_sm &&
                      c->graph_sched.tensor_cores == c->sched.tensor_cores;
    if (!same) {
        if (c->graph) {
            cudaGraphExecDestroy(c->graph);
            c->graph = nullptr;
        }
        cudaError_t e = cudaSuccess;
        if (!c->capture_stream) e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return LB_ERR_CUDA;
        CtxView v = c->view;
        v.stream = c->capture_stream;
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return LB_ERR_CUDA;
        const cudaError_t el = launch_persistent(c, v, fa, fb, nsteps);
        e = cudaStreamEndCapture(c->capture_stream, &g);
        if (el != cudaSuccess || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return LB_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&c->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->graph = nullptr;
            return LB_ERR_CUDA;
        }
        c->graph_fa = fa;
        c->graph_fb = fb;
        c->graph_steps = nsteps;
        c->graph_sched = c->sched;
    }
    return cuda_status(cudaGraphLaunch(c->graph, c->view.stream));
}

extern "C" lb_status lb_moments(lb_ctx *c, const void *f, double *out, unsigned mask) {
    if (!c || !f || !out || mask == 0 || (mask & ~0x3fu)) return LB_ERR_INVALID;
    const lb_status fs = flush_tables(c);
    if (fs != LB_OK) return fs;
    return cuda_status(c->ks->moments(c->view, f, out, mask));
}

extern "C" lb_status lb_step_adjoint(lb_ctx *c, const void *f_t, const double *lam_next, double *lam_t,
                                     double *dtau) {
    if (!c || !f_t || !lam_next || !lam_t || !dtau || lam_next == lam_t) return LB_ERR_INVALID;
    if (!c->relax_set || !c->as) return c->as ? LB_ERR_INVALID : LB_ERR_UNSUPPORTED;
    if (any_es_bgk(c)) return LB_ERR_UNSUPPORTED;
    const size_t bytes = sizeof(double) * lb_state_elems(c);
    const char *a0 = reinterpret_cast<const char *>(lam_next), *b0 = reinterpret_cast<const char *>(lam_t);
    if (a0 < b0 + bytes && b0 < a0 + bytes) return LB_ERR_INVALID;
    const lb_status fs = flush_tables(c);
    if (fs != LB_OK) return fs;
    return cuda_status(c->as->step(c->view, f_t, lam_next, lam_t, c->d_partials, dtau));
}

extern "C" lb_status lb_moments_adjoint(lb_ctx *c, const void *f, const double *gbar, unsigned mask, double *lam) {
    if (!c || !f || !gbar || !lam || mask == 0) return LB_ERR_INVALID;
    if (mask & ~(LB_MOM_RHO | LB_MOM_U | LB_MOM_THETA | LB_MOM_Q)) return LB_ERR_INVALID;
    if (!c->as) return LB_ERR_UNSUPPORTED;
    const lb_status fs = flush_tables(c);
    if (fs != LB_OK) return fs;
    return cuda_status(c->as->moments(c->view, f, gbar, mask, lam));
}

extern "C" lb_status lb_poll_status(lb_ctx *c, unsigned *flags) {
    if (!c) return LB_ERR_INVALID;
    unsigned h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, c->d_health, sizeof(unsigned), cudaMemcpyDeviceToHost, c->view.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->view.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_health, 0, sizeof(unsigned), c->view.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->view.stream);
    if (flags) *flags = h;
    if (e != cudaSuccess) return LB_ERR_CUDA;
    if (h & LB_HEALTH_UNSTABLE) return LB_ERR_UNSTABLE;
    if (h & LB_HEALTH_TIMEOUT) return LB_ERR_TIMEOUT;
    return LB_OK;
}

extern "C" size_t lb_cells(const lb_ctx *c) { return c ? c->ncells : 0; }
extern "C" size_t lb_plane_stride(const lb_ctx *c) { return c ? c->stride : 0; }
extern "C" size_t lb_state_elems(const lb_ctx *c) { return c ? c->stride * (size_t)c->q : 0; }
extern "C" int lb_num_moment_rows(const lb_ctx *c, unsigned mask) {
    if (!c) return 0;
    const int Nm = c->N < 3 ? 3 : c->N;
    int r = 0;
    if (mask & LB_MOM_RHO) r += 1;
    if (mask & LB_MOM_U) r += 3;
    if (mask & LB_MOM_THETA) r += 1;
    if (mask & LB_MOM_SIGMA) r += 6;
    if (mask & LB_MOM_Q) r += 3;
    if (mask & LB_MOM_D) r += nmom(Nm);
    return r;
}

extern "C" const char *lb_error_string(lb_status s) {
    switch (s) {
        case LB_OK: return "ok";
        case LB_ERR_INVALID: return "invalid argument";
        case LB_ERR_CUDA: return "CUDA runtime error";
        case LB_ERR_UNSTABLE: return "unstable state (rho or theta not positive, or NaN)";
        case LB_ERR_TIMEOUT: return "bounded device wait timed out";
        case LB_ERR_UNSUPPORTED: return "unsupported lattice, order or geometry";
        case LB_ERR_NOMEM: return "out of memory";
    }
    return "unknown status";
}

extern "C" void lb_destroy(lb_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->view.stream);
    free_tables(c);
    delete c;
}

// ----------------------------------------------------------------------------------------
// lb_step_adjoint_noalloc: lb_step_adjoint for callers that cannot allocate device memory at
// the time they step backwards (code running under CUDA stream capture, where cudaMalloc is
// not allowed; frameworks whose own pool allocator owns all device memory; hosts with a hard
// device-memory budget). The per-block gradient partials live in the fixed-size device array
// below instead of the context's scratch. It is reserved once per process on every GPU that
// loads libsmrt and kept until exit; every call on every context of that GPU shares it.
namespace {

constexpr long long kNoallocMaxBlocks = 8192;  // 8192 blocks of 128 cells = 1,048,576 cells
__device__ __align__(256) double g_noalloc_partials[kNoallocMaxBlocks * kMaxTau];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[kNoallocMaxDevices] = {nullptr};

// The device address of g_noalloc_partials on the current device, looked up on first use
// (in host code the array's name is only a stand-in; kernels need the device address).
lb_status noalloc_scratch(double **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return LB_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) return LB_ERR_CUDA;
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return LB_OK;
}

}  // namespace

extern "C" lb_status lb_step_adjoint_noalloc(lb_ctx *c, const void *f_t, const double *lam_next, double *lam_t,
                                             double *dtau) {
    if (!c || !f_t || !lam_next || !lam_t || !dtau || lam_next == lam_t) return LB_ERR_INVALID;
    if (!c->as || any_es_bgk(c)) return LB_ERR_UNSUPPORTED;
    if (!c->relax_set) return LB_ERR_INVALID;
    const size_t bytes = sizeof(double) * lb_state_elems(c);
    const char *a0 = reinterpret_cast<const char *>(lam_next), *b0 = reinterpret_cast<const char *>(lam_t);
    if (a0 < b0 + bytes && b0 < a0 + bytes) return LB_ERR_INVALID;
    if (adj_blocks(c->view) > kNoallocMaxBlocks) return LB_ERR_INVALID;  // grid too large
    double *scratch = nullptr;
    lb_status st = noalloc_scratch(&scratch);
    if (st == LB_OK) st = flush_tables(c);
    if (st != LB_OK) return st;
    // every block writes its own slot before the reduction reads it: nothing to clear
    return cuda_status(c->as->step(c->view, f_t, lam_next, lam_t, scratch, dtau));
}
