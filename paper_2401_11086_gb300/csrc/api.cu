// api.cu -- the extern "C" entry points of libsmrt (declared and documented in smrt.h).
// Host-side validation, the context's small device tables, and dispatch to the kernels
// instantiated per velocity set and precision.
#include <cuda_runtime.h>

#include <algorithm>
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
}  // namespace smrt

using namespace smrt;

struct lb_ctx {
    int kind;  // 0 D3Q39, 1 D3Q103
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
    // device tables owned by the context
    InstanceInfo *d_inst;
    int2 *d_tiles;
    void *d_ghosts;
    double *d_ghostsd;
    double *d_states;
    unsigned *d_health;
    double *d_partials;  // per-block relaxation-time gradients of lb_step_adjoint
};

namespace {

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
    cudaFree(c->d_ghosts);
    cudaFree(c->d_ghostsd);
    cudaFree(c->d_states);
    cudaFree(c->d_health);
    cudaFree(c->d_partials);
}

}  // namespace

extern "C" lb_status lb_init_lattice(lb_ctx **out, const lb_lattice_desc *lat, const lb_grid_desc *grid,
                                     int N, lb_precision prec, void *stream) {
    if (!out || !lat || !grid || !lat->e || !lat->w) return LB_ERR_INVALID;
    *out = nullptr;
    if (prec != LB_F64 && prec != LB_F32 && prec != LB_F32_CONS64) return LB_ERR_INVALID;
    if (!(lat->c > 0.0) || lat->q <= 0 || lat->q > kMaxQ) return LB_ERR_INVALID;
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
    if (match_set<D3Q39>(lat, c->perm)) {
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
        if (line)
            for (int x0 = 0; x0 < in.nx; x0 += kTile) tiles.push_back(make_int2(j, x0));
        ncells += line ? (size_t)in.nx : (size_t)grid->nx * grid->ny * grid->nz;
    }
    c->ncells = ncells;
    c->stride = (ncells + 63) / 64 * 64;  // planes start on 256-byte boundaries (float)
    c->h_states.assign((size_t)grid->batch * 10, 0.0);

    CtxView &v = c->view;
    std::memset(&v, 0, sizeof(v));
    v.stream = static_cast<cudaStream_t>(stream);
    for (int i = 0; i < c->q; ++i) v.plane[i] = (long long)c->perm[i] * (long long)c->stride;
    v.wp[0] = lat->w[c->perm[0]];
    for (int p = 0; p < c->np; ++p) v.wp[p + 1] = lat->w[c->perm[2 * p + 1]];
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

    cudaError_t e = cudaSuccess;
    e = cudaMalloc(&c->d_inst, sizeof(InstanceInfo) * grid->batch);
    if (e == cudaSuccess && !tiles.empty()) e = cudaMalloc(&c->d_tiles, sizeof(int2) * tiles.size());
    if (e == cudaSuccess) e = cudaMalloc(&c->d_ghosts, c->elem * c->q * 2 * grid->batch);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_ghostsd, sizeof(double) * c->q * 2 * grid->batch);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_states, sizeof(double) * 10 * grid->batch);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_health, 16);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_partials, sizeof(double) * kMaxTau * std::max(1LL, adj_blocks(v)));
    if (e != cudaSuccess) {
        free_tables(c);
        delete c;
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? LB_ERR_NOMEM : LB_ERR_CUDA;
    }
    if (!tiles.empty())
        e = cudaMemcpyAsync(c->d_tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, v.stream);
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
    v.ghosts = c->d_ghosts;
    v.ghostsd = c->d_ghostsd;
    v.health = c->d_health;
    c->relax_set = false;
    *out = c;
    return LB_OK;
}

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
    cudaStream_t st = c->view.stream;
    cudaError_t e = cudaMemcpyAsync(c->d_inst, c->h_inst.data(), sizeof(InstanceInfo) * c->batch,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && c->view.fixedx) {
        e = cudaMemcpyAsync(c->d_states, c->h_states.data(), sizeof(double) * 10 * c->batch,
                            cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = c->ks->ghost(c->view, c->d_states, c->batch, c->d_ghosts, c->d_ghostsd);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host tables are reused next call
    if (e != cudaSuccess) return LB_ERR_CUDA;
    c->relax_set = true;
    return LB_OK;
}

extern "C" lb_status lb_set_frame_shift(lb_ctx *c, int instance, int kx) {
    if (!c || instance < -1 || instance >= c->batch) return LB_ERR_INVALID;
    if (!c->view.line && instance != -1) return LB_ERR_INVALID;
    const int j0 = instance < 0 ? 0 : instance, j1 = instance < 0 ? c->batch : instance + 1;
    for (int j = j0; j < j1; ++j) c->h_inst[j].kx = kx;
    if (!c->view.line) c->view.kx = kx;
    cudaError_t e = cudaMemcpyAsync(c->d_inst, c->h_inst.data(), sizeof(InstanceInfo) * c->batch,
                                    cudaMemcpyHostToDevice, c->view.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->view.stream);
    return cuda_status(e);
}

extern "C" lb_status lb_fill_equilibrium(lb_ctx *c, void *f, const double *rho, const double *u,
                                         const double *theta) {
    if (!c || !f || !rho || !u || !theta) return LB_ERR_INVALID;
    return cuda_status(c->ks->fill(c->view, f, rho, u, theta));
}

extern "C" lb_status lb_step(lb_ctx *c, void *fa, void *fb, int nsteps) {
    if (!c || !fa || !fb || fa == fb || nsteps < 1) return LB_ERR_INVALID;
    if (!c->relax_set) return LB_ERR_INVALID;
    const size_t bytes = c->elem * lb_state_elems(c);
    const char *a0 = static_cast<const char *>(fa), *b0 = static_cast<const char *>(fb);
    if (a0 < b0 + bytes && b0 < a0 + bytes) return LB_ERR_INVALID;  // overlap
    void *src = fa, *dst = fb;
    for (int s = 0; s < nsteps; ++s) {
        c->view.step++;
        const cudaError_t e = c->ks->step(c->view, src, dst);
        if (e != cudaSuccess) return LB_ERR_CUDA;
        std::swap(src, dst);
    }
    return LB_OK;
}

extern "C" lb_status lb_moments(lb_ctx *c, const void *f, double *out, unsigned mask) {
    if (!c || !f || !out || mask == 0 || (mask & ~0x3fu)) return LB_ERR_INVALID;
    return cuda_status(c->ks->moments(c->view, f, out, mask));
}

extern "C" lb_status lb_step_adjoint(lb_ctx *c, const void *f_t, const double *lam_next, double *lam_t,
                                     double *dtau) {
    if (!c || !f_t || !lam_next || !lam_t || !dtau || lam_next == lam_t) return LB_ERR_INVALID;
    if (!c->relax_set || !c->as) return c->as ? LB_ERR_INVALID : LB_ERR_UNSUPPORTED;
    const size_t bytes = sizeof(double) * lb_state_elems(c);
    const char *a0 = reinterpret_cast<const char *>(lam_next), *b0 = reinterpret_cast<const char *>(lam_t);
    if (a0 < b0 + bytes && b0 < a0 + bytes) return LB_ERR_INVALID;
    return cuda_status(c->as->step(c->view, f_t, lam_next, lam_t, c->d_partials, dtau));
}

extern "C" lb_status lb_moments_adjoint(lb_ctx *c, const void *f, const double *gbar, unsigned mask, double *lam) {
    if (!c || !f || !gbar || !lam || mask == 0) return LB_ERR_INVALID;
    if (mask & ~(LB_MOM_RHO | LB_MOM_U | LB_MOM_THETA | LB_MOM_Q)) return LB_ERR_INVALID;
    if (!c->as) return LB_ERR_UNSUPPORTED;
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
    if (!c->as) return LB_ERR_UNSUPPORTED;
    if (!c->relax_set) return LB_ERR_INVALID;
    const size_t bytes = sizeof(double) * lb_state_elems(c);
    const char *a0 = reinterpret_cast<const char *>(lam_next), *b0 = reinterpret_cast<const char *>(lam_t);
    if (a0 < b0 + bytes && b0 < a0 + bytes) return LB_ERR_INVALID;
    if (adj_blocks(c->view) > kNoallocMaxBlocks) return LB_ERR_INVALID;  // grid too large
    double *scratch = nullptr;
    const lb_status st = noalloc_scratch(&scratch);
    if (st != LB_OK) return st;
    // every block writes its own slot before the reduction reads it: nothing to clear
    return cuda_status(c->as->step(c->view, f_t, lam_next, lam_t, scratch, dtau));
}
