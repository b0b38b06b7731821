/*
 * smrt.h -- C ABI of libsmrt, the GB300 (sm_103a) implementation of the LB-SMRT
 * collide-and-stream step of Yan & Shan, "Lattice Boltzmann simulation of non-equilibrium
 * flows using spectral multiple-relaxation-time collision model" (arXiv 2401.11086).
 *
 * Conventions shared by every call
 * --------------------------------
 * Units.   Lattice units: one time step, cell size c. Population i has the lattice abscissa
 *          xi_i = c e_i (e_i an integer vector) relative to the frame velocity u_bar = c k,
 *          k = lattice->shift (Sec. 4.1, "shifted stencil"); its physical velocity is
 *          xi_i + u_bar and it streams by e_i + k cells per step. Velocities passed in or out
 *          of the library (lb_state.u, lb_fill_equilibrium's u, lb_moments' u) are PHYSICAL
 *          (they include u_bar); theta is the temperature in units of the reference
 *          temperature ("energy units", Sec. 2).
 * State.   A state is the set of post-collision populations of every cell, stored as their
 *          deviations from the weights, df_i = f_i - w_i (the populations of the rest state
 *          rho = 1, u = u_bar, theta = 1 are exactly w_i, so rounding acts only on the
 *          deviation), structure of arrays: element  df[i * plane_stride + cell]  for population
 *          i (the caller's lattice order) and cell = instance_offset + (z * ny + y) * nx + x,
 *          x fastest.
 *          Instances (batched 1D problems) are concatenated in order. plane_stride and the
 *          element count of a state are given by lb_plane_stride / lb_state_elems.
 *          The element type is double for LB_F64 and float otherwise.
 * Memory.  Every pointer argument named f*, out, rho, u, theta, lam*, dtau is DEVICE memory
 *          owned by the caller. The library owns only the context and its small device tables.
 *          lb_step, lb_moments and lb_fill_equilibrium allocate nothing.
 * Streams. All device work of a context is enqueued on the stream given to lb_init_lattice
 *          (a cudaStream_t passed as void*, NULL = legacy default stream) and is asynchronous;
 *          only lb_poll_status synchronises. One context per stream; calls on one context are
 *          not thread-safe.
 * Errors.  Arguments are validated before any launch (LB_ERR_INVALID, nothing enqueued).
 *          Device-side trouble is recorded in a health word read by lb_poll_status. No C++
 *          exception crosses this ABI.
 */
#ifndef SMRT_H
#define SMRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_ctx lb_ctx; /* opaque; created by lb_init_lattice, freed by lb_destroy */

typedef enum {
    LB_OK = 0,
    LB_ERR_INVALID = 1,     /* bad pointer, size, lattice or parameter; nothing was enqueued */
    LB_ERR_CUDA = 2,        /* a CUDA runtime call failed                                     */
    LB_ERR_UNSTABLE = 3,    /* a cell reached rho <= 0, theta <= 0 or NaN (health word)       */
    LB_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up (health word)               */
    LB_ERR_UNSUPPORTED = 5, /* valid request the library has no kernel for                    */
    LB_ERR_NOMEM = 6        /* allocation of the context's own tables failed                  */
} lb_status;

typedef enum {
    LB_F64 = 0,        /* populations and all arithmetic in double                           */
    LB_F32 = 1,        /* populations and all arithmetic in float                            */
    LB_F32_CONS64 = 2  /* float populations; the conserved sums (rho, rho u, energy) and the
                          equilibrium part of the rebuild in double                          */
} lb_precision;

/* Health-word bits returned by lb_poll_status. */
#define LB_HEALTH_UNSTABLE 0x1u /* some cell had rho <= 0, theta <= 0 or a NaN moment */
#define LB_HEALTH_TIMEOUT 0x2u

/* Velocity set: a degree-`degree` Gauss-Hermite quadrature (Sec. 3, Eq. an): abscissae
 * xi_i = c e_i, weights w_i. e is q*3 int8 (row i = e_i), w is q doubles; both host memory,
 * copied by lb_init_lattice. shift = k, the integer frame shift of Sec. 4.1. */
typedef struct {
    int q;
    const int8_t *e;
    const double *w;
    double c;
    int degree;
    int shift[3];
} lb_lattice_desc;

/* Grid. Single instance: nx, ny, nz cells, batch = 1, nx_per_instance = NULL.
 * Batched 1D problems: ny = nz = 1, batch = B, nx_per_instance = B lengths (host memory,
 * copied), nx ignored. bc_x: 0 periodic in x, 1 fixed end states in x (cells beyond either
 * end hold the order-N equilibrium of the left/right state; Sec. 4.2). y and z are periodic. */
typedef struct {
    int nx, ny, nz;
    int batch;
    const int *nx_per_instance;
    int bc_x;
} lb_grid_desc;

/* A macroscopic state: density, PHYSICAL velocity, temperature (Sec. 2, Eq. Maxwellian). */
typedef struct {
    double rho, u[3], theta;
} lb_state;

/* lb_init_lattice -- create a context for one velocity set, grid, truncation order and
 * precision. The velocity set must integrate every monomial of degree <= 2N exactly (Sec. 3,
 * the exactness remark after Eq. fi); the library checks this by brute force and also
 * matches e against the velocity sets it has kernels for (LB_ERR_UNSUPPORTED otherwise):
 *   D3Q39 (N = 3), D3Q103 (N = 3, 4): every geometry and precision;
 *   D3Q729 and D3Q4913, the tensor products of D1Q9-P1 and D1Q17-P1 (Sec. 4.2, Table 3:
 *   d = 9, degree 11; d = 17, degree 19), N = 4, 5:
 *     batched 1D lines (ny = nz = 1), frame shift along x only, LB_F64 or LB_F32; weights
 *     must factor as w_a w_b w_c with equal weights for +e and -e. The states
 *     passed to the stepping calls must start on 16-byte boundaries (LB_ERR_INVALID
 *     otherwise): the kernel stages population segments with the bulk-copy engine. When e
 *     lists the velocities in the library order (i = a + d b + d^2 c over the 1D order rest,
 *     +1, -1, +2, -2, ..., the order lb_lattice_named returns), each group of d planes is
 *     staged as one box of a 2D tensor map of the state; any other order works, staged plane
 *     by plane, with the same results bit for bit.
 * hermite_order N: truncation order of Eqs. an/fi.
 * cuda_stream: cudaStream_t used for every later call on this context.
 * On success *out is a new context (relaxation times unset: lb_set_relaxation must follow).
 * Errors: LB_ERR_INVALID (null/size/quadrature), LB_ERR_UNSUPPORTED, LB_ERR_NOMEM, LB_ERR_CUDA. */
lb_status lb_init_lattice(lb_ctx **out, const lb_lattice_desc *lattice, const lb_grid_desc *grid,
                          int hermite_order, lb_precision precision, void *cuda_stream);

/* lb_set_relaxation -- relaxation times of the SMRT operator (Eq. SMRT) and end states.
 * tau: continuous relaxation times tau_c,nm in time steps at density rho_ref, one per
 *      irreducible part (n, m), n = 2..N, m = 0..floor(n/2), in the order
 *      (2,0) (2,1) (3,0) (3,1) (4,0) (4,1) (4,2) (5,0) (5,1) (5,2) (host memory; 2 entries for
 *      N=2, 4 for N=3, 7 for N=4, 10 for N=5). Table 4 gives tau_nm / tau_20 for Maxwell molecules.
 *      The discrete time of part (n,m) at a cell is tau_c,nm * s + 1/2, with s = rho_ref/rho
 *      when maxwell_molecule_law is 1 (viscosity proportional to temperature, Sec. 4.2) and
 *      s = 1 when it is 0. Every tau must be > 0.
 * left, right: end states of a grid with bc_x = 1 (host memory; may be NULL when bc_x = 0).
 * instance: which instance of a batch to set (-1 = all).
 * Validates and stores the settings on the host. The instance table and the end-state
 * populations of every instance set since the last launch are uploaded and computed, in one
 * launch, on the context's stream by the next call that launches work (lb_fill_equilibrium,
 * lb_step, lb_step_graph, lb_autotune, lb_moments, the adjoint calls), which then synchronises
 * once; setting many instances one by one therefore costs one launch.
 * Errors: LB_ERR_INVALID (null, tau <= 0, rho or theta <= 0, bad instance), LB_ERR_CUDA. */
lb_status lb_set_relaxation(lb_ctx *ctx, const double *tau, int maxwell_molecule_law,
                            double rho_ref, const lb_state *left, const lb_state *right,
                            int instance);

/* lb_set_frame_shift -- change the integer frame shift k_x of one instance (-1 = all) after
 * lb_init_lattice (Sec. 4.1: each shock chooses k_x = round(((u1 + u2)/2) / c)). Call before
 * lb_set_relaxation so that the end-state populations use the new frame (end states already set
 * are recomputed in the new frame). Stored on the host and uploaded as lb_set_relaxation's
 * settings are.
 * Errors: LB_ERR_INVALID (bad instance; a single box accepts only -1), LB_ERR_CUDA. */
lb_status lb_set_frame_shift(lb_ctx *ctx, int instance, int kx);

/* Collision models of lb_set_collision_model. */
#define LB_MODEL_SMRT 0   /* Eq. SMRT: each irreducible part (n, m) with its own time (default) */
#define LB_MODEL_ES_BGK 1 /* Eq. ES-BGK: one time, target = Holway's ellipsoidal Gaussian    */

/* lb_set_collision_model -- choose the collision model of one instance (-1 = all).
 * LB_MODEL_ES_BGK (Sec. 3, Eq. ES-BGK; the paper notes that its covariance
 * Lambda = theta delta + b sigma / rho is a weighted sum of two order-2 irreducible tensors):
 * every order n >= 2 of the local-frame coefficients relaxes at the one discrete rate
 * 1/tau_20 (tau_20 = the first time given to lb_set_relaxation, + 1/2, with its density law)
 * toward the coefficients of that Gaussian, truncated at N. The discrete scheme uses
 * b' = 1 - (1 - b) tau_20 / (tau_20 - b/2), which keeps the continuous model's stress rate
 * (1 - b)/tau_c under the second-order discretisation, so Pr = 1/(1 - b) (2/3 at b = -1/2).
 * Requires -1/2 <= b < 1. Every velocity set and precision (with LB_F32_CONS64 the relaxation
 * acts on the non-equilibrium part, which in the local frame is the whole of orders >= 2). The
 * adjoint calls (lb_step_adjoint, lb_step_adjoint_noalloc) differentiate SMRT only and return
 * LB_ERR_UNSUPPORTED while any instance uses ES-BGK. Stored on the host and uploaded as
 * lb_set_relaxation's settings are.
 * Errors: LB_ERR_INVALID (instance, model or b), LB_ERR_CUDA. */
lb_status lb_set_collision_model(lb_ctx *ctx, int instance, int model, double b);

/* lb_fill_equilibrium -- f = order-N truncated Maxwellian of the given fields at every cell
 * (Sec. 3: f_i^eq is the truncated Hermite expansion of Eq. Maxwellian evaluated at xi_i,
 * built through Eq. fi). rho, theta: ncells doubles; u: 3*ncells doubles (row k = component
 * k of the PHYSICAL velocity), all device memory; f: a state (device). This is the
 * post-collision state of an equilibrium, i.e. a valid initial state.
 * Errors: LB_ERR_INVALID, LB_ERR_CUDA. */
lb_status lb_fill_equilibrium(lb_ctx *ctx, void *f, const double *rho, const double *u,
                              const double *theta);

/* lb_step -- advance nsteps collide-and-stream steps (Sec. 3: stream f_i along e_i + k, then
 * the SMRT collision of Eq. SMRT through the irreducible decomposition of Appendix A and the
 * rebuild of Eq. fi). The state enters in f_a. Steps alternate f_a -> f_b -> f_a ...; after
 * the call the newest state is in f_b when nsteps is odd and in f_a when nsteps is even
 * (for nsteps = 1, f_a is read only). f_a and f_b must be distinct, non-overlapping states.
 * Errors: LB_ERR_INVALID (null, nsteps < 1, relaxation unset), LB_ERR_CUDA. */
lb_status lb_step(lb_ctx *ctx, void *f_a, void *f_b, int nsteps);

/* Launch schedule of the 1D-line (batched) kernels. tile_width: cells per block (32, 64, 128;
 * on D3Q729 and D3Q4913 a block of tile_width / 32 warps steps a tile of tile_width cells whose
 * pulls it stages once for all its warps, one 32-cell row per warp -- lb_init_lattice sets 128
 * for LB_F32, 32 (D3Q729) or 64 (D3Q4913) for LB_F64, 128 on the other sets; on D3Q729 the value
 * 1 selects one block per cell -- its populations in shared memory, the factored sums spread
 * over the block -- which lb_init_lattice picks for problems of at most 48 (LB_F64) or 32 (LB_F32)
 * cells per SM, and
 * which runs one launch per step only);
 * persistent = 1: lb_step runs all its steps in one cooperative launch of blocks_per_sm
 * blocks per SM (0 = as many as fit), tiles spread over the blocks, a grid-wide barrier between
 * steps (its wait is bounded: on timeout the health word gets LB_HEALTH_TIMEOUT and the
 * launch ends); persistent = 0: one launch per step. tensor_cores = 1 (LB_F32 D3Q729 / D3Q4913
 * lines with fixed ends, tile width 32): the x-row sums of the projection (Eq. an, the
 * first of its three factored passes) run as warp-wide TF32 matrix products on the tensor
 * cores, with each population split into two TF32 parts and each power e^j into two, three
 * products per tile, for single-precision accuracy; 0: on the CUDA cores. ms_per_step: measured
 * by lb_autotune. */
typedef struct {
    int tile_width;
    int blocks_per_sm;
    int persistent;
    int tensor_cores;
    double ms_per_step;
} lb_schedule;

/* lb_set_schedule / lb_get_schedule -- apply or read a schedule (a periodic box accepts only
 * {128, 0, 0, 0}). Setting a new tile width rebuilds the context's tile table (synchronises).
 * Errors: LB_ERR_INVALID, LB_ERR_UNSUPPORTED (persistent kernel cannot be resident; tensor_cores
 * on any other context), LB_ERR_CUDA. */
lb_status lb_set_schedule(lb_ctx *ctx, const lb_schedule *schedule);
lb_status lb_get_schedule(const lb_ctx *ctx, lb_schedule *schedule);

/* lb_autotune -- time every candidate schedule (tile widths 32/64/128, and 1 on D3Q729; one
 * launch per step or persistent with 1, 2, 4 or all resident blocks per SM; x-row sums on the
 * CUDA cores and, where allowed, the tensor cores) for trial_steps steps on the states
 * f_a / f_b (which it ADVANCES: pass copies), apply the fastest and return it in *best with
 * its ms_per_step. Synchronises. Errors: as lb_step, LB_ERR_CUDA. */
lb_status lb_autotune(lb_ctx *ctx, void *f_a, void *f_b, int trial_steps, lb_schedule *best);

/* lb_step_graph -- lb_step of a 1D-line context as a replay of a CUDA graph holding one
 * persistent launch of nsteps steps (captured on first use for this (f_a, f_b, nsteps,
 * schedule) and cached in the context; capture needs no allocation of device memory). Same
 * buffer convention as lb_step. Errors: as lb_step, LB_ERR_UNSUPPORTED (box, a D3Q729 context
 * on its one-cell-per-block schedule, or a persistent kernel that cannot be resident),
 * LB_ERR_CUDA. */
lb_status lb_step_graph(lb_ctx *ctx, void *f_a, void *f_b, int nsteps);

/* lb_test_barrier_timeout -- failure-detection test of the persistent launch: runs two steps
 * with the barrier's arrival count preset so that the barrier can never complete. Every block
 * waits out its bounded spin (about a second), sets LB_HEALTH_TIMEOUT and returns; the next
 * lb_poll_status reports LB_ERR_TIMEOUT and the context stays usable. f_a/f_b contents are
 * undefined afterwards. Synchronises. Errors: as lb_step, LB_ERR_UNSUPPORTED (box). */
lb_status lb_test_barrier_timeout(lb_ctx *ctx, void *f_a, void *f_b);

/* Row groups of lb_moments' output, selected by which_mask. */
#define LB_MOM_RHO 0x1u   /* 1 row:  rho                                                    */
#define LB_MOM_U 0x2u     /* 3 rows: physical velocity u_x, u_y, u_z                        */
#define LB_MOM_THETA 0x4u /* 1 row:  theta                                                  */
#define LB_MOM_SIGMA 0x8u /* 6 rows: sigma = theta d^(2): xx yy zz xy xz yz                 */
#define LB_MOM_Q 0x10u    /* 3 rows: heat flux q_k = theta^(3/2)/2 sum_l d^(3)_kll          */
#define LB_MOM_D 0x20u    /* M rows: local coefficients d_beta, |beta| <= max(N,3)          */

/* lb_moments -- macroscopic moments of the PRE-collision populations (the state streamed by
 * one step, without colliding) at every cell: rho, u, theta (Sec. 2, Eq. hermite), and the
 * local-frame Hermite coefficients d_beta = sum_i f_i He_beta((xi_i - u)/sqrt(theta)) of the
 * expansion that defines SMRT (Sec. 3), with sigma and q derived from them (Sec. 2.2:
 * a^(2) = P/p - delta, q_i = Q_ikk/2). Multi-indices beta are ordered by order, then
 * descending lexicographically ((2,0,0) (1,1,0) (1,0,1) (0,2,0) (0,1,1) (0,0,2) ...).
 * out: device doubles, rows of lb_cells(ctx) values, the selected groups in the order of
 * the bits above. Errors: LB_ERR_INVALID, LB_ERR_CUDA. */
lb_status lb_moments(lb_ctx *ctx, const void *f, double *out, unsigned which_mask);

/* lb_step_adjoint -- one step of the discrete adjoint (reverse mode) of lb_step, for gradients
 * of a loss L with respect to the state and to the relaxation times of Eq. SMRT. With
 * h^{t+1} = C(S h^t) (S: pull streaming of Sec. 3, C: per-cell collision):
 *   lam_t = S^T J_C(S h^t)^T lam_next,   dtau[k] += sum_cells (d h^{t+1} / d tau_c,k)^T lam_next.
 * f_t: the forward state h^t entering the step (a state of this context, device).
 * lam_next: dL/dh^{t+1}, lam_t: dL/dh^t (output, overwritten): device doubles with the state
 * layout (lb_state_elems values; plane i = population i). dtau: device doubles, one per (n,m)
 * in lb_set_relaxation's order, ACCUMULATED (+=) -- derivatives with respect to the continuous
 * times tau_c,nm. Arithmetic is double whatever the precision of f_t. Populations pulled from
 * beyond a fixed x end are constants (no gradient). The per-block gradient partials live in a
 * scratch array owned by the context; calls on one context must not overlap.
 * Every set has adjoint kernels; on D3Q729 and D3Q4913 the projection of lam_next and the
 * evaluation of the raw moments' adjoint factor over the axes as the forward step does
 * (one thread per cell, 32-cell tiles, the per-tile gradient partials reduced in tile order).
 * Errors: LB_ERR_INVALID (null, lam_next overlapping lam_t, relaxation unset), LB_ERR_UNSUPPORTED
 * (an instance using the ES-BGK model), LB_ERR_CUDA. */
lb_status lb_step_adjoint(lb_ctx *ctx, const void *f_t, const double *lam_next, double *lam_t,
                          double *dtau);

/* lb_step_adjoint_noalloc -- lb_step_adjoint for callers that may not allocate device memory
 * when they run it: work captured into a CUDA graph (cudaMalloc cannot be captured), code
 * whose device memory all belongs to its own pool allocator, or a process with a fixed
 * device-memory budget. The paper has no counterpart; the arguments, results and errors are
 * those of lb_step_adjoint, and the call allocates nothing. Instead of the context's scratch
 * it uses one fixed array of 8192 x 10 doubles (640 KB) that every GPU loading libsmrt holds
 * until the process exits, enough for grids of up to 8192 blocks: a box of up to 8192 blocks
 * of 128 cells along x (1,048,576 cells), or batched lines of up to 8192 tiles of the
 * scheduled tile width (lb_set_schedule: 32, 64 or 128 cells per tile, so at most 262,144
 * cells at width 32 and 1,048,576 at width 128); larger grids return LB_ERR_INVALID and
 * touch neither lam_t nor dtau. The first call on a device looks up that array's device
 * address, and settings changed since the context's last launch (lb_set_relaxation and its
 * kin) are uploaded first with a synchronising copy: make the first call, and a launching call
 * after any change of settings, before any stream capture. All calls share
 * the array and it keeps the last call's partial sums (each call overwrites the slots it reads,
 * so nothing needs clearing), hence calls that may overlap on the GPU -- on different streams
 * or contexts of one device -- race and must be ordered by the caller. */
lb_status lb_step_adjoint_noalloc(lb_ctx *ctx, const void *f_t, const double *lam_next,
                                  double *lam_t, double *dtau);

/* lb_moments_adjoint -- reverse mode of lb_moments for the row groups LB_MOM_RHO, LB_MOM_U,
 * LB_MOM_THETA and LB_MOM_Q: given gbar = dL/d(moments) in lb_moments' layout for which_mask
 * (rows x lb_cells doubles, device), writes lam = dL/df (device doubles, state layout,
 * overwritten), including the transpose of the streaming that lb_moments applies.
 * Errors: LB_ERR_INVALID (null, empty mask or a row group without an adjoint), LB_ERR_CUDA. */
lb_status lb_moments_adjoint(lb_ctx *ctx, const void *f, const double *gbar, unsigned which_mask,
                             double *lam);

/* lb_poll_status -- synchronise the context's stream, return and clear its health word.
 * Returns LB_ERR_UNSTABLE / LB_ERR_TIMEOUT when the corresponding bit was set, LB_ERR_CUDA
 * when the stream reports an error, LB_OK otherwise. health_flags may be NULL. */
lb_status lb_poll_status(lb_ctx *ctx, unsigned *health_flags);

/* Sizes of a context's arrays. */
size_t lb_cells(const lb_ctx *ctx);       /* total cells over all instances              */
size_t lb_plane_stride(const lb_ctx *ctx); /* elements between population planes          */
size_t lb_state_elems(const lb_ctx *ctx);  /* elements of one state = q * plane_stride    */
int lb_num_moment_rows(const lb_ctx *ctx, unsigned which_mask);

/* lb_lattice_named -- the library's own velocity sets, solved from the even-moment
 * conditions of a degree-Q Gauss-Hermite rule (Sec. 3, Eq. an): "D3Q39" (degree 7),
 * "D3Q103" (degree 9) and "D3Q729" (degree 11, the 3D tensor product of the 1D rule D1Q9-P1
 * on c {0, +-1, +-2, +-3, +-5} of Sec. 4.2 / Table 3, in the order i = a + 9 b + 81 c over the
 * 1D indices a, b, c = rest, +1, -1, +2, -2, +3, -3, +5, -5) and "D3Q4913" (degree 19, the
 * product of D1Q17-P1 on c {0, +-1, .., +-7, +-9}, i = a + 17 b + 289 c, 1D order rest, +1, -1,
 * .., +7, -7, +9, -9).
 * Writes up to capacity velocities: e_out (capacity*3 int8), w_out
 * (capacity doubles), *c_out, *q_out, *degree_out (host memory).
 * Errors: LB_ERR_INVALID (unknown name, null, capacity too small). */
lb_status lb_lattice_named(const char *name, int8_t *e_out, double *w_out, double *c_out,
                           int *q_out, int *degree_out, int capacity);

/* lb_hermite_convergence -- the convergence study of Appendix B (Eq. fexp): for each of npts
 * points (theta[p] > 0, u[p]) the smallest order N <= nmax whose truncated Hermite expansion
 * f_N = omega(xi) sum_{n<=N} a^(n) He_n(xi)/n! of the 1D Maxwellian of temperature theta and
 * velocity u has L1 error int |f - f_N| dxi < tol (the paper's figure uses tol = 0.01).
 * order[p] = that N, or nmax + 1 when no order up to nmax reaches tol (-1 for a point with
 * theta <= 0 or a non-finite value); err[p] = the error at order[p] (at nmax when not reached;
 * NaN for invalid points). The integral is composite Simpson on 4097 points of [-L, L],
 * L = max(|u| + 12 sqrt(theta), 2 sqrt(nmax + 1) + 10); a^(n) and He_n come from their
 * recurrences scaled by sqrt(n!). theta, u (npts doubles), order (npts ints) and err (npts
 * doubles) are device memory; asynchronous on cudaStream_t stream; no context needed.
 * Errors: LB_ERR_INVALID (npts < 0, nmax outside 0..LB_HERMITE_MAX_ORDER, tol <= 0, null
 * pointers), LB_ERR_CUDA. */
#define LB_HERMITE_MAX_ORDER 200
lb_status lb_hermite_convergence(const double *theta, const double *u, int npts, double tol, int nmax,
                                 int *order, double *err, void *stream);

/* lb_rankine_hugoniot -- end states of a normal shock (Eq. rankine, temperature ratio read
 * with Ma^2 in the denominator) for upstream Mach number Ma, ratio of specific heats gamma,
 * upstream rho1 and theta1; velocities in the shock frame, along +x (host memory out). */
lb_status lb_rankine_hugoniot(double Ma, double gamma, double rho1, double theta1,
                              lb_state *left, lb_state *right);

/* lb_shock_frame -- reference temperature and frame shift of a normal shock (Sec. 4.1-4.2):
 * *theta1 = min(1, theta2_max / (theta2/theta1)): 1 when the downstream temperature stays at
 * or below theta2_max, else the upstream temperature that puts the downstream one at
 * theta2_max (well below 2, the Hermite convergence bound);
 * *kx = round(((u1 + u2)/2) / c), the integer shift minimising the largest relative speed.
 * Host memory out. Errors: LB_ERR_INVALID. */
lb_status lb_shock_frame(double Ma, double gamma, double c, double theta2_max, double *theta1, int *kx);

/* lb_shock_shift -- the frame shift of lb_shock_frame for a given upstream temperature theta1
 * (e.g. Table 3's): *kx = round(((u1 + u2)/2) / c) with (u1 + u2)/2 =
 * (gamma Ma^2 + 1) / ((gamma + 1) Ma) sqrt(gamma theta1) (Sec. 4.1-4.2). Host memory out.
 * Errors: LB_ERR_INVALID (null, Ma < 1, gamma <= 1, c <= 0, theta1 <= 0). */
lb_status lb_shock_shift(double Ma, double gamma, double c, double theta1, int *kx);

const char *lb_error_string(lb_status status);
void lb_destroy(lb_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SMRT_H */
