"""Parity of the tensor-product kernels (D3Q729 = D1Q9-P1^3, N = 4 and 5: the paper's own
configuration, Sec. 4.2 / Table 3) with the FP64 oracle, through the C ABI.

Every expected value comes from ``oracle/`` or from a golden file written by
tests/golden/make_shock_golden.py (oracle only). FP64 kernels agree with the oracle to
round-off (1e-11 relative to the population scale); FP32 kernels to 2e-6 per step.
"""
import os

import numpy as np
import pytest

import synthetic
from oracle import lattice as OL
from oracle import shock as OK
from oracle import smrt as OS
from _lb import download, lib_from_oracle, upload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2401_11086_gb300 as P  # noqa: E402
from paper_2401_11086_gb300 import shocks  # noqa: E402

# Table 3 rows on the D1Q9-P1 product set, ragged lengths (several 32/64/128-cell tiles)
MACHS = [1.5, 3.0, 5.0]
LENGTHS = [100, 37, 150]


@pytest.fixture(scope="module")
def lat():
    o = OL.d3q729()
    d = P.lb_lattice_named("D3Q729")
    return o, d, lib_from_oracle(o, d)


def _desc(d, shift):
    return P.LatticeDesc(e=d.e, w=d.w, c=d.c, degree=d.degree, shift=tuple(shift))


def _tau(model):
    keys = [(n, m) for n in range(2, model.N + 1) for m in range(n // 2 + 1)]
    return [model.tau_star[k] * model.tau_ref for k in keys]


def _oracle_case(olat, N, Ma, L, tau_star=None):
    case = OK.shock_case(olat, N, Ma, L, theta1=shocks.TABLE3_THETA1[Ma], tau_star=tau_star)
    st = case.states
    h = OK.initial_state(case, *[synthetic.step_blend(L, st[k + "1"], st[k + "2"])
                                 for k in ("rho", "u", "theta")])
    return case, h


def _upload_batch(ctx, d, idx, hs):
    flat = np.concatenate([h.reshape(h.shape[0], -1) for h in hs], axis=1)
    st = ctx.new_state()
    ctx.planes(st)[:] = torch.from_numpy(np.ascontiguousarray(flat[idx] - d.w[:, None])).to(ctx.device, ctx.dtype)
    return st


def _download_batch(ctx, d, idx, st, lengths):
    arr = ctx.planes(st).double().cpu().numpy() + d.w[:, None]
    out = np.empty_like(arr)
    out[idx] = arr
    offs = np.concatenate([[0], np.cumsum(lengths)])
    return [out[:, offs[j]:offs[j + 1]] for j in range(len(lengths))]


def _batch(olat, d, N, prec, tau_star=None, ratios=shocks.TAU_RATIOS_SMRT):
    ctx, _, params = shocks.setup_batch(d, N, MACHS, LENGTHS, precision=prec, width=0.0,
                                        ratios=ratios, theta1=[shocks.TABLE3_THETA1[m] for m in MACHS])
    cases, hs = zip(*[_oracle_case(olat, N, Ma, L, tau_star) for Ma, L in zip(MACHS, LENGTHS)])
    return ctx, params, list(cases), list(hs)


@pytest.mark.parametrize("N", [4, 5])
@pytest.mark.parametrize("table", ["smrt", "shakhov", "reduced"])
@pytest.mark.parametrize("width", [1, 64])
def test_table3_shocks_match_oracle(lat, N, table, width):
    """FP64, the three Table 3 rows (Ma 1.5/3/5, theta1 = 0.714/0.333/0.167, k_x = 2) in one
    batch from the step initial condition, 12 steps, each instance vs its own oracle run;
    SMRT, Shakhov and the 'reduced' tau_41 = tau_42 table of Sec. 4.3."""
    olat, d, idx = lat
    star = {"smrt": OS.TAU_STAR_SMRT, "shakhov": OS.TAU_STAR_SHAKHOV,
            "reduced": {**OS.TAU_STAR_SMRT, (4, 2): 6.0 / 7.0}}[table]
    ratios = {"smrt": shocks.TAU_RATIOS_SMRT, "shakhov": shocks.TAU_RATIOS_SHAKHOV,
              "reduced": shocks.TAU_RATIOS_REDUCED}[table]
    ctx, params, cases, hs = _batch(olat, d, N, "f64", star, ratios)
    P.lb_set_schedule(ctx, width, 0, 0)   # one block per cell, or warps of 32-cell tiles
    for p, case in zip(params, cases):
        assert p["kx"] == case.k == 2
        np.testing.assert_allclose(p["taus"], _tau(case.model), rtol=1e-14)
    fa = _upload_batch(ctx, d, idx, hs)
    nsteps = 12
    out = P.lb_step(ctx, fa, ctx.new_state(), nsteps)
    assert P.lb_poll_status(ctx)[0] == 0
    got = _download_batch(ctx, d, idx, out, LENGTHS)
    for j, (case, h) in enumerate(zip(cases, hs)):
        for _ in range(nsteps):
            h = OS.step(h, case.model, case.geom)
        want = h.reshape(olat.q, -1)
        assert np.abs(got[j] - want).max() / np.abs(want).max() < 1e-11, (j, MACHS[j])


def test_fill_equilibrium_matches_oracle(lat):
    olat, d, idx = lat
    for prec, tol in (("f64", 1e-14), ("f32", 1e-7)):
        ctx, f, params, = shocks.setup_batch(d, 5, MACHS, LENGTHS, precision=prec, width=0.0,
                                             theta1=[shocks.TABLE3_THETA1[m] for m in MACHS])
        got = _download_batch(ctx, d, idx, f, LENGTHS)
        for j, (Ma, L) in enumerate(zip(MACHS, LENGTHS)):
            _, h = _oracle_case(olat, 5, Ma, L)
            want = h.reshape(olat.q, -1)
            assert np.abs(got[j] - want).max() / np.abs(want).max() < tol


def test_moments_match_oracle(lat):
    """lb_moments (rho, u, theta, sigma, q and every local coefficient d up to order 5) of a
    perturbed periodic line vs the oracle's macroscopic()."""
    olat, d, idx = lat
    nx, N = 90, 5
    rho, u, th = synthetic.taylor_green(0, amplitude=0.1, noise=3e-3, seed=4, shape=(1, 1, nx))
    f0 = OS.equilibrium(rho.ravel(), u.reshape(3, -1), th.ravel(), olat, N)
    rng = np.random.default_rng(4)
    f0 = (f0 * (1.0 + 0.05 * rng.standard_normal(f0.shape))).reshape(olat.q, 1, 1, nx)
    shift = (2, 0, 0)
    ctx = P.lb_init_lattice(_desc(d, shift), nx, N=N, precision="f64")
    f = upload(ctx, f0, idx)
    mask = P.LB_MOM_RHO | P.LB_MOM_U | P.LB_MOM_THETA | P.LB_MOM_SIGMA | P.LB_MOM_Q | P.LB_MOM_D
    out = P.lb_moments(ctx, f, mask).cpu().numpy()
    m = OS.macroscopic(f0, OS.Model(olat, N, tau_ref=1.0), OS.Geometry(shape=(1, 1, nx), shift=shift))
    want = np.concatenate([m["rho"][None], m["u"], m["theta"][None], m["sigma"], m["q"], m["d"]])
    assert out.shape == want.shape
    np.testing.assert_allclose(out, want, rtol=1e-10, atol=1e-11)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-6)])
@pytest.mark.parametrize("width", [1, 64])
def test_periodic_line_matches_oracle(lat, prec, tol, width):
    """Periodic line of 133 cells (a ragged 5-cell tail), shift 2, perturbed populations,
    1 and 4 steps."""
    olat, d, idx = lat
    nx, N = 133, 5
    rho, u, th = synthetic.taylor_green(0, amplitude=0.08, noise=2e-3, seed=9, shape=(1, 1, nx))
    f0 = OS.equilibrium(rho.ravel(), u.reshape(3, -1), th.ravel(), olat, N)
    rng = np.random.default_rng(9)
    f0 = (f0 * (1.0 + 0.02 * rng.standard_normal(f0.shape))).reshape(olat.q, 1, 1, nx)
    shift = (2, 0, 0)
    model = OS.Model(olat, N, tau_ref=0.7)
    geom = OS.Geometry(shape=(1, 1, nx), shift=shift)
    ctx = P.lb_init_lattice(_desc(d, shift), nx, N=N, precision=prec)
    P.lb_set_relaxation(ctx, _tau(model), True, 1.0)
    P.lb_set_schedule(ctx, width, 0, 0)
    fa = upload(ctx, f0, idx)
    h = download(ctx, fa, idx).reshape(f0.shape)     # start from the stored (rounded) state
    for nsteps in (1, 4):
        want = h
        for _ in range(nsteps):
            want = OS.step(want, model, geom)
        got = download(ctx, P.lb_step(ctx, fa.clone(), ctx.new_state(), nsteps), idx)
        assert np.abs(got - want.reshape(olat.q, -1)).max() / np.abs(want).max() < tol * nsteps


def test_schedules_and_graph_agree(lat):
    """FP64, 12 steps. Blocks of 32, 64 and 128 threads run the same per-step kernel and give
    the same bits; the persistent cooperative launch and its CUDA-graph replay are one other
    kernel (same bits as each other) whose compiled multiply-add fusion may differ, so it
    agrees with the per-step kernel to round-off (1e-14 relative)."""
    olat, d, idx = lat
    ctx, params, cases, hs = _batch(olat, d, 5, "f64")
    f0 = _upload_batch(ctx, d, idx, hs)
    runs = []
    for mode, sched in [("step", (128, 0, 0)), ("step", (32, 0, 0)), ("step", (64, 0, 0)),
                        ("step", (64, 1, 1)), ("graph", (32, 2, 1)), ("step", (1, 0, 0))]:
        P.lb_set_schedule(ctx, *sched)
        fa, fb = f0.clone(), ctx.new_state()
        out = P.lb_step_graph(ctx, fa, fb, 12) if mode == "graph" else P.lb_step(ctx, fa, fb, 12)
        assert P.lb_poll_status(ctx)[0] == 0
        runs.append(out.clone())
    for r in runs[1:3]:
        assert torch.equal(r, runs[0])
    assert torch.equal(runs[4], runs[3])
    scale = runs[0].abs().max()
    assert ((runs[3] - runs[0]).abs().max() / scale).item() < 1e-14
    # one block per cell sums in another order
    assert ((runs[5] - runs[0]).abs().max() / scale).item() < 1e-13


@pytest.mark.parametrize("width", [1, 64])
def test_caller_velocity_order_is_free(lat, width):
    """A context built on the oracle's own velocity order (any order is allowed) gives the
    same populations as one in library order, under the one-cell kernel and the block-staged
    one. In library order the block-staged kernel stages whole x-row groups with tensor-map
    boxes, in another order plane by plane: the data moved is the same, so the two agree
    bit for bit."""
    olat, d, idx = lat
    nx, N = 64, 4
    case, h = _oracle_case(olat, N, 3.0, nx)
    left, right = P.lb_rankine_hugoniot(3.0, theta1=case.theta1)
    w_oracle_order = np.empty(olat.q)
    w_oracle_order[idx] = d.w  # the same weights and c in both contexts, only the order differs
    outs = []
    for desc, order in ((_desc(d, (2, 0, 0)), idx),
                        (P.LatticeDesc(e=olat.e.astype(np.int8), w=w_oracle_order, c=d.c, degree=11,
                                       shift=(2, 0, 0)), np.arange(olat.q))):
        ctx = P.lb_init_lattice(desc, nx, N=N, precision="f64", bc_x=1)
        P.lb_set_relaxation(ctx, _tau(case.model), True, 1.0, left, right)
        P.lb_set_schedule(ctx, tile_width=width, blocks_per_sm=0, persistent=0)
        fa = upload(ctx, h, order)
        outs.append(download(ctx, P.lb_step(ctx, fa, ctx.new_state(), 5), order))
        assert P.lb_poll_status(ctx)[0] == 0
    want = h
    for _ in range(5):
        want = OS.step(want, case.model, case.geom)
    for g in outs:
        assert np.abs(g - want.reshape(olat.q, -1)).max() / np.abs(want).max() < 1e-11
    assert np.array_equal(outs[0], outs[1])


def test_paper_configuration_ma3_n5_against_golden(lat):
    """The paper's Ma = 3 run (Table 3 row, D3Q729, N = 5, 100 cells, step start, SMRT
    times), FP64, 1000 steps: moments vs the oracle's stored profiles."""
    path = os.path.join(os.path.dirname(__file__), "golden", "ma3_d3q729_n5.npz")
    gold = np.load(path)
    olat, d, idx = lat
    ctx, f0, params = shocks.setup_batch(d, 5, [3.0], [100], precision="f64", width=0.0,
                                         theta1=[0.333])
    assert params[0]["kx"] == int(gold["k"])
    np.testing.assert_allclose(params[0]["taus"][0], float(gold["tau_ref"]), rtol=1e-14)
    mask = P.LB_MOM_RHO | P.LB_MOM_U | P.LB_MOM_THETA | P.LB_MOM_Q
    fa, fb = f0, ctx.new_state()
    done = 0
    for cp in (200, 1000):
        out = P.lb_step(ctx, fa, fb, cp - done)
        fa, fb = out, (fb if out is fa else fa)
        done = cp
        assert P.lb_poll_status(ctx)[0] == 0
        m = P.lb_moments(ctx, fa, mask).cpu().numpy()
        assert np.abs(m[0] / gold[f"rho_{cp}"] - 1).max() < 1e-10
        assert np.abs(m[1] - gold[f"u_{cp}"]).max() < 1e-10
        assert np.abs(m[4] / gold[f"theta_{cp}"] - 1).max() < 1e-10
        assert np.abs(m[5] - gold[f"q_{cp}"]).max() < 1e-10


# ------------------------------------------------------------------ D3Q4913: Table 3, Ma = 7
@pytest.fixture(scope="module")
def lat17():
    o = OL.d3q4913()
    d = P.lb_lattice_named("D3Q4913")
    return o, d, lib_from_oracle(o, d)


def _ma7_case(olat, N, L):
    case = OK.shock_case(olat, N, 7.0, L, theta1=shocks.TABLE3_THETA1_D1Q17[7.0])
    st = case.states
    h = OK.initial_state(case, *[synthetic.step_blend(L, st[k + "1"], st[k + "2"])
                                 for k in ("rho", "u", "theta")])
    return case, h


@pytest.mark.parametrize("N", [4, 5])
def test_table3_ma7_d3q4913_matches_oracle(lat17, N):
    """FP64, Table 3's Ma = 7 row (D1Q17-P1 product, theta1 = 0.071, k_x = 3), two shocks of
    40 and 70 cells (ragged 32-cell tiles) from the step start, 6 steps, populations and
    moments vs the oracle."""
    olat, d, idx = lat17
    lengths = [40, 70]
    ctx, _, params = shocks.setup_batch(d, N, [7.0, 7.0], lengths, precision="f64", width=0.0,
                                        theta1=[0.071, 0.071])
    cases, hs = zip(*[_ma7_case(olat, N, L) for L in lengths])
    assert all(p["kx"] == c.k == 3 for p, c in zip(params, cases))
    fa = _upload_batch(ctx, d, idx, hs)
    out = P.lb_step(ctx, fa, ctx.new_state(), 6)
    assert P.lb_poll_status(ctx)[0] == 0
    got = _download_batch(ctx, d, idx, out, lengths)
    mom = P.lb_moments(ctx, out, P.LB_MOM_RHO | P.LB_MOM_U | P.LB_MOM_THETA | P.LB_MOM_Q).cpu().numpy()
    off = 0
    for j, (case, h) in enumerate(zip(cases, hs)):
        for _ in range(6):
            h = OS.step(h, case.model, case.geom)
        want = h.reshape(olat.q, -1)
        assert np.abs(got[j] - want).max() / np.abs(want).max() < 1e-11, j
        m = OS.macroscopic(h, case.model, case.geom)
        L = lengths[j]
        np.testing.assert_allclose(mom[0, off:off + L], m["rho"], rtol=1e-11)
        np.testing.assert_allclose(mom[4, off:off + L], m["theta"], rtol=1e-11)
        np.testing.assert_allclose(mom[5, off:off + L], m["q"][0], atol=1e-10)
        off += L


def test_d3q4913_periodic_line_f32(lat17):
    """FP32 periodic line of 45 cells (shift 3), perturbed populations, 2 steps."""
    olat, d, idx = lat17
    nx, N = 45, 5
    rho, u, th = synthetic.taylor_green(0, amplitude=0.08, noise=2e-3, seed=3, shape=(1, 1, nx))
    f0 = OS.equilibrium(rho.ravel(), u.reshape(3, -1), th.ravel(), olat, N)
    rng = np.random.default_rng(3)
    f0 = (f0 * (1.0 + 0.02 * rng.standard_normal(f0.shape))).reshape(olat.q, 1, 1, nx)
    shift = (3, 0, 0)
    model = OS.Model(olat, N, tau_ref=0.7)
    geom = OS.Geometry(shape=(1, 1, nx), shift=shift)
    ctx = P.lb_init_lattice(_desc(d, shift), nx, N=N, precision="f32")
    P.lb_set_relaxation(ctx, _tau(model), True, 1.0)
    fa = upload(ctx, f0, idx)
    h = download(ctx, fa, idx).reshape(f0.shape)
    for _ in range(2):
        h = OS.step(h, model, geom)
    got = download(ctx, P.lb_step(ctx, fa, ctx.new_state(), 2), idx)
    assert np.abs(got - h.reshape(olat.q, -1)).max() / np.abs(h).max() < 2e-6 * 2


def test_paper_configuration_ma7_n5_against_golden(lat17):
    """The paper's Ma = 7 run (Table 3 row, D3Q4913, N = 5, 100 cells, step start, SMRT
    times), FP64, 400 steps: moments vs the oracle's stored profiles."""
    gold = np.load(os.path.join(os.path.dirname(__file__), "golden", "ma7_d3q4913_n5.npz"))
    olat, d, idx = lat17
    ctx, f0, params = shocks.setup_batch(d, 5, [7.0], [100], precision="f64", width=0.0, theta1=[0.071])
    assert params[0]["kx"] == int(gold["k"])
    mask = P.LB_MOM_RHO | P.LB_MOM_U | P.LB_MOM_THETA | P.LB_MOM_Q
    fa, fb = f0, ctx.new_state()
    done = 0
    for cp in (100, 400):
        out = P.lb_step(ctx, fa, fb, cp - done)
        fa, fb = out, (fb if out is fa else fa)
        done = cp
        assert P.lb_poll_status(ctx)[0] == 0
        m = P.lb_moments(ctx, fa, mask).cpu().numpy()
        assert np.abs(m[0] / gold[f"rho_{cp}"] - 1).max() < 1e-10
        assert np.abs(m[1] - gold[f"u_{cp}"]).max() < 1e-10
        assert np.abs(m[4] / gold[f"theta_{cp}"] - 1).max() < 1e-10
        assert np.abs(m[5] - gold[f"q_{cp}"]).max() < 1e-10


# ------------------------------------------------------------------ ES-BGK target (Sec. 3)
@pytest.mark.parametrize("b", [-0.5, 0.4])
@pytest.mark.parametrize("width", [1, 64])
def test_es_bgk_table3_matches_oracle(lat, b, width):
    """FP64 ES-BGK (Eq. ES-BGK, one relaxation time, Holway's Gaussian target) on the three
    Table 3 rows, N = 5, 12 steps, each instance vs the oracle's ES-BGK run."""
    olat, d, idx = lat
    ctx, params, cases, hs = _batch(olat, d, 5, "f64")
    P.lb_set_schedule(ctx, width, 0, 0)
    P.lb_set_collision_model(ctx, -1, P.LB_MODEL_ES_BGK, b)
    fa = _upload_batch(ctx, d, idx, hs)
    out = P.lb_step(ctx, fa, ctx.new_state(), 12)
    assert P.lb_poll_status(ctx)[0] == 0
    got = _download_batch(ctx, d, idx, out, LENGTHS)
    for j, (case, h) in enumerate(zip(cases, hs)):
        case.model.es_b = b
        for _ in range(12):
            h = OS.step(h, case.model, case.geom)
        want = h.reshape(olat.q, -1)
        assert np.abs(got[j] - want).max() / np.abs(want).max() < 1e-11, (j, MACHS[j])


def test_es_bgk_periodic_f32_and_model_switch(lat):
    """FP32 ES-BGK on a perturbed periodic line (3 steps vs the oracle); switching the
    instance back to SMRT restores the SMRT step."""
    olat, d, idx = lat
    nx, N = 70, 5
    rho, u, th = synthetic.taylor_green(0, amplitude=0.08, noise=2e-3, seed=12, shape=(1, 1, nx))
    f0 = OS.equilibrium(rho.ravel(), u.reshape(3, -1), th.ravel(), olat, N)
    rng = np.random.default_rng(12)
    f0 = (f0 * (1.0 + 0.02 * rng.standard_normal(f0.shape))).reshape(olat.q, 1, 1, nx)
    shift = (2, 0, 0)
    geom = OS.Geometry(shape=(1, 1, nx), shift=shift)
    model = OS.Model(olat, N, tau_ref=0.8, es_b=-0.5)
    ctx = P.lb_init_lattice(_desc(d, shift), nx, N=N, precision="f32")
    P.lb_set_relaxation(ctx, _tau(model), True, 1.0)
    P.lb_set_collision_model(ctx, 0, P.LB_MODEL_ES_BGK, -0.5)
    fa = upload(ctx, f0, idx)
    h0 = download(ctx, fa, idx).reshape(f0.shape)
    h = h0
    for _ in range(3):
        h = OS.step(h, model, geom)
    got = download(ctx, P.lb_step(ctx, fa.clone(), ctx.new_state(), 3), idx)
    assert np.abs(got - h.reshape(olat.q, -1)).max() / np.abs(h).max() < 2e-6 * 3
    P.lb_set_collision_model(ctx, -1, P.LB_MODEL_SMRT, 0.0)
    model.es_b = None
    want = OS.step(h0, model, geom)
    got = download(ctx, P.lb_step(ctx, fa.clone(), ctx.new_state(), 1), idx)
    assert np.abs(got - want.reshape(olat.q, -1)).max() / np.abs(want).max() < 2e-6


def test_persistent_barrier_timeout_is_reported_and_recoverable(lat):
    """D3Q729 persistent launch whose grid barrier can never complete: every block gives up
    after its bounded wait, the health word says LB_HEALTH_TIMEOUT, and the context keeps
    working afterwards (the step then matches a fresh per-step run)."""
    olat, d, idx = lat
    ctx, params, cases, hs = _batch(olat, d, 5, "f64")
    f0 = _upload_batch(ctx, d, idx, hs)
    P.lb_set_schedule(ctx, 64, 1, 1)
    P.lb_test_barrier_timeout(ctx, f0.clone(), ctx.new_state())
    st, flags = P.lb_poll_status(ctx)
    assert st == 4 and flags & 2
    a = P.lb_step(ctx, f0.clone(), ctx.new_state(), 3)
    st, flags = P.lb_poll_status(ctx)
    assert st == 0 and flags == 0
    P.lb_set_schedule(ctx, 64, 0, 0)
    b = P.lb_step(ctx, f0.clone(), ctx.new_state(), 3)
    assert ((a - b).abs().max() / b.abs().max()).item() < 1e-14


def test_graph_needs_a_persistent_schedule(lat):
    """A small D3Q729 context starts on the one-cell-per-block schedule, which has no
    persistent form: the graph path refuses it instead of launching."""
    olat, d, idx = lat
    ctx, f0, _ = shocks.setup_batch(d, 5, [3.0], [100], precision="f64", width=0.0, theta1=[0.333])
    assert P.lb_get_schedule(ctx)["tile_width"] == 1
    with pytest.raises(P.SmrtError) as e:
        P.lb_step_graph(ctx, f0.clone(), ctx.new_state(), 4)
    assert e.value.status == 5
    with pytest.raises(P.SmrtError):
        P.lb_set_schedule(ctx, 1, 0, 1)
    P.lb_set_schedule(ctx, 32, 1, 1)
    out = P.lb_step_graph(ctx, f0.clone(), ctx.new_state(), 4)
    assert P.lb_poll_status(ctx)[0] == 0 and torch.isfinite(out).all()


# ------------------------------------------------------------------ mixed-Mach batch, graph path
@pytest.mark.parametrize("prec,tol_rho,tol_q", [("f64", 1e-10, 1e-9), ("f32", 5e-5, 1e-4)])
def test_mixed_mach_batch_graph_replay_against_golden(lat, prec, tol_rho, tol_q):
    """Shocks at Ma 1.5 / 2.5 / 4 / 5 on D3Q729 (N = 5, reference temperature of reading 11,
    tanh width 10, 80-140 cells), batched in one context and run as one persistent launch of
    1000 steps captured in a CUDA graph (lb_step_graph): rho, theta and q_x of every instance
    against the oracle's stored profiles (tests/golden/make_shock_golden.py mixed_d3q729_n5).
    FP64 to round-off; FP32 populations (no split precision on this set) to the stated
    tolerances, relative to rho, theta and to the instance's largest |q_x|."""
    path = os.path.join(os.path.dirname(__file__), "golden", "mixed_d3q729_n5.npz")
    gold = np.load(path)
    olat, d, idx = lat
    machs = [float(m) for m in gold["machs"]]
    lengths = [int(n) for n in gold["nx"]]
    ctx, f0, params = shocks.setup_batch(d, 5, machs, lengths, precision=prec, width=10.0)
    for j, p in enumerate(params):
        assert p["kx"] == int(gold[f"k_{j}"]) and abs(p["theta1"] - float(gold[f"theta1_{j}"])) < 1e-14
    P.lb_set_schedule(ctx, 64, 0, 1)
    fb = ctx.new_state()
    out = P.lb_step_graph(ctx, f0, fb, 1000)
    assert P.lb_poll_status(ctx)[0] == 0
    m = P.lb_moments(ctx, out, P.LB_MOM_RHO | P.LB_MOM_U | P.LB_MOM_THETA | P.LB_MOM_Q).cpu().numpy()
    off = np.concatenate([[0], np.cumsum(lengths)])
    for j in range(len(machs)):
        s = slice(off[j], off[j + 1])
        rho, th, q = gold[f"rho_1000_{j}"], gold[f"theta_1000_{j}"], gold[f"q_1000_{j}"]
        assert np.abs(m[0][s] / rho - 1).max() < tol_rho, (j, machs[j])
        assert np.abs(m[4][s] / th - 1).max() < tol_rho, (j, machs[j])
        assert np.abs(m[5][s] - q).max() / np.abs(q).max() < tol_q, (j, machs[j])
    ctx.close()


# ------------------------------------------------------------------ x-row sums on tensor cores
@pytest.mark.parametrize("sched", [(32, 0, 0), (32, 2, 1)])
def test_tensor_core_xrows_table3_f32(lat, sched):
    """FP32 with the x-row sums of the projection on the tensor cores (TF32 operands split in
    two, three products): the three Table 3 rows in one batch from the step start, 8 steps,
    vs the oracle at the FP32 bound of 2e-6 per step, and vs the CUDA-core x-rows."""
    olat, d, idx = lat
    ctx, params, cases, hs = _batch(olat, d, 5, "f32")
    fa = _upload_batch(ctx, d, idx, hs)
    nsteps = 8
    P.lb_set_schedule(ctx, *sched, tensor_cores=0)
    ref = P.lb_step(ctx, fa.clone(), ctx.new_state(), nsteps).clone()
    P.lb_set_schedule(ctx, *sched, tensor_cores=1)
    assert P.lb_get_schedule(ctx)["tensor_cores"] == 1
    out = P.lb_step(ctx, fa, ctx.new_state(), nsteps)
    assert P.lb_poll_status(ctx)[0] == 0
    got = _download_batch(ctx, d, idx, out, LENGTHS)
    for j, (case, h) in enumerate(zip(cases, hs)):
        for _ in range(nsteps):
            h = OS.step(h, case.model, case.geom)
        want = h.reshape(olat.q, -1)
        assert np.abs(got[j] - want).max() / np.abs(want).max() < 2e-6 * nsteps, (j, MACHS[j])
    scale = ref.abs().max()
    assert 0 < ((out - ref).abs().max() / scale).item() < 2e-6 * nsteps


def test_tensor_core_xrows_ma7_d3q4913_f32(lat17):
    """D3Q4913 (two k-steps of 8 velocities per x-row), Table 3's Ma = 7 row, FP32 with the
    tensor-core x-rows, two shocks of 40 and 70 cells, 6 steps, plain and persistent launches
    and a graph replay vs the oracle."""
    olat, d, idx = lat17
    lengths = [40, 70]
    ctx, _, params = shocks.setup_batch(d, 5, [7.0, 7.0], lengths, precision="f32", width=0.0,
                                        theta1=[0.071, 0.071])
    cases, hs = zip(*[_ma7_case(olat, 5, L) for L in lengths])
    f0 = _upload_batch(ctx, d, idx, hs)
    nsteps = 6
    wants = []
    for case, h in zip(cases, hs):
        for _ in range(nsteps):
            h = OS.step(h, case.model, case.geom)
        wants.append(h.reshape(olat.q, -1))
    for mode, sched in [("step", (32, 0, 0)), ("step", (32, 1, 1)), ("graph", (32, 2, 1))]:
        P.lb_set_schedule(ctx, *sched, tensor_cores=1)
        fa, fb = f0.clone(), ctx.new_state()
        out = P.lb_step_graph(ctx, fa, fb, nsteps) if mode == "graph" else P.lb_step(ctx, fa, fb, nsteps)
        assert P.lb_poll_status(ctx)[0] == 0
        got = _download_batch(ctx, d, idx, out, lengths)
        for j, want in enumerate(wants):
            assert np.abs(got[j] - want).max() / np.abs(want).max() < 2e-6 * nsteps, (mode, sched, j)


def test_tensor_core_xrows_refused_where_not_built(lat):
    """tensor_cores applies to float tensor-product lines with fixed ends, one warp per block."""
    olat, d, idx = lat
    ctx64, _, _ = shocks.setup_batch(d, 5, [3.0], [40], precision="f64", width=0.0, theta1=[0.333])
    with pytest.raises(P.SmrtError):
        P.lb_set_schedule(ctx64, 64, 0, 0, tensor_cores=1)
    ctx32, _, _ = shocks.setup_batch(d, 5, [3.0], [40], precision="f32", width=0.0, theta1=[0.333])
    with pytest.raises(P.SmrtError):
        P.lb_set_schedule(ctx32, 1, 0, 0, tensor_cores=1)   # one block per cell
    with pytest.raises(P.SmrtError):
        P.lb_set_schedule(ctx32, 32, 0, 0, tensor_cores=2)
    with pytest.raises(P.SmrtError):
        P.lb_set_schedule(ctx32, 64, 0, 0, tensor_cores=1)   # block tiles of two warps
    P.lb_set_schedule(ctx32, 32, 0, 0, tensor_cores=1)
    per = P.lb_init_lattice(_desc(d, (2, 0, 0)), 40, N=5, precision="f32")
    with pytest.raises(P.SmrtError):
        P.lb_set_schedule(per, 32, 0, 0, tensor_cores=1)  # periodic line
