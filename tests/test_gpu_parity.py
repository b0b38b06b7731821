"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Inputs are seeded and synthetic; every expected value comes from ``oracle/`` (or a golden file
written by a script that calls only the oracle). Tolerances: FP64 kernels agree with the oracle
to round-off (1e-11 relative to the population scale); FP32 kernels to 2e-6 per step relative
to the population scale; FP32 runs of many steps are held to the mass-conservation
bound |delta rho| / rho <= 1e-5.
"""
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


@pytest.fixture(scope="module")
def lats():
    out = {}
    for name in ("D3Q39", "D3Q103"):
        o = OL.by_name(name)
        d = P.lb_lattice_named(name)
        out[name] = (o, d, lib_from_oracle(o, d))
    return out


def _desc(d, shift):
    return P.LatticeDesc(e=d.e, w=d.w, c=d.c, degree=d.degree, shift=tuple(shift))


def _tau(model):
    N = model.N
    keys = [(n, m) for n in range(2, N + 1) for m in range(n // 2 + 1)]
    return [model.tau_star[k] * model.tau_ref for k in keys]


def _perturbed_box(olat, N, shape, seed=5, eps=0.02):
    rho, u, th = synthetic.taylor_green(0, amplitude=0.08, noise=2e-3, seed=seed, shape=shape)
    f = OS.equilibrium(rho.ravel(), u.reshape(3, -1), th.ravel(), olat, N)
    rng = np.random.default_rng(seed)
    return f * (1.0 + eps * rng.standard_normal(f.shape))


@pytest.mark.parametrize("name,N,prec,tol", [("D3Q39", 3, "f64", 1e-12), ("D3Q39", 3, "f32", 2e-6),
                                              ("D3Q103", 4, "f64", 1e-12), ("D3Q103", 4, "f32", 2e-6),
                                              ("D3Q103", 3, "f32c64", 2e-6), ("D3Q39", 3, "f32c64", 2e-6)])
def test_box_steps_match_oracle(lats, name, N, prec, tol):
    """Periodic box (several x-blocks and a ragged tail): 1 and 3 steps from a perturbed state."""
    olat, d, idx = lats[name]
    shape = (5, 6, 133)                     # nz, ny, nx: 2 blocks of 128 cells + ragged 5
    model = OS.Model(olat, N, tau_ref=0.9)
    geom = OS.Geometry(shape=shape, shift=(1, 0, 0))
    f0 = _perturbed_box(olat, N, shape).reshape(olat.q, *shape)
    ctx = P.lb_init_lattice(_desc(d, (1, 0, 0)), shape[2], shape[1], shape[0], N=N, precision=prec)
    P.lb_set_relaxation(ctx, _tau(model), True, 1.0)
    fa = upload(ctx, f0, idx)
    fb = ctx.new_state()
    if prec != "f64":   # compare against the oracle started from the rounded input
        f0 = download(ctx, fa, idx).reshape(f0.shape)
    want = f0
    for nsteps in (1, 3):
        want_n = want
        for _ in range(nsteps):
            want_n = OS.step(want_n, model, geom)
        fa2 = upload(ctx, f0, idx)
        got = download(ctx, P.lb_step(ctx, fa2, fb, nsteps), idx)
        scale = np.abs(want_n).max()
        err = np.abs(got - want_n.reshape(olat.q, -1)).max() / scale
        assert err < tol * nsteps, (nsteps, err)
    assert P.lb_poll_status(ctx)[0] == 0


@pytest.mark.parametrize("name,N,nx,shift", [("D3Q103", 4, 150, 1), ("D3Q39", 3, 70, 2), ("D3Q103", 4, 20, 0)])
def test_periodic_line_split_precision_matches_oracle(lats, name, N, nx, shift):
    """Split precision on a periodic line (staged pulls; wrapped pulls read the state directly):
    several 32-cell warp parts and a ragged tail, and a line shorter than one warp, 1 and 3
    steps from a perturbed state."""
    olat, d, idx = lats[name]
    shape = (1, 1, nx)
    model = OS.Model(olat, N, tau_ref=0.9)
    geom = OS.Geometry(shape=shape, shift=(shift, 0, 0))
    f0 = _perturbed_box(olat, N, shape).reshape(olat.q, *shape)
    ctx = P.lb_init_lattice(_desc(d, (shift, 0, 0)), nx, N=N, precision="f32c64", bc_x=0)
    P.lb_set_relaxation(ctx, _tau(model), True, 1.0)
    fa = upload(ctx, f0, idx)
    f0 = download(ctx, fa, idx).reshape(f0.shape)
    fb = ctx.new_state()
    for nsteps in (1, 3):
        want = f0
        for _ in range(nsteps):
            want = OS.step(want, model, geom)
        got = download(ctx, P.lb_step(ctx, upload(ctx, f0, idx), fb, nsteps), idx)
        err = np.abs(got - want.reshape(olat.q, -1)).max() / np.abs(want).max()
        assert err < 2e-6 * nsteps, (nsteps, err)
    assert P.lb_poll_status(ctx)[0] == 0


@pytest.mark.parametrize("name,N,prec,tol", [("D3Q39", 3, "f64", 1e-13), ("D3Q39", 3, "f32", 1e-7),
                                              ("D3Q103", 4, "f64", 1e-13)])
def test_fill_equilibrium_matches_oracle(lats, name, N, prec, tol):
    olat, d, idx = lats[name]
    shape = (4, 5, 130)
    rho, u, th = synthetic.taylor_green(0, amplitude=0.1, noise=1e-2, seed=2, shape=shape)
    shift = (1, 0, 0)
    ctx = P.lb_init_lattice(_desc(d, shift), shape[2], shape[1], shape[0], N=N, precision=prec)
    ubar = d.c * np.array(shift, dtype=float)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()  # noqa: E731
    f = ctx.new_state()
    P.lb_fill_equilibrium(ctx, f, dev(rho.ravel()), dev((u.reshape(3, -1) + ubar[:, None])),
                          dev(th.ravel()))
    want = OS.equilibrium(rho.ravel(), u.reshape(3, -1), th.ravel(), olat, N)
    got = download(ctx, f, idx)
    assert np.abs(got - want).max() / np.abs(want).max() < tol


@pytest.mark.parametrize("name,N", [("D3Q39", 3), ("D3Q103", 4)])
def test_moments_match_oracle(lats, name, N):
    olat, d, idx = lats[name]
    shape = (4, 5, 140)
    shift = (1, 0, 0)
    f0 = _perturbed_box(olat, N, shape, eps=0.05).reshape(olat.q, *shape)
    model = OS.Model(olat, N, tau_ref=1.0)
    geom = OS.Geometry(shape=shape, shift=shift)
    ctx = P.lb_init_lattice(_desc(d, shift), shape[2], shape[1], shape[0], N=N, precision="f64")
    f = upload(ctx, f0, idx)
    mask = P.LB_MOM_RHO | P.LB_MOM_U | P.LB_MOM_THETA | P.LB_MOM_SIGMA | P.LB_MOM_Q | P.LB_MOM_D
    out = P.lb_moments(ctx, f, mask).cpu().numpy()
    m = OS.macroscopic(f0, model, geom)
    want = np.concatenate([m["rho"][None], m["u"], m["theta"][None], m["sigma"], m["q"], m["d"]])
    assert out.shape == want.shape
    np.testing.assert_allclose(out, want, rtol=1e-10, atol=1e-11)


def _shock_setup(olat, d, N, Ma, nx, width, prec, ell=2.0):
    case = OK.shock_case(olat, N, Ma, nx, ell_cells=ell)
    st = case.states
    fields = [synthetic.tanh_blend(nx, width, st[k + "1"], st[k + "2"]) for k in ("rho", "u", "theta")]
    h0 = OK.initial_state(case, *fields)
    left, right = P.lb_rankine_hugoniot(Ma, theta1=case.theta1)
    ctx = P.lb_init_lattice(_desc(d, (case.k, 0, 0)), nx, N=N, precision=prec, bc_x=1)
    P.lb_set_relaxation(ctx, _tau(case.model), True, 1.0, left, right)
    return case, h0, ctx


def test_shock_ma12_d3q39_fp64_full_run(lats):
    """Ma = 1.2 shock, D3Q39, N = 3, FP64, 400 cells, 2000 steps: whole run vs the oracle."""
    olat, d, idx = lats["D3Q39"]
    case, h, ctx = _shock_setup(olat, d, 3, 1.2, 400, 10.0, "f64")
    fa = upload(ctx, h, idx)
    fb = ctx.new_state()
    for _ in range(2000):
        h = OS.step(h, case.model, case.geom)
    got = P.lb_step(ctx, fa, fb, 2000)
    assert P.lb_poll_status(ctx)[0] == 0
    g = download(ctx, got, idx)
    assert np.abs(g - h.reshape(olat.q, -1)).max() / np.abs(h).max() < 1e-11
    mom = P.lb_moments(ctx, got, P.LB_MOM_RHO | P.LB_MOM_U | P.LB_MOM_THETA | P.LB_MOM_Q).cpu().numpy()
    m = OS.macroscopic(h, case.model, case.geom)
    np.testing.assert_allclose(mom[0], m["rho"], rtol=1e-11)
    np.testing.assert_allclose(mom[1], m["u"][0], rtol=1e-11)
    np.testing.assert_allclose(mom[4], m["theta"], rtol=1e-11)
    np.testing.assert_allclose(mom[5], m["q"][0], atol=1e-11)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32c64", 3e-6), ("f32", 3e-6)])
def test_shock_ma3_d3q103_n4_steps(lats, prec, tol):
    """Ma = 3 shock on the degree-9 set, N = 4, 300 cells (3 blocks, ragged tail), 40 steps."""
    olat, d, idx = lats["D3Q103"]
    case, h, ctx = _shock_setup(olat, d, 4, 3.0, 300, 20.0, prec)
    fa = upload(ctx, h, idx)
    if prec != "f64":
        h = download(ctx, fa, idx).reshape(h.shape)
    fb = ctx.new_state()
    for _ in range(40):
        h = OS.step(h, case.model, case.geom)
    got = download(ctx, P.lb_step(ctx, fa, fb, 40), idx)
    assert np.abs(got - h.reshape(olat.q, -1)).max() / np.abs(h).max() < tol * 40


def test_shock_ma3_full_run_against_golden(lats):
    """Ma = 3, 2048 cells, D3Q103, N = 4, FP32 with FP64 sums, 20000 steps vs the oracle's
    stored profiles: |delta rho|/rho <= 1e-5, and theta, q_x alike."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "ma3_d3q103_n4.npz")
    if not os.path.exists(path):
        pytest.skip("golden profile not generated")
    gold = np.load(path)
    olat, d, idx = lats["D3Q103"]
    case, h, ctx = _shock_setup(olat, d, 4, 3.0, 2048, 20.0, "f32c64")
    fa = upload(ctx, h, idx)
    fb = ctx.new_state()
    cur = P.lb_step(ctx, fa, fb, 2000)
    mom = P.lb_moments(ctx, cur, P.LB_MOM_RHO | P.LB_MOM_U | P.LB_MOM_THETA | P.LB_MOM_Q).cpu().numpy()
    assert np.abs(mom[0] / gold["rho_2000"] - 1).max() < 1e-5
    other = fa if cur is fb else fb
    cur = P.lb_step(ctx, cur, other, 18000)
    assert P.lb_poll_status(ctx)[0] == 0
    mom = P.lb_moments(ctx, cur, P.LB_MOM_RHO | P.LB_MOM_U | P.LB_MOM_THETA | P.LB_MOM_Q).cpu().numpy()
    assert np.abs(mom[0] / gold["rho_20000"] - 1).max() < 1e-5
    assert np.abs(mom[4] / gold["theta_20000"] - 1).max() < 1e-5
    qs = np.abs(gold["q_20000"]).max()
    assert np.abs(mom[5] - gold["q_20000"]).max() / qs < 1e-4


def test_box_256_sampled_one_step(lats):
    """Full-size periodic box (256^3, D3Q39, N = 3, FP32) in the benchmark's launch shape:
    one step from the oracle's Taylor-Green equilibrium, 4096 sampled cells vs the oracle."""
    olat, d, idx = lats["D3Q39"]
    n = 256
    rho, u, th = synthetic.taylor_green(n)
    model = OS.Model(olat, 3, tau_ref=2.0 * olat.c)
    geom = OS.Geometry(shape=(n, n, n))
    ctx = P.lb_init_lattice(_desc(d, (0, 0, 0)), n, n, n, N=3, precision="f32")
    P.lb_set_relaxation(ctx, _tau(model), True, 1.0)
    fa = ctx.new_state()
    planes = ctx.planes(fa)
    h0 = np.empty((olat.q, n, n, n))
    for z0 in range(0, n, 32):       # build the oracle equilibrium in slabs
        sl = slice(z0, z0 + 32)
        fz = OS.equilibrium(rho[sl].ravel(), u[:, sl].reshape(3, -1), th[sl].ravel(), olat, 3)
        h0[:, sl] = fz.reshape(olat.q, 32, n, n)
    for i_lib, i_or in enumerate(idx):     # the oracle starts from the rounded deviations
        h0[i_or] = (h0[i_or] - d.w[i_lib]).astype(np.float32).astype(np.float64) + d.w[i_lib]
    for i_lib, i_or in enumerate(idx):     # states hold f_i - w_i
        planes[i_lib] = torch.from_numpy((h0[i_or].ravel() - d.w[i_lib]).astype(np.float32)).cuda()
    fb = ctx.new_state()
    got_t = P.lb_step(ctx, fa, fb, 1)
    rng = np.random.default_rng(11086)
    cells = np.concatenate([rng.choice(n ** 3, 4000, replace=False),
                            [0, n - 1, n * n - 1, n ** 3 - 1, n ** 3 - n, 255 * n * n]])
    pre = OS.pull_cells(h0, olat, geom, cells)
    want = OS.collide(pre, model)
    got = ctx.planes(got_t)[:, torch.from_numpy(cells).cuda()].double().cpu().numpy() + d.w[:, None]
    got_o = np.empty_like(got)
    got_o[idx] = got
    assert np.abs(got_o - want).max() / np.abs(want).max() < 2e-6
    # 1000 further steps: total mass sum_cells (1 + sum_i df_i) kept to FP32 round-off (the
    # states store deviations, so the float rounding of w_i leaves no systematic drift)
    m0 = ctx.planes(got_t).double().sum().item()
    cur = P.lb_step(ctx, got_t, fa if got_t is fb else fb, 1000)
    assert P.lb_poll_status(ctx)[0] == 0
    m1 = ctx.planes(cur).double().sum().item()
    assert abs(m1 - m0) / n ** 3 < 1e-7


def test_unstable_state_sets_health_flag(lats):
    """Failure detection on the host-made bad input: a negative-density cell is reported."""
    olat, d, idx = lats["D3Q39"]
    shape = (4, 4, 8)
    f0 = _perturbed_box(olat, 3, shape).reshape(olat.q, -1)
    f0[:, 17] = -0.1
    ctx = P.lb_init_lattice(_desc(d, (0, 0, 0)), shape[2], shape[1], shape[0], N=3, precision="f64")
    P.lb_set_relaxation(ctx, [1.0, 1.0, 1.0, 1.0], True, 1.0)
    fa = upload(ctx, f0, idx)
    P.lb_step(ctx, fa, ctx.new_state(), 1)
    st, flags = P.lb_poll_status(ctx)
    assert st == 3 and flags & 1
    st, flags = P.lb_poll_status(ctx)        # cleared by the previous poll
    assert st == 0 and flags == 0


def test_invalid_calls_are_rejected(lats):
    olat, d, idx = lats["D3Q39"]
    ctx = P.lb_init_lattice(_desc(d, (0, 0, 0)), 8, 8, 8, N=3, precision="f32")
    f = ctx.new_state()
    with pytest.raises(P.SmrtError):            # relaxation not set yet
        P.lb_step(ctx, f, ctx.new_state(), 1)
    with pytest.raises(P.SmrtError):
        P.lb_set_relaxation(ctx, [1.0, -1.0, 1.0, 1.0], True, 1.0)
    P.lb_set_relaxation(ctx, [1.0, 1.0, 1.0, 1.0], True, 1.0)
    with pytest.raises(P.SmrtError):            # same buffer twice
        P.lb_step(ctx, f, f, 1)
    with pytest.raises(P.SmrtError):            # reach 3 does not fit a 2-cell axis
        P.lb_init_lattice(_desc(d, (0, 0, 0)), 8, 2, 8, N=3)
    with pytest.raises(P.SmrtError):            # N = 4 needs degree 8
        P.lb_init_lattice(_desc(d, (0, 0, 0)), 8, 8, 8, N=4)


# ---------------------------------------------------------------------------- ES-BGK
@pytest.mark.parametrize("name,N,prec,tol", [("D3Q39", 3, "f64", 1e-12), ("D3Q39", 3, "f32", 2e-6),
                                              ("D3Q103", 4, "f64", 1e-12), ("D3Q103", 4, "f32", 2e-6),
                                              ("D3Q103", 4, "f32c64", 2e-6)])
def test_es_bgk_box_steps_match_oracle(lats, name, N, prec, tol):
    """The ES-BGK model (Sec. 3, Eq. ES-BGK, b = -1/2: Pr = 2/3) on the D3Q39 / D3Q103 kernels:
    periodic box (two x-blocks and a ragged tail), 1 and 3 steps from a perturbed state."""
    olat, d, idx = lats[name]
    shape = (4, 5, 133)
    model = OS.Model(olat, N, tau_ref=0.9, es_b=-0.5)
    geom = OS.Geometry(shape=shape, shift=(1, 0, 0))
    f0 = _perturbed_box(olat, N, shape).reshape(olat.q, *shape)
    ctx = P.lb_init_lattice(_desc(d, (1, 0, 0)), shape[2], shape[1], shape[0], N=N, precision=prec)
    P.lb_set_relaxation(ctx, _tau(model), True, 1.0)
    P.lb_set_collision_model(ctx, -1, P.LB_MODEL_ES_BGK, -0.5)
    fa = upload(ctx, f0, idx)
    fb = ctx.new_state()
    if prec != "f64":
        f0 = download(ctx, fa, idx).reshape(f0.shape)
    for nsteps in (1, 3):
        want = f0
        for _ in range(nsteps):
            want = OS.step(want, model, geom)
        got = download(ctx, P.lb_step(ctx, upload(ctx, f0, idx), fb, nsteps), idx)
        err = np.abs(got - want.reshape(olat.q, -1)).max() / np.abs(want).max()
        assert err < tol * nsteps, (nsteps, err)
    assert P.lb_poll_status(ctx)[0] == 0


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32c64", 3e-6)])
def test_es_bgk_shock_steps_match_oracle(lats, prec, tol):
    """ES-BGK on a Ma = 2 shock (D3Q103, N = 4, 300 cells, fixed ends; the split precision runs
    the staged line kernel), 40 steps; the adjoint, written for SMRT, refuses such a context."""
    olat, d, idx = lats["D3Q103"]
    case, h, ctx = _shock_setup(olat, d, 4, 2.0, 300, 10.0, prec)
    case.model.es_b = -0.5
    P.lb_set_collision_model(ctx, -1, P.LB_MODEL_ES_BGK, -0.5)
    fa = upload(ctx, h, idx)
    if prec != "f64":
        h = download(ctx, fa, idx).reshape(h.shape)
    fb = ctx.new_state()
    for _ in range(40):
        h = OS.step(h, case.model, case.geom)
    got = download(ctx, P.lb_step(ctx, fa, fb, 40), idx)
    assert np.abs(got - h.reshape(olat.q, -1)).max() / np.abs(h).max() < tol * 40
    assert P.lb_poll_status(ctx)[0] == 0
    if prec == "f64":
        lam = torch.zeros(ctx.state_elems, dtype=torch.float64, device="cuda")
        dtau = torch.zeros(7, dtype=torch.float64, device="cuda")
        with pytest.raises(P.SmrtError):
            P.lb_step_adjoint(ctx, fa, lam, torch.zeros_like(lam), dtau)
