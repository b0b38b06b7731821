"""Batched 1D shocks (many Mach numbers and lengths in one context): per-instance parity with
the oracle under every launch schedule (one launch per step with 32/64/128-cell tiles, the
persistent cooperative launch, its CUDA-graph replay), the split precision against FP64, the
autotuner and its cache, and failure detection of the persistent launch's bounded barrier."""
import numpy as np
import pytest

import synthetic
from oracle import lattice as OL
from oracle import shock as OK
from oracle import smrt as OS
from _lb import lib_from_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2401_11086_gb300 as P  # noqa: E402
from paper_2401_11086_gb300 import shocks  # noqa: E402
from paper_2401_11086_gb300.autotune import tuned_schedule  # noqa: E402

MACHS = [1.2, 2.0, 3.0, 4.5, 6.5]
LENGTHS = [40, 130, 64, 200, 96]


@pytest.fixture(scope="module")
def lat():
    olat = OL.d3q103()
    d = P.lb_lattice_named("D3Q103")
    return olat, d, lib_from_oracle(olat, d)


def _oracle_batch(olat, machs, lengths, N=4):
    cases, hs = [], []
    for Ma, L in zip(machs, lengths):
        case = OK.shock_case(olat, N, Ma, L)
        st = case.states
        W = 10.0
        h = OK.initial_state(case, *[synthetic.tanh_blend(L, W, st[k + "1"], st[k + "2"])
                                     for k in ("rho", "u", "theta")])
        cases.append(case)
        hs.append(h)
    return cases, hs


def _upload_batch(ctx, d, idx, hs):
    flat = np.concatenate([h.reshape(h.shape[0], -1) for h in hs], axis=1)
    st = ctx.new_state()
    ctx.planes(st)[:] = torch.from_numpy(np.ascontiguousarray(flat[idx] - d.w[:, None])).to(ctx.device, ctx.dtype)
    return st


def _download_instances(ctx, d, idx, st, lengths):
    arr = ctx.planes(st).double().cpu().numpy() + d.w[:, None]
    out = np.empty_like(arr)
    out[idx] = arr
    offs = np.concatenate([[0], np.cumsum(lengths)])
    return [out[:, offs[j]:offs[j + 1]] for j in range(len(lengths))]


def test_batch_frame_matches_oracle(lat):
    olat, d, idx = lat
    for Ma, L in zip(MACHS, LENGTHS):
        p = shocks.shock_params(Ma, d.c, 4)
        case = OK.shock_case(olat, 4, Ma, L)
        assert p["kx"] == case.k and abs(p["theta1"] - case.theta1) < 1e-14
        want = [case.model.tau_star[k] * case.model.tau_ref for k in
                [(2, 0), (2, 1), (3, 0), (3, 1), (4, 0), (4, 1), (4, 2)]]
        np.testing.assert_allclose(p["taus"], want, rtol=1e-14)


SCHEDULES = [("per-step", dict(tile_width=32, blocks_per_sm=0, persistent=0)),
             ("per-step", dict(tile_width=64, blocks_per_sm=0, persistent=0)),
             ("per-step", dict(tile_width=128, blocks_per_sm=0, persistent=0)),
             ("persistent", dict(tile_width=64, blocks_per_sm=1, persistent=1)),
             ("persistent", dict(tile_width=128, blocks_per_sm=0, persistent=1)),
             ("graph", dict(tile_width=32, blocks_per_sm=2, persistent=1))]


@pytest.mark.parametrize("mode,sched", SCHEDULES)
def test_batch_matches_oracle_under_every_schedule(lat, mode, sched):
    """FP64, 5 shocks (Ma 1.2..6.5, 40..200 cells, ragged tiles), 25 steps, each instance vs its
    own oracle run to 1e-11 -- identical for every schedule."""
    olat, d, idx = lat
    ctx, _, _ = shocks.setup_batch(d, 4, MACHS, LENGTHS, precision="f64")
    cases, hs = _oracle_batch(olat, MACHS, LENGTHS)
    P.lb_set_schedule(ctx, **sched)
    fa = _upload_batch(ctx, d, idx, hs)
    fb = ctx.new_state()
    nsteps = 25
    out = P.lb_step_graph(ctx, fa, fb, nsteps) if mode == "graph" else P.lb_step(ctx, fa, fb, nsteps)
    st, flags = P.lb_poll_status(ctx)
    assert st == 0, flags
    got = _download_instances(ctx, d, idx, out, LENGTHS)
    for j, (case, h) in enumerate(zip(cases, hs)):
        for _ in range(nsteps):
            h = OS.step(h, case.model, case.geom)
        want = h.reshape(olat.q, -1)
        assert np.abs(got[j] - want).max() / np.abs(want).max() < 1e-11, (j, MACHS[j])


def test_graph_replays_continue_the_run(lat):
    """Two replays of a 10-step graph equal 20 plain steps (FP64, bitwise)."""
    olat, d, idx = lat
    ctx, f0, _ = shocks.setup_batch(d, 4, MACHS, LENGTHS, precision="f64")
    P.lb_set_schedule(ctx, tile_width=64, blocks_per_sm=0, persistent=1)
    fa, fb = f0.clone(), ctx.new_state()
    P.lb_step_graph(ctx, fa, fb, 10)
    P.lb_step_graph(ctx, fa, fb, 10)
    ga, gb = f0.clone(), ctx.new_state()
    P.lb_set_schedule(ctx, tile_width=128, blocks_per_sm=0, persistent=0)
    P.lb_step(ctx, ga, gb, 20)
    assert torch.equal(fa, ga)


def test_split_batch_tracks_fp64(lat):
    olat, d, idx = lat
    machs, lengths = [1.5, 3.0, 5.0], [256, 384, 512]
    runs = {}
    for prec in ("f64", "f32c64"):
        ctx, f0, _ = shocks.setup_batch(d, 4, machs, lengths, precision=prec)
        P.lb_set_schedule(ctx, tile_width=128, blocks_per_sm=0, persistent=1)
        out = P.lb_step(ctx, f0, ctx.new_state(), 1000)
        assert P.lb_poll_status(ctx)[0] == 0
        runs[prec] = P.lb_moments(ctx, out, P.LB_MOM_RHO).cpu().numpy()[0]
    assert np.abs(runs["f32c64"] / runs["f64"] - 1).max() < 1e-5


def test_autotune_and_schedule_cache(lat, tmp_path):
    olat, d, idx = lat
    ctx, f0, _ = shocks.setup_batch(d, 4, MACHS, LENGTHS, precision="f32c64")
    path = str(tmp_path / "sched.json")
    s1 = tuned_schedule(ctx, f0, LENGTHS, trial_steps=6, path=path)
    assert s1["tile_width"] in (32, 64, 128) and s1["ms_per_step"] > 0
    assert P.lb_get_schedule(ctx)["tile_width"] == s1["tile_width"]
    P.lb_set_schedule(ctx, tile_width=128, blocks_per_sm=0, persistent=0)
    s2 = tuned_schedule(ctx, f0, LENGTHS, trial_steps=6, path=path)   # from the cache
    assert s2 == s1 and P.lb_get_schedule(ctx)["persistent"] == s1["persistent"]
    out = P.lb_step(ctx, f0.clone(), ctx.new_state(), 11)
    assert P.lb_poll_status(ctx)[0] == 0 and torch.isfinite(out).all()
    # the persistent-only choice (what lb_step_graph replays) is cached under its own key
    s3 = tuned_schedule(ctx, f0, LENGTHS, trial_steps=4, path=path, persistent=True)
    assert s3["persistent"] == 1 and P.lb_get_schedule(ctx)["persistent"] == 1
    assert tuned_schedule(ctx, f0, LENGTHS, trial_steps=4, path=path, persistent=True) == s3
    assert tuned_schedule(ctx, f0, LENGTHS, trial_steps=6, path=path) == s1
    a, b = f0.clone(), ctx.new_state()
    g = P.lb_step_graph(ctx, a, b, 5)
    assert P.lb_poll_status(ctx)[0] == 0 and torch.isfinite(g).all()


def test_persistent_barrier_timeout_is_reported_and_recoverable(lat):
    """A barrier that can never complete: every block gives up after its bounded wait, the
    health word says LB_HEALTH_TIMEOUT, and the context keeps working afterwards."""
    olat, d, idx = lat
    ctx, f0, _ = shocks.setup_batch(d, 4, MACHS, LENGTHS, precision="f64")
    P.lb_set_schedule(ctx, tile_width=64, blocks_per_sm=1, persistent=1)
    P.lb_test_barrier_timeout(ctx, f0.clone(), ctx.new_state())
    st, flags = P.lb_poll_status(ctx)
    assert st == 4 and flags & 2
    out = P.lb_step(ctx, f0.clone(), ctx.new_state(), 5)
    st, flags = P.lb_poll_status(ctx)
    assert st == 0 and flags == 0 and torch.isfinite(out).all()


def test_batched_shocks_64_instances_full_run(lat):
    """The batched workload: 64 shocks, Ma ~ U[1.2, 3] (the stable range of the degree-9 set),
    lengths from {512..8192} by seed,
    D3Q103, N = 4, FP32 with FP64 sums, 10000 steps, autotuned schedule: stays healthy and
    every instance keeps its Rankine-Hugoniot far fields."""
    olat, d, idx = lat
    machs, lengths = synthetic.batched_shocks(ma_range=(1.2, shocks.MA_STABLE_DEGREE9))
    ctx, f0, params = shocks.setup_batch(d, 4, machs, lengths, precision="f32c64")
    best = P.lb_autotune(ctx, f0.clone(), ctx.new_state(), 10)
    out = P.lb_step(ctx, f0, ctx.new_state(), 10000)
    st, flags = P.lb_poll_status(ctx)
    assert st == 0, (flags, best)
    m = P.lb_moments(ctx, out, P.LB_MOM_RHO | P.LB_MOM_THETA).cpu().numpy()
    offs = np.concatenate([[0], np.cumsum(lengths)])
    for j, p in enumerate(params):
        rho = m[0, offs[j]:offs[j + 1]]
        assert abs(rho[3] / p["left"]["rho"] - 1) < 1e-4, (j, machs[j])
        assert abs(rho[-4] / p["right"]["rho"] - 1) < 1e-4, (j, machs[j])
