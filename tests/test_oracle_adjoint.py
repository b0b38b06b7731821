"""Pins of the oracle's discrete adjoint: complex-step Jacobian products against central finite
differences, the streaming transpose against the dot-product identity, whole-run gradients with
checkpointing against finite differences of the loss, and the inert bulk time (Sec. 4.2)."""
import numpy as np
import pytest

import synthetic
from oracle import adjoint as A
from oracle import lattice as L
from oracle import shock as K
from oracle import smrt as S


@pytest.fixture(scope="module")
def lat39():
    return L.d3q39()


def test_stream_transpose_is_the_adjoint(lat39):
    rng = np.random.default_rng(0)
    for geom in (S.Geometry(shape=(4, 5, 7), shift=(1, 0, 0)),
                 S.Geometry(shape=(1, 1, 12), shift=(2, 0, 0), fixed_x=True,
                            ghost_left=np.zeros(lat39.q), ghost_right=np.zeros(lat39.q))):
        h = rng.random((lat39.q,) + geom.shape)
        g = rng.random((lat39.q,) + geom.shape)
        lhs = np.sum(S.stream(h, lat39, geom) * g)
        rhs = np.sum(h * A.stream_transpose(g, lat39, geom))
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("name,N", [("D3Q39", 3), ("D3Q103", 4)])
def test_collide_vjp_matches_central_differences(name, N):
    lat = L.by_name(name)
    rng = np.random.default_rng(1)
    rho, u, th = 1 + 0.1 * rng.random(4), 0.2 * rng.standard_normal((3, 4)), 0.9 + 0.2 * rng.random(4)
    f = S.equilibrium(rho, u, th, lat, N) * (1 + 0.05 * rng.standard_normal((lat.q, 4)))
    model = S.Model(lat, N, tau_ref=1.0)
    taus = A.model_taus(model) * (1 + 0.1 * rng.random(len(A.tau_keys(N))))
    lam = rng.standard_normal(f.shape)
    fbar, gtau = A.collide_vjp(f, lam, model, taus)
    m = A.model_with_taus(model, taus)
    v = rng.standard_normal(f.shape)
    eps = 1e-6
    fd = np.sum(lam * (S.collide(f + eps * v, m) - S.collide(f - eps * v, m))) / (2 * eps)
    assert abs(fd - np.sum(fbar * v)) < 1e-7 * max(1.0, abs(fd))
    for p in range(len(taus)):
        tp, tm = taus.copy(), taus.copy()
        tp[p] += eps
        tm[p] -= eps
        fd = np.sum(lam * (S.collide(f, A.model_with_taus(model, tp)) -
                           S.collide(f, A.model_with_taus(model, tm)))) / (2 * eps)
        assert abs(fd - gtau[p]) < 1e-7 * max(1.0, abs(fd)), p
    # the bulk part (2,1) is identically zero for the full 3-dof temperature
    assert abs(gtau[1]) < 1e-12


def _small_shock(Ma=1.5, nx=40, N=3):
    lat = L.d3q39()
    case = K.shock_case(lat, N, Ma, nx)
    st = case.states
    h0 = K.initial_state(case, *[synthetic.tanh_blend(nx, 4.0, st[k + "1"], st[k + "2"])
                                 for k in ("rho", "u", "theta")])
    return lat, case, h0


def test_run_gradient_matches_finite_differences():
    """Loss of the differentiable shock after 24 steps (checkpoint every 10) against central
    differences of whole runs, h = 1e-4 relative, for every relaxation parameter."""
    lat, case, h0 = _small_shock()
    model, geom = case.model, case.geom
    taus0 = A.model_taus(model)
    target_taus = taus0 * (1 + synthetic.perturbed(np.zeros(len(taus0)) + 1, 0.2, seed=7) - 1)
    mt = A.model_with_taus(model, target_taus)
    h = h0
    for _ in range(24):
        h = S.step(h, mt, geom)
    target = A.loss_moments(h, mt, geom)
    Lval, g, _ = A.run_gradient(h0, model, geom, taus0, 24, target, checkpoint_every=10)
    assert Lval > 0
    gmax = np.abs(g).max()
    for p in range(len(taus0)):
        hstep = 1e-4 * taus0[p]
        vals = []
        for sgn in (1, -1):
            t = taus0.copy()
            t[p] += sgn * hstep
            mm = A.model_with_taus(model, t)
            hh = h0
            for _ in range(24):
                hh = S.step(hh, mm, geom)
            vals.append(A.shock_loss(hh, mm, geom, target))
        fd = (vals[0] - vals[1]) / (2 * hstep)
        assert abs(fd - g[p]) <= 1e-4 * abs(fd) + 1e-9 * gmax, (p, fd, g[p])
    assert abs(g[1]) < 1e-10 * max(1.0, np.abs(g).max())
