"""Pins of the oracle's collision (Eq. SMRT), frames (binomial transform) and rebuild (Eq. fi)."""
import numpy as np
import pytest
from numpy.polynomial.hermite_e import hermegauss

import synthetic
from oracle import hermite as H
from oracle import lattice as L
from oracle import smrt as S
from oracle import tensors as T
from _golden import frac, rows

CASES = [("D3Q39", 3), ("D3Q103", 4), ("D3Q103", 3), ("D3Q729", 5), ("D3Q729", 4), ("D3Q4913", 5)]


@pytest.fixture(scope="module")
def lats():
    return {n: L.by_name(n) for n in ("D3Q39", "D3Q103", "D3Q729", "D3Q4913")}


def _random_state(lat, N, ncell=7, seed=1, eps=0.05):
    rng = np.random.default_rng(seed)
    rho = 0.8 + 0.4 * rng.random(ncell)
    u = 0.3 * rng.standard_normal((3, ncell))
    th = 0.7 + 0.6 * rng.random(ncell)
    feq = S.equilibrium(rho, u, th, lat, N)
    f = feq * (1.0 + eps * rng.standard_normal(feq.shape))
    return f, feq


def test_table4_ratios_match_golden():
    for model, n, m, r in rows("table4_relaxation.txt"):
        table = S.TAU_STAR_SMRT if model == "SMRT" else S.TAU_STAR_SHAKHOV
        assert abs(table[(int(n), int(m))] - float(frac(r))) < 1e-15


@pytest.mark.parametrize("name,N", CASES)
def test_route_a_equals_route_b(lats, name, N):
    """Direct local projection = absolute projection followed by the binomial transform."""
    lat = lats[name]
    f, _ = _random_state(lat, N, eps=0.2)
    rho, u, th = S.conserved(f, lat)
    dA = S.local_direct(f, lat, N, u, th)
    dB = S.to_local(S.absolute(f, lat, N), N, u, th)
    np.testing.assert_allclose(dA, dB, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(S.to_absolute(dB, N, u, th), S.absolute(f, lat, N), atol=1e-13)
    # d^(0) = rho, d^(1) = 0, tr d^(2) = 0 (theta is the full 3-dof kinetic temperature)
    np.testing.assert_allclose(dA[0], rho, rtol=1e-14)
    np.testing.assert_allclose(dA[1:4], 0.0, atol=1e-13)
    np.testing.assert_allclose(dA[4] + dA[7] + dA[9], 0.0, atol=1e-13)


def test_equilibrium_coefficients_against_numerical_integration():
    """Appendix B: a^(n) of a 1D Maxwellian equals its Hermite projection by quadrature."""
    x, wq = hermegauss(80)                     # integrates p(x) exp(-x^2/2) exactly, deg <= 159
    wq = wq / np.sqrt(2 * np.pi)
    for u, th in [(0.0, 1.0), (0.7, 0.6), (-1.1, 1.4), (0.3, 1.9)]:
        ratio = np.exp(x * x / 2 - (x - u) ** 2 / (2 * th)) / np.sqrt(th)   # f / omega
        he = H.he_1d(8, x)
        for n in range(9):
            want = np.sum(wq * ratio * he[n])
            got = S.g_coef(n, u, th)
            assert abs(got - want) < 1e-9 * max(1.0, abs(want)), (u, th, n)


@pytest.mark.parametrize("name,N", CASES)
def test_discrete_equilibrium_has_maxwellian_moments(lats, name, N):
    """sum_i f^eq_i xi^alpha = integral of the Maxwellian times xi^alpha for |alpha| <= N."""
    lat = lats[name]
    rho, u, th = np.array([1.3]), np.array([[0.4], [-0.2], [0.1]]), np.array([0.85])
    f = S.equilibrium(rho, u, th, lat, N)[:, 0]
    x, wq = hermegauss(40)
    wq = wq / np.sqrt(2 * np.pi)
    for a in H.multi_indices_upto(N):
        got = np.sum(f * np.prod(lat.xi ** np.array(a), axis=1))
        want = rho[0]
        for k in range(3):     # 1D moment of N(u_k, th): integrate (u + sqrt(th) x)^a dN(0,1)
            want *= np.sum(wq * (u[k, 0] + np.sqrt(th[0]) * x) ** a[k])
        assert abs(got - want) < 1e-12 * max(1, abs(want)), a


@pytest.mark.parametrize("name,N", CASES)
def test_collision_conserves_mass_momentum_energy(lats, name, N):
    lat = lats[name]
    f, _ = _random_state(lat, N, eps=0.3)
    model = S.Model(lat, N, tau_ref=0.7)
    h = S.collide(f, model)
    for x0, x1 in zip(S.conserved(f, lat), S.conserved(h, lat)):
        np.testing.assert_allclose(x1, x0, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("name,N", CASES)
def test_equilibrium_is_fixed_point(lats, name, N):
    lat = lats[name]
    _, feq = _random_state(lat, N)
    h = S.collide(feq, S.Model(lat, N, tau_ref=1.3))
    np.testing.assert_allclose(h, feq, atol=1e-14)


@pytest.mark.parametrize("name,N", CASES)
def test_equal_times_reduce_to_regularised_bgk(lats, name, N):
    """Sec. 3: all tau equal gives BGK, here f' = f^eq,N + (1 - 1/tau) Pi_N (f - f^eq,N).

    Pi_N is the absolute-frame Hermite projection truncated at N written out directly from
    Eqs. an and fi: no frames, no binomial transform, no irreducible projectors.
    """
    lat = lats[name]
    f, _ = _random_state(lat, N, eps=0.2)
    tau_c = 0.9
    model = S.Model(lat, N, tau_ref=tau_c, tau_star={k: 1.0 for k in S.TAU_STAR_SMRT},
                    maxwell_law=False)
    rho, u, th = S.conserved(f, lat)
    feq = S.equilibrium(rho, u, th, lat, N)
    al = H.multi_indices_upto(N)
    He = H.he_multi(al, lat.xi)
    fact = np.array([H.alpha_factorial(a) for a in al], dtype=float)
    proj = lat.w[:, None] * (He / fact) @ (He.T @ (f - feq))
    want = feq + (1.0 - 1.0 / (tau_c + 0.5)) * proj
    np.testing.assert_allclose(S.collide(f, model), want, atol=1e-13)


def _harmonic_part(X):
    """Traceless part of a symmetric tensor found by a linear solve rather than Appendix A's
    closed form: H = X - sym(delta Y) with Y chosen so that tr H = 0 (least squares over every
    rank r-2 tensor Y; the solution is exact because the trace map is onto)."""
    r = X.ndim
    basis = np.eye(3 ** (r - 2))
    cols = [T.trace(T.sprod(np.eye(3), b.reshape((3,) * (r - 2)))).ravel() for b in basis]
    y, *_ = np.linalg.lstsq(np.stack(cols, axis=1), T.trace(X).ravel(), rcond=None)
    H = X - T.sprod(np.eye(3), y.reshape((3,) * (r - 2)))
    assert np.abs(T.trace(H)).max() < 1e-12
    return H


def _pure_mode(n, m, rng):
    """A random pure irreducible mode A delta^m of order n, built from Appendix A's formulas."""
    d = np.eye(3)
    if n - 2 * m == 0:
        core = np.array(1.0)
    elif n - 2 * m == 1:
        core = rng.standard_normal(3)
    else:
        r = n - 2 * m
        X = T.sym(rng.standard_normal((3,) * r))
        if r == 2:
            core = X - np.trace(X) / 3 * d
        elif r == 3:
            core = X - 3 / 5 * T.sprod(d, T.trace(X))
        elif r == 4:
            core = (X - 6 / 7 * T.sprod(d, T.trace(X))
                    + 3 / 35 * T.sprod(T.delta_power(2), T.trace_pow(X, 2)))
        else:
            core = _harmonic_part(X)
    return T.sprod(core, T.delta_power(m)) if m else core


@pytest.mark.parametrize("name,N,n,m", [("D3Q39", 3, 2, 0), ("D3Q39", 3, 3, 0), ("D3Q39", 3, 3, 1),
                                         ("D3Q103", 4, 2, 0), ("D3Q103", 4, 3, 0), ("D3Q103", 4, 3, 1),
                                         ("D3Q103", 4, 4, 0), ("D3Q103", 4, 4, 1), ("D3Q103", 4, 4, 2),
                                         ("D3Q729", 5, 4, 1), ("D3Q729", 5, 5, 0), ("D3Q729", 5, 5, 1),
                                         ("D3Q729", 5, 5, 2)])
def test_single_mode_decays_at_its_own_rate(lats, name, N, n, m):
    """Eq. SMRT: a pure (n, m) mode on a moving, non-unit-temperature state is multiplied by
    exactly 1 - 1/tau_nm per collision, all other coefficients untouched (Galilean invariant)."""
    lat = lats[name]
    rng = np.random.default_rng(10 * n + m)
    rho, u, th = 1.1, np.array([0.35, -0.2, 0.15]), 0.9
    mode = _pure_mode(n, m, rng)
    comp = H.components(mode)
    al = H.multi_indices_upto(N)
    d = np.zeros((len(al), 1))
    d[0, 0] = rho
    eps = 1e-3
    for k, a in enumerate(al):
        if sum(a) == n:
            d[k, 0] = eps * comp[a]
    a_abs = S.to_absolute(d, N, u[:, None], np.array([th]))
    f = S.rebuild(a_abs, lat, N)
    r0, u0, t0 = S.conserved(f, lat)
    np.testing.assert_allclose([r0[0], t0[0]], [rho, th], rtol=1e-13)
    np.testing.assert_allclose(u0[:, 0], u, atol=1e-13)
    model = S.Model(lat, N, tau_ref=0.8)
    h = S.collide(f, model)
    d_after = S.local_direct(h, lat, N, u0, t0)
    tau = S.tau_discrete(model, np.array([rho]))[(n, m)][0]
    want = d.copy()
    want[1:, 0] *= 0.0
    for k, a in enumerate(al):
        if sum(a) == n:
            want[k, 0] = (1.0 - 1.0 / tau) * d[k, 0]
    want[0, 0] = rho
    np.testing.assert_allclose(d_after, want, atol=1e-14)


@pytest.mark.parametrize("table", ["smrt", "shakhov"])
def test_prandtl_two_thirds_from_decay_rates(lats, table):
    """Sec. 3 / Table 4: tau_31 = tau_20 / Pr with Pr = 2/3, read off measured decay factors."""
    lat = lats["D3Q39"]
    star = S.TAU_STAR_SMRT if table == "smrt" else S.TAU_STAR_SHAKHOV
    model = S.Model(lat, 3, tau_ref=1.7, tau_star=star, maxwell_law=False)
    rng = np.random.default_rng(5)
    rates = {}
    for n, m in [(2, 0), (3, 1)]:
        mode = H.components(_pure_mode(n, m, rng))
        al = H.multi_indices_upto(3)
        d = np.zeros((len(al), 1))
        d[0, 0] = 1.0
        k0 = [k for k, a in enumerate(al) if sum(a) == n and abs(mode[a]) > 1e-3][0]
        for k, a in enumerate(al):
            if sum(a) == n:
                d[k, 0] = 1e-3 * mode[a]
        f = S.rebuild(S.to_absolute(d, 3, np.zeros((3, 1)), np.ones(1)), lat, 3)
        dh = S.local_direct(S.collide(f, model), lat, 3, np.zeros((3, 1)), np.ones(1))
        lam = dh[k0, 0] / d[k0, 0]
        rates[(n, m)] = 1.0 / (1.0 - lam) - 0.5       # continuous relaxation time
    assert abs(rates[(2, 0)] / rates[(3, 1)] - 2.0 / 3.0) < 1e-12


def test_bulk_mode_is_inert(lats):
    """Sec. 4.2: tau_21 is absent for a monatomic gas -- changing it changes nothing."""
    lat = lats["D3Q103"]
    f, _ = _random_state(lat, 4, eps=0.3)
    s1 = dict(S.TAU_STAR_SMRT)
    s2 = dict(S.TAU_STAR_SMRT)
    s2[(2, 1)] = 7.0
    h1 = S.collide(f, S.Model(lat, 4, tau_ref=0.6, tau_star=s1))
    h2 = S.collide(f, S.Model(lat, 4, tau_ref=0.6, tau_star=s2))
    np.testing.assert_allclose(h1, h2, atol=1e-14)


def test_periodic_uniform_equilibrium_invariant(lats):
    lat = lats["D3Q39"]
    model = S.Model(lat, 3, tau_ref=0.9)
    geom = S.Geometry(shape=(3, 4, 5))
    feq = S.equilibrium(np.array([1.2]), np.array([[0.1], [0.05], [-0.1]]), np.array([0.95]), lat, 3)
    h = np.broadcast_to(feq[:, :, None, None], (lat.q, 3, 4, 5)).copy()
    h2 = S.step(h, model, geom)
    np.testing.assert_allclose(h2, h, atol=1e-14)


def test_streaming_is_a_permutation(lats):
    """Pull streaming by e_i + k moves populations without changing any value (periodic)."""
    lat = lats["D3Q39"]
    rng = np.random.default_rng(2)
    h = rng.random((lat.q, 4, 5, 6))
    geom = S.Geometry(shape=(4, 5, 6), shift=(1, 0, 0))
    f = S.stream(h, lat, geom)
    for i in range(lat.q):
        assert np.allclose(np.sort(f[i].ravel()), np.sort(h[i].ravel()))
        sx, sy, sz = lat.e[i] + np.array([1, 0, 0])
        assert f[i][sz % 4, sy % 5, sx % 6] == h[i][0, 0, 0]


def test_pull_cells_matches_stream(lats):
    lat = lats["D3Q39"]
    rng = np.random.default_rng(4)
    h = rng.random((lat.q, 5, 6, 7))
    geom = S.Geometry(shape=(5, 6, 7), shift=(1, 0, 0))
    full = S.stream(h, lat, geom).reshape(lat.q, -1)
    cells = rng.choice(5 * 6 * 7, size=20, replace=False)
    np.testing.assert_array_equal(S.pull_cells(h, lat, geom, cells), full[:, cells])


# ---------------------------------------------------------------------------- ES-BGK
def test_es_target_matches_gaussian_integration(lats):
    """Sec. 3, Eq. ES-BGK: the target's local-frame Hermite coefficients equal rho E[He_beta(v)]
    for v ~ N(0, A), A = I + (b/rho) D2, here integrated directly by a 3D Gauss-Hermite rule on
    v = L z (A = L L^T) with numpy's own Hermite evaluation (no generating function)."""
    from numpy.polynomial.hermite_e import hermeval
    lat = lats["D3Q729"]
    N, b = 5, -0.5
    f, _ = _random_state(lat, N, ncell=2, eps=0.2)
    rho, u, th = S.conserved(f, lat)
    d = S.local_direct(f, lat, N, u, th)
    got = S.es_target(d, N, rho, b)
    al = H.multi_indices_upto(N)
    pos = {a: k for k, a in enumerate(al)}
    z, wz = hermegauss(12)
    wz = wz / wz.sum()
    Z = np.stack(np.meshgrid(z, z, z, indexing="ij"), axis=-1).reshape(-1, 3)
    WZ = np.einsum("i,j,k->ijk", wz, wz, wz).ravel()
    for c in range(2):
        D2 = np.zeros((3, 3))
        for k in range(3):
            for l in range(3):
                e = [0, 0, 0]
                e[k] += 1
                e[l] += 1
                D2[k, l] = d[pos[tuple(e)], c]
        A = np.eye(3) + (b / rho[c]) * D2
        V = Z @ np.linalg.cholesky(A).T
        for beta in al:
            hv = np.ones(len(V))
            for k in range(3):
                hv = hv * hermeval(V[:, k], [0] * beta[k] + [1])
            want = rho[c] * (WZ * hv).sum()
            assert abs(got[pos[beta], c] - want) < 1e-12 * max(1.0, abs(want)), beta


@pytest.mark.parametrize("name,N", [("D3Q729", 5), ("D3Q103", 4), ("D3Q39", 3)])
def test_es_b_zero_is_bgk(lats, name, N):
    """ES-BGK with b = 0 is the BGK model: the regularised-BGK formula written without frames."""
    lat = lats[name]
    f, _ = _random_state(lat, N, eps=0.2)
    tau_c = 0.9
    model = S.Model(lat, N, tau_ref=tau_c, maxwell_law=False, es_b=0.0)
    rho, u, th = S.conserved(f, lat)
    feq = S.equilibrium(rho, u, th, lat, N)
    al = H.multi_indices_upto(N)
    He = H.he_multi(al, lat.xi)
    fact = np.array([H.alpha_factorial(a) for a in al], dtype=float)
    proj = lat.w[:, None] * (He / fact) @ (He.T @ (f - feq))
    np.testing.assert_allclose(S.collide(f, model), feq + (1.0 - 1.0 / (tau_c + 0.5)) * proj, atol=1e-13)


@pytest.mark.parametrize("name,N", [("D3Q729", 5), ("D3Q103", 4), ("D3Q39", 3)])
@pytest.mark.parametrize("b", [-0.5, 0.3])
def test_es_prandtl_number_from_decay_rates(lats, b, name, N):
    """Holway's model: Pr = 1/(1 - b) (2/3 at b = -1/2), read off the continuous relaxation
    times of a shear and a heat-flux mode measured from one collision."""
    lat = lats[name]
    model = S.Model(lat, N, tau_ref=1.3, maxwell_law=False, es_b=b)
    rng = np.random.default_rng(8)
    rates = {}
    for n, m in [(2, 0), (3, 1)]:
        mode = H.components(_pure_mode(n, m, rng))
        al = H.multi_indices_upto(N)
        d = np.zeros((len(al), 1))
        d[0, 0] = 1.0
        k0 = [k for k, a in enumerate(al) if sum(a) == n and abs(mode[a]) > 1e-3][0]
        for k, a in enumerate(al):
            if sum(a) == n:
                d[k, 0] = 1e-4 * mode[a]
        f = S.rebuild(S.to_absolute(d, N, np.zeros((3, 1)), np.ones(1)), lat, N)
        dh = S.local_direct(S.collide(f, model), lat, N, np.zeros((3, 1)), np.ones(1))
        lam = dh[k0, 0] / d[k0, 0]
        rates[(n, m)] = 1.0 / (1.0 - lam) - 0.5
    # the order-4 part of the target is quadratic in the 1e-4 amplitude: Pr to ~1e-8
    assert abs(rates[(2, 0)] / rates[(3, 1)] - 1.0 / (1.0 - b)) < 1e-7


@pytest.mark.parametrize("name,N", [("D3Q729", 5), ("D3Q103", 4), ("D3Q39", 3)])
def test_es_collision_conserves(lats, name, N):
    lat = lats[name]
    f, _ = _random_state(lat, N, eps=0.2)
    h = S.collide(f, S.Model(lat, N, tau_ref=0.7, es_b=-0.5))
    for a, b in zip(S.conserved(f, lat), S.conserved(h, lat)):
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-14)


# ---------------------------------------------------------------------------- Maxwell molecules
def _measured_viscosity(lat, model, rho, theta, u=(0.2, -0.1, 0.05), eps=1e-4):
    """mu = p tau_c of a pure shear mode (the (2,0) component d_xy), with tau_c read off one
    collision: the mode is multiplied by 1 - 1/tau and tau = tau_c + 1/2 (second-order scheme).
    Nothing here calls the oracle's relaxation-time formula."""
    N = model.N
    al = H.multi_indices_upto(N)
    k0 = al.index((1, 1, 0))
    d = np.zeros((len(al), 1))
    d[0, 0] = rho
    d[k0, 0] = eps * rho
    uu = np.array(u, dtype=float)[:, None]
    f = S.rebuild(S.to_absolute(d, N, uu, np.array([theta])), lat, N)
    dh = S.local_direct(S.collide(f, model), lat, N, uu, np.array([theta]))
    lam = dh[k0, 0] / d[k0, 0]
    tau_c = 1.0 / (1.0 - lam) - 0.5
    return rho * theta * tau_c


def _viscosity_law_error(lat, model):
    """Largest relative departure of the measured mu(rho, theta) from mu = mu_ref theta: the
    viscosity of Maxwell molecules is proportional to the temperature and independent of the
    density (Sec. 4.2), mu_ref being the value at rho_ref and theta = 1."""
    mu_ref = _measured_viscosity(lat, model, model.rho_ref, 1.0)
    err = 0.0
    for rho in (0.5, 1.0, 2.0, 3.7):
        for theta in (0.8, 1.0, 1.2):
            mu = _measured_viscosity(lat, model, rho, theta)
            err = max(err, abs(mu / (mu_ref * theta) - 1.0))
    return err, mu_ref


@pytest.mark.parametrize("rho_ref", [1.0, 1.5])
def test_maxwell_molecule_viscosity_law(lats, rho_ref):
    """Maxwell molecules (Sec. 4.2; viscosity proportional to temperature): the shear viscosity
    measured from one collision is mu = p tau_c = rho_ref tau_ref theta at every density; at the
    reference density and theta = 1 the continuous time is tau_ref itself."""
    lat = lats["D3Q39"]
    model = S.Model(lat, 3, tau_ref=1.3, rho_ref=rho_ref)
    err, mu_ref = _viscosity_law_error(lat, model)
    assert err < 1e-9
    assert abs(mu_ref - rho_ref * 1.3) < 1e-9


def test_viscosity_law_detects_an_inverted_density_ratio(lats, monkeypatch):
    """The pin above fails when the oracle scales tau by rho/rho_ref instead of rho_ref/rho
    (the mistake planted in the oracle on the CPU), and also with the density law switched off
    (mu would then grow with rho)."""
    lat = lats["D3Q39"]

    def inverted(model, rho):
        return {nm: model.tau_star[nm] * model.tau_ref * (rho / model.rho_ref) + 0.5
                for nm in model.tau_star}
    monkeypatch.setattr(S, "tau_discrete", inverted)
    err, _ = _viscosity_law_error(lat, S.Model(lat, 3, tau_ref=1.3))
    assert err > 1.0
    monkeypatch.undo()
    err, _ = _viscosity_law_error(lat, S.Model(lat, 3, tau_ref=1.3, maxwell_law=False))
    assert err > 1.0


# ---------------------------------------------------------------------------- stress and heat flux
def _sigma_q_error(lat, N, macroscopic, seed=3):
    """Largest difference between macroscopic()'s sigma and q and their definitions as direct
    moments of the populations (Sec. 2.2): with the peculiar velocity c_i = xi_i + u_bar - u,
    sigma = sum_i f_i c_i c_i - p delta (p = rho theta) and q = 1/2 sum_i f_i |c_i|^2 c_i. A
    one-cell periodic grid makes streaming the identity, so the populations are f itself."""
    rng = np.random.default_rng(seed)
    err = 0.0
    for k in range(3):
        rho = 0.8 + 0.5 * rng.random(1)
        u = 0.3 * rng.standard_normal((3, 1))
        th = 0.7 + 0.6 * rng.random(1)
        f = S.equilibrium(rho, u, th, lat, N)
        f = f * (1.0 + 0.2 * rng.standard_normal(f.shape))
        shift = (k, 0, 0)
        geom = S.Geometry(shape=(1, 1, 1), shift=shift)
        m = macroscopic(f.reshape(lat.q, 1, 1, 1), S.Model(lat, N, tau_ref=1.0), geom)
        ubar = lat.c * np.asarray(shift, dtype=float)
        vel = lat.xi + ubar[None, :]                       # physical velocities
        fc = f[:, 0]
        rho_d = fc.sum()
        u_d = (fc[:, None] * vel).sum(0) / rho_d
        c = vel - u_d[None, :]
        p_d = (fc * (c * c).sum(1)).sum() / 3.0
        S2 = np.einsum("i,ik,il->kl", fc, c, c) - p_d * np.eye(3)
        q_d = 0.5 * np.einsum("i,i,ik->k", fc, (c * c).sum(1), c)
        pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
        sig_d = np.array([S2[a, b] for a, b in pairs])
        scale = max(1.0, np.abs(sig_d).max(), np.abs(q_d).max())
        err = max(err, abs(m["theta"][0] * m["rho"][0] - p_d) / scale,
                  np.abs(m["sigma"][:, 0] - sig_d).max() / scale,
                  np.abs(m["q"][:, 0] - q_d).max() / scale)
    return err


@pytest.mark.parametrize("name,N", [("D3Q39", 3), ("D3Q103", 4), ("D3Q729", 5)])
def test_macroscopic_stress_and_heat_flux_are_direct_moments(lats, name, N):
    assert _sigma_q_error(lats[name], N, S.macroscopic) < 1e-12


@pytest.mark.parametrize("mutation", ["sigma_theta_squared", "q_theta_half", "q_without_half"])
def test_stress_and_heat_flux_pin_detects_mistakes(lats, mutation):
    """Plausible mistakes in macroscopic() (a wrong power of theta in sigma or q, the 1/2 of q
    dropped), planted in a wrapper around the oracle, fail the direct-moment pin."""
    def planted(h, model, geom):
        m = dict(S.macroscopic(h, model, geom))
        if mutation == "sigma_theta_squared":
            m["sigma"] = m["sigma"] * m["theta"]
        elif mutation == "q_theta_half":
            m["q"] = m["q"] / m["theta"]
        else:
            m["q"] = 2.0 * m["q"]
        return m
    assert _sigma_q_error(lats["D3Q39"], 3, planted) > 1e-3
