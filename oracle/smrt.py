"""The LB-SMRT collide-and-stream step, written step by step (oracle; test infrastructure only).

Lattice units: one time step, cell size c (a population with abscissa xi_i = c e_i moves e_i
cells per step). The abscissae are shifted by the constant frame velocity u_bar = c k (Sec. 4.1,
shifted stencil), so the physical velocity of population i is xi_i + u_bar, it streams by the
integer vector e_i + k, and every velocity used in the collision is relative to u_bar.

Per cell, per step (``collide``), in the order of Sec. 3:

1. moments: rho = sum f_i, rho u = sum f_i xi_i, rho(|u|^2 + 3 theta) = sum f_i |xi_i|^2
   (Eqs. hermite/hermite1 with D = 3 degrees of freedom);
2. local-frame coefficients d_beta = sum_i f_i He_beta(v_i), v_i = (xi_i - u)/sqrt(theta), for
   |beta| <= N: the discrete form of the local expansion that defines SMRT (Sec. 3, the
   expansion before Eq. SMRT), exact for a degree >= 2N rule (Eq. an);
3. irreducible split of each order n >= 2 and relaxation of each part with its own time,
   d'^(n) = sum_m (1 - 1/tau_nm) d^(n,m) delta^m; orders 0 and 1 untouched (Eq. SMRT,
   Appendix A projectors);
4. back to the absolute frame, truncated at order N (binomial transform, below);
5. rebuild f_i' = w_i sum_{|alpha|<=N} a'_alpha He_alpha(xi_i)/alpha! (Eq. fi).

Streaming (``stream``) is a pull: the pre-collision population at x is the post-collision one at
x - e_i - k; the buffers hold post-collision populations. Periodic axes wrap; on an axis with
fixed ends the cells beyond the domain hold the order-N equilibrium of the end states
(Sec. 4.2: Maxwellian at both x ends), and they are never collided or updated.

Binomial transform. With g_j(u, theta) = sum_l j!/(l! (j-2l)!) u^(j-2l) ((theta-1)/2)^l, the
one-dimensional absolute coefficient of a Maxwellian (Appendix B closed form for a^(n)), the
shifted-and-scaled Hermite polynomials obey the generating-function identities
  He_j(u + sqrt(theta) v) = sum_b C(j,b) g_{j-b}(u, theta) theta^(b/2) He_b(v),
  theta^(b/2) He_b((xi-u)/sqrt(theta)) = sum_c C(b,c) g_{b-c}(-u, 2-theta) He_c(xi),
so, axis by axis for multi-indices,
  a_alpha = sum_{beta<=alpha} prod_k C(alpha_k,beta_k) g_{alpha_k-beta_k}(u_k,theta)
            theta^(|beta|/2) d_beta,
  d_beta  = theta^(-|beta|/2) sum_{gamma<=beta} prod_k C(beta_k,gamma_k)
            g_{beta_k-gamma_k}(-u_k, 2-theta) a_gamma.
These are polynomial identities, so route A (step 2) and route B (``absolute`` then
``to_local``) agree for any f; the tests check both that and the Appendix B reduction.

Relaxation times: tau_c,nm(x) = tau*_nm tau_ref (rho_ref / rho(x)) for Maxwell molecules
(viscosity proportional to temperature, Sec. 4.2) or tau*_nm tau_ref without the density law;
the discrete relaxation time is tau_nm = tau_c,nm + 1/2 (second-order time discretisation).

ES-BGK (Model.es_b set): step 3 instead relaxes every order n >= 2 at the single rate 1/tau_20
toward the local-frame coefficients of Holway's anisotropic Gaussian (``es_target``).

Parity: pinned (conservation, equilibrium fixed point, BGK reduction against an independent
regularised-BGK formula, single-mode decay, the Maxwell-molecule law mu = p tau_c proportional
to theta at every density measured from one collision, sigma and q of ``macroscopic`` against
their direct moments, Rankine-Hugoniot steady shock with uniform face fluxes of mass,
momentum and energy; for ES-BGK the target against direct numerical integration of the
Gaussian, b = 0 against BGK, Pr = 1/(1-b)).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from math import comb, factorial

import numpy as np

from .hermite import alpha_factorial, he_multi, multi_indices, multi_indices_upto
from .lattice import Lattice
from .tensors import projector_matrices

# Table 4, SMRT columns (Maxwell molecules), tau*_{n,m} = tau_{n,m} / tau_{2,0}.
# tau_{2,1} is absent for a monatomic gas; its mode is identically zero, any value is inert.
TAU_STAR_SMRT = {(2, 0): 1.0, (2, 1): 1.0,
                 (3, 0): 2.0 / 3.0, (3, 1): 3.0 / 2.0,
                 (4, 0): 432.0 / 763.0, (4, 1): 6.0 / 7.0, (4, 2): 3.0 / 2.0,
                 (5, 0): 864.0 / 1655.0, (5, 1): 108.0 / 163.0, (5, 2): 1.0}
# Table 4, Shakhov columns: tau*_{3,1} = 1/Pr = 3/2, every other ratio 1.
TAU_STAR_SHAKHOV = {k: 1.0 for k in TAU_STAR_SMRT}
TAU_STAR_SHAKHOV[(3, 1)] = 3.0 / 2.0


@dataclass
class Model:
    lat: Lattice
    N: int
    tau_ref: float                      # continuous tau_c,2,0 (in steps) at rho_ref
    tau_star: dict = field(default_factory=lambda: dict(TAU_STAR_SMRT))
    rho_ref: float = 1.0
    maxwell_law: bool = True
    es_b: float | None = None           # None: SMRT; else the ES-BGK model with parameter b


@dataclass
class Geometry:
    shape: tuple                        # (nz, ny, nx) cells
    shift: tuple = (0, 0, 0)            # integer k (x, y, z): u_bar = c k
    fixed_x: bool = False               # fixed end states in x (else periodic)
    ghost_left: np.ndarray | None = None   # (Q,) populations beyond x < 0
    ghost_right: np.ndarray | None = None  # (Q,) populations beyond x >= nx


def alphas(N: int):
    return multi_indices_upto(N)


def g_coef(j: int, u, theta):
    """g_j(u, theta) = sum_l j!/(l!(j-2l)!) u^(j-2l) ((theta-1)/2)^l."""
    s = 0.0 * u
    for l in range(j // 2 + 1):
        s = s + factorial(j) / (factorial(l) * factorial(j - 2 * l)) * u ** (j - 2 * l) * ((theta - 1.0) / 2.0) ** l
    return s


# ---------------------------------------------------------------------------- step 1
def conserved(f, lat: Lattice):
    """rho, u (relative to u_bar), theta of f with shape (Q, ncell)."""
    xi = lat.xi
    rho = f.sum(axis=0)
    j = xi.T @ f
    E = (xi ** 2).sum(axis=1) @ f
    u = j / rho
    theta = (E / rho - (u ** 2).sum(axis=0)) / 3.0
    return rho, u, theta


# ---------------------------------------------------------------------------- step 2
def local_direct(f, lat: Lattice, N: int, u, theta):
    """d_beta = sum_i f_i He_beta((xi_i - u)/sqrt(theta)), shape (M, ncell)."""
    v = (lat.xi[:, None, :] - u.T[None, :, :]) / np.sqrt(theta)[None, :, None]   # (Q, ncell, 3)
    H = he_multi(alphas(N), v)                                                   # (Q, ncell, M)
    return np.einsum("ic,icm->mc", f, H)


def absolute(f, lat: Lattice, N: int):
    """a_alpha = sum_i f_i He_alpha(xi_i) (Eq. an), shape (M, ncell)."""
    H = he_multi(alphas(N), lat.xi)                                              # (Q, M)
    return H.T @ f


def _binomial_sum(coefs, N: int, uu, tt):
    """out_alpha = sum_{beta<=alpha} prod_k C(alpha_k,beta_k) g_{alpha_k-beta_k}(uu_k, tt) coefs_beta."""
    al = alphas(N)
    pos = {a: k for k, a in enumerate(al)}
    g = [[g_coef(j, uu[k], tt) for j in range(N + 1)] for k in range(3)]
    out = np.zeros_like(coefs)
    for alpha in al:
        acc = 0.0 * coefs[0]
        for beta in al:
            if any(b > a for a, b in zip(alpha, beta)):
                continue
            w = 1.0
            for k in range(3):
                w = w * comb(alpha[k], beta[k]) * g[k][alpha[k] - beta[k]]
            acc = acc + w * coefs[pos[beta]]
        out[pos[alpha]] = acc
    return out


def to_absolute(d, N: int, u, theta):
    """a_alpha = sum_{beta<=alpha} prod C(alpha_k,beta_k) g(u_k,theta) theta^(|beta|/2) d_beta."""
    sq = np.sqrt(theta)
    scaled = np.stack([d[k] * sq ** sum(b) for k, b in enumerate(alphas(N))])
    return _binomial_sum(scaled, N, u, theta)


def to_local(a, N: int, u, theta):
    """d_beta = theta^(-|beta|/2) sum_{gamma<=beta} prod C g(-u_k, 2-theta) a_gamma."""
    sq = np.sqrt(theta)
    out = _binomial_sum(a, N, -u, 2.0 - theta)
    return np.stack([out[k] / sq ** sum(b) for k, b in enumerate(alphas(N))])


# ---------------------------------------------------------------------------- step 3
def order_slices(N: int):
    """Positions of order-n components inside the multi-index vector of orders <= N."""
    out, start = {}, 0
    for n in range(N + 1):
        k = (n + 1) * (n + 2) // 2
        out[n] = slice(start, start + k)
        start += k
    return out


def tau_discrete(model: Model, rho):
    """tau_nm(x) = tau*_nm tau_ref (rho_ref/rho) [Maxwell molecules] + 1/2."""
    scale = model.rho_ref / rho if model.maxwell_law else 1.0 + 0.0 * rho
    return {nm: model.tau_star[nm] * model.tau_ref * scale + 0.5 for nm in model.tau_star}


def relax(d, N: int, tau):
    """d'^(n) = sum_m (1 - 1/tau_nm) P^(n)_m d^(n) for 2 <= n <= N; orders 0, 1 unchanged."""
    out = d.copy()
    sl = order_slices(N)
    for n in range(2, N + 1):
        block = d[sl[n]]
        acc = 0.0 * block
        for m, P in enumerate(projector_matrices(n)):
            acc = acc + (1.0 - 1.0 / tau[(n, m)]) * (P @ block)
        out[sl[n]] = acc
    return out


def es_target(d, N: int, rho, b: float):
    """Local-frame coefficients (undivided, like d) of the ES-BGK target (Sec. 3, Eq. ES-BGK):
    the Gaussian of covariance Lambda = theta delta + b sigma / rho. In the scaled variable
    v = (xi - u)/sqrt(theta) its covariance is A = I + B, B = (b / rho) D2 with D2 the order-2
    coefficient tensor of f (sigma = theta D2), and the Hermite coefficients of a Gaussian
    follow from E[exp(t.v - |t|^2/2)] = exp(t.B.t / 2): the coefficient of t^beta / beta! is
    the target's d_beta / rho. Only even orders are nonzero."""
    al = alphas(N)
    pos = {a: k for k, a in enumerate(al)}
    ncell = d.shape[1]
    # the quadratic form Q(t) = t.B.t / 2 as a monomial dictionary (exponent -> per-cell value)
    Bf = {}
    for k in range(3):
        for l in range(3):
            e = [0, 0, 0]
            e[k] += 1
            e[l] += 1
            Bf[tuple(e)] = Bf.get(tuple(e), 0.0) + 0.5 * (b / rho) * d[pos[tuple(e)]]
    out = np.zeros_like(d)
    out[pos[(0, 0, 0)]] = rho
    term = {(0, 0, 0): np.ones(ncell)}
    for k in range(1, N // 2 + 1):
        nxt = {}
        for e1, c1 in term.items():
            for e2, c2 in Bf.items():
                e = tuple(x + y for x, y in zip(e1, e2))
                nxt[e] = nxt.get(e, 0.0) + c1 * c2 / k        # Q^k / k! built as (Q^(k-1)/(k-1)!) Q / k
        term = nxt
        for e, c in term.items():
            out[pos[e]] = rho * alpha_factorial(e) * c
    return out


def es_discrete_b(tau20, b: float):
    """The ES parameter of the discrete-time scheme. The continuous model relaxes the stress
    at (1 - b)/tau_c and the heat flux at 1/tau_c; the second-order scheme turns each such
    continuous time into tau + 1/2 (as for every SMRT mode), so with one discrete rate 1/tau_20
    (tau_20 = tau_c + 1/2) the target uses b' with (1 - b')/tau_20 = 1/(tau_c/(1 - b) + 1/2)."""
    return 1.0 - (1.0 - b) * tau20 / (tau20 - 0.5 * b)


def relax_es(d, N: int, tau20, rho, b: float):
    """ES-BGK in the local frame: every order n >= 2 relaxes at the one discrete rate
    1/tau_20 toward the ES target of parameter es_discrete_b(tau_20, b) (orders 0 and 1 are
    the target's own)."""
    target = es_target(d, N, rho, es_discrete_b(tau20, b))
    out = d.copy()
    sl = order_slices(N)
    for n in range(2, N + 1):
        out[sl[n]] = d[sl[n]] - (d[sl[n]] - target[sl[n]]) / tau20
    return out


# ---------------------------------------------------------------------------- step 5
def rebuild(a, lat: Lattice, N: int):
    """f_i = w_i sum_{|alpha|<=N} a_alpha He_alpha(xi_i) / alpha!  (Eq. fi)."""
    al = alphas(N)
    H = he_multi(al, lat.xi)                                                     # (Q, M)
    inv_fact = np.array([1.0 / alpha_factorial(a) for a in al])
    return lat.w[:, None] * (H * inv_fact[None, :]) @ a


# ---------------------------------------------------------------------------- collision
def collide(f, model: Model):
    """Post-collision populations of pre-collision f (shape (Q, ncell))."""
    lat, N = model.lat, model.N
    rho, u, theta = conserved(f, lat)
    d = local_direct(f, lat, N, u, theta)
    if model.es_b is None:
        d2 = relax(d, N, tau_discrete(model, rho))
    else:
        d2 = relax_es(d, N, tau_discrete(model, rho)[(2, 0)], rho, model.es_b)
    a2 = to_absolute(d2, N, u, theta)
    return rebuild(a2, lat, N)


def equilibrium(rho, u, theta, lat: Lattice, N: int):
    """Order-N truncated Maxwellian: a_alpha = rho prod_k g_{alpha_k}(u_k, theta), then Eq. fi.

    rho, theta shape (ncell,), u shape (3, ncell), u relative to u_bar.
    """
    rho = np.asarray(rho)
    u = np.asarray(u)
    theta = np.asarray(theta)
    a = np.stack([rho * g_coef(al[0], u[0], theta) * g_coef(al[1], u[1], theta) * g_coef(al[2], u[2], theta)
                  for al in alphas(N)])
    return rebuild(a, lat, N)


# ---------------------------------------------------------------------------- streaming
def stream(h, lat: Lattice, geom: Geometry):
    """Pull streaming of post-collision h (Q, nz, ny, nx) by e_i + k."""
    Q = lat.q
    nz, ny, nx = geom.shape
    kx, ky, kz = geom.shift
    out = np.empty_like(h)
    for i in range(Q):
        sx, sy, sz = int(lat.e[i, 0]) + kx, int(lat.e[i, 1]) + ky, int(lat.e[i, 2]) + kz
        src = np.roll(h[i], shift=(sz, sy), axis=(0, 1))
        if not geom.fixed_x:
            out[i] = np.roll(src, shift=sx, axis=2)
            continue
        x = np.arange(nx)
        xs = x - sx
        inside = (xs >= 0) & (xs < nx)
        res = np.empty_like(src)
        res[..., inside] = src[..., xs[inside]]
        res[..., xs < 0] = geom.ghost_left[i]
        res[..., xs >= nx] = geom.ghost_right[i]
        out[i] = res
    return out


def pull_cells(h, lat: Lattice, geom: Geometry, cells):
    """Pre-collision populations (Q, len(cells)) at the listed flat cell indices of a periodic
    field h (Q, nz, ny, nx): f_i(x) = h_i(x - e_i - k), each axis wrapped. The same rule as
    ``stream``, evaluated only where asked."""
    nz, ny, nx = geom.shape
    cells = np.asarray(cells)
    z, rem = np.divmod(cells, ny * nx)
    y, x = np.divmod(rem, nx)
    kx, ky, kz = geom.shift
    out = np.empty((lat.q, len(cells)), dtype=h.dtype)
    for i in range(lat.q):
        xs = (x - lat.e[i, 0] - kx) % nx
        ys = (y - lat.e[i, 1] - ky) % ny
        zs = (z - lat.e[i, 2] - kz) % nz
        out[i] = h[i][zs, ys, xs]
    return out


def collide_field(f, model: Model, chunk: int = 4096):
    """Collide every cell of a (Q, nz, ny, nx) field, in chunks of cells."""
    Q = f.shape[0]
    flat = f.reshape(Q, -1)
    out = np.empty_like(flat)
    for s in range(0, flat.shape[1], chunk):
        out[:, s:s + chunk] = collide(flat[:, s:s + chunk], model)
    return out.reshape(f.shape)


def step(h, model: Model, geom: Geometry):
    """One collide-and-stream step on post-collision state h: collide(stream(h))."""
    return collide_field(stream(h, model.lat, geom), model)


# ---------------------------------------------------------------------------- diagnostics
def macroscopic(h, model: Model, geom: Geometry):
    """Moments of the pre-collision (streamed) populations at every cell.

    Returns a dict of arrays over cells (flattened z, y, x): rho, u (physical, 3), theta,
    sigma (6 components xx yy zz xy xz yz, sigma = theta d^(2)), q (3, q_k = 1/2
    theta^(3/2) sum_l d^(3)_kll), and the local coefficients d (M) for |beta| <= max(N, 3).
    """
    lat = model.lat
    f = stream(h, lat, geom).reshape(lat.q, -1)
    rho, u, theta = conserved(f, lat)
    Nd = max(model.N, 3)
    d = local_direct(f, lat, Nd, u, theta)
    al = alphas(Nd)
    pos = {a: k for k, a in enumerate(al)}
    pairs = [(2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1)]
    sigma = np.stack([theta * d[pos[p]] for p in pairs])
    q = []
    for k in range(3):
        t = 0.0
        for l in range(3):
            b = [0, 0, 0]
            b[k] += 1
            b[l] += 2
            t = t + d[pos[tuple(b)]]
        q.append(0.5 * theta ** 1.5 * t)
    ubar = lat.c * np.asarray(geom.shift, dtype=np.float64)
    return {"rho": rho, "u": u + ubar[:, None], "theta": theta, "sigma": sigma,
            "q": np.stack(q), "d": d}
