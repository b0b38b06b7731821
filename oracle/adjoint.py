"""Discrete adjoint of the LB-SMRT step (oracle; test infrastructure only).

One step maps the post-collision state h^t to h^{t+1} = C(S h^t; tau): S is the pull streaming
(a permutation, plus constant end-state populations beyond fixed x ends) and C the per-cell
collision of ``smrt.collide``. For a loss L(h^T) the adjoint recursion is

    lambda^T = dL/dh^T,
    lambda^t = S^T ( J_C(S h^t)^T lambda^{t+1} ),
    dL/dtau += sum_cells (dC/dtau)^T lambda^{t+1}.

This module evaluates it plainly: the per-cell Jacobian-transpose products are taken by
complex-step differentiation of the oracle's own collision, d/dx g(x) = Im g(x + i h)/h with
h = 1e-30, which is exact to rounding for real-analytic g (no subtractive cancellation), one
complex collision per population (or per relaxation parameter); S^T is the push that undoes the
pull. Central finite differences of whole runs are provided for the tests as a second, fully
independent check.

Relaxation parameters are the continuous times tau_c,nm = tau*_nm tau_ref (Table 4 ratios times
the reference time), one per irreducible part (n, m) of orders 2..N, in the order
(2,0) (2,1) (3,0) (3,1) (4,0) (4,1) (4,2).

The loss of the differentiable-shock workload is
    L = sum_x (rho - rho*)^2 + (theta - theta*)^2 + (q_x - q_x*)^2
on the moments of the pre-collision populations S h^T (``smrt.macroscopic``).

Parity: pinned (complex-step vs central differences of single steps and of whole runs; the
tau_21 gradient vanishes, Sec. 4.2).
"""
from __future__ import annotations

import numpy as np

from . import smrt as S

H_CS = 1e-30


def tau_keys(N: int):
    return [(n, m) for n in range(2, N + 1) for m in range(n // 2 + 1)]


def model_with_taus(model: S.Model, taus) -> S.Model:
    """A copy of model whose continuous times tau_c,nm are the given values (tau_ref = 1)."""
    star = dict(model.tau_star)
    for k, t in zip(tau_keys(model.N), taus):
        star[k] = t
    return S.Model(lat=model.lat, N=model.N, tau_ref=1.0, tau_star=star, rho_ref=model.rho_ref,
                   maxwell_law=model.maxwell_law)


def model_taus(model: S.Model) -> np.ndarray:
    return np.array([model.tau_star[k] * model.tau_ref for k in tau_keys(model.N)])


def collide_vjp(f, lam, model: S.Model, taus):
    """(J_C^T lam per cell, dL/dtau summed over cells) at pre-collision f (Q, ncell)."""
    Q, n = f.shape
    m = model_with_taus(model, taus)
    fbar = np.zeros((Q, n))
    for k in range(Q):
        fc = f.astype(np.complex128)
        fc[k] += 1j * H_CS
        fbar[k] = np.sum(lam * S.collide(fc, m).imag, axis=0) / H_CS
    gtau = np.zeros(len(taus))
    for p in range(len(taus)):
        tc = np.asarray(taus, dtype=np.complex128)
        tc[p] += 1j * H_CS
        gtau[p] = np.sum(lam * S.collide(f.astype(np.complex128), model_with_taus(model, tc)).imag) / H_CS
    return fbar, gtau


def stream_transpose(g, lat, geom: S.Geometry):
    """S^T: push g (Q, nz, ny, nx) back to where the pull read it; pulls from the constant
    end-state cells beyond fixed x ends carry no dependence and are dropped."""
    nz, ny, nx = geom.shape
    kx, ky, kz = geom.shift
    out = np.zeros_like(g)
    for i in range(lat.q):
        sx, sy, sz = int(lat.e[i, 0]) + kx, int(lat.e[i, 1]) + ky, int(lat.e[i, 2]) + kz
        src = np.roll(g[i], shift=(-sz, -sy), axis=(0, 1))
        if not geom.fixed_x:
            out[i] = np.roll(src, shift=-sx, axis=2)
            continue
        x = np.arange(nx)
        xs = x - sx                      # cell x pulled from xs
        inside = (xs >= 0) & (xs < nx)
        res = np.zeros_like(src)
        res[..., xs[inside]] = src[..., inside]
        out[i] = res
    return out


def step_vjp(h, lam_next, model: S.Model, geom: S.Geometry, taus):
    """lambda^t and dL/dtau contribution of one step, given lambda^{t+1}."""
    lat = model.lat
    f = S.stream(h, lat, geom).reshape(lat.q, -1)
    mu, gtau = collide_vjp(f, lam_next.reshape(lat.q, -1), model, taus)
    return stream_transpose(mu.reshape(h.shape), lat, geom), gtau


def loss_moments(h, model: S.Model, geom: S.Geometry):
    m = S.macroscopic(h, model, geom)
    return m["rho"], m["theta"], m["q"][0]


def shock_loss(h, model, geom, target):
    rho, th, q = loss_moments(h, model, geom)
    return float(np.sum((rho - target[0]) ** 2 + (th - target[1]) ** 2 + (q - target[2]) ** 2))


def shock_loss_grad(h, model, geom, target):
    """dL/dh of the shock loss: per-cell complex-step gradient of the moments, then S^T."""
    lat = model.lat
    f = S.stream(h, lat, geom).reshape(lat.q, -1)
    rho, th, q = loss_moments(h, model, geom)
    wr, wt, wq = 2 * (rho - target[0]), 2 * (th - target[1]), 2 * (q - target[2])
    gbar = np.zeros_like(f)
    Nd = max(model.N, 3)
    from .hermite import multi_indices_upto
    al = multi_indices_upto(Nd)
    pos = {a: k for k, a in enumerate(al)}
    for k in range(lat.q):
        fc = f.astype(np.complex128)
        fc[k] += 1j * H_CS
        r, u, t = S.conserved(fc, lat)
        d = S.local_direct(fc, lat, Nd, u, t)
        qx = 0.5 * t ** 1.5 * (d[pos[(3, 0, 0)]] + d[pos[(1, 2, 0)]] + d[pos[(1, 0, 2)]])
        gbar[k] = (wr * r.imag + wt * t.imag + wq * qx.imag) / H_CS
    return stream_transpose(gbar.reshape(h.shape), lat, geom)


def run_gradient(h0, model, geom, taus, nsteps, target, checkpoint_every=250):
    """L and dL/dtau of an nsteps run from h0, by checkpointed reverse sweeps."""
    m = model_with_taus(model, taus)
    ckpt = {0: h0.copy()}
    h = h0
    for t in range(nsteps):
        h = S.step(h, m, geom)
        if (t + 1) % checkpoint_every == 0 and t + 1 < nsteps:
            ckpt[t + 1] = h.copy()
    L = shock_loss(h, m, geom, target)
    lam = shock_loss_grad(h, m, geom, target)
    gtau = np.zeros(len(taus))
    starts = sorted(ckpt)
    for s0 in reversed(starts):
        s1 = min(s0 + checkpoint_every, nsteps)
        states = [ckpt[s0]]
        for _ in range(s0, s1 - 1):
            states.append(S.step(states[-1], m, geom))
        for t in range(s1 - 1, s0 - 1, -1):
            lam, g = step_vjp(states[t - s0], lam, m, geom, taus)
            gtau += g
    return L, gtau, lam
