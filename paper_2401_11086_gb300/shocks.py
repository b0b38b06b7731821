"""Set-up of 1D normal-shock problems on libsmrt contexts (Sec. 4.2 of Yan & Shan).

Problem set-up only (end states, frame shift, relaxation times, initial fields); every step of
the method runs in libsmrt. A shock of upstream Mach number Ma in a monatomic gas
(gamma = 5/3) has Rankine-Hugoniot end states (lb_rankine_hugoniot), a reference temperature
and integer frame shift chosen by lb_shock_frame, and relaxation times from Table 4 scaled by
the upstream mean free path: ell cells = tau_c,20 sqrt(theta1) / c.
"""
from __future__ import annotations

import numpy as np

from . import api

GAMMA = 5.0 / 3.0

# Largest upstream Mach number whose uniform states stay linearly stable on the degree-9
# velocity set (D3Q103, N = 4, theta2 = 1.2, ell = 2 cells): seeded 1e-6 noise on a periodic
# line at the upstream state stays flat at Ma = 3.0 and grows tenfold every 300 steps at 3.25;
# at Ma = 5 it overflows within 600 steps. Long domains (thousands of cells) let that growth
# run to completion, so batched long shocks on this set use Ma <= 3. The paper's own runs at
# Ma 5 and 7 use degree-11 and degree-19 sets.
MA_STABLE_DEGREE9 = 3.0

# Table 4: tau*_{n,m} = tau_{n,m} / tau_{2,0}, Maxwell molecules (SMRT) and the Shakhov model,
# in lb_set_relaxation's order (2,0) (2,1) (3,0) (3,1) (4,0) (4,1) (4,2) (5,0) (5,1) (5,2).
# tau_{2,1} (bulk) is absent for a monatomic gas; its mode vanishes identically, 1 is used.
TAU_RATIOS_SMRT = (1.0, 1.0, 2.0 / 3.0, 3.0 / 2.0, 432.0 / 763.0, 6.0 / 7.0, 3.0 / 2.0,
                   864.0 / 1655.0, 108.0 / 163.0, 1.0)
TAU_RATIOS_SHAKHOV = (1.0, 1.0, 1.0, 3.0 / 2.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0)
# Sec. 4.3's "reduced" operator: the SMRT table with tau*_{4,1} = tau*_{4,2} = 6/7, so that the
# two traced parts of the order-4 tensor relax together.
TAU_RATIOS_REDUCED = (1.0, 1.0, 2.0 / 3.0, 3.0 / 2.0, 432.0 / 763.0, 6.0 / 7.0, 6.0 / 7.0,
                      864.0 / 1655.0, 108.0 / 163.0, 1.0)

# Table 3: reference temperature (upstream theta1) of the paper's runs on the D1Q9-P1 product
# set, by upstream Mach number; the frame shift is k_x = 2 in these rows.
TABLE3_THETA1 = {1.5: 0.714, 3.0: 0.333, 5.0: 0.167}
# Table 3's Ma = 7 row runs on the D1Q17-P1 product set: theta1 = 0.071, k_x = 3.
TABLE3_THETA1_D1Q17 = {7.0: 0.071}


def ntau(N: int) -> int:
    return sum(n // 2 + 1 for n in range(2, N + 1))


def shock_params(Ma: float, c: float, N: int, ell_cells: float = 2.0, ratios=TAU_RATIOS_SMRT,
                 theta2_max: float = 1.2, theta1: float | None = None):
    """End states, frame shift and continuous relaxation times of one shock. theta1 overrides
    the reference temperature (e.g. a Table 3 value); the frame shift follows it."""
    if theta1 is None:
        theta1, kx = api.lb_shock_frame(Ma, c, GAMMA, theta2_max)
    else:
        kx = api.lb_shock_shift(Ma, c, theta1, GAMMA)
    left, right = api.lb_rankine_hugoniot(Ma, GAMMA, 1.0, theta1)
    tau20 = ell_cells * c / np.sqrt(theta1)
    taus = [r * tau20 for r in ratios[: ntau(N)]]
    return {"Ma": Ma, "theta1": theta1, "kx": kx, "left": left, "right": right, "taus": taus}


def tanh_fields(params, L: int, width: float):
    """rho, u_x, theta of the tanh blend between the end states (x0 = L/2); width <= 0 gives
    the step of the paper's runs (Sec. 4.2): upstream on x < L/2, downstream beyond."""
    x = np.arange(L, dtype=np.float64)
    if width > 0:
        s = 0.5 * (1.0 + np.tanh((x - L / 2.0) / width))
    else:
        s = (x >= L // 2).astype(np.float64)
    lf, rt = params["left"], params["right"]
    rho = lf["rho"] + (rt["rho"] - lf["rho"]) * s
    u = lf["u"][0] + (rt["u"][0] - lf["u"][0]) * s
    th = lf["theta"] + (rt["theta"] - lf["theta"]) * s
    return rho, u, th


def setup_batch(lattice: api.LatticeDesc, N: int, machs, lengths, precision: str = "f32c64",
                ell_cells: float = 2.0, width: float = 10.0, stream=None, ratios=TAU_RATIOS_SMRT,
                theta1=None):
    """A batched context with one shock per (Ma, L) and its initial state: the equilibrium of
    the tanh blend of width `width` cells (10 by default: a wider blend puts intermediate
    (u, theta) states into the cells that, above Ma ~ 3.5, leave the stable range of a degree-9
    velocity set; width <= 0: a step). ratios: tau*_{n,m} table; theta1: optional per-instance
    upstream temperatures (e.g. Table 3's). Returns (ctx, state, per-instance params)."""
    import torch
    lat = api.LatticeDesc(lattice.e, lattice.w, lattice.c, lattice.degree, (0, 0, 0))
    ctx = api.lb_init_lattice(lat, 0, N=N, precision=precision, bc_x=1,
                              nx_per_instance=[int(L) for L in lengths], stream=stream)
    params = []
    rho, ux, th = [], [], []
    for j, (Ma, L) in enumerate(zip(machs, lengths)):
        t1 = None if theta1 is None else float(theta1[j])
        p = shock_params(float(Ma), lattice.c, N, ell_cells, ratios=ratios, theta1=t1)
        api.lb_set_frame_shift(ctx, j, p["kx"])
        api.lb_set_relaxation(ctx, p["taus"], True, 1.0, p["left"], p["right"], instance=j)
        r, u, t = tanh_fields(p, int(L), width)
        rho.append(r)
        ux.append(u)
        th.append(t)
        params.append(p)
    rho, ux, th = np.concatenate(rho), np.concatenate(ux), np.concatenate(th)
    u = np.stack([ux, np.zeros_like(ux), np.zeros_like(ux)])
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(ctx.device)  # noqa: E731
    f = ctx.new_state()
    api.lb_fill_equilibrium(ctx, f, dev(rho), dev(u), dev(th))
    ctx.relax_args = None  # per-instance relaxation: lb_set_relaxation was called per instance
    return ctx, f, params
