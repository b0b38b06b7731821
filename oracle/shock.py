"""Normal-shock problem set-up (oracle; test infrastructure only).

* ``rankine_hugoniot``: Eq. rankine with the temperature ratio read as
  (2 gamma Ma^2 - gamma + 1)((gamma-1) Ma^2 + 2) / ((gamma+1)^2 Ma^2). The printed denominator
  has Ma to the first power; only the squared form reproduces Table 3 (pinned in the tests).
* ``mean_speed``: (u1 + u2)/2 = (gamma Ma^2 + 1)/((gamma+1) Ma) c1 (Sec. 4.2).
* ``shift``: k_x = round(((u1 + u2)/2) / c), the integer frame shift of Sec. 4.1; reproduces
  every k_x and u_bar_x of Table 3.
* ``theta_scale``: the reference temperature is chosen so that the hottest state stays well
  below the Hermite convergence bound theta < 2 (Sec. 4.1): theta1 = 1 when the downstream
  state is at most ``theta2_target`` (1.2) at theta1 = 1, otherwise theta2 = ``theta2_target``,
  i.e. theta1 = min(1, theta2_target / (theta2/theta1)). The paper lowers theta1 below 1 even
  where theta2 would stay below 2 (Table 3, Ma = 1.5: theta1 = 0.714, theta2 = 1.07), and a
  downstream state at theta2 = 1.94 (Ma = 1.89 with theta1 = 1) is unstable on D3Q729.
* ``tau_from_mean_free_path``: the upstream mean free path in cells is
  ell = tau_c sqrt(theta1) / c (time in steps, cell size c), so tau_c = ell c / sqrt(theta1).
  The paper's Kn definition (Sec. 4.2) is dimensionally garbled; this is the reading used.
* ``shock_case``: model, geometry and end states of a 1D shock on nx cells with Maxwellian
  (order-N equilibrium) end states; the initial fields are supplied by the caller.

Parity: pinned (Table 3 rows; steady shock reached with RH end states).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .lattice import Lattice
from .smrt import TAU_STAR_SMRT, Geometry, Model, equilibrium

GAMMA = 5.0 / 3.0


def rankine_hugoniot(Ma: float, gamma: float = GAMMA, rho1: float = 1.0, theta1: float = 1.0):
    """Downstream (rho2, u2, theta2) and upstream u1 of a normal shock (shock frame)."""
    r = (gamma + 1.0) * Ma ** 2 / ((gamma - 1.0) * Ma ** 2 + 2.0)
    t = (2.0 * gamma * Ma ** 2 - gamma + 1.0) * ((gamma - 1.0) * Ma ** 2 + 2.0) / ((gamma + 1.0) ** 2 * Ma ** 2)
    u1 = Ma * np.sqrt(gamma * theta1)
    return {"rho1": rho1, "u1": u1, "theta1": theta1,
            "rho2": rho1 * r, "u2": u1 / r, "theta2": theta1 * t}


def mean_speed(Ma: float, theta1: float, gamma: float = GAMMA) -> float:
    return (gamma * Ma ** 2 + 1.0) / ((gamma + 1.0) * Ma) * np.sqrt(gamma * theta1)


def half_jump(Ma: float, theta1: float, gamma: float = GAMMA) -> float:
    return (Ma ** 2 - 1.0) / ((gamma + 1.0) * Ma) * np.sqrt(gamma * theta1)


def theta_scale(Ma: float, theta2_target: float = 1.2, gamma: float = GAMMA) -> float:
    """Upstream theta1 in units of the reference temperature."""
    ratio = rankine_hugoniot(Ma, gamma)["theta2"]
    return min(1.0, theta2_target / ratio)


def shift(Ma: float, theta1: float, c: float, gamma: float = GAMMA) -> int:
    return int(np.round(mean_speed(Ma, theta1, gamma) / c))


def tau_from_mean_free_path(ell_cells: float, c: float, theta1: float) -> float:
    return ell_cells * c / np.sqrt(theta1)


@dataclass
class ShockCase:
    model: Model
    geom: Geometry
    states: dict            # physical end states (shock frame)
    k: int                  # frame shift, u_bar = c k
    theta1: float


def shock_case(lat: Lattice, N: int, Ma: float, nx: int, ell_cells: float = 2.0,
               tau_star: dict | None = None, theta1: float | None = None,
               gamma: float = GAMMA) -> ShockCase:
    th1 = theta_scale(Ma, gamma=gamma) if theta1 is None else theta1
    st = rankine_hugoniot(Ma, gamma, 1.0, th1)
    k = shift(Ma, th1, lat.c, gamma)
    ubar = lat.c * k
    tau_ref = tau_from_mean_free_path(ell_cells, lat.c, th1)
    model = Model(lat=lat, N=N, tau_ref=tau_ref, tau_star=dict(tau_star or TAU_STAR_SMRT),
                  rho_ref=1.0, maxwell_law=True)
    zero = np.zeros(1)
    left = equilibrium(np.array([st["rho1"]]), np.array([[st["u1"] - ubar], zero, zero]),
                       np.array([st["theta1"]]), lat, N)[:, 0]
    right = equilibrium(np.array([st["rho2"]]), np.array([[st["u2"] - ubar], zero, zero]),
                        np.array([st["theta2"]]), lat, N)[:, 0]
    geom = Geometry(shape=(1, 1, nx), shift=(k, 0, 0), fixed_x=True, ghost_left=left, ghost_right=right)
    return ShockCase(model=model, geom=geom, states=st, k=k, theta1=th1)


def initial_state(case: ShockCase, rho, u_phys, theta):
    """Post-collision state h0 = order-N equilibrium of the given fields (length nx each)."""
    lat = case.model.lat
    nx = case.geom.shape[2]
    ubar = lat.c * case.k
    u = np.stack([np.asarray(u_phys) - ubar, np.zeros(nx), np.zeros(nx)])
    f = equilibrium(np.asarray(rho), u, np.asarray(theta), lat, case.model.N)
    return f.reshape(lat.q, 1, 1, nx)
