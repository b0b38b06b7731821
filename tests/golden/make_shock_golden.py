"""Write oracle reference profiles of 1D normal shocks to tests/golden/*.npz.

Calls only ``oracle/`` and the shared input generators in ``synthetic.py``; nothing here
touches the CUDA path. Usage:

    python tests/golden/make_shock_golden.py ma3_d3q103_n4          # Ma = 3, 2048 cells, 20000 steps
    python tests/golden/make_shock_golden.py ma5_d3q103_n4_target   # Ma = 5, 1024 cells, 5000 steps
    python tests/golden/make_shock_golden.py ma3_d3q729_n5          # Table 3 row Ma = 3, 100 cells
    python tests/golden/make_shock_golden.py ma7_d3q4913_n5         # Table 3 row Ma = 7, 100 cells
    python tests/golden/make_shock_golden.py mixed_d3q729_n5        # batch of Ma 1.5 / 2.5 / 4 / 5

Each case stores, at the listed step counts, the moments of the pre-collision populations
(rho, physical u_x, theta, q_x) on every cell, float64.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synthetic  # noqa: E402
from oracle import lattice as L  # noqa: E402
from oracle import shock as K  # noqa: E402
from oracle import smrt as S  # noqa: E402

CASES = {
    # SMRT, Table 4 times, ell = 2 upstream cells, tanh width 20, theta2 = 1.2 reference
    "ma3_d3q103_n4": dict(lattice="D3Q103", N=4, Ma=3.0, nx=2048, width=20.0,
                          checkpoints=(2000, 20000)),
    # target of the differentiable shock: Ma = 5, 1024 cells, Table 4 times, 5000 steps
    "ma5_d3q103_n4_target": dict(lattice="D3Q103", N=4, Ma=5.0, nx=1024, width=10.0,
                                 checkpoints=(5000,)),
    # the paper's own configuration (Sec. 4.2, Table 3 row Ma = 3): D3Q729, N = 5, 100 cells,
    # theta1 = 0.333, k_x = 2, step initial condition, Table 4 SMRT times, ell = 2 cells
    "ma3_d3q729_n5": dict(lattice="D3Q729", N=5, Ma=3.0, nx=100, width=0.0, theta1=0.333,
                          checkpoints=(200, 1000)),
    # Table 3 row Ma = 7: D3Q4913 (D1Q17-P1 product), N = 5, theta1 = 0.071, k_x = 3
    "ma7_d3q4913_n5": dict(lattice="D3Q4913", N=5, Ma=7.0, nx=100, width=0.0, theta1=0.071,
                           checkpoints=(100, 400)),
}


# A batch of shocks of different Mach numbers on the paper's D3Q729 set (N = 5), each with the
# reference temperature of reading 11 (theta2 = 1.2 above Ma 1.9: Table 3's own theta1 = 0.167
# makes the Ma = 5 upstream state linearly unstable on long domains), tanh width 10, SMRT times
# of Table 4 with ell = 2 upstream cells; profiles after 1000 steps, one entry per instance.
BATCHES = {
    "mixed_d3q729_n5": dict(lattice="D3Q729", N=5, machs=(1.5, 2.5, 4.0, 5.0), nx=(80, 100, 120, 140),
                            width=10.0, checkpoints=(1000,)),
}


def run_batch(name: str):
    cfg = BATCHES[name]
    lat = L.by_name(cfg["lattice"])
    out = {"machs": np.array(cfg["machs"]), "nx": np.array(cfg["nx"])}
    t0 = time.time()
    for j, (Ma, nx) in enumerate(zip(cfg["machs"], cfg["nx"])):
        case = K.shock_case(lat, cfg["N"], Ma, nx)
        st = case.states
        h = K.initial_state(case, *[synthetic.tanh_blend(nx, cfg["width"], st[k + "1"], st[k + "2"])
                                    for k in ("rho", "u", "theta")])
        done = 0
        for cp in cfg["checkpoints"]:
            for _ in range(cp - done):
                h = S.step(h, case.model, case.geom)
            done = cp
            m = S.macroscopic(h, case.model, case.geom)
            for key in ("rho", "theta"):
                out[f"{key}_{cp}_{j}"] = m[key]
            out[f"q_{cp}_{j}"] = m["q"][0]
        out[f"theta1_{j}"] = case.theta1
        out[f"k_{j}"] = case.k
        print(f"{name}: instance {j} (Ma {Ma}) after {time.time() - t0:.0f} s", flush=True)
    np.savez_compressed(os.path.join(HERE, f"{name}.npz"), **out)


def run(name: str):
    if name in BATCHES:
        run_batch(name)
        return
    cfg = CASES[name]
    lat = L.by_name(cfg["lattice"])
    case = K.shock_case(lat, cfg["N"], cfg["Ma"], cfg["nx"], theta1=cfg.get("theta1"))
    st = case.states
    nx, W = cfg["nx"], cfg["width"]
    if W > 0:
        prof = lambda k: synthetic.tanh_blend(nx, W, st[k + "1"], st[k + "2"])  # noqa: E731
    else:
        prof = lambda k: synthetic.step_blend(nx, st[k + "1"], st[k + "2"])  # noqa: E731
    h = K.initial_state(case, prof("rho"), prof("u"), prof("theta"))
    out = {"theta1": case.theta1, "k": case.k, "tau_ref": case.model.tau_ref}
    t0 = time.time()
    done = 0
    for cp in cfg["checkpoints"]:
        for _ in range(cp - done):
            h = S.step(h, case.model, case.geom)
        done = cp
        m = S.macroscopic(h, case.model, case.geom)
        for key in ("rho", "theta"):
            out[f"{key}_{cp}"] = m[key]
        out[f"u_{cp}"] = m["u"][0]
        out[f"q_{cp}"] = m["q"][0]
        print(f"{name}: step {cp} after {time.time() - t0:.0f} s", flush=True)
    np.savez_compressed(os.path.join(HERE, f"{name}.npz"), **out)


if __name__ == "__main__":
    for n in sys.argv[1:] or list(CASES) + list(BATCHES):
        run(n)
