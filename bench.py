#!/usr/bin/env python
"""Throughput of the LB-SMRT fused collide-and-stream step on GB300.

Workload (the HBM-roofline case): a 256^3 periodic box, D3Q39 velocity set, SMRT truncated at
order N = 3 with the Maxwell-molecule relaxation times of Table 4, populations and arithmetic
in FP32. Initial state: the order-3 equilibrium of rho = 1 + N(0, 1e-3^2) (seed 11086),
theta = 1 and a Taylor-Green velocity field of amplitude 0.05 (synthetic.taylor_green), made on
the device by lb_fill_equilibrium. One step = one launch of the fused kernel over all cells;
the two 2.6 GB state buffers (5.2 GB) are far larger than the 129 MB L2, so every timed step
streams from HBM.

Metric: GLUPSxQ = cells x Q x steps / s (cell-velocity updates per second), with the fraction
of the HBM roofline taken from the algorithmic traffic 2 Q 4 bytes per cell-step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 oracle (the plain CPU restatement of the method) on the host
cores on a bounded sample of the same workload: the 32^3 corner block of the same Taylor-Green
field stepped as its own periodic box. With N > 1 (torchrun), every rank runs its own box
(replicas: the step has no exchange on one GPU) and value = all ranks' updates / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

Q = 39
N_ORDER = 3
METRIC = "GLUPSxQ (cell-velocity updates/s) and % HBM roofline"
UNIT = "G cell-velocity updates/s"
# the device code of the box and batched-line kernels (launch set-up excluded)
KERNEL_SOURCES = ["core.cuh", "kernels.cuh", "lattices.cuh"]
PROFILE = os.path.join(ROOT, "profiles", "collide_stream_d3q39_f32_box.txt")
PROFILE_BATCHED = os.path.join(ROOT, "profiles", "collide_stream_d3q103_n4_batched.txt")


def kernel_hash() -> str:
    h = hashlib.sha256()
    for n in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2401_11086_gb300", "csrc", n), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profile_value(path: str, key: str):
    """A number recorded in a committed ncu summary ("key: value" line), or None when the
    summary is missing or was taken on different kernel sources."""
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_sources_sha256_12") != kernel_hash():
        return None
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


def profile_traffic(n: int):
    """DRAM bytes per launch from the committed ncu summary of the box, scaled to n^3 cells."""
    per_cell = profile_value(PROFILE, "dram_bytes_per_cell")
    return None if per_cell is None else per_cell * n ** 3


def tau_table():
    # Table 4 (SMRT, Maxwell molecules) times tau_20; tau_20 from an upstream mean free path of
    # 2 cells at theta = 1: tau_c = 2 c / sqrt(theta).
    return [1.0, 1.0, 2.0 / 3.0, 1.5]


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        # raw samples go to SMRT_CLOCK_DIR (default: the system temporary directory); the
        # JSON line carries their summary
        self.path = os.path.join(os.environ.get("SMRT_CLOCK_DIR", tempfile.gettempdir()),
                                 f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = max(mx, float(parts[2]))
                except ValueError:
                    continue
                for name, flag in zip(names, parts[5:9]):
                    if flag.lower() == "active":
                        reasons.add(name)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample_rate(block: int, steps: int, warmup: int = 1) -> dict:
    """FP64 oracle on the block^3 corner of the 256^3 Taylor-Green workload (own periodic box),
    single-threaded BLAS; returns cell-velocity updates/s. Runs in a fresh spawned process."""
    code = f"""
import os, sys, time, json
sys.path.insert(0, {ROOT!r})
import numpy as np
import synthetic
from oracle import lattice as L, smrt as S
lat = L.d3q39()
rho, u, th = synthetic.taylor_green(256)
b = {block}
rho, u, th = rho[:b, :b, :b], u[:, :b, :b, :b], th[:b, :b, :b]
model = S.Model(lat, 3, tau_ref=2.0 * lat.c)
geom = S.Geometry(shape=(b, b, b))
h = S.equilibrium(rho.ravel(), u.reshape(3, -1), th.ravel(), lat, 3).reshape(lat.q, b, b, b)
for _ in range({warmup}):
    h = S.step(h, model, geom)
t0 = time.perf_counter()
for _ in range({steps}):
    h = S.step(h, model, geom)
dt = time.perf_counter() - t0
print(json.dumps({{"rate": b ** 3 * lat.q * {steps} / dt, "seconds": dt}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if res.returncode != 0:
        raise RuntimeError(f"oracle baseline failed: {res.stderr[-2000:]}")
    return json.loads(res.stdout.strip().splitlines()[-1])


def oracle_sample_rate_all_cores(block: int, steps: int, warmup: int = 1) -> dict:
    """The same oracle sample run as one process per host core at once (independent samples,
    single-threaded BLAS each): the aggregate rate of the host's cores, with their count."""
    ncores = os.cpu_count() or 1
    code = f"""
import sys, json
sys.path.insert(0, {ROOT!r})
import bench
print(json.dumps(bench.oracle_sample_rate({block}, {steps}, {warmup})))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    t0 = time.perf_counter()
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                              text=True, env=env) for _ in range(ncores)]
    rates = []
    for pr in procs:
        out, err = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError(f"oracle baseline failed: {err[-2000:]}")
        rates.append(json.loads(out.strip().splitlines()[-1])["rate"])
    return {"rate": float(sum(rates)), "cores": ncores, "seconds": time.perf_counter() - t0}


# The other workloads, each timed by its own bench.py run after the box on the same GPU (one
# GPU only), reported in the box line under "secondary": the 64 batched shocks on D3Q103 in the
# split precision, the 512 Table 3 shocks on D3Q729 in FP32, the mixed-Mach batch (Ma 1.2 to 7 on
# D3Q729 / D3Q4913) as one graph replay of 1000 steps per set, and the adjoint (its step kernel
# on the batched shocks; the 5000-step differentiable shock forward and backward).
SECONDARY_WORKLOADS = [
    ["--workload", "batched", "--steps", "200", "--warmup", "5"],
    ["--workload", "table3", "--precision", "f32", "--steps", "100", "--warmup", "5"],
    ["--workload", "mixed_mach", "--steps", "1000", "--warmup", "3"],
    ["--workload", "adjoint", "--steps", "5000", "--warmup", "3"],
]


def run_secondary(extra: list, timeout: float = 600.0) -> dict:
    """One other workload's bench.py line, condensed: its own CUDA-event timing, roofline and
    clocks, run as a child process (no oracle baseline)."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), *extra, "--no-cpu-baseline", "--no-secondary"]
    out = {"args": " ".join(extra)}
    try:
        res = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout)
    except subprocess.TimeoutExpired:
        out["error"] = f"no result within {timeout:.0f} s"
        return out
    lines = [x for x in res.stdout.splitlines() if x.startswith("{")]
    if res.returncode != 0 or not lines:
        out["error"] = (res.stderr or res.stdout)[-400:]
        return out
    d = json.loads(lines[-1])
    roof = d.get("roofline") or {}
    out.update({"workload": d["config"]["workload"], "value": d["value"], "unit": d["unit"],
                "ms_per_step": d["ms_per_step"], "steps": d["steps"], "dtype": d["dtype"],
                "roofline": {k: roof.get(k) for k in ("bound", "achieved", "peak", "unit", "frac")},
                "clocks": d.get("clocks")})
    return out


def run_reference(args, rank: int) -> None:
    if rank != 0:
        return
    # size the sampled block so that warm-up + timed steps stay near 90 s of oracle work
    # (about 24 us per cell-step for the FP64 oracle on one core)
    budget_cells = 90.0 / max(1, args.steps + args.warmup) / 24e-6
    block = int(max(8, min(32, round(budget_cells ** (1.0 / 3.0)))))
    t0 = time.perf_counter()
    r = oracle_sample_rate(block, args.steps, args.warmup)
    wall = time.perf_counter() - t0
    value = r["rate"] / 1e9
    sample = f"{block}^3 corner block of the 256^3 Taylor-Green box, {args.steps} oracle steps"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * r["seconds"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "box256_d3q39_n3_f32", "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


def batched_instances(rank: int):
    """The 64 shocks of one rank: Mach numbers and lengths drawn with seed 11086 + rank (each
    rank owns its own independent instances), Ma within the degree-9 set's stable range."""
    import synthetic
    from paper_2401_11086_gb300.shocks import MA_STABLE_DEGREE9
    return synthetic.batched_shocks(seed=synthetic.SEED + rank, ma_range=(1.2, MA_STABLE_DEGREE9))


def job_rate(units: float, ms: float, dist=None, device="cuda"):
    """Whole-job throughput: all ranks' units / the slowest rank's time. Returns (units per
    second, max ms). Without a process group, the local numbers."""
    if dist is None:
        return units / (ms * 1e-3), ms
    import torch
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()) / (float(t.item()) * 1e-3), float(t.item())


def oracle_shock_rate(L: int, steps: int) -> dict:
    """FP64 oracle on one Ma = 3 shock of L cells (D3Q103, N = 4), single-threaded BLAS."""
    code = f"""
import sys, time, json
sys.path.insert(0, {ROOT!r})
import synthetic
from oracle import lattice as Lt, shock as K, smrt as S
lat = Lt.d3q103()
case = K.shock_case(lat, 4, 3.0, {L})
st = case.states
h = K.initial_state(case, *[synthetic.tanh_blend({L}, 10.0, st[k + "1"], st[k + "2"]) for k in ("rho", "u", "theta")])
h = S.step(h, case.model, case.geom)
t0 = time.perf_counter()
for _ in range({steps}):
    h = S.step(h, case.model, case.geom)
dt = time.perf_counter() - t0
print(json.dumps({{"rate": {L} * lat.q * {steps} / dt, "seconds": dt}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if res.returncode != 0:
        raise RuntimeError(f"oracle baseline failed: {res.stderr[-2000:]}")
    return json.loads(res.stdout.strip().splitlines()[-1])


def run_batched(args, world: int, rank: int, local: int) -> None:
    """64 independent 1D shocks (Ma ~ U[1.2, 3], lengths from {512..8192}, seed 11086), D3Q103,
    N = 4, FP32 populations with exact fixed-point conserved sums and a two-float equilibrium,
    autotuned launch schedule. With N ranks the instances are split between them (no data
    exchange: the problems are independent)."""
    import numpy as np
    import torch

    import paper_2401_11086_gb300 as P
    import synthetic
    from paper_2401_11086_gb300 import shocks
    from paper_2401_11086_gb300.autotune import tuned_schedule

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    # weak scaling: every rank runs its own 64 shocks; instances are independent, so there is
    # no exchange
    machs, lengths = batched_instances(rank)
    d = P.lb_lattice_named("D3Q103")
    stream = torch.cuda.current_stream()
    ctx, f0, _ = shocks.setup_batch(d, 4, machs, lengths, precision="f32c64", stream=stream)
    sched = tuned_schedule(ctx, f0, lengths, trial_steps=10)
    fa, fb = f0, ctx.new_state()
    cur = P.lb_step(ctx, fa, fb, args.warmup)
    other = fb if cur is fa else fa
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    K = args.steps
    # the two state buffers (2 x ~81 MB) fit in the 129 MB L2 together with little else, so
    # every timed step starts after a 256 MB write that flushes L2; only the step is timed
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f0.device)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    for i in range(K):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        cur = P.lb_step(ctx, cur, other, 1)
        ev[i][1].record(stream)
        other = fa if cur is fb else fb
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    st, flags = P.lb_poll_status(ctx)
    if st != 0:
        raise SystemExit(f"health word reports status {st} (flags {flags})")
    cells = int(lengths.sum())
    q = 103
    rate, ms = job_rate(cells * q * K, ms, dist)
    value = rate / 1e9
    peak, peak_kind = measured_peak()
    achieved = 2.0 * q * 4 * cells * K / (ms * 1e-3) / 1e9
    # the FP64 pipe bounds this kernel: its double-precision operations per cell-step (ncu
    # instruction counts, an FMA counted as two) against the nominal FP64 rate
    # the kernel is bound by instruction issue (ncu: 26 % issue-active, instruction-fetch stalls
    # first): its warp instructions per cell-step against one per clock per scheduler
    ginst = BATCHED_WARP_INST_PER_CELL * cells * K / (ms * 1e-3) / 1e9
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        r = oracle_shock_rate(512, 40)
        cpu = {"value": r["rate"] / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "one Ma = 3 shock of 512 cells (D3Q103, N = 4), 40 FP64 oracle steps"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (exact fixed-point moments and conserved sums, two-float equilibrium)", "data": "synthetic",
            "config": {"workload": "batched_shocks_64_d3q103_n4", "instances_per_gpu": int(len(machs)),
                       "cells_per_gpu": cells, "velocities": q, "hermite_order": 4,
                       "schedule": sched,
                       "l2": "L2 flushed (256 MB write) before every timed step; steps timed one by one"},
            "roofline": {"bound": "alu", "achieved": ginst, "peak": ISSUE_PEAK_GINST,
                         "unit": "G warp-instructions/s", "frac": ginst / ISSUE_PEAK_GINST,
                         "traffic": profile_value(PROFILE_BATCHED, "dram_bytes_per_launch"),
                         "peak_kind": "instruction issue: 4 schedulers x 152 SMs x 2070 MHz, one warp "
                                      "instruction per clock each",
                         "warp_inst_per_cell": BATCHED_WARP_INST_PER_CELL,
                         "hbm_achieved_gbs": achieved, "hbm_frac": achieved / peak,
                         "note": "instruction issue (fetch-bound), not HBM, limits this workload"},
            "cpu_baseline": cpu, "gpu_launches": K,
            "clocks": clk}
    print(json.dumps(line), flush=True)


# double-precision operations per cell-step of the D3Q729, N = 5 step kernel (ncu: DFMA x 2 +
# DADD + DMUL over one launch of the 512-shock workload, divided by its cells), and the
# nominal FP64 rate of a GB300
TP_FP64_FLOP_PER_CELL = 14949.0
FP64_PEAK_GFLOPS = 1250.0
# warp instructions per cell-step of the split-precision D3Q103, N = 4 staged line kernel on the
# 64 batched shocks (ncu smsp__inst_executed.sum of one launch / cells: 499.9 for the persistent
# form, 501.9 for one plain launch per step), and the issue rate of a GB300 (4 schedulers per SM,
# 152 SMs, 2070 MHz, one warp instruction per clock each)
BATCHED_WARP_INST_PER_CELL = 499.9
ISSUE_PEAK_GINST = 4 * 152 * 2.07


def table3_instances(rank: int, count: int = 512, length: int = 0, lattice: str = "D3Q729"):
    """The Table 3 workload of one rank: count shocks cycling over the D3Q729 rows (Ma 3, 1.5,
    5 with their theta1), or all on the D3Q4913 row (Ma 7), lengths 100..400 cells drawn with
    seed 11086 + rank, or all `length` cells when given (a single shock is then the paper's
    run of that row)."""
    import numpy as np
    from paper_2401_11086_gb300 import shocks
    if lattice == "D3Q4913":
        machs = [7.0] * count
    else:
        machs = [(3.0, 1.5, 5.0)[j % 3] for j in range(count)]
    if length > 0:
        lengths = np.full(count, length)
    else:
        lengths = np.random.default_rng(11086 + rank).integers(100, 401, count)
    th = {**shocks.TABLE3_THETA1, **shocks.TABLE3_THETA1_D1Q17}
    return machs, lengths, [th[m] for m in machs]


def oracle_table3_rate(steps: int, lattice: str = "D3Q729") -> dict:
    """FP64 oracle on one Table 3 shock (Ma = 3 on D3Q729, Ma = 7 on D3Q4913; 100 cells,
    N = 5), single-threaded."""
    mk, Ma, th1, q = {"D3Q729": ("d3q729", 3.0, 0.333, 729), "D3Q4913": ("d3q4913", 7.0, 0.071, 4913)}[lattice]
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import synthetic
from oracle import lattice as L, shock as K, smrt as S
lat = L.{mk}()
case = K.shock_case(lat, 5, {Ma}, 100, theta1={th1})
st = case.states
h = K.initial_state(case, *[synthetic.step_blend(100, st[k + "1"], st[k + "2"]) for k in ("rho", "u", "theta")])
h = S.step(h, case.model, case.geom)
t0 = time.perf_counter()
for _ in range({steps}):
    h = S.step(h, case.model, case.geom)
dt = time.perf_counter() - t0
print(json.dumps({{"rate": 100 * {q} * {steps} / dt, "seconds": dt}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_table3(args, world: int, rank: int, local: int) -> None:
    """The paper's configuration (Sec. 4.2, Table 3): D3Q729 = D1Q9-P1^3, N = 5, SMRT times of
    Table 4, step initial condition, fixed end states; 512 shocks per GPU cycling over the
    rows Ma = 1.5, 3, 5 (theta1 = 0.714, 0.333, 0.167, k_x = 2), 100..400 cells each."""
    import torch

    import paper_2401_11086_gb300 as P
    from paper_2401_11086_gb300 import shocks

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    machs, lengths, theta1 = table3_instances(rank, args.instances, args.length, args.lattice)
    d = P.lb_lattice_named(args.lattice)
    stream = torch.cuda.current_stream()
    prec = args.precision
    ctx, f0, _ = shocks.setup_batch(d, 5, machs, lengths, precision=prec, width=0.0, theta1=theta1,
                                    stream=stream)
    if args.es_b is not None:          # the ES-BGK model (Sec. 3) instead of SMRT
        P.lb_set_collision_model(ctx, -1, P.LB_MODEL_ES_BGK, args.es_b)
    if args.tensor_cores:              # the projection's x-row sums on the tensor cores
        P.lb_set_schedule(ctx, 32, 0, 0, tensor_cores=1)   # (one warp per block)
    elif args.tile_width:
        P.lb_set_schedule(ctx, args.tile_width, 0, 0)
    sched = P.lb_get_schedule(ctx)   # the library's choice for this size
    fa, fb = f0, ctx.new_state()
    cur = P.lb_step(ctx, fa, fb, args.warmup)
    other = fb if cur is fa else fa
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    K = args.steps
    cells = int(sum(lengths))
    q = d.q
    elem = 8 if prec == "f64" else 4
    # states that fit in the 129 MB L2 are flushed (256 MB write) before every timed step
    small = 2 * q * elem * cells < 129e6
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f0.device) if small else None
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    for i in range(K):
        if small:
            flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        cur = P.lb_step(ctx, cur, other, 1)
        ev[i][1].record(stream)
        other = fa if cur is fb else fb
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    st, flags = P.lb_poll_status(ctx)
    if st != 0:
        raise SystemExit(f"health word reports status {st} (flags {flags})")
    kern_ms = ms / K
    rate, ms = job_rate(cells * q * K, ms, dist)
    if rank != 0:
        return
    peak, peak_kind = measured_peak()
    alg_bytes = 2.0 * q * elem * cells
    achieved = alg_bytes / (kern_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None, "peak_kind": f"{peak_kind} (copy bandwidth)",
            "algorithmic_bytes_per_launch": alg_bytes, "kernel_ms": kern_ms,
            "note": "issue-bound: the HBM fraction says how far from the memory roofline"}
    if prec == "f64" and args.lattice == "D3Q729":
        # the FP64 pipe bounds the double kernel: its double-precision operations per
        # cell-step (ncu instruction counts, an FMA counted as two) against the nominal rate
        gflop = TP_FP64_FLOP_PER_CELL * cells / (kern_ms * 1e-3) / 1e9
        roof = {"bound": "alu", "achieved": gflop, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s (fp64)",
                "frac": gflop / FP64_PEAK_GFLOPS, "traffic": None, "peak_kind": "nominal FP64 rate",
                "flop_per_cell": TP_FP64_FLOP_PER_CELL, "kernel_ms": kern_ms,
                "hbm_frac": achieved / peak}
    cpu = None
    if not args.no_cpu_baseline:
        nst = 40 if args.lattice == "D3Q729" else 6
        r = oracle_table3_rate(nst, args.lattice)
        row = "Ma = 3, 100 cells, D3Q729" if args.lattice == "D3Q729" else "Ma = 7, 100 cells, D3Q4913"
        cpu = {"value": r["rate"] / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one Table 3 shock ({row}, N = 5), {nst} FP64 oracle steps"}
    line = {"metric": METRIC, "value": rate / 1e9, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": f"table3_{args.lattice.lower()}_n5_{prec}" + ("" if args.es_b is None else "_es_bgk")
                                   + ("_tensor_core_xrows" if args.tensor_cores else ""),
                       "collision": "SMRT" if args.es_b is None else f"ES-BGK b={args.es_b}",
                       "instances_per_gpu": len(machs),
                       "cells_per_gpu": cells, "velocities": q, "hermite_order": 5,
                       "state_bytes": elem * int(ctx.state_elems), "schedule": sched,
                       "l2": "L2 flushed (256 MB write) before every timed step" if small else
                             "inputs larger than L2"},
            "roofline": roof, "cpu_baseline": cpu, "gpu_launches": K, "clocks": clk}
    print(json.dumps(line), flush=True)


def run_mixed_mach(args, world: int, rank: int, local: int) -> None:
    """The batched configuration as specified: 64 shocks with Ma ~ U[1.2, 7] and lengths from
    {512, ..., 8192} (seed 11086 + rank), each run for K steps by one persistent launch captured
    in a CUDA graph (lb_step_graph), launch schedule from the autotuner (the fastest persistent
    one: the graph replays a persistent launch). The degree-9 set holds
    uniform states only up to Ma 3, so the shocks run on the paper's own sets: Ma <= 5 on
    D3Q729 (D1Q9-P1 cubed, degree 11), Ma > 5 on D3Q4913 (D1Q17-P1 cubed, degree 19); N = 5,
    SMRT times of Table 4 with ell = 2 upstream cells, reference temperatures with theta2 = 1.2
    (Table 3's own theta1 = 0.167 leaves the Ma 5 upstream state linearly unstable), tanh width
    10. Populations: FP32 on D3Q729; FP64 on D3Q4913, where the float rounding seeds a
    long-wave instability of the Ma > 5 upstream states that blows up the 8192-cell lines within
    1000 steps (it grows in FP64 too, ~30x per 250 steps, from round-off; these sets have no
    split precision). K defaults to 1000: the configuration's 10000 steps at these Mach numbers
    on 8192-cell lines exceed the stable range of every set here. The graph of each context is
    replayed once untimed on the initial state (the warm-up), the state is reset, and the graph
    is replayed once timed."""
    import numpy as np
    import torch

    import paper_2401_11086_gb300 as P
    import synthetic
    from paper_2401_11086_gb300 import shocks
    from paper_2401_11086_gb300.autotune import tuned_schedule

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    machs, lengths = synthetic.batched_shocks(seed=synthetic.SEED + rank, ma_range=(1.2, 7.0))
    stream = torch.cuda.current_stream()
    K = args.steps
    runs = []
    for name, sel, prec in (("D3Q729", machs <= 5.0, "f32"), ("D3Q4913", machs > 5.0, "f64")):
        if not sel.any():
            continue
        d = P.lb_lattice_named(name)
        ctx, f0, _ = shocks.setup_batch(d, 5, machs[sel], lengths[sel], precision=prec, width=10.0,
                                        stream=stream)
        sched = tuned_schedule(ctx, f0, lengths[sel], trial_steps=10, persistent=True)  # as replayed
        init = f0.clone()
        fb = ctx.new_state()
        P.lb_step_graph(ctx, f0, fb, K)          # capture + warm-up replay of K steps
        f0.copy_(init)                           # the timed replay starts from the initial state
        del init
        runs.append({"set": name, "ctx": ctx, "fa": f0, "fb": fb, "q": int(d.q), "dtype": prec,
                     "elem": 4 if prec == "f32" else 8,
                     "cells": int(lengths[sel].sum()), "instances": int(sel.sum()), "schedule": sched,
                     "mach_range": [float(machs[sel].min()), float(machs[sel].max())]})
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for r in runs:
        P.lb_step_graph(r["ctx"], r["fa"], r["fb"], K)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    for r in runs:
        st, flags = P.lb_poll_status(r["ctx"])
        if st != 0:
            raise SystemExit(f"{r['set']}: health word reports status {st} (flags {flags})")
    units = sum(r["cells"] * r["q"] for r in runs) * K
    rate, ms = job_rate(units, ms, dist)
    if rank != 0:
        return
    peak, peak_kind = measured_peak()
    alg_bytes = sum(2.0 * r["q"] * r["elem"] * r["cells"] for r in runs) * K
    achieved = alg_bytes / (ms * 1e-3) / 1e9
    cpu = None
    if not args.no_cpu_baseline:
        rr = oracle_table3_rate(40)
        cpu = {"value": rr["rate"] / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "one Ma = 3 shock of 100 cells (D3Q729, N = 5), 40 FP64 oracle steps"}
    line = {"metric": METRIC, "value": rate / 1e9, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": K, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (D3Q729) / f64 (D3Q4913)", "data": "synthetic",
            "config": {"workload": "batched_shocks_64_ma1.2-7_graph",
                       "instances_per_gpu": int(len(machs)), "cells_per_gpu": int(lengths.sum()),
                       "sets": [{k: r[k] for k in ("set", "dtype", "instances", "cells", "q", "mach_range",
                                                   "schedule")}
                                for r in runs],
                       "hermite_order": 5, "launch": "one lb_step_graph replay of K steps per set",
                       "l2": "states larger than L2 (no flush inside the replay)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "peak_kind": f"{peak_kind} (copy bandwidth)",
                         "algorithmic_bytes_per_step": alg_bytes / K,
                         "note": "the tensor-product kernels are issue-bound; the fraction says how far "
                                 "from the memory roofline"},
            "cpu_baseline": cpu, "gpu_launches": 2 * len(runs), "clocks": clk}
    print(json.dumps(line), flush=True)


def run_adjoint(args, world: int, rank: int, local: int) -> None:
    """The reverse mode of the step (lb_step_adjoint, Sec. 3's collision and the streaming
    transposed; FP64 adjoint arithmetic on the FP32 forward states of the split precision):
    (1) the adjoint step kernel alone on the 64 batched D3Q103, N = 4 shocks, one launch per
    step, its HBM roofline counting the forward state read in float and the adjoint state read
    and written in double; (2) the differentiable shock (Ma = 5, 1024 cells, D3Q103, N = 4,
    tanh width 10, K steps, a checkpoint every 250): one checkpointed forward run and its
    backward pass through torch.autograd (relaxation_run), timed end to end: the loss is the
    squared distance of the final rho, theta and q_x profiles to a run at the Table 4 times, the
    start every time perturbed by up to +-20 % by seed."""
    import numpy as np
    import torch

    import paper_2401_11086_gb300 as P
    import synthetic
    from paper_2401_11086_gb300 import shocks
    from paper_2401_11086_gb300.autograd import relaxation_run

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    d = P.lb_lattice_named("D3Q103")
    q = int(d.q)
    stream = torch.cuda.current_stream()
    # (1) the adjoint step kernel on the batched shocks
    machs, lengths = batched_instances(rank)
    ctx, f0, params = shocks.setup_batch(d, 4, machs, lengths, precision="f32c64", stream=stream)
    cells = int(sum(lengths))
    gen = torch.Generator(device=f0.device).manual_seed(synthetic.SEED + rank)
    lam = 1e-3 * torch.randn(ctx.state_elems, dtype=torch.float64, device=f0.device, generator=gen)
    lam2 = torch.empty_like(lam)
    dtau = torch.zeros(len(params[0]["taus"]), dtype=torch.float64, device=f0.device)
    for _ in range(args.warmup):
        P.lb_step_adjoint(ctx, f0, lam, lam2, dtau)
        lam, lam2 = lam2, lam
    KA = args.adjoint_steps
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(KA):
        P.lb_step_adjoint(ctx, f0, lam, lam2, dtau)
        lam, lam2 = lam2, lam
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    if P.lb_poll_status(ctx)[0] != 0 or not bool(torch.isfinite(lam).all()):
        raise SystemExit("adjoint steps: health word or non-finite adjoint state")
    kern_ms = ms / KA
    rate, ms = job_rate(cells * q * KA, ms, dist)
    # (2) the differentiable shock, forward and backward, end to end
    K = args.steps
    ctx1, h0, p1 = shocks.setup_batch(d, 4, [5.0], [1024], precision="f32c64", width=10.0, stream=stream)
    P.lb_set_relaxation(ctx1, p1[0]["taus"], True, 1.0, p1[0]["left"], p1[0]["right"])
    taus_ref = np.asarray(p1[0]["taus"], dtype=np.float64)
    with torch.no_grad():
        tgt = relaxation_run(ctx1, torch.tensor(taus_ref), h0, K, checkpoint_every=250).clone()
    tau = torch.tensor(synthetic.perturbed(taus_ref, 0.2, seed=synthetic.SEED + rank), requires_grad=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = relaxation_run(ctx1, tau, h0, K, checkpoint_every=250)
    loss = ((out - tgt) ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    run_ms = (time.perf_counter() - t0) * 1e3
    grad_ok = bool(torch.isfinite(tau.grad).all()) and P.lb_poll_status(ctx1)[0] == 0
    if rank != 0:
        return
    peak, peak_kind = measured_peak()
    alg_bytes = float(cells) * q * (4 + 8 + 8)
    achieved = alg_bytes / (kern_ms * 1e-3) / 1e9
    line = {"metric": METRIC, "value": rate / 1e9, "unit": UNIT, "n_gpus": world, "steps": KA,
            "warmup": args.warmup, "ms_per_step": ms / KA, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 adjoint of f32 forward states (exact fixed-point sums)",
            "data": "synthetic",
            "config": {"workload": "adjoint_step_batched_shocks_64_d3q103_n4", "instances_per_gpu": len(machs),
                       "cells_per_gpu": cells, "velocities": q, "hermite_order": 4,
                       "schedule": P.lb_get_schedule(ctx),
                       "l2": "inputs larger than L2 (81 MB forward state, two 162 MB adjoint states)",
                       "differentiable_shock": {
                           "workload": "differentiable_shock_ma5_1024_d3q103_n4_f32c64", "steps": K,
                           "checkpoint_every": 250, "ms_forward_and_backward": run_ms,
                           "ms_per_differentiated_step": run_ms / K,
                           "launches": "K forward steps, K - K/250 recomputed, K adjoint steps, one "
                                       "launch each (1024 cells: launch-latency bound)",
                           "gradient_finite": grad_ok}},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": f"{peak_kind} (copy bandwidth)",
                         "algorithmic_bytes_per_launch": alg_bytes, "kernel_ms": kern_ms,
                         "note": "forward state read in float, adjoint state read and written in double"},
            "cpu_baseline": None, "gpu_launches": KA, "clocks": clk}
    print(json.dumps(line), flush=True)


def run_convergence(args, rank: int, local: int) -> None:
    """The Appendix B study: smallest Hermite order of the 1D Maxwellian's expansion with L1
    error below 0.01, on a 200 x 200 grid of theta in [0.1, 2] and u in [0, 4], orders <= 99."""
    import numpy as np
    import torch

    import paper_2401_11086_gb300 as P

    torch.cuda.set_device(local)
    th = np.linspace(0.1, 2.0, 200)
    uu = np.linspace(0.0, 4.0, 200)
    T, U = np.meshgrid(th, uu, indexing="ij")
    t = torch.from_numpy(T.ravel()).cuda()
    u = torch.from_numpy(U.ravel()).cuda()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        P.lb_hermite_convergence(t, u)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        order, err = P.lb_hermite_convergence(t, u)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    npts = t.numel()
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        code = f"""
import json, sys, time
import numpy as np
sys.path.insert(0, {ROOT!r})
from oracle import convergence as CV
pts = [(float(a), float(b)) for a in np.linspace(0.1, 2.0, 5) for b in np.linspace(0.0, 4.0, 4)]
t0 = time.perf_counter()
for th, u in pts:
    CV.min_order(u, th)
print(json.dumps({{"rate": len(pts) / (time.perf_counter() - t0)}}))
"""
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
        r = json.loads(out.stdout.strip().splitlines()[-1])
        cpu = {"value": r["rate"], "unit": "points/s", "cores": 1, "kind": "oracle",
               "sample": "20 (theta, u) points of the same axes (5 x 4), orders <= 99, exact coefficients"}
    if rank != 0:
        return
    o = order.cpu().numpy()
    line = {"metric": "Appendix B convergence study throughput", "value": npts / (ms * 1e-3), "unit": "points/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "hermite_convergence_200x200", "points": npts, "nmax": 99, "tol": 0.01,
                       "quadrature": "Simpson, 4097 points", "orders_min_max": [int(o.min()), int(o.max())],
                       "not_reached": int((o == 100).sum()),
                       "l2": "inputs and outputs of a few hundred KB; the work is arithmetic"},
            "roofline": {"bound": "alu", "note": "FP64 arithmetic on the recurrences and the Simpson sums",
                         "achieved": None, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s (fp64)", "frac": None,
                         "traffic": None},
            "cpu_baseline": cpu, "gpu_launches": args.steps, "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--e2e-steps", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="box workload: skip the other workloads' runs reported under 'secondary'")
    ap.add_argument("--workload", default="box",
                    choices=["box", "batched", "table3", "convergence", "mixed_mach", "adjoint"],
                    help="box: the 256^3 roofline case (default); batched: 64 1D shocks on "
                         "D3Q103; table3: 512 Table 3 shocks on D3Q729, N = 5; convergence: the "
                         "Appendix B study; adjoint: the adjoint step on the batched shocks and the "
                         "differentiable shock; mixed_mach: 64 shocks with Ma in [1.2, 7] on D3Q729 / "
                         "D3Q4913, K steps in one graph-captured persistent launch per set")
    ap.add_argument("--es-b", type=float, default=None,
                    help="table3 workload: run the ES-BGK model with this b instead of SMRT")
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"],
                    help="table3 workload only")
    ap.add_argument("--instances", type=int, default=512, help="table3 workload: number of shocks")
    ap.add_argument("--lattice", default="D3Q729", choices=["D3Q729", "D3Q4913"],
                    help="table3 workload: the D3Q729 rows (Ma 1.5/3/5) or the D3Q4913 row (Ma 7)")
    ap.add_argument("--tensor-cores", action="store_true",
                    help="table3 workload, f32: the projection's x-row sums on the tensor cores")
    ap.add_argument("--adjoint-steps", type=int, default=200,
                    help="adjoint workload: timed adjoint steps on the batched shocks")
    ap.add_argument("--tile-width", type=int, default=0,
                    help="table3 workload: block tile width (32, 64, 128; 0: the library's default)")
    ap.add_argument("--length", type=int, default=0,
                    help="table3 workload: cells per shock (0: 100..400 by seed)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "ours" and args.workload == "batched":
        run_batched(args, world, rank, local)
        return
    if args.impl == "ours" and args.workload == "table3":
        run_table3(args, world, rank, local)
        return
    if args.impl == "ours" and args.workload == "adjoint":
        run_adjoint(args, world, rank, local)
        return
    if args.impl == "ours" and args.workload == "mixed_mach":
        run_mixed_mach(args, world, rank, local)
        return
    if args.impl == "ours" and args.workload == "convergence":
        run_convergence(args, rank, local)
        return
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import numpy as np
    import torch

    import paper_2401_11086_gb300 as P
    import synthetic

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    n = args.n
    d = P.lb_lattice_named("D3Q39")
    stream = torch.cuda.current_stream()
    ctx = P.lb_init_lattice(P.LatticeDesc(d.e, d.w, d.c, d.degree), n, n, n, N=N_ORDER,
                            precision="f32", stream=stream)
    tau20 = 2.0 * d.c
    P.lb_set_relaxation(ctx, [r * tau20 for r in tau_table()], True, 1.0)
    rho, u, th = synthetic.taylor_green(n)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()  # noqa: E731
    fa, fb = ctx.new_state(), ctx.new_state()
    P.lb_fill_equilibrium(ctx, fa, dev(rho.ravel()), dev(u.reshape(3, -1)), dev(th.ravel()))
    del rho, u, th
    torch.cuda.synchronize()

    cur, other = fa, fb
    for _ in range(args.warmup):
        cur = P.lb_step(ctx, cur, other, 1)
        other = fa if cur is fb else fb
    torch.cuda.synchronize()
    if dist:
        dist.barrier()

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    t_start.record(stream)
    for k in range(K):
        ev[k][0].record(stream)
        cur = P.lb_step(ctx, cur, other, 1)
        ev[k][1].record(stream)
        other = fa if cur is fb else fb
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    kern_ms = sum(a.elapsed_time(b) for a, b in ev) / K
    st, flags = P.lb_poll_status(ctx)
    if st != 0:
        raise SystemExit(f"health word reports status {st} (flags {flags})")

    cells = n ** 3
    rate, total_ms = job_rate(cells * Q * K, total_ms, dist)
    value = rate / 1e9

    # end to end through the public API with host buffers: every step copies its state in from
    # pinned host memory, steps once, and copies the new state back. Steps are independent
    # batches, pipelined as a user streaming them would: two device state pairs, the copy in on
    # one stream, the step on the context's stream, the copy out on a third, so that one step's
    # copy in runs while the previous one's copy out does (the host link is full duplex).
    state_bytes = ctx.state_elems * 4
    E = args.e2e_steps
    host_in = [torch.empty(ctx.state_elems, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    host_out = [torch.empty(ctx.state_elems, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    for h in host_in:
        h.copy_(cur)
    # a context of its own on a non-default stream: work on the legacy default stream would
    # serialise with the copy streams
    s_comp, s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ctx_e = P.lb_init_lattice(P.LatticeDesc(d.e, d.w, d.c, d.degree), n, n, n, N=N_ORDER,
                              precision="f32", stream=s_comp)
    P.lb_set_relaxation(ctx_e, [r * tau20 for r in tau_table()], True, 1.0)
    dev_in, dev_out = [fa, ctx_e.new_state()], [fb, ctx_e.new_state()]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_step = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def pipeline(nsteps):
        for k in range(nsteps):
            b = k & 1
            if k >= 2:
                s_in.wait_event(ev_step[b])        # the step two back has read dev_in[b]
            with torch.cuda.stream(s_in):
                dev_in[b].copy_(host_in[b], non_blocking=True)
            ev_in[b].record(s_in)
            s_comp.wait_event(ev_in[b])
            if k >= 2:
                s_comp.wait_event(ev_out[b])       # the copy out two back has read dev_out[b]
            res = P.lb_step(ctx_e, dev_in[b], dev_out[b], 1)
            ev_step[b].record(s_comp)
            s_out.wait_event(ev_step[b])
            with torch.cuda.stream(s_out):
                host_out[b].copy_(res, non_blocking=True)
            ev_out[b].record(s_out)
        s_comp.wait_event(ev_out[(nsteps - 1) & 1])
        if nsteps > 1:
            s_comp.wait_event(ev_out[nsteps & 1])

    pipeline(E)                                 # untimed: the first passes over fresh pinned pages
    torch.cuda.synchronize()
    e0.record(s_comp)
    s_in.wait_event(e0)
    s_out.wait_event(e0)
    pipeline(E)
    e1.record(s_comp)
    torch.cuda.synchronize()
    st_e, flags_e = P.lb_poll_status(ctx_e)
    if st_e != 0:
        raise SystemExit(f"end-to-end run: health word reports status {st_e} (flags {flags_e})")
    ctx_e.close()
    e2e_ms = e0.elapsed_time(e1) / E
    e2e_value = world * cells * Q / (e2e_ms * 1e-3) / 1e9

    peak, peak_kind = measured_peak()
    alg_bytes = 2.0 * Q * 4 * cells
    achieved = alg_bytes / (kern_ms * 1e-3) / 1e9
    traffic = profile_traffic(n)

    if rank != 0:
        ctx.close()
        return
    secondary = None
    if world == 1 and not args.no_secondary:
        ctx.close()                              # the children get the GPU's memory
        del cur, other, fa, fb, dev_in, dev_out, host_in, host_out
        torch.cuda.empty_cache()
        secondary = [run_secondary(a) for a in SECONDARY_WORKLOADS]
    cpu = None
    if not args.no_cpu_baseline:
        r = oracle_sample_rate(32, 20)
        ra = oracle_sample_rate_all_cores(24, 10)
        cpu = {"value": r["rate"] / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "32^3 corner block of the 256^3 Taylor-Green box stepped as its own "
                         "periodic box, 20 FP64 oracle steps, single-threaded BLAS",
               "all_cores": {"value": ra["rate"] / 1e9, "unit": UNIT, "cores": ra["cores"],
                             "sample": "one 24^3 corner block, 10 oracle steps, per host core, "
                                       "all at once (independent samples, one BLAS thread each)"}}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"box{n}_d3q39_n3_f32", "cells": cells, "velocities": Q,
                   "hermite_order": N_ORDER, "init": "Taylor-Green A=0.05, rho noise 1e-3",
                   "l2": "inputs larger than L2 (two 2.6 GB state buffers)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": f"{peak_kind} (copy bandwidth)",
                     "algorithmic_bytes_per_launch": alg_bytes, "kernel_ms": kern_ms},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes, "steps": E,
                "pipeline": "independent steps, double-buffered: copy in, step and copy out on "
                            "three streams"},
        "gpu_launches": K,
        "clocks": clk,
    }
    if secondary is not None:
        line["secondary"] = secondary
    print(json.dumps(line), flush=True)
    if secondary is None:
        ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
