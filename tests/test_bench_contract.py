"""bench.py's host logic on the CPU: the reference arm's JSON line (the oracle timed on the host
cores), the rule that a committed ncu figure is reported only while the kernel sources it was
taken on are unchanged, and the secondary workloads of the default run."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_one_complete_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 3
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_profile_figures_follow_the_kernel_sources(tmp_path):
    p = tmp_path / "summary.txt"
    p.write_text(f"kernel_sources_sha256_12: {bench.kernel_hash()}\ndram_bytes_per_cell: 289.3\n")
    assert bench.profile_value(str(p), "dram_bytes_per_cell") == 289.3
    assert bench.profile_value(str(p), "missing_key") is None
    p.write_text("kernel_sources_sha256_12: 000000000000\ndram_bytes_per_cell: 289.3\n")
    assert bench.profile_value(str(p), "dram_bytes_per_cell") is None
    assert bench.profile_value(str(tmp_path / "absent.txt"), "dram_bytes_per_cell") is None


def test_committed_profiles_match_the_kernel_sources():
    """The box and batched summaries under profiles/ were captured on the kernels as committed,
    so the bench line reports their DRAM traffic (it would print null after a kernel edit)."""
    assert bench.profile_traffic(256) is not None
    assert bench.profile_value(bench.PROFILE_BATCHED, "dram_bytes_per_launch") is not None


def test_secondary_workloads_parse_and_failures_are_reported():
    """Every secondary workload is a valid bench.py command line, and a child that fails is
    reported in the box line instead of ending the run."""
    for extra in bench.SECONDARY_WORKLOADS:
        assert extra[0] == "--workload" and extra[1] in ("batched", "table3", "mixed_mach", "adjoint")
        assert int(extra[extra.index("--steps") + 1]) > 0 and int(extra[extra.index("--warmup") + 1]) >= 3
    out = bench.run_secondary(["--workload", "no_such_workload"], timeout=120)
    assert out["args"] == "--workload no_such_workload" and "error" in out and "value" not in out
