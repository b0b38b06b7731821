"""The N > 1 path of bench.py on CPU: two gloo ranks (no GPU). Each rank owns its own batched
shocks (independent instances, no exchange), and the whole-job rate is all ranks' updates
divided by the slowest rank's time."""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    machs, lengths = bench.batched_instances(rank)
    # rank r pretends to have processed (r + 1) * 100 units in 10 (r + 1) ms
    rate, ms = bench.job_rate((rank + 1) * 100.0, 10.0 * (rank + 1), dist, device="cpu")
    dist.barrier()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
        json.dump({"machs": list(map(float, machs)), "lengths": list(map(int, lengths)),
                   "rate": rate, "ms": ms}, fh)
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    # each rank owns 64 shocks of its own; the sets differ
    assert all(len(r["machs"]) == 64 for r in res)
    assert res[0]["machs"] != res[1]["machs"]
    assert all(1.2 <= m <= 3.0 for r in res for m in r["machs"])
    # whole-job rate: (100 + 200) units over the slowest rank's 20 ms, the same on both ranks
    for r in res:
        assert r["ms"] == 20.0
        assert abs(r["rate"] - 300.0 / 20e-3) < 1e-9


def test_single_process_rate_is_local():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(500.0, 5.0) == (500.0 / 5e-3, 5.0)
