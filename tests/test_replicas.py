"""The N > 1 path of bench.py (one replica per rank, no data-path collective)
on the CPU with the gloo backend, world size 2: the job's time is the
slowest rank's, every rank gets it, and each replica solves its own seeded
problem."""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    worst = bench.max_over_ranks(10.0 * rank + 1.5, world)
    dist.barrier()
    pr, c = bench.make_problem("c1", bench.replica_seed(7, rank))
    digest = float(np.abs(pr.X[:, :3]).sum())
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump({"worst": worst, "digest": digest, "c": c, "shape": list(pr.X.shape)}, f)
    dist.destroy_process_group()


def test_two_gloo_replicas(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(2)]
    assert r[0]["worst"] == r[1]["worst"] == 11.5
    assert r[0]["shape"] == r[1]["shape"] == [500, 500] and r[0]["c"] == r[1]["c"] == 25
    assert r[0]["digest"] != r[1]["digest"]          # different problems per replica


def test_single_rank_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.replica_seed(5, 0) == 5 and bench.replica_seed(5, 3) == 8


@pytest.mark.parametrize("workload", ["c4", "c5", "spectral"])
def test_reference_arm_without_oracle_workload_says_unavailable(workload):
    """bench.py --impl reference prints one JSON line with an `unavailable`
    reason (and exits 0) for the workloads that have no oracle arm."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--workload", workload], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unavailable"]
