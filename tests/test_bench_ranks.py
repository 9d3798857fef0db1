"""bench.py's multi-process path on CPU (gloo, world size 2): the barrier and the max over
ranks that its timings use, and the reference arm launched with torchrun, where rank 0
alone runs the oracle sample and prints the one JSON line and the other rank exits."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup("gloo")
    bench.barrier(w)
    v = bench.allmax(w, 1.5 * (r + 1), "cpu")
    with open(os.path.join(out_dir, f"rank{r}.txt"), "w") as f:
        f.write(f"{w} {r} {v}")
    dist.destroy_process_group()


def test_allmax_over_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(2)]
    assert [g[:2] for g in got] == [["2", "0"], ["2", "1"]]
    assert [float(g[2]) for g in got] == [3.0, 3.0]   # max of 1.5 and 3.0 on both ranks


def test_allmax_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.allmax(1, 2.5, "cpu") == 2.5


@pytest.mark.timeout(600)
def test_reference_arm_two_ranks_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--cpu-slices", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=580)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
