"""The N > 1 path of the benchmark on CPU: world size 2 over gloo.

The solver has no exchange step, so several GPUs run independent replicas; what the
multi-rank path must get right is the whole-job aggregate -- the work of all ranks over
the slowest rank's time -- and that only rank 0 prints.  Both are checked here with two
gloo processes on 127.0.0.1; no GPU is used.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    rep = bench.Replicas(dist, torch.device("cpu"))
    rep.barrier()
    ms = [10.0, 25.0][rank]           # the slower rank sets the job time
    units = [3.0e9, 5.0e9][rank]      # unequal work, so a sum differs from world * own
    res = {"max": rep.max(ms), "sum": rep.sum(units), "rate": rep.rate(units, ms)}
    rep.barrier()
    out[rank] = res
    dist.destroy_process_group()


def test_replica_aggregates_over_two_gloo_ranks():
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        assert res[r]["max"] == 25.0
        assert res[r]["sum"] == 8.0e9
        assert res[r]["rate"] == pytest.approx(8.0e9 / 25e-3, rel=1e-15)


def test_replicas_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    rep = bench.Replicas(None, torch.device("cpu"))
    rep.barrier()
    assert rep.max(7.5) == 7.5 and rep.sum(2.0) == 2.0
    assert rep.rate(2.0e9, 1000.0) == pytest.approx(2.0e9)


def test_reference_arm_under_torchrun_prints_once():
    """`bench.py --impl reference` launched as two ranks: rank 0 alone times the oracle on a
    small cell and prints one line carrying the reference-arm keys; rank 1 exits 0."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--ncell", "2",
           "--steps", "1", "--warmup", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["n_atoms"] == 64 and d["higher_is_better"] is True
