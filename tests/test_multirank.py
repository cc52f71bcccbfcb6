"""The multi-GPU path of bench.py on the CPU: two gloo ranks on 127.0.0.1.

The step does not shard (one domain per GPU, independent replicas), so the only
cross-rank work is the timing: every rank takes the slowest rank's time, and the
whole-job throughput counts the cells of all ranks.  The reference arm (the oracle) runs
on rank 0 only; the other ranks exit at once with no output."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    seconds = [2.0, 3.5][rank]                      # the slower rank sets the time
    t = bench.max_over_ranks(torch, seconds, ws, device="cpu")
    q.put((rank, t, bench.whole_job_mlups(ws, 1000, 10, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_timing_takes_the_slowest_rank_and_counts_all_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == 3.5
        assert v == pytest.approx(2 * 1000 * 10 / 3.5 / 1e6)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    import torch
    assert bench.max_over_ranks(torch, 1.25, 1) == 1.25


def _reference(rank, ws):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", str(ws),
                           "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env, timeout=300,
                          cwd=ROOT)


def test_reference_arm_runs_on_rank_zero_only():
    r1 = _reference(1, 2)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    r0 = _reference(0, 2)
    assert r0.returncode == 0, r0.stderr
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
