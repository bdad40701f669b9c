"""The N > 1 path of bench.py on CPU: world-size-2 process groups over gloo
(one process per rank, as torchrun launches them).  The factorization does
not shard, so N GPUs run N independent replicas; what is shared is the
host-side protocol: distinct problems per rank, the slowest rank's step time
(an all-reduce MAX), and the whole-job value."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, times, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], world, dist, "cpu")
        seeds = bench.replica_seeds(bench.SIZES["full"], rank)
        out.put((rank, t, seeds, bench.job_value(t, world)))
    finally:
        dist.destroy_process_group()


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_take_the_slowest_step_and_distinct_replicas():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    times = [1.25, 2.5]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(out.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [2.5, 2.5]               # max over ranks on every rank
    assert res[0][2] != res[1][2]                           # independent problems per replica
    assert res[0][3] == pytest.approx(2.5 / 2)              # whole-job seconds per factorization


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1, None, "cpu") == 3.0
    assert bench.replica_seeds(bench.SIZES["full"], 0) == (301, 302)
    assert bench.job_value(3.0, 1) == 3.0


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    """`bench.py --impl reference` launched as the N > 1 driver launches it:
    rank 0 times the oracle on the host and prints the one JSON line, the
    other rank exits 0 without work; no GPU and no process group needed."""
    import json
    import subprocess
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(s) for s in r.stdout.splitlines() if s.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["steps"] == 1
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["higher_is_better"] is False
