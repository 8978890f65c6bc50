"""The N > 1 host path of bench.py on CPU ranks (gloo, world size 2): every
rank sweeps its own seeds, the job time is the slowest rank's and the units
are summed exactly; only rank 0 runs the oracle reference arm."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        times = [10.0 + rank, 1.5 - rank]
        counts = [2**40 + 7 * rank, 3 + rank]
        q.put((rank, bench.reduce_over_ranks(world, times, counts)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_gloo_world_2():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        times, counts = got[r]
        assert times == [11.0, 1.5]
        assert counts == [2 * 2**40 + 7, 7]


def test_single_rank_is_identity():
    assert bench.reduce_over_ranks(1, [2.5], [5]) == ([2.5], [5])


def test_ranks_sweep_disjoint_seeds():
    s0 = {c["seed"] for c in bench.sweep_configs(0, 1000)}
    s1 = {c["seed"] for c in bench.sweep_configs(1, 1000)}
    assert len(s0) == 21 and len(s1) == 21 and not (s0 & s1)
    assert [c["Vd"] for c in bench.sweep_configs(1, 1000)] == [float(v) for v in range(21)]


def test_reference_arm_only_on_rank_0(capsys):
    class A:
        steps, warmup = 1, 3
    assert bench.run_reference(A(), world=2, rank=1) is None
    assert capsys.readouterr().out == ""


def test_reference_arm_under_torchrun_two_ranks(tmp_path):
    """bench.py --impl reference launched as the multi-GPU driver launches it
    (torch.distributed.run, two ranks; gloo here): rank 0 alone prints one
    JSON line, both ranks exit 0."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, EMC_BENCH_BACKEND="gloo", OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", "bench.py", "--impl", "reference",
           "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
