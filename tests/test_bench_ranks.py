"""The N > 1 form of bench.py on CPU: two gloo ranks, as torchrun would launch them.

The path is not sharded; every rank advances its own box (replicas). What N > 1 adds is host
logic: the timed region's max over ranks, the whole-job rate, and the reference arm's rule that
only rank 0 runs. That is checked here without a GPU.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 20.0][rank]  # rank 1 is the slow one
    t = bench.max_over_ranks(ms, dist, torch.device("cpu"))
    rate = bench.whole_job_rate(1000, world, t)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t, rate))


def test_replica_aggregation_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate in res:
        assert t == 20.0  # every rank sees the slowest rank's time
        assert rate == pytest.approx(2 * 1000 / 0.020)  # all ranks' units over that time


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(7.0, None, None) == 7.0
    assert bench.whole_job_rate(500, 1, 250.0) == pytest.approx(2000.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_bench_module_names_resolve():
    """Every global name a function of bench.py loads is defined in the module or a builtin (the
    GPU legs cannot run here, so a missing helper would surface only on the GPU machine)."""
    import builtins
    import dis
    import types

    sys.path.insert(0, ROOT)
    import bench

    def globals_used(code):
        for ins in dis.get_instructions(code):
            if ins.opname in ("LOAD_GLOBAL", "LOAD_NAME"):
                yield ins.argval
        for c in code.co_consts:
            if isinstance(c, types.CodeType):
                yield from globals_used(c)

    src = open(os.path.join(ROOT, "bench.py")).read()
    missing = sorted({n for n in globals_used(compile(src, "bench.py", "exec"))
                      if not hasattr(bench, n) and not hasattr(builtins, n)})
    assert not missing, missing
