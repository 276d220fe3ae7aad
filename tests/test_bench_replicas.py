"""Replica (N > 1) path of bench.py on CPU: two gloo ranks with different step times.

Each rank runs an independent CGP instance, so the job's time is the slowest rank's and
its throughput is the steps of all ranks over that time, for the device-timed value and
the end-to-end one alike.  The ranks here are processes with made-up timings; nothing
touches a GPU.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, results):
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        ms, e2e_ms = times[rank]
        out = {"ms_per_step": ms, "value": 1000.0 / ms,
               "e2e": {"value": 1000.0 / e2e_ms, "unit": "steps/s", "ms_per_step": e2e_ms}}
        bench.aggregate_ranks(out, world, "cpu")
        results[rank] = (out["ms_per_step"], out["value"], out["e2e"]["ms_per_step"], out["e2e"]["value"])
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_replica_timing_is_the_slowest_rank(world):
    times = [(2.0 + 0.5 * r, 2.6 - 0.3 * r) for r in range(world)]   # the slowest rank differs per metric
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        results = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, times, results)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        codes = [p.exitcode for p in procs]
        for p in procs:
            if p.is_alive():
                p.kill()
        assert codes == [0] * world, codes
        res = dict(results)
    t_max = max(t for t, _ in times)
    e_max = max(e for _, e in times)
    for r in range(world):
        ms, value, e2e_ms, e2e_value = res[r]
        assert ms == pytest.approx(t_max) and e2e_ms == pytest.approx(e_max)
        assert value == pytest.approx(1000.0 * world / t_max, rel=1e-6)
        assert e2e_value == pytest.approx(1000.0 * world / e_max, rel=1e-6)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm (the CPU oracle) runs on rank 0 alone; the other
    ranks exit 0 without work."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
