"""The benchmark's multi-rank path (replicas: every rank steps its own scene,
the job's time is the slowest rank's): max over ranks and the aggregate
ms/step, run as two gloo ranks on the CPU."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    local = 10.0 + 5.0 * rank  # the ranks' own timed totals (ms)
    t = b.max_over_ranks(local, world, torch.device("cpu"))
    out[rank] = (t, b.aggregate_ms_per_step(t, 4, world))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_and_aggregate():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(2):
            t, ms = out[r]
            assert t == 15.0
            assert ms == 15.0 / (4 * 2)


def test_single_rank_is_unchanged():
    b = _bench()
    assert b.max_over_ranks(12.5, 1, None) == 12.5
    assert b.aggregate_ms_per_step(100.0, 10, 1) == 10.0
