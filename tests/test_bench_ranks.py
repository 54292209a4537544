"""The multi-process path of bench.py on CPU: ranks as torchrun launches them
(one process each, rendezvous on 127.0.0.1), over the gloo backend.  The
whole-job rate is the units of all ranks over the slowest rank's time, and
every rank computes the same figure; the reference arm runs on rank 0 only."""
import os
import socket
import types

import pytest

import bench


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, seconds, units, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = bench.job_rate(dist, seconds[rank], units[rank], "cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()
    q.put((rank, out))


def _run_ranks(seconds, units):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = len(seconds)
    procs = [ctx.Process(target=_worker, args=(r, world, port, seconds, units, q))
             for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = dict(q.get(timeout=120) for _ in range(world))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    return res


def test_job_rate_single_process():
    assert bench.job_rate(None, 2.0, 4000) == (2.0, 4000.0, 2000.0)


@pytest.mark.parametrize("seconds,units", [((0.5, 2.0), (1000, 3000)),
                                           ((3.0, 1.5), (2000, 2000))])
def test_job_rate_two_gloo_ranks(seconds, units):
    res = _run_ranks(seconds, units)
    want = (max(seconds), float(sum(units)), sum(units) / max(seconds))
    for r in range(len(seconds)):
        assert res[r] == pytest.approx(want, rel=1e-15)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    # a rank other than 0 returns before building or timing the oracle
    monkeypatch.setenv("RANK", "1")
    args = types.SimpleNamespace(gpus=2, steps=1, warmup=3)
    assert bench.run_reference(args) is None
