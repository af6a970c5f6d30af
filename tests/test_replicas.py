"""The multi-GPU path is replicas (independent solves per rank, no data-path
collective); its host logic, the rank environment and the whole-job timing
reduction, runs here as two gloo processes on the CPU."""
import socket

import pytest

from paper_1706_00692_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, units, seconds, q):
    import os
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, replicas.dist_env(), replicas.job_throughput(units[rank], seconds[rank])))
    finally:
        dist.destroy_process_group()


def test_two_rank_throughput_is_units_over_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    units, seconds = [56.0, 112.0], [1.5, 2.0]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, units, seconds, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict((r, (env, res)) for r, env, res in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        env, (u, s, v) = out[r]
        assert env == (r, 2, r)
        assert (u, s) == (168.0, 2.0)  # every rank's units over the slowest rank's time
        assert v == pytest.approx(84.0)


def test_single_process_and_bad_environment(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert replicas.dist_env() == (0, 1, 0)
    assert replicas.job_throughput(10, 2.0) == (10.0, 2.0, 5.0)
    monkeypatch.setenv("RANK", "3")
    monkeypatch.setenv("WORLD_SIZE", "2")
    with pytest.raises(ValueError):
        replicas.dist_env()
