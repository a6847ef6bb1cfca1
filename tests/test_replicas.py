"""Host logic of the replica runs on CPU: two gloo ranks (world size 2) agree
on the maximum of their timings; a single process needs no group."""
import multiprocessing as mp
import os
import socket

import pytest

from paper_2505_00384_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, values, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank),
                      LOCAL_RANK=str(rank))
    pg = replicas.init("gloo")
    replicas.barrier(pg)
    m = replicas.max_over_ranks(pg, values[rank])
    replicas.barrier(pg)
    q.put((rank, m, replicas.env()))
    pg.destroy_process_group()


def test_max_over_two_gloo_ranks():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    values = [1.25, 3.5]
    procs = [ctx.Process(target=_rank, args=(r, port, values, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [3.5, 3.5]
    assert [o[2] for o in out] == [(2, 0, 0), (2, 1, 1)]


def test_single_process_has_no_group(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert replicas.init("gloo") is None
    assert replicas.max_over_ranks(None, 2.5) == 2.5
