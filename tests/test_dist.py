"""Multi-process host logic of multi-GPU runs, on CPU with gloo ranks."""
import os
import socket

import numpy as np
import pytest

from paper_2602_21911_gb300 import dist as D
from paper_2602_21911_gb300 import inputs as I


def test_lpt_partition_is_a_balanced_partition():
    n = I.batched_params(4096, 2602)["n"]
    for world in (1, 2, 3, 8):
        parts = D.lpt_partition(n, world)
        allp = np.concatenate(parts)
        assert sorted(allp.tolist()) == list(range(len(n)))
        loads = [int(n[p].sum()) for p in parts]
        assert max(loads) - min(loads) <= int(n.max())


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = I.batched_params(512, 2602)["n"]
    mine = D.lpt_partition(n, world)[rank]
    ms, upd = D.reduce_time_and_work(10.0 + rank, float(n[mine].sum()))
    out.put((rank, ms, upd, mine.tolist()))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_work():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    n = I.batched_params(512, 2602)["n"]
    for rank, ms, upd, mine in res:
        assert ms == 11.0                           # max over ranks
        assert upd == float(n.sum())                # every domain counted once
    assert set(res[0][3]).isdisjoint(res[1][3])
