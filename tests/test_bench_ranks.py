"""The multi-rank logic of bench.py on CPU (gloo, world size 2): each rank
fits an independent batch (own seed), the job time is the max over ranks and
the particle count the sum."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.rank_info()
    t = bench.reduce_max(1.5 + rank, dist)
    n = bench.reduce_sum(100.0 * (rank + 1), dist)
    wl = bench.make_workload("two_stream_1d1v", r)
    out[rank] = (r, w, lr, t, n, bench.rank_seed(r), float(wl.v[0, :8].sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][:3] == (0, 2, 0) and res[1][:3] == (1, 2, 1)
    assert res[0][3] == res[1][3] == 2.5          # max over ranks
    assert res[0][4] == res[1][4] == 300.0        # sum over ranks
    assert res[0][5] != res[1][5]                 # independent batches
    assert res[0][6] != res[1][6]
