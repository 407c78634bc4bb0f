"""Host logic of bench.py's multi-GPU path on CPU: two gloo ranks, each with
its own source position, and the job time taken as the maximum over ranks
(no data-path collective: the solves are independent)."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    from paper_2103_16073_gb300 import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    wl = W.cfg_small()
    src = bench.rank_source(W, wl, r)
    t = bench.reduce_max_ms(10.0 * (r + 1), dist, "cpu")
    out[rank] = (ws, r, tuple(np.round(src, 12)), t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    port = 29500 + (os.getpid() % 1000)
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == 2 and res[1][0] == 2
    assert res[0][1] == 0 and res[1][1] == 1
    assert res[0][2] != res[1][2]              # independent source positions
    assert res[0][3] == res[1][3] == 20.0      # max over ranks
    from paper_2103_16073_gb300 import workloads as W
    inside = np.array(res[1][2])
    assert np.all(inside > 0.25) and np.all(inside < np.array(W.cfg_small().room) - 0.25)
