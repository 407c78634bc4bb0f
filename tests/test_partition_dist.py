"""Host logic of a sweep sharded over ranks, on CPU: the largest-first
partition of (frequency, source) keys (fb_batch_partition, host only), and
two gloo ranks that each solve their own keys (here with the oracle's dense
solve of a small room), write one result file per key and let rank 0 gather
them after one barrier.  The gathered results must equal a serial solve of
every key, and every key must be solved exactly once."""
import itertools
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

import paper_2103_16073_gb300 as fb


def brute_force_makespan(costs, nranks):
    best = float("inf")
    for assign in itertools.product(range(nranks), repeat=len(costs)):
        load = [0.0] * nranks
        for c, r in zip(costs, assign):
            load[r] += c
        best = min(best, max(load))
    return best


def test_partition_assigns_every_key_once_within_grahams_bound():
    rng = np.random.default_rng(5)
    for nranks in (2, 3):
        for trial in range(4):
            costs = rng.uniform(0.1, 10.0, size=8)
            owner, load = fb.fb_batch_partition(costs, nranks)
            assert owner.shape == (8,) and set(owner.tolist()) <= set(range(nranks))
            for r in range(nranks):
                assert load[r] == pytest.approx(costs[owner == r].sum())
            opt = brute_force_makespan(costs.tolist(), nranks)
            assert max(load) <= 4.0 / 3.0 * opt + 1e-12


def test_partition_largest_first_example_and_errors():
    # 2 ranks; by cost 7 -> r0, 5 -> r1, 4 -> r1 (5 < 7), 3 -> r0 (7 < 9), 1 -> r1 (9 < 10): loads 10, 10
    owner, load = fb.fb_batch_partition([3.0, 7.0, 1.0, 5.0, 4.0], 2)
    assert owner.tolist() == [0, 0, 1, 1, 1]
    assert load.tolist() == [10.0, 10.0]
    owner, load = fb.fb_batch_partition([], 3)
    assert owner.size == 0 and load.tolist() == [0.0, 0.0, 0.0]
    with pytest.raises(fb.FBError):
        fb.fb_batch_partition([1.0, -1.0], 2)
    with pytest.raises(fb.FBError):
        fb.fb_batch_partition([1.0], 0)


ROOM = (1.0, 0.8, 0.6)
FREQS = (150.0, 250.0, 350.0)


def small_problem():
    from paper_2103_16073_gb300 import workloads as W
    verts, tris, wall = W.shoebox_mesh(*ROOM, 4, 3, 3)
    beta = np.asarray([0.1, 0.3, 0.2, 0.25, 0.15, 0.05], dtype=np.complex128)[wall]
    rng = W.seeded_rng(70)
    srcs = W.uniform_points_in_box(rng, [0, 0, 0], list(ROOM), 2, 0.2)
    rcv = W.uniform_points_in_box(rng, [0, 0, 0], list(ROOM), 4, 0.2, avoid=srcs, avoid_dist=0.1)
    return verts, tris, beta, srcs, rcv


def solve_key(problem, key):
    """Oracle dense solve of Eq. (dbem4) for one (frequency, source) key and
    its field at the receivers (Eq. dbem1)."""
    from oracle import bem
    from paper_2103_16073_gb300 import workloads as W
    verts, tris, beta, srcs, rcv = problem
    fi, si = key
    k = W.wavenumber(FREQS[fi])
    m = bem.Mesh(verts, tris)
    L, M, _ = bem.dense_operators(m, k)
    A = bem.system_matrix(L, M, k, beta)
    g = bem.gamma_monopole(m, k, beta, srcs[si])
    psi = np.linalg.solve(A, L @ g)
    field = bem.receiver_field(m, k, beta, psi, g, rcv, xs=srcs[si])
    return psi, field


def _worker(rank, world, port, out_dir, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_2103_16073_gb300 import distributed as Dd
    from paper_2103_16073_gb300 import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    problem = small_problem()
    keys = [(fi, si) for fi in range(len(FREQS)) for si in range(2)]
    n = problem[1].shape[0]
    diam = float(np.linalg.norm(ROOM))
    costs = [Dd.predicted_cost(n, W.wavenumber(FREQS[fi]), diam) for fi, _ in keys]
    owner, load = Dd.partition(costs, world)
    mine = Dd.rank_keys(owner, rank)
    for i in mine:
        psi, field = solve_key(problem, keys[i])
        Dd.write_result(out_dir, keys[i], psi=psi, field=field, rank=np.array(rank))
    dist.barrier()        # the only synchronisation: every rank's files are written
    if rank == 0:
        got = Dd.gather(out_dir, keys)
        out["gathered"] = {k: (v["psi"], v["field"], int(v["rank"])) for k, v in got.items()}
    out[f"mine{rank}"] = [keys[i] for i in mine]
    out[f"owner{rank}"] = owner
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo_sweep(tmp_path):
    port = 29600 + (os.getpid() % 1000)
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, str(tmp_path), out), nprocs=2, join=True)
        res = dict(out)
    keys = [(fi, si) for fi in range(len(FREQS)) for si in range(2)]
    assert res["owner0"] == res["owner1"]                     # every rank computes the same partition
    mine = res["mine0"] + res["mine1"]
    assert sorted(mine) == sorted(keys)                       # every key solved exactly once
    assert res["mine0"] and res["mine1"]                      # both ranks work
    problem = small_problem()
    for key in keys:
        psi, field, r = res["gathered"][key]
        assert key in (res["mine0"] if r == 0 else res["mine1"])
        ref_psi, ref_field = solve_key(problem, key)
        assert np.allclose(psi, ref_psi, rtol=0, atol=1e-12 * np.abs(ref_psi).max())
        assert np.allclose(field, ref_field, rtol=0, atol=1e-12 * np.abs(ref_field).max())
