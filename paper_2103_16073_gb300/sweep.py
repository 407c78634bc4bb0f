"""Frequency sweep through the batch scheduler (fb_batch_solve): the L-shaped
room at log-spaced frequencies, each meshed at lambda/8 (uneven N), several
interior sources per frequency, all solved to a true relative residual by
the lockstep batched FGMRES.  Mesh and octree setup stays with the caller
(here); operators, preconditioner, autotuning and solves run in the library.

Under torchrun the frequencies are sharded over the ranks (one GPU each):
the library's largest-first partition on the predicted cost N x (kD)^(1/2)
x sources, no exchange while solving, one result file per (frequency,
source) key with the field at seeded receivers (Eq. dbem1), and rank 0
gathers the files after one barrier.

    python -m paper_2103_16073_gb300.sweep --nfreq 16 --fhi 600 --nsrc 8
    torchrun --nproc-per-node N -m paper_2103_16073_gb300.sweep --out-dir DIR ...
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import torch

import paper_2103_16073_gb300 as fb
from paper_2103_16073_gb300 import distributed as D
from paper_2103_16073_gb300 import workloads as W

LROOM_DIAMETER = float(np.linalg.norm([8.0, 4.0, 3.0]))


def sweep_receivers(n=16, seed=71):
    """Seeded receivers inside the L-room, >= 0.3 m from every wall."""
    rng = W.seeded_rng(seed)
    out = []
    while len(out) < n:
        p = np.array([8.0, 4.0, 3.0]) * rng.random(3)
        if W.lroom_inside(p, 0.3)[0]:
            out.append(p)
    return np.asarray(out)


def run(nfreq, f_lo, f_hi, nsrc, tol=1e-4, max_rhs=8, autotune=True, lookahead=True, rank=0, world=1,
        out_dir=None, inner_iters=0):
    wls = W.lroom_sweep(nfreq=nfreq, f_lo=f_lo, f_hi=f_hi, nsrc=nsrc)
    costs = [D.predicted_cost(wl.n, wl.k, LROOM_DIAMETER, nsrc) for wl in wls]
    owner, load = D.partition(costs, world)
    mine = D.rank_keys(owner, rank)
    rcv = sweep_receivers()
    t0 = time.perf_counter()
    built = []
    for i in mine:
        wl = wls[i]
        mesh = fb.fb_mesh_create(wl.verts, wl.tris)
        fb.fb_mesh_set_admittance(mesh, wl.beta)
        tree = fb.fb_tree_build(mesh, 64)
        x = torch.zeros((nsrc, wl.n), dtype=torch.complex128, device="cuda")
        built.append(dict(mesh=mesh, tree=tree, k=wl.k, src=wl.sources, x=x))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    res = fb.fb_batch_solve(built, tol=tol, max_rhs=max_rhs, autotune=autotune, lookahead=lookahead,
                            inner_iters=inner_iters)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    if out_dir:
        rd = torch.tensor(rcv, device="cuda")
        field = torch.empty(rcv.shape[0], dtype=torch.complex128, device="cuda")
        g = None
        for i, b, r in zip(mine, built, res):
            wl = wls[i]
            g = torch.empty(wl.n, dtype=torch.complex128, device="cuda")
            for si in range(nsrc):
                fb.fb_gamma_monopole(b["mesh"], wl.k, wl.sources[si], g)
                fb.fb_eval_field(b["mesh"], wl.k, b["x"][si], g, rd, field, src=wl.sources[si])
                D.write_result(out_dir, (i, si), field=field.cpu().numpy(), f_hz=np.array(wl.freq_hz),
                               n=np.array(wl.n), iters=np.array(r["infos"][si]["iters"]),
                               true_relres=np.array(r["infos"][si]["true_relres"]), rank=np.array(rank))
    out = {"workload": f"L-room sweep {nfreq} freqs {f_lo:g}-{f_hi:g} Hz, lambda/8, {nsrc} sources each",
           "preconditioner": (f"inner-outer, {inner_iters} GMRES steps on a low-accuracy FMM" if inner_iters
                              else "block Jacobi"),
           "rank": rank, "ranks": world, "predicted_load": load,
           "n_elements": [wls[i].n for i in mine], "mesh_tree_s": round(t1 - t0, 3), "batch_s": round(t2 - t1, 3),
           "solves": len(mine) * nsrc, "solves_per_s": round(len(mine) * nsrc / max(t2 - t1, 1e-9), 3),
           "jobs": [{"f_hz": round(wls[i].freq_hz, 1), "n": wls[i].n, "order": r["order"], "status": r["status"],
                     "setup_ms": round(r["setup_ms"], 1), "solve_ms": round(r["solve_ms"], 1),
                     "iters": [q["iters"] for q in r["infos"]],
                     "max_true_relres": max(q["true_relres"] for q in r["infos"])} for i, r in zip(mine, res)]}
    for b in built:
        fb.fb_tree_destroy(b["tree"])
        fb.fb_mesh_destroy(b["mesh"])
    return out, built, [wls[i] for i in mine]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nfreq", type=int, default=16)
    ap.add_argument("--flo", type=float, default=100.0)
    ap.add_argument("--fhi", type=float, default=600.0)
    ap.add_argument("--nsrc", type=int, default=8)
    ap.add_argument("--max-rhs", type=int, default=8)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-lookahead", action="store_true")
    ap.add_argument("--out-dir", default="", help="one result file per (frequency, source) key")
    ap.add_argument("--inner", type=int, default=0, help="inner-outer preconditioner with this many inner steps")
    a = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if world > 1 and not a.out_dir:
        raise SystemExit("--out-dir is required with several ranks (a directory every rank writes to)")
    out_dir = a.out_dir
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    t0 = time.perf_counter()
    out, _, _ = run(a.nfreq, a.flo, a.fhi, a.nsrc, max_rhs=a.max_rhs, autotune=not a.no_autotune,
                    lookahead=not a.no_lookahead, rank=rank, world=world, out_dir=out_dir, inner_iters=a.inner)
    if world > 1:
        dist.barrier()   # every rank's result files are written
    if rank == 0:
        if out_dir:
            keys = [(i, si) for i in range(a.nfreq) for si in range(a.nsrc)]
            got = D.gather(out_dir, keys)
            out["gathered_keys"] = len(got)
            out["wall_s"] = round(time.perf_counter() - t0, 3)
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
