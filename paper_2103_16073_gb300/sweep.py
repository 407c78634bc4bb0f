"""Frequency sweep through the batch scheduler (fb_batch_solve): the L-shaped
room at log-spaced frequencies, each meshed at lambda/8 (uneven N), several
interior sources per frequency, all solved to a true relative residual by
the lockstep batched FGMRES.  Mesh and octree setup stays with the caller
(here); operators, preconditioner, autotuning and solves run in the library.

    python -m paper_2103_16073_gb300.sweep --nfreq 16 --fhi 600 --nsrc 8
"""
from __future__ import annotations

import argparse
import json
import time

import torch

import paper_2103_16073_gb300 as fb
from paper_2103_16073_gb300 import workloads as W


def run(nfreq, f_lo, f_hi, nsrc, tol=1e-4, max_rhs=8, autotune=True, lookahead=True):
    wls = W.lroom_sweep(nfreq=nfreq, f_lo=f_lo, f_hi=f_hi, nsrc=nsrc)
    t0 = time.perf_counter()
    built = []
    for wl in wls:
        mesh = fb.fb_mesh_create(wl.verts, wl.tris)
        fb.fb_mesh_set_admittance(mesh, wl.beta)
        tree = fb.fb_tree_build(mesh, 64)
        x = torch.zeros((nsrc, wl.n), dtype=torch.complex128, device="cuda")
        built.append(dict(mesh=mesh, tree=tree, k=wl.k, src=wl.sources, x=x))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    res = fb.fb_batch_solve(built, tol=tol, max_rhs=max_rhs, autotune=autotune, lookahead=lookahead)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    out = {"workload": f"L-room sweep {nfreq} freqs {f_lo:g}-{f_hi:g} Hz, lambda/8, {nsrc} sources each",
           "n_elements": [wl.n for wl in wls], "mesh_tree_s": round(t1 - t0, 3), "batch_s": round(t2 - t1, 3),
           "solves": nfreq * nsrc, "solves_per_s": round(nfreq * nsrc / (t2 - t1), 3),
           "jobs": [{"f_hz": round(wl.freq_hz, 1), "n": wl.n, "order": r["order"], "status": r["status"],
                     "setup_ms": round(r["setup_ms"], 1), "solve_ms": round(r["solve_ms"], 1),
                     "iters": [i["iters"] for i in r["infos"]],
                     "max_true_relres": max(i["true_relres"] for i in r["infos"])} for wl, r in zip(wls, res)]}
    for b in built:
        fb.fb_tree_destroy(b["tree"])
        fb.fb_mesh_destroy(b["mesh"])
    return out, built, wls


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nfreq", type=int, default=16)
    ap.add_argument("--flo", type=float, default=100.0)
    ap.add_argument("--fhi", type=float, default=600.0)
    ap.add_argument("--nsrc", type=int, default=8)
    ap.add_argument("--max-rhs", type=int, default=8)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-lookahead", action="store_true")
    a = ap.parse_args()
    out, _, _ = run(a.nfreq, a.flo, a.fhi, a.nsrc, max_rhs=a.max_rhs, autotune=not a.no_autotune,
                    lookahead=not a.no_lookahead)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
