"""Profiling driver: builds one workload and applies an operator a few times.

Meant to run under a profiler (ncu) or alone to print per-phase CUDA-event
times of the FMM matvec:

    python -m paper_2103_16073_gb300.profile --workload 1khz --prec mixed --matvecs 3

Workloads: "1khz" (shoebox 3.0 x 2.4 x 2.0 m, 1 kHz, N = 39,368), "sub"
(same room, N = 3,984), "small" (125 Hz, N = 3,072).
"""
from __future__ import annotations

import argparse
import json

import torch

import paper_2103_16073_gb300 as fb
from paper_2103_16073_gb300 import workloads as W

PRECS = {"mixed": fb.FB_PREC_MIXED_FMM, "fp64": fb.FB_PREC_FP64_FMM, "dense": fb.FB_PREC_FP64_DENSE}
KINDS = {"A": fb.FB_OP_A, "L": fb.FB_OP_L, "M": fb.FB_OP_M, "LP": fb.FB_OP_LP}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="1khz", choices=["1khz", "sub", "small", "high_order"])
    ap.add_argument("--prec", default="mixed", choices=list(PRECS))
    ap.add_argument("--kind", default="A", choices=list(KINDS))
    ap.add_argument("--matvecs", type=int, default=3)
    ap.add_argument("--pmin", type=int, default=12)
    ap.add_argument("--autotune", action="store_true", help="autotune the translation forms first (as bench.py)")
    ap.add_argument("--forms", default="", help="fixed per-level choice, comma-separated ints by level "
                                                "(bit 0 M2L on tensor cores, bit 1 M2M/L2L), e.g. 0,0,0,2,0,1")
    args = ap.parse_args()
    wl = {"1khz": W.cfg_1khz, "sub": W.cfg_1khz_sub, "small": W.cfg_small,
          "high_order": W.cfg_high_order}[args.workload]()
    torch.cuda.set_device(0)
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = None if args.prec == "dense" else fb.fb_tree_build(mesh, 64)
    op = fb.fb_operator_create(mesh, tree, wl.k, KINDS[args.kind], PRECS[args.prec], 6.0, args.pmin)
    if args.autotune and args.prec == "mixed":
        fb.fb_operator_autotune(op, 1)
    if args.forms and args.prec == "mixed":
        fb.fb_operator_set_forms(op, [int(v) for v in args.forms.split(",")])
    x = torch.randn(wl.n, dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    times = []
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("apply")   # ncu --nvtx --nvtx-include apply/
    for _ in range(args.matvecs):
        times.append(fb.fb_operator_apply_timed(op, x, y))
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    n, L, p = fb.fb_operator_info(op)
    print(json.dumps({"workload": wl.name, "n": n, "leaf_level": L, "p": p.tolist(), "phase_ms": times[-1]}))
    fb.fb_operator_destroy(op)
    if tree is not None:
        fb.fb_tree_destroy(tree)
    fb.fb_mesh_destroy(mesh)


if __name__ == "__main__":
    main()
