"""Learned-preconditioner comparison on the door-and-baffle room.

Geometry: shoebox 5 x 4 x 3 m, walls of admittance 0.2, a door (0.9 x 2.0 m)
and a 2.0 x 1.5 m baffle of admittance 1.0, legs lambda/10 at 2 kHz
(N = 685,272).  The network is trained on residual/error pairs logged from
plain block-Jacobi FGMRES solves at training frequencies (default 1.6, 1.8,
2.2 and 2.4 kHz) on the same mesh, the parameters passing from one
frequency's operator to the next in blocks of Adam steps, and is then used
at 2 kHz for source positions it has not seen.  Compared there on FGMRES
iterations and time to a true relative residual (FP64 FMM) of 1e-4:
block Jacobi alone, the learned network over block Jacobi, the inner-outer
preconditioner of Sec. 4, and the plain FP64 path.

With --cross-validate it instead solves the same room twice for one
source: the 2 cm baffle box in the direct formulation (Eq. dbem4) and a
zero-thickness baffle sheet in the indirect one (Eq. ibem5, two unknowns per
element, walls and door with the same admittance on both sides), each with
the inner-outer preconditioner (block Jacobi inside: leaf blocks, 2 x 2 for
the indirect system) and an FP64 true residual, and compares the
fields at 64 receivers (Sec. 4 compares its direct and indirect solutions
the same way).

Orchestration only: every solve, matvec, network pass and Adam step runs in
the library.

    python -m paper_2103_16073_gb300.baffle_study [--train-freqs 1600,1800,2200,2400]
        [--train-sources 2] [--eval-sources 3] [--steps 200] [--out result.json]
    python -m paper_2103_16073_gb300.baffle_study --cross-validate [--out result.json]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

import paper_2103_16073_gb300 as fb
from paper_2103_16073_gb300 import training
from paper_2103_16073_gb300 import workloads as W

TOL = 1e-4
RESTART = 40
D0, PMIN = 6.0, 12
INNER = (2.0, 4, 8)   # low-accuracy FMM (d0, p_min) and GMRES steps of the inner-outer preconditioner


def _now():
    torch.cuda.synchronize()
    return time.perf_counter()


def _rhs(mesh, Lop, k, src, n):
    g = torch.empty(n, dtype=torch.complex128, device="cuda")
    fb.fb_gamma_monopole(mesh, k, src, g)
    b = torch.empty_like(g)
    fb.fb_operator_apply(Lop, g, b)
    return b


def _solve(A, b, pc, true_op):
    x = torch.zeros_like(b)
    t0 = _now()
    info = fb.fb_fgmres_solve(A, b, x, pc=pc, tol=TOL, restart=RESTART, maxit=3000, max_refine=4, true_op=true_op)
    info["ms"] = (_now() - t0) * 1e3
    return info


def run(train_freqs, ntrain, neval, steps, every=10, lr=1e-3, batch=8, log=print):
    wl = W.cfg_baffle(nsrc=ntrain + 1 + neval)
    out = {"workload": wl.name, "n": wl.n, "train_freqs_hz": list(train_freqs), "eval_freq_hz": wl.freq_hz}
    t0 = _now()
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = fb.fb_tree_build(mesh, 64)
    handles = []

    def op(k, kind, prec, d0=D0, pmin=PMIN):
        h = fb.fb_operator_create(mesh, tree, k, kind, prec, d0, pmin)
        handles.append(("op", h))
        return h

    def pc_of(A, kind=fb.FB_PC_BLOCK_JACOBI):
        h = fb.fb_precond_create(A, kind)
        handles.append(("pc", h))
        return h

    # ---- training data: truncated block-Jacobi solves at every training frequency
    train = []
    for f in train_freqs:
        k = W.wavenumber(f)
        A = op(k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM)
        fb.fb_operator_autotune(A, 1)
        fb.fb_operator_use_graphs(A, True)
        Lm = fb.fb_operator_create(mesh, tree, k, fb.FB_OP_L, fb.FB_PREC_MIXED_FMM, D0, PMIN)
        bj = pc_of(A)
        Rs, Es = [], []
        for s in range(ntrain):
            R, E = training.collect_pairs(A, bj, _rhs(mesh, Lm, k, wl.sources[s], wl.n))
            Rs.append(R)
            Es.append(E)
        fb.fb_operator_destroy(Lm)
        R = torch.cat(Rs)
        E = torch.cat(Es)
        npairs = int(R.shape[0])
        R, E = training.augment_noise(R, E, npairs, seed=int(f))
        lp = fb.fb_precond_create_learned(A, bj)
        handles.append(("pc", lp))
        fb.fb_learned_set_objective(lp, fb.FB_LOSS_RESIDUAL)
        train.append({"f": f, "A": A, "pc": lp, "R": R, "E": E, "pairs": npairs})
        log(f"pairs at {f:.0f} Hz: {npairs} (+{npairs} noise), {_now() - t0:.1f} s")
    t_collect = _now() - t0

    # ---- operators at the evaluation frequency
    k = wl.k
    A32 = op(k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM)
    tune = fb.fb_operator_autotune(A32, 1)
    A64 = op(k, fb.FB_OP_A, fb.FB_PREC_FP64_FMM)
    L64 = op(k, fb.FB_OP_L, fb.FB_PREC_FP64_FMM)
    for h in (A32, A64):
        fb.fb_operator_use_graphs(h, True)
    bj32 = pc_of(A32)
    bj64 = pc_of(A64)
    Alow = op(k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, INNER[0], INNER[1])
    fb.fb_operator_autotune(Alow, 1)
    fb.fb_operator_use_graphs(Alow, True)
    inner = fb.fb_precond_create_inner(A32, Alow, pc_of(Alow), INNER[2])
    handles.append(("pc", inner))
    learned = fb.fb_precond_create_learned(A32, bj32)
    handles.append(("pc", learned))
    rhs = [_rhs(mesh, L64, k, wl.sources[s], wl.n) for s in range(ntrain, ntrain + 1 + neval)]
    bval, beval = rhs[0], rhs[1:]

    x = torch.zeros_like(bval)
    base_its = fb.fb_fgmres_solve(A32, bval, x, pc=bj32, tol=TOL, restart=RESTART, maxit=3000, max_refine=4)["iters"]
    cap = 2 * base_its   # a candidate that needs more is not kept: stop early

    def validate(params):
        fb.fb_learned_params(learned, params)
        x = torch.zeros_like(bval)
        info = fb.fb_fgmres_solve(A32, bval, x, pc=learned, tol=TOL, restart=RESTART, maxit=cap, max_refine=1)
        return info["iters"] if info["status"] == 0 else cap + 1

    # ---- round-robin Adam over the training frequencies
    t1 = _now()
    g = torch.Generator(device="cpu")
    g.manual_seed(0)
    params = fb.fb_learned_params(train[0]["pc"])
    best = (validate(params), params.copy())
    vlog = [(0, best[0])]
    hist = []
    for blk in range((steps + every - 1) // every):
        tr = train[blk % len(train)]
        fb.fb_learned_params(tr["pc"], params)
        for _ in range(min(every, steps - blk * every)):
            idx = torch.randperm(tr["R"].shape[0], generator=g)[:batch].to(tr["R"].device)
            hist.append(fb.fb_learned_train_step(tr["pc"], tr["R"].index_select(0, idx).contiguous(),
                                                 tr["E"].index_select(0, idx).contiguous(), lr))
        params = fb.fb_learned_params(tr["pc"])
        it = validate(params)
        vlog.append((min(steps, (blk + 1) * every), it))
        if it < best[0]:
            best = (it, params.copy())
        log(f"block {blk} at {tr['f']:.0f} Hz: loss {np.mean(hist[-every:]):.4f}, validation {it} iterations")
    fb.fb_learned_params(learned, best[1])
    t_train = _now() - t1
    out["training"] = {"sources_per_freq": ntrain, "pairs_per_freq": train[0]["pairs"], "noise_inputs": "equal",
                       "objective": "residual", "adam_steps": steps, "batch": batch, "lr": lr,
                       "loss_first": round(float(np.mean(hist[:every])), 5),
                       "loss_last": round(float(np.mean(hist[-every:])), 5), "validation_iterations": vlog,
                       "block_jacobi_validation_iterations": base_its,
                       "selected_iterations": best[0], "collect_s": round(t_collect, 1),
                       "train_s": round(t_train, 1)}

    # ---- evaluation at 2 kHz on unseen sources
    forms = {"mixed_block_jacobi": (A32, bj32, A64), "mixed_learned_over_block_jacobi": (A32, learned, A64),
             "mixed_inner_outer": (A32, inner, A64)}
    res = {}
    for name, (A, pc, tru) in forms.items():
        _solve(A, beval[0], pc, tru)   # warm-up (graph capture)
        runs = [_solve(A, b, pc, tru) for b in beval]
        res[name] = {"iterations": [r["iters"] for r in runs], "ms": [round(r["ms"], 1) for r in runs],
                     "true_relres": [float(f"{r['true_relres']:.3e}") for r in runs],
                     "mean_ms": round(float(np.mean([r["ms"] for r in runs])), 1)}
        log(f"{name}: {res[name]}")
    r = _solve(A64, beval[0], bj64, None)
    res["plain_fp64_block_jacobi"] = {"iterations": [r["iters"]], "ms": [round(r["ms"], 1)],
                                      "true_relres": [float(f"{r['true_relres']:.3e}")], "mean_ms": round(r["ms"], 1)}
    log(f"plain_fp64_block_jacobi: {res['plain_fp64_block_jacobi']}")
    out["solves"] = res
    out["autotune_m2l_rcr_ms"] = {int(l): v["m2l_rcr"] for l, v in tune.items()}
    # matvec times
    x = torch.randn(wl.n, dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    mv = {}
    for name, h in (("mixed", A32), ("fp64", A64), ("inner_low_accuracy", Alow)):
        fb.fb_operator_apply(h, x, y)
        t = _now()
        for _ in range(5):
            fb.fb_operator_apply(h, x, y)
        mv[name] = round((_now() - t) / 5 * 1e3, 2)
    out["matvec_ms"] = mv
    for kind, h in reversed(handles):
        (fb.fb_operator_destroy if kind == "op" else fb.fb_precond_destroy)(h)
    fb.fb_tree_destroy(tree)
    fb.fb_mesh_destroy(mesh)
    return out


def cross_validate(log=print):
    thick = W.cfg_baffle(nsrc=1, nrec=64)
    thin = W.baffle_workload(2000.0, 10.0, nsrc=1, nrec=64, thickness=0.0)
    src = thick.sources[0]
    rcv = torch.tensor(thick.receivers, device="cuda")
    k = thick.k
    out = {"freq_hz": thick.freq_hz, "source": src.tolist(), "receivers": int(rcv.shape[0])}
    fields = {}
    for name, wl in (("direct_thick_baffle", thick), ("indirect_thin_baffle", thin)):
        t0 = _now()
        mesh = fb.fb_mesh_create(wl.verts, wl.tris)
        fb.fb_mesh_set_admittance(mesh, wl.beta)
        tree = fb.fb_tree_build(mesh, 64)
        indirect = name.startswith("indirect")
        kind = fb.FB_OP_IBEM if indirect else fb.FB_OP_A
        pmin = 14 if indirect else PMIN   # M' and L' need 14 for 1e-5 (the single operators' rule)
        A32 = fb.fb_operator_create(mesh, tree, k, kind, fb.FB_PREC_MIXED_FMM, D0, pmin)
        fb.fb_operator_autotune(A32, 1)
        fb.fb_operator_use_graphs(A32, True)
        A64 = fb.fb_operator_create(mesh, tree, k, kind, fb.FB_PREC_FP64_FMM, D0, pmin)
        fb.fb_operator_use_graphs(A64, True)
        Alow = fb.fb_operator_create(mesh, tree, k, kind, fb.FB_PREC_MIXED_FMM, INNER[0], INNER[1])
        fb.fb_operator_autotune(Alow, 1)
        fb.fb_operator_use_graphs(Alow, True)
        pclow = fb.fb_precond_create(Alow, fb.FB_PC_BLOCK_JACOBI)   # 2 x 2 leaf blocks for the indirect system
        inner = fb.fb_precond_create_inner(A32, Alow, pclow, INNER[2])
        L64 = None
        if indirect:
            gp, gm = fb.fb_ibem_gammas_monopole(A64, src)
            b = fb.fb_ibem_rhs(A64, gp, gm)
        else:
            L64 = fb.fb_operator_create(mesh, tree, k, fb.FB_OP_L, fb.FB_PREC_FP64_FMM, D0, PMIN)
            g = torch.empty(wl.n, dtype=torch.complex128, device="cuda")
            fb.fb_gamma_monopole(mesh, k, src, g)
            b = torch.empty_like(g)
            fb.fb_operator_apply(L64, g, b)
        t_setup = _now() - t0
        _solve(A32, b, inner, A64)   # warm-up (graph capture)
        x = torch.zeros_like(b)
        t1 = _now()
        info = fb.fb_fgmres_solve(A32, b, x, pc=inner, tol=TOL, restart=RESTART, maxit=3000, max_refine=4,
                                  true_op=A64)
        info["ms"] = (_now() - t1) * 1e3
        if indirect:
            f = fb.fb_ibem_field(A64, x, gp, gm, rcv)
            # plus the incident field: Eq. (dbem1) with zero surface densities
            zero = torch.zeros(wl.n, dtype=torch.complex128, device="cuda")
            inc = torch.empty_like(f)
            fb.fb_eval_field(mesh, k, zero, zero, rcv, inc, src=src)
            f = f + inc
        else:
            f = torch.empty(rcv.shape[0], dtype=torch.complex128, device="cuda")
            fb.fb_eval_field(mesh, k, x, g, rcv, f, src=src)
        fields[name] = f.cpu().numpy()
        out[name] = {"n_elements": wl.n, "unknowns": int(b.numel()), "setup_s": round(t_setup, 1),
                     "iterations": info["iters"], "solve_ms": round(info["ms"], 1),
                     "true_relres": float(f"{info['true_relres']:.3e}")}
        log(f"{name}: {out[name]}")
        fb.fb_precond_destroy(inner)
        fb.fb_precond_destroy(pclow)
        for h in (A32, A64, Alow, L64):
            if h is not None:
                fb.fb_operator_destroy(h)
        fb.fb_tree_destroy(tree)
        fb.fb_mesh_destroy(mesh)
    a, c = fields["direct_thick_baffle"], fields["indirect_thin_baffle"]
    out["receiver_rel_difference"] = float(np.linalg.norm(a - c) / np.linalg.norm(a))
    out["receiver_rel_difference_median"] = float(np.median(np.abs(a - c) / np.abs(a)))
    log(f"receiver difference {out['receiver_rel_difference']:.3e}")
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--train-freqs", default="1600,1800,2200,2400")
    ap.add_argument("--train-sources", type=int, default=2)
    ap.add_argument("--eval-sources", type=int, default=3)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--cross-validate", action="store_true")
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    freqs = [float(v) for v in a.train_freqs.split(",")]
    if a.cross_validate:
        res = cross_validate(log=lambda s: print(s, flush=True))
        txt = json.dumps(res)
        print(txt)
        if a.out:
            with open(a.out, "w") as f:
                f.write(txt + "\n")
        return
    res = run(freqs, a.train_sources, a.eval_sources, a.steps, lr=a.lr, log=lambda s: print(s, flush=True))
    txt = json.dumps(res)
    print(txt)
    if a.out:
        with open(a.out, "w") as f:
            f.write(txt + "\n")


if __name__ == "__main__":
    main()
