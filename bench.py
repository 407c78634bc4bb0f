"""Benchmark: FGMRES time-to-solve at true relative residual 1e-4 and
matvecs/s of the FMM-accelerated Helmholtz BEM on one GB300.

Workload (default): the largest room, shoebox 6.5 x 5.5 x 4.2 m at 5 kHz
(kD ~ 870), flat triangles with legs lambda/6 (569 x 482 x 368 rectangles)
-> N = 2,644,104 elements, one admittance per wall drawn uniform in
[0.05, 0.3] (seeded), one seeded monopole; octree leaves <= 64 elements; FMM
order per level from the excess-bandwidth rule (d0 = 6, p_min = 12): orders
159 / 89 / 52 / 32 / 20 / 14 on levels 2-7.  Synthetic input: a structured
mesh; ranks other than 0 solve for their own seeded source positions.  The
1 kHz shoebox (3.0 x 2.4 x 2.0 m, N = 39,368) is measured beside it as a
secondary workload.

A step is one solve A x = b of Eq. (dbem4), b = L gamma, with the mixed
operator (FP32 near field, P2M/L2P and translations, FP64 Arnoldi) right-
preconditioned by the inner-outer preconditioner of Sec. 4 (a few GMRES
steps on a low-accuracy mixed FMM with its own block Jacobi), judged by the
true residual of the FP64 FMM operator.  The plain FP64 path (FP64 FMM +
FP64 block Jacobi) is timed beside it.  N GPUs (torchrun) each solve their
own source position: weak scaling, no data-path collective.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload largest|shoebox_1khz]
"""
from __future__ import annotations

import os

# the host work of this process (and of the oracle worker processes it
# spawns, which inherit the environment) runs one BLAS thread per process
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FGMRES time-to-solve @1e-4 & matvecs/s: mixed+learned vs plain FP64, 1 GB300"
TOL = 1e-4
RESTART = 40
D0, PMIN = 6.0, 12                              # order rule of the operators (1e-5 FP64 FMM target)
INNER_D0, INNER_PMIN, INNER_ITERS = 0.5, 2, 14  # inner-outer preconditioner (low-accuracy FMM)

WORKLOADS = {
    "largest": ("cfg_largest", "shoebox 6.5x5.5x4.2 m, 5 kHz, N=2644104 flat triangles (lambda/6), "
                               "per-wall beta ~ U[0.05,0.3]"),
    "shoebox_1khz": ("cfg_1khz", "shoebox 3.0x2.4x2.0 m, 1 kHz, N=39368 flat triangles (lambda/8), beta=0.2"),
    "high_order": ("cfg_high_order", "shoebox 3.0x2.4x2.0 m, 7.5 kHz, N=3072 (orders 116 / 66)"),
}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    def __init__(self, gpu_index=0):
        # raw samples go to FB_BENCH_LOG_DIR (default: the temporary directory);
        # the JSON line carries their summary
        out_dir = os.environ.get("FB_BENCH_LOG_DIR", tempfile.gettempdir())
        self.path = os.path.join(out_dir, f"clocks_gpu{gpu_index}.csv")
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.cmd = ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                    "-lms", "200"]
        self.proc = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(self.cmd, stdout=self.f, stderr=subprocess.DEVNULL)
            # the timed region starts once sampling runs (first line written)
            t0 = time.time()
            while time.time() - t0 < 3.0:
                self.f.flush()
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self, max_mhz):
        rows = []
        try:
            for ln in open(self.path):
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": max_mhz, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else max_mhz, "reasons": reasons, "samples": len(rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_source(W, wl, rank):
    """Source position solved by `rank`: rank 0 the workload's own monopole,
    every other rank its own seeded position (independent solves, weak scaling)."""
    if rank == 0:
        return np.asarray(wl.sources[0], dtype=np.float64)
    rng = W.seeded_rng(100 + rank)
    return W.uniform_points_in_box(rng, [0, 0, 0], list(wl.room), 1, 0.25)[0]


def reduce_max_ms(ms, dist, device):
    """Max over ranks of a rank-local time (the job's wall time is its slowest rank)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def load_workload(name):
    from paper_2103_16073_gb300 import workloads as W
    return getattr(W, WORKLOADS[name][0])()


def bench_config(name, wl, ws):
    """The `config` object of the JSON line (identical for both arms)."""
    return {"workload": WORKLOADS[name][1], "n_elements": int(wl.n), "frequency_hz": wl.freq_hz,
            "fmm": f"leaf<=64, order rule d0={D0:g} p_min={PMIN}",
            "solver": "FGMRES(40), FP64 Arnoldi (CGS2), tol 1e-4 on the FP64 FMM true residual",
            "step": "one solve A x = b (Eq. dbem4), b = L gamma of a monopole",
            "precond": (f"inner-outer (Sec. 4): {INNER_ITERS} GMRES steps on a low-accuracy mixed FMM "
                        f"(d0={INNER_D0:g}, p_min={INNER_PMIN}, BF16 near-field entries) with block Jacobi"),
            "operator": "mixed: FP32 near field, P2M/L2P and translations (3xTF32 tensor-core and FP32 forms, "
                        "autotuned per level); FP64 true residual: FP64 or double-FP32 translations, autotuned",
            "l2": "inputs larger than L2 (near-field entries and translation data of GB size)",
            "parallelism": f"replicas x{ws} (one (f, source) solve per GPU)"}


def build_problem(fb, W, torch, wl, rank, forms="", forms_inner="", forms_fp64=""):
    """Mesh, tree and the operators of a solve: mixed A (autotuned translation
    forms, graph replay), FP64 A (true residual, plain method), FP64 L
    (b = L gamma), block Jacobi of each, and the inner-outer preconditioner
    on a low-accuracy mixed FMM."""
    wl.sources = rank_source(W, wl, rank)[None, :]
    t0 = time.perf_counter()
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = fb.fb_tree_build(mesh, 64)
    A64 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_FP64_FMM, D0, PMIN)
    A32 = fb.fb_operator_create_like(A64, fb.FB_PREC_MIXED_FMM, D0, PMIN)   # near-field entries copied
    L64 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_L, fb.FB_PREC_FP64_FMM, D0, PMIN)
    pc32 = fb.fb_precond_create(A32, fb.FB_PC_BLOCK_JACOBI)
    pc64 = fb.fb_precond_create(A64, fb.FB_PC_BLOCK_JACOBI)
    # per-level translation forms timed on the device (or a saved choice, e.g.
    # under a profiler, whose serialisation would distort the timing), then
    # graph replay of the matvecs
    if forms:
        fb.fb_operator_set_forms(A32, [int(v) for v in forms.split(",")])
        tune = {"fixed_forms": forms}
    else:
        tune = {"mixed": fb.fb_operator_autotune(A32, 1)}
    if forms_fp64 or forms:
        f64 = [int(v) for v in forms_fp64.split(",")] if forms_fp64 else [int(v) & 12 for v in forms.split(",")]
        fb.fb_operator_set_forms(A64, f64)
        tune["fp64_fixed_forms"] = ",".join(str(v) for v in f64)
        a64_forms = f64
    else:
        tune["fp64"] = fb.fb_operator_autotune(A64, 1)
        a64_forms = [tune["fp64"][l]["choice"] if l in tune["fp64"] else 0 for l in range(13)]
    for op in (A32, A64):
        fb.fb_operator_use_graphs(op, True)
    Alow = fb.fb_operator_create_like(A64, fb.FB_PREC_MIXED_FMM, INNER_D0, INNER_PMIN)
    if forms_inner:
        fb.fb_operator_set_forms(Alow, [int(v) for v in forms_inner.split(",")])
        tune["inner_fixed_forms"] = forms_inner
    else:
        tune["inner"] = fb.fb_operator_autotune(Alow, 1)
    pclow = fb.fb_precond_create(Alow, fb.FB_PC_BLOCK_JACOBI)
    fb.fb_operator_set_near_bf16(Alow, True)   # low-accuracy operator: 16-bit near-field entries
    fb.fb_operator_use_graphs(Alow, True)
    inner = fb.fb_precond_create_inner(A32, Alow, pclow, INNER_ITERS)
    fb.fb_precond_use_graphs(inner, True)
    g = torch.empty(wl.n, dtype=torch.complex128, device="cuda")
    fb.fb_gamma_monopole(mesh, wl.k, wl.sources[0], g)
    b = torch.empty_like(g)
    fb.fb_operator_apply(L64, g, b)
    torch.cuda.synchronize()
    return dict(wl=wl, mesh=mesh, tree=tree, A32=A32, A64=A64, L64=L64, pc32=pc32, pc64=pc64, b=b, tune=tune,
                Alow=Alow, pclow=pclow, inner=inner, A64_forms=a64_forms, setup_s=time.perf_counter() - t0)


def destroy_problem(fb, P):
    for pc in ("inner", "pclow", "pc32", "pc64"):
        fb.fb_precond_destroy(P[pc])
    for op in ("Alow", "A32", "A64", "L64"):
        fb.fb_operator_destroy(P[op])
    fb.fb_tree_destroy(P["tree"])
    fb.fb_mesh_destroy(P["mesh"])


def level_counts(fb, op, tree):
    """(p, tensor-core flag, M2L pairs, boxes) per level."""
    L, org, side, nb = fb.fb_tree_info(tree)
    n, L2, p = fb.fb_operator_info(op)
    tc = fb.fb_operator_export(op, 7).real.astype(int)
    pairs = [0, 0] + [fb.fb_tree_export(tree, 4, lev).shape[0] for lev in range(2, L + 1)]
    return L, p, tc, pairs, nb


def rot_flops(p_out, p_in):
    """Algorithmic flops of the two rotations of one RCR translation: sum
    (2n+1)^2 over n < p_in (rotate) and n < p_out (rotate back), complex-by-
    real MACs counted as complex MACs x 8 (the unfolded count; the folded
    kernels execute about half)."""
    return 8.0 * (sum((2 * n + 1) ** 2 for n in range(p_in)) + sum((2 * n + 1) ** 2 for n in range(p_out)))


def coax_flops(p_out, p_in):
    """Algorithmic flops of the coaxial step: sum over m of (p_out-|m|)(p_in-|m|) complex MACs x 8."""
    q = min(p_out, p_in)
    return 8.0 * sum((p_out - abs(m)) * (p_in - abs(m)) for m in range(-q + 1, q))


def rcr_flops(p_out, p_in):
    """Algorithmic flops of one RCR translation (rotations + coaxial step),
    about (10/3) p^3 x 8 for p_out = p_in."""
    return rot_flops(p_out, p_in) + coax_flops(p_out, p_in)


# double-FP32 multiply-accumulate: 12 FP32-pipe operations (df.cuh)
DF_OPS_PER_MAC = 12

FAMILY = {("f32", "tiles"): "k_rcr<float>", ("f32", "tc"): "k_trans_tc", ("f64", "tiles"): "k_rcr<double>",
          ("f64", "tiles_df"): "k_rcr<df>"}
FAMILY_WHAT = {
    "k_stg_tc": "staged RCR rotation passes on the tensor cores (k_stg_tc<0> rotate, k_stg_tc<1> rotate back; "
                "tcgen05 3xTF32 GEMMs per polar-angle group and degree)",
    "k_stg_coax<float>": "staged RCR coaxial pass (FP32 CUDA-core GEMMs per |t| and order)",
    "k_stc_coax": "staged RCR coaxial pass on the tensor cores (tcgen05 3xTF32, complex blocks in real form per "
                  "|t| and order)",
    "k_stg_rot+back<float>": "staged RCR rotation passes on CUDA cores (FP32)",
    "k_stg_prep<float>": "staged RCR pre-pass (folded phased inputs, FP32)",
    "k_stg<double>": "staged RCR passes in FP64 (true residual)",
    "k_stg<df>": "staged RCR passes in double-FP32 arithmetic (FP64 true residual; 48-bit significand)",
    "k_stg_prep<df>": "staged RCR pre-pass of the double-FP32 levels",
    "k_stg_prep<double>": "staged RCR pre-pass (FP64)",
    "k_rcr<float>": "per-pair RCR M2L tiles (FP32)",
    "k_trans_tc": "tensor-core M2L (tcgen05 3xTF32, composed matrices)",
    "k_rcr<double>": "per-pair RCR M2L tiles (FP64, true residual)",
    "k_rcr<df>": "per-pair RCR M2L tiles in double-FP32 arithmetic (FP64 true residual; 48-bit significand)",
}


def fp64_only_forms(tune):
    """Per-level forms of an FP64 operator restricted to FP64 arithmetic
    (per-pair tiles or staged passes, whichever the autotuner timed faster),
    for the plain FP64 baseline."""
    out = [0] * 13
    for l, t in (tune or {}).items():
        l = int(l)
        c = 0
        a, b = t["m2l_rcr"], t["m2l_staged"]
        if b is not None and (a is None or b < a):
            c |= 4
        a, b = t["m2m_l2l_rcr"], t["m2m_l2l_staged"]
        if b is not None and (a is None or b < a):
            c |= 8
        out[l] = c
    return out


def m2l_levels(tune, p, pairs):
    """Per level of an autotuned operator whose M2L is not staged: (form,
    device ms of its M2L pass, algorithmic flops) from the autotuner's
    timings of the installed form."""
    out = {}
    for l, t in (tune or {}).items():
        l = int(l)
        ch = t["choice"]
        if ch & 4 and not ch & 1:
            continue   # staged: timed pass by pass (fb_operator_staged_pass_times)
        if ch & 1:
            form, ms = "tc", t["m2l_tensor"]
        elif ch & 256:
            form, ms = "tiles_df", t["m2l_tiles_df"]
        else:
            form, ms = "tiles", t["m2l_rcr"]
        if ms is None:
            continue
        out[l] = (form, ms, float(pairs[l]) * rcr_flops(int(p[l]), int(p[l])))
    return out


def roofline(fb, P, iters, true_mv, pk, fp32_peak, fp64_peak):
    """Rooflines of the M2L kernels of a solve and the dominant one.  The
    staged levels are timed pass by pass with CUDA events
    (fb_operator_staged_pass_times: each pass launched alone); the per-pair
    tiles and composed tensor-core levels by the autotuner's device timings.
    A kernel's achieved rate is its algorithmic work (flops, or bytes for
    the pre-pass) over its device time, both summed over the launches of one
    solve: outer iterations for the mixed operator, outer x inner iterations
    for the low-accuracy inner operator, true residuals for FP64."""
    tune = P["tune"]
    L, _, _, pairs, _ = level_counts(fb, P["A32"], P["tree"])
    tf32 = float(pk.get("bf16_tflops", 1990.0)) * (1.1 / 2.25)
    hbm = float(pk.get("hbm_gbs", 6790.7))
    peaks_ = {
        "tensor": (tf32 / 3.0, "TFLOP/s", "measured BF16 burst x 1.1/2.25 (TF32) / 3 split passes, of measured"),
        "f32": (fp32_peak, "TFLOP/s", "FP32 FMA throughput measured by fb_measure_alu_peaks"),
        "f64": (fp64_peak, "TFLOP/s", "FP64 FMA throughput measured by fb_measure_alu_peaks"),
        "df": (fp32_peak / DF_OPS_PER_MAC, "TFLOP/s",
               f"measured FP32 FMA throughput x 2 flops / {DF_OPS_PER_MAC} FP32 operations per double-FP32 MAC"),
        "hbm": (hbm / 1e3, "TB/s", "measured HBM copy bandwidth (MEASURED_PEAKS.json), of measured"),
    }
    fam = {}

    def add(name, kind, key, l, count, ms, work):
        if ms is None or ms <= 0:
            return
        f = fam.setdefault(name, {"ms": 0.0, "work": 0.0, "kind": kind, "per_op": {}})
        f["ms"] += ms * count
        f["work"] += work * count
        po = f["per_op"].setdefault(key, {"levels": [], "launch_ms": 0.0, "work": 0.0, "per_step": count})
        po["levels"].append(l)
        po["launch_ms"] = round(po["launch_ms"] + ms, 4)
        po["work"] += work

    for key, op, prec, count in (("mixed", "A32", "f32", iters), ("inner", "Alow", "f32", iters * INNER_ITERS),
                                 ("fp64", "A64", "f64", true_mv)):
        p = fb.fb_operator_info(P[op])[2]
        for l, d in fb.fb_operator_staged_pass_times(P[op]).items():
            pl, npair = int(p[l]), float(pairs[l])
            rot, cox = npair * rot_flops(pl, pl), npair * coax_flops(pl, pl)
            cw = 16 if prec == "f32" else 32   # bytes per complex coefficient read + written
            if d["form"] == "df":
                add("k_stg<df>", "df", key, l, count, d["rot"] + d["coax"] + d["back"], rot + cox)
                add("k_stg_prep<df>", "hbm", key, l, count, d["prep"], npair * pl * pl * cw)
                continue
            if prec == "f64":
                add("k_stg<double>", "f64", key, l, count, d["rot"] + d["coax"] + d["back"], rot + cox)
                add("k_stg_prep<double>", "hbm", key, l, count, d["prep"], npair * pl * pl * cw)
                continue
            if d["form"] == "tensor_rot_coax":
                add("k_stg_tc", "tensor", key, l, count, d["rot"] + d["back"], rot)
                add("k_stc_coax", "tensor", key, l, count, d["coax"], cox)
            elif d["form"] == "tensor_rot":
                add("k_stg_tc", "tensor", key, l, count, d["rot"] + d["back"], rot)
                add("k_stg_coax<float>", "f32", key, l, count, d["coax"], cox)
            else:
                add("k_stg_rot+back<float>", "f32", key, l, count, d["rot"] + d["back"], rot)
                add("k_stg_coax<float>", "f32", key, l, count, d["coax"], cox)
            add("k_stg_prep<float>", "hbm", key, l, count, d["prep"], npair * pl * pl * cw)
        for l, (form, ms, alg) in m2l_levels(tune.get(key), p, pairs).items():
            add(FAMILY[(prec, form)], {"tc": "tensor", "tiles_df": "df"}.get(form, prec), key, l, count, ms, alg)
    out = {}
    for name, f in fam.items():
        peak, unit, kind = peaks_[f["kind"]]
        ach = f["work"] / (f["ms"] / 1e3) / 1e12   # TFLOP/s or TB/s
        bound = {"tensor": "tensor", "hbm": "hbm"}.get(f["kind"], "alu")
        out[name] = {"what": FAMILY_WHAT.get(name, name), "bound": bound, "achieved": round(ach, 3),
                     "peak": round(peak, 3), "unit": unit, "frac": round(ach / peak, 4) if peak else None,
                     "est_ms_per_step": round(f["ms"], 2), "per_operator": f["per_op"], "peak_kind": kind}
    if not out:
        return None, out
    dom = max(out, key=lambda k: out[k]["est_ms_per_step"])
    d = out[dom]
    if d["unit"] == "TB/s":
        work = "algorithmic bytes per box pair: 16 B per complex coefficient read and written (32 B in FP64)"
    elif dom in ("k_stg_tc", "k_stg_rot+back<float>"):
        work = "algorithmic flops per box pair: rotations 8 x 2 sum_{n<p}(2n+1)^2 (unfolded count)"
    elif dom in ("k_stc_coax", "k_stg_coax<float>"):
        work = "algorithmic flops per box pair: coaxial step 8 x sum_m (p-|m|)^2"
    else:
        work = "algorithmic flops per box pair: rotations 8 x 2 sum_{n<p}(2n+1)^2 + coaxial 8 x sum_m (p-|m|)^2"
    rf = {"kernel": dom, "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"], "unit": d["unit"],
          "frac": d["frac"], "traffic": traffic_for(dom), "peak_kind": d["peak_kind"], "what": d["what"],
          "est_ms_per_step": d["est_ms_per_step"],
          "launch": {k: {"levels": v["levels"], "launch_ms": v["launch_ms"], "work": v["work"]}
                     for k, v in d["per_operator"].items()},
          "work": work}
    return rf, out


def traffic_for(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or
    None when the kernel source changed since the counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path)).get(kernel)
    if not d:
        return None
    src = os.path.join(ROOT, d["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != d["sha256"]:
        return None
    return d["dram_bytes_per_launch"]


def timed(torch, stream, fn, reps=1):
    """Device time (s) of `reps` calls of fn on `stream` (CUDA events, synchronised)."""
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = [fn() for _ in range(reps)]
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps, out


def matvec_rate(fb, torch, stream, op, n, reps):
    xv = torch.randn(n, dtype=torch.complex128, device="cuda")
    yv = torch.empty_like(xv)
    for _ in range(2):
        fb.fb_operator_apply(op, xv, yv)
    t, _ = timed(torch, stream, lambda: fb.fb_operator_apply(op, xv, yv), reps)
    ph = [fb.fb_operator_apply_timed(op, xv, yv) for _ in range(3)]
    return t, {k: statistics.median(p[k] for p in ph) for k in ph[0]}


def secondary(fb, W, torch, stream, name):
    """Mixed + inner-outer and plain FP64 on a second workload (median of 3
    mixed solves, one plain solve)."""
    wl = load_workload(name)
    P = build_problem(fb, W, torch, wl, 0)
    try:
        def solve(pc, A, T):
            x = torch.zeros_like(P["b"])
            return fb.fb_fgmres_solve(A, P["b"], x, pc=pc, tol=TOL, restart=RESTART, maxit=3000, max_refine=4,
                                      true_op=T)
        solve(P["inner"], P["A32"], P["A64"])
        ts = [timed(torch, stream, lambda: solve(P["inner"], P["A32"], P["A64"])) for _ in range(3)]
        t_io = statistics.median(t for t, _ in ts)
        mv32, _ = matvec_rate(fb, torch, stream, P["A32"], wl.n, 20)
        fb.fb_operator_set_forms(P["A64"], fp64_only_forms(P["tune"]["fp64"]))   # FP64 arithmetic
        t64, (i64,) = timed(torch, stream, lambda: solve(P["pc64"], P["A64"], None))
        mv64, _ = matvec_rate(fb, torch, stream, P["A64"], wl.n, 5)
        info = ts[-1][1][0]
        return {"workload": WORKLOADS[name][1], "n_elements": wl.n,
                "mixed_inner_outer": {"time_to_solve_s": round(t_io, 5), "solves_per_s": round(1 / t_io, 3),
                                      "iterations": info["iters"], "true_relres": info["true_relres"],
                                      "matvecs_per_s": round(1 / mv32, 2)},
                "plain_fp64": {"time_to_solve_s": round(t64, 4), "iterations": i64["iters"],
                               "true_relres": i64["true_relres"], "matvecs_per_s": round(1 / mv64, 2)},
                "speedup_vs_plain_fp64": round(t64 / t_io, 2)}
    finally:
        destroy_problem(fb, P)


def run_matvecs(args):
    """Profiling mode: one operator of the workload (autotuned forms unless
    --forms), `--matvec-only` applications on the device and the per-phase
    CUDA-event split of one more; prints one JSON line."""
    import torch
    import paper_2103_16073_gb300 as fb
    torch.cuda.set_device(0)
    wl = load_workload(args.workload)
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = fb.fb_tree_build(mesh, 64)
    prec = {"mixed": fb.FB_PREC_MIXED_FMM, "fp64": fb.FB_PREC_FP64_FMM}[args.prec]
    d0, pmin = (INNER_D0, INNER_PMIN) if args.inner_operator else (D0, PMIN)
    op = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, prec, d0, pmin)
    tune = None
    if args.forms:
        fb.fb_operator_set_forms(op, [int(v) for v in args.forms.split(",")])
    else:
        tune = fb.fb_operator_autotune(op, 1)
    if args.inner_operator:
        fb.fb_operator_set_near_bf16(op, True)   # as the solve's inner operator
    stream = torch.cuda.current_stream()
    t, ph = matvec_rate(fb, torch, stream, op, wl.n, args.matvec_only)
    passes = fb.fb_operator_staged_pass_times(op)
    print(json.dumps({"workload": WORKLOADS[args.workload][1], "precision": args.prec, "d0": d0, "pmin": pmin,
                      "orders": [int(v) for v in fb.fb_operator_info(op)[2][2:]], "matvec_ms": round(t * 1e3, 4),
                      "phase_ms": {k: round(v, 4) for k, v in ph.items()},
                      "staged_pass_ms": {l: {k: (round(v, 4) if isinstance(v, float) else v) for k, v in d.items()}
                                         for l, d in passes.items()},
                      "forms": args.forms or ",".join(str(tune[l]["choice"] if l in tune else 0) for l in range(13)),
                      "autotune": tune}))
    fb.fb_operator_destroy(op)
    fb.fb_tree_destroy(tree)
    fb.fb_mesh_destroy(mesh)


def run_ours(args):
    import torch
    import paper_2103_16073_gb300 as fb
    from paper_2103_16073_gb300 import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if dist.is_nccl_available() else "gloo")
    wl = load_workload(args.workload)
    P = build_problem(fb, W, torch, wl, rank, args.forms, args.forms_inner, args.forms_fp64)
    n = wl.n
    stream = torch.cuda.current_stream()
    pc_main = P["inner"]

    def solve_mixed(x, pc=pc_main):
        return fb.fb_fgmres_solve(P["A32"], P["b"], x, pc=pc, tol=TOL, restart=RESTART, maxit=3000,
                                  max_refine=4, true_op=P["A64"])

    x = torch.zeros_like(P["b"])
    for _ in range(args.warmup):
        info = solve_mixed(x)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    pk, pk_kind = peaks()
    sampler = ClockSampler(local)
    launches0 = fb.fb_kernel_launches()
    infos = []
    with sampler:
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("bench_timed")     # ncu --nvtx-include bench_timed/
        e0.record(stream)
        for _ in range(args.steps):
            infos.append(solve_mixed(x))
        e1.record(stream)
        barrier()
        torch.cuda.nvtx.range_pop()
    launches = fb.fb_kernel_launches() - launches0
    ms_total = reduce_max_ms(e0.elapsed_time(e1), dist, "cuda" if dist is not None and
                             dist.get_backend() == "nccl" else "cpu")
    ms_step = ms_total / args.steps
    iters = statistics.mean(i["iters"] for i in infos)
    relres = max(i["true_relres"] for i in infos)
    ok = all(i["status"] == 0 for i in infos)
    clocks = sampler.summary(pk.get("sm_max_mhz"))

    # matvecs/s and phase split of the three operators of the solve
    mv_s, ph = matvec_rate(fb, torch, stream, P["A32"], n, args.matvecs)
    mv64_s, ph64 = matvec_rate(fb, torch, stream, P["A64"], n, max(2, args.matvecs // 5))
    mvlow_s, ph_low = matvec_rate(fb, torch, stream, P["Alow"], n, args.matvecs)

    # plain FP64 path: FP64 FMM + FP64 block Jacobi, one solve, with the
    # FP64 operator restricted to FP64 arithmetic; then the same method with
    # the operator's autotuned forms (double-FP32 translations included)
    fp64_forms = fp64_only_forms(P["tune"].get("fp64")) if "fp64" in P["tune"] else \
        [int(v) & 12 for v in P["tune"]["fp64_fixed_forms"].split(",")]
    tuned_forms = P["A64_forms"]

    def plain_solve():
        x64 = torch.zeros_like(P["b"])
        t, (inf,) = timed(torch, stream, lambda: fb.fb_fgmres_solve(
            P["A64"], P["b"], x64, pc=P["pc64"], tol=TOL, restart=RESTART, maxit=3000))
        return t, inf, x64
    fb.fb_operator_set_forms(P["A64"], fp64_forms)
    mv64p_s, _ = matvec_rate(fb, torch, stream, P["A64"], n, max(2, args.matvecs // 5))
    t64, info64, x64 = plain_solve()
    fb.fb_operator_set_forms(P["A64"], tuned_forms)
    t64d, info64d, x64d = plain_solve()
    # agreement of the solutions (all judged by the FP64 operator)
    sol_diff = float((x - x64).norm() / x64.norm())
    sol_diff_df = float((x64d - x64).norm() / x64.norm())

    # end to end through the public API with host (pinned) buffers
    bh = torch.empty(n, dtype=torch.complex128, pin_memory=True)
    bh.copy_(P["b"].cpu())
    xh = torch.zeros(n, dtype=torch.complex128, pin_memory=True)
    xn = xh.numpy()
    e2e_t = []
    for _ in range(max(1, min(args.steps, args.e2e_steps))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fb.fb_fgmres_solve(P["A32"], bh, xn, pc=pc_main, tol=TOL, restart=RESTART, maxit=3000,
                           max_refine=4, true_op=P["A64"])
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = statistics.median(e2e_t)

    fp32_peak, fp64_peak = fb.fb_measure_alu_peaks()
    rf, kernels = roofline(fb, P, iters, res_true_matvecs(infos), pk, fp32_peak, fp64_peak)
    L, p, tc, pairs, nb = level_counts(fb, P["A32"], P["tree"])
    setup_s = P["setup_s"]
    destroy_problem(fb, P)
    sec = None
    if rank == 0 and args.secondary and args.workload != "shoebox_1khz":
        sec = secondary(fb, W, torch, stream, "shoebox_1khz")
    res = {
        "metric": METRIC,
        "value": round(ws / (ms_step / 1e3), 5),
        "unit": "solves/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": bench_config(args.workload, wl, ws),
        "time_to_solve_s": round(ms_step / 1e3, 5),
        "iterations": iters,
        "inner_iterations_per_outer": INNER_ITERS,
        "true_relres": relres,
        "true_matvecs_per_solve": res_true_matvecs(infos),
        "converged": ok,
        "setup_s": round(setup_s, 2),
        "orders_per_level": [int(v) for v in p[2:]],
        "m2l_pairs_per_level": [int(v) for v in pairs[2:]],
        "matvecs_per_s": {"mixed": round(1 / mv_s, 3), "fp64": round(1 / mv64_s, 3),
                          "fp64_arithmetic_only": round(1 / mv64p_s, 3),
                          "inner_low_accuracy": round(1 / mvlow_s, 3)},
        "matvec_ms": {"mixed": round(mv_s * 1e3, 3), "fp64": round(mv64_s * 1e3, 3),
                      "fp64_arithmetic_only": round(mv64p_s * 1e3, 3),
                      "inner_low_accuracy": round(mvlow_s * 1e3, 3)},
        "phase_ms": {"mixed": {k: round(v, 3) for k, v in ph.items()},
                     "fp64": {k: round(v, 3) for k, v in ph64.items()},
                     "inner_low_accuracy": {k: round(v, 3) for k, v in ph_low.items()}},
        "plain_fp64": {"time_to_solve_s": round(t64, 4), "iterations": info64["iters"],
                       "true_relres": info64["true_relres"], "preconditioner": "FP64 block Jacobi"},
        "plain_fp64_df_translations": {
            "time_to_solve_s": round(t64d, 4), "iterations": info64d["iters"],
            "true_relres": info64d["true_relres"], "solution_rel_diff_vs_plain_fp64": sol_diff_df,
            "what": "the plain method with the FP64 operator's autotuned forms (translations in double-FP32 "
                    "arithmetic, 48-bit significand, where faster); the mixed solve's true residual uses them"},
        "speedup_vs_plain_fp64": round(t64 / (ms_step / 1e3), 2),
        "solution_rel_diff_mixed_vs_plain": sol_diff,
        "learned": "side study, not in the timed step (the trained network did not reduce the outer "
                   "iterations of the inner-outer solve)",
        "autotune": P["tune"],
        "graphs": True,
        "measured_alu_peaks_tflops": {"fp32": round(fp32_peak, 2), "fp64": round(fp64_peak, 3)},
        "e2e": {"value": round(1.0 / e2e_s, 5), "unit": "solves/s", "h2d_bytes_per_step": 16 * n,
                "d2h_bytes_per_step": 16 * n},
        "gpu_launches": int(launches),
        "roofline": rf,
        "kernels": kernels,
        "clocks": clocks,
        "secondary": sec,
    }
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle's dense matvec, counted like the plain method's solve
        # (block-Jacobi iterations + one true residual)
        res["cpu_baseline"] = cpu_baseline(wl, info64["iters"] + 1, budget_s=args.cpu_seconds)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(res))


def res_true_matvecs(infos):
    return int(round(statistics.mean(i["true_matvecs"] for i in infos)))


# ---------------------------------------------------------------- oracle leg
_ORACLE = {}


def _oracle_init(verts, tris, k, beta):
    """Worker set-up: the oracle's mesh (geometry of every element)."""
    from oracle import bem
    _ORACLE.update(mesh=bem.Mesh(verts, tris), k=k, beta=beta)
    rng = np.random.default_rng(0)
    n = tris.shape[0]
    _ORACLE["x"] = rng.standard_normal(n) + 1j * rng.standard_normal(n)


def _oracle_rows(rows):
    """Rows of the dense FP64 system matrix of Eq. (dbem4), assembled on the
    fly by the oracle and applied to a fixed vector."""
    from oracle import bem
    A = bem.system_rows(_ORACLE["mesh"], _ORACLE["k"], _ORACLE["beta"], np.asarray(rows))
    return len(rows), complex(np.sum(A @ _ORACLE["x"]))


def _ready(_):
    return os.getpid()


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_workers(n_elements):
    """One worker per host core, as many as the free host memory holds (the
    oracle's geometry and one dense row take about 1 KB per element)."""
    cores = cpu_cores()
    try:
        free = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        cores = max(1, min(cores, int(0.6 * free / (1100.0 * n_elements + 3e8))))
    except (ValueError, OSError, AttributeError):
        pass
    return cores


class OraclePool:
    """Worker processes (started with spawn, each holding the oracle's mesh)
    that time seeded random rows of the dense FP64 system matrix of
    Eq. (dbem4), assembled on the fly and applied to a fixed vector."""

    def __init__(self, wl, workers=None):
        import multiprocessing as mp
        self.wl = wl
        self.cores = workers or oracle_workers(wl.n)
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_init,
                                                 initargs=(wl.verts, wl.tris, wl.k, wl.beta))
        self.pool.map(_ready, range(self.cores), chunksize=1)   # workers started and initialised
        self.rng = np.random.default_rng(1)

    def sample(self, budget_s):
        """(rows, wall seconds): rows submitted for `budget_s` seconds, all
        cores busy, every submitted row waited for."""
        pending, rows = [], 0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < budget_s:
            while len(pending) < 2 * self.cores:
                pending.append(self.pool.apply_async(_oracle_rows, (self.rng.integers(0, self.wl.n, size=1),)))
            still = []
            for r in pending:
                if r.ready():
                    rows += r.get()[0]
                else:
                    still.append(r)
            pending = still
            time.sleep(0.01)
        for r in pending:
            rows += r.get()[0]
        return rows, time.perf_counter() - t0

    def close(self):
        self.pool.terminate()
        self.pool.join()


def extrapolate(wl, rows, dt, cores, matvecs_per_solve):
    per_matvec = dt / max(rows, 1) * wl.n
    per_solve = per_matvec * max(1, matvecs_per_solve)
    return {"value": 1.0 / per_solve, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{rows} seeded random rows of the dense FP64 matrix-free A (Eq. dbem4, N={wl.n}) "
                      f"in {dt:.1f} s on {cores} worker processes; extrapolated x N rows per matvec x "
                      f"{matvecs_per_solve} matvecs per solve (the plain method's block-Jacobi iterations "
                      f"+ 1 true residual)",
            "matvec_s_extrapolated": per_matvec}


def cpu_baseline(wl, matvecs_per_solve, budget_s=15.0):
    """The oracle timed on the host cores for about `budget_s` seconds of wall
    time; the row rate is extrapolated to N rows per matvec and to
    `matvecs_per_solve` matvecs per solve."""
    pool = OraclePool(wl)
    try:
        rows, dt = pool.sample(budget_s)
    finally:
        pool.close()
    return extrapolate(wl, rows, dt, pool.cores, matvecs_per_solve)


def run_reference(args):
    """The oracle as it stands on the host cores: each step a bounded sample of
    dense matrix-free rows of the same workload, extrapolated to one solve."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    wl = load_workload(args.workload)
    matvecs = args.ref_matvecs
    vals = []
    budget = max(3.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    pool = OraclePool(wl)
    try:
        for i in range(args.warmup + args.steps):
            rows, dt = pool.sample(budget)
            if i >= args.warmup:
                vals.append(extrapolate(wl, rows, dt, pool.cores, matvecs))
    finally:
        pool.close()
    v = statistics.mean(c["value"] for c in vals)
    res = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": bench_config(args.workload, wl, ws),
           "arm": "dense FP64 collocation oracle (CPU), extrapolated from sampled rows",
           "matvecs_per_solve": matvecs,
           "cpu_baseline": {"value": v, "unit": "solves/s", "cores": vals[-1]["cores"], "kind": "oracle",
                            "sample": vals[-1]["sample"]},
           "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="largest", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", dest="secondary", action="store_false",
                    help="skip the 1 kHz shoebox measured beside the main workload")
    ap.add_argument("--matvecs", type=int, default=10, help="matvecs timed per operator for matvecs/s")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--forms", default="", help="fixed per-level translation forms of the mixed and FP64 "
                                                "operators instead of autotuning (comma-separated choice ints "
                                                "by level, as fb_operator_set_forms; the FP64 one takes bits 2-3)")
    ap.add_argument("--forms-inner", default="", help="the same for the low-accuracy inner operator")
    ap.add_argument("--forms-fp64", default="", help="the same for the FP64 operator (default: --forms)")
    ap.add_argument("--ref-matvecs", type=int, default=52,
                    help="matvecs per solve used to extrapolate the reference arm (default: the plain "
                         "method's 51 block-Jacobi iterations on the largest room + 1 true residual)")
    ap.add_argument("--matvec-only", type=int, default=0,
                    help="profiling mode: time this many matvecs of one operator and exit")
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"], help="operator of --matvec-only")
    ap.add_argument("--inner-operator", action="store_true", help="--matvec-only on the low-accuracy inner operator")
    args = ap.parse_args()
    if args.matvec_only > 0:
        run_matvecs(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
