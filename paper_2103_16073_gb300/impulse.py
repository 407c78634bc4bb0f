"""Broadband room response (Sec. 4): Helmholtz solutions at equispaced
frequencies turned into the response to the pulse of Eq. (an3), compared
with the image-source method (Eqs. an1, an2) in the frequency and the time
domain, on the paper's 8 x 6 x 3 m room with zeta = 9 (R = 0.8) and the
source at (3, 2, 1.75) m; receivers on a grid in the plane z = 1.75 m.

Every frequency is meshed at lambda/8 (legs at most 0.5 m) and solved to a
true relative residual of 1e-4 through the batch scheduler; the receiver
field, the image sums and the synthesis run in the library.  The image
method assumes angle-independent reflection while the BEM imposes a locally
reacting impedance, so the two differ by the order of 10 % (Sec. 4 reports
16 % in frequency and 15 % in time).

    python -m paper_2103_16073_gb300.impulse [--fmax 640] [--df 10] [--out result.json]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

import paper_2103_16073_gb300 as fb
from paper_2103_16073_gb300 import workloads as W


def run(f_max=640.0, df=10.0, tol=1e-4, log=print):
    wls = W.ir_sweep(f_max, df)
    src = np.asarray(W.IR_SOURCE)
    rcv_h = wls[0].receivers
    rcv = torch.tensor(rcv_h, device="cuda")
    nr = rcv_h.shape[0]
    t0 = time.perf_counter()
    built = []
    for wl in wls:
        mesh = fb.fb_mesh_create(wl.verts, wl.tris)
        fb.fb_mesh_set_admittance(mesh, wl.beta)
        tree = fb.fb_tree_build(mesh, 64)
        built.append(dict(mesh=mesh, tree=tree, k=wl.k, src=wl.sources,
                          x=torch.zeros((1, wl.n), dtype=torch.complex128, device="cuda")))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    res = fb.fb_batch_solve(built, tol=tol, max_rhs=1, autotune=True, lookahead=True)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    psi = torch.empty((len(wls), nr), dtype=torch.complex128, device="cuda")
    for m, (wl, b) in enumerate(zip(wls, built)):
        g = torch.empty(wl.n, dtype=torch.complex128, device="cuda")
        fb.fb_gamma_monopole(b["mesh"], wl.k, src, g)
        fb.fb_eval_field(b["mesh"], wl.k, b["x"][0].contiguous(), g, rcv, psi[m], src=src)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    R = (W.IR_ZETA - 1.0) / (W.IR_ZETA + 1.0)
    ks = np.array([wl.k for wl in wls])
    img = fb.fb_image_field(W.IR_ROOM, src, [R] * 6, ks, rcv, a_th=1e-7)
    t4 = time.perf_counter()
    freqs = np.array([wl.freq_hz for wl in wls])
    nt = 2 * len(wls)
    T = 1.0 / df
    dt = T / nt
    p_bem = fb.fb_pulse_synthesis(psi, freqs, df, dt, nt, dt)
    p_img = fb.fb_pulse_synthesis(img, freqs, df, dt, nt, dt)
    torch.cuda.synchronize()
    e_f = float(torch.linalg.norm(psi - img) / torch.linalg.norm(img))
    e_t = float(torch.linalg.norm(p_bem - p_img) / torch.linalg.norm(p_img))
    per_f = (torch.linalg.norm(psi - img, dim=1) / torch.linalg.norm(img, dim=1)).cpu().numpy()
    out = {"room": list(W.IR_ROOM), "zeta": W.IR_ZETA, "reflection": R, "source": list(W.IR_SOURCE),
           "frequencies": [float(freqs[0]), float(freqs[-1]), len(freqs)], "df_hz": df, "receivers": nr,
           "n_elements": [wl.n for wl in wls], "time_samples": nt, "dt_ms": dt * 1e3,
           "solves_converged": int(sum(r["status"] == 0 for r in res)),
           "max_true_relres": max(i["true_relres"] for r in res for i in r["infos"]),
           "mesh_tree_s": round(t1 - t0, 2), "batch_solve_s": round(t2 - t1, 2), "receivers_s": round(t3 - t2, 2),
           "images_s": round(t4 - t3, 2),
           "rel_l2_frequency_domain": round(e_f, 4), "rel_l2_time_domain": round(e_t, 4),
           "rel_l2_per_frequency": {f"{f:.0f}": round(float(e), 4) for f, e in zip(freqs[::8], per_f[::8])}}
    log(json.dumps(out))
    for b in built:
        fb.fb_tree_destroy(b["tree"])
        fb.fb_mesh_destroy(b["mesh"])
    return out, (psi, img, p_bem, p_img)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--fmax", type=float, default=640.0)
    ap.add_argument("--df", type=float, default=10.0)
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    out, _ = run(a.fmax, a.df, log=lambda s: None)
    txt = json.dumps(out)
    print(txt)
    if a.out:
        with open(a.out, "w") as f:
            f.write(txt + "\n")


if __name__ == "__main__":
    main()
