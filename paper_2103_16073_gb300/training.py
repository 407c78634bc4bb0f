"""Training driver of the learned octree preconditioner.

Orchestration only: every step runs in the library (FGMRES solves, operator
and preconditioner applications, the network's forward/backward kernels and
Adam).  Pairs (r, e) come from the plain method's own solves: FGMRES with
block Jacobi is stopped after j iterations for several j, giving iterates x_j
with r_j = b - A x_j and e_j = x* - x_j, where x* is the converged solution,
so A e_j = r_j holds for the operator A the preconditioner will serve.

The default objective is the residual one, ||A z(r) - r||^2 / ||r||^2, which
does not use e; for it the logged residuals can be joined by white-noise
inputs (``augment_noise``) so that the network does not trade accuracy on
the directions the Krylov basis also contains for accuracy on the logged
residuals.  ``train`` can keep the parameters that did best on a validation
solve (``validate``), the block-Jacobi-like initial state included.
"""
from __future__ import annotations

import numpy as np
import torch

import paper_2103_16073_gb300 as fb


def collect_pairs(A, bj, b, iterates=(1, 2, 3, 4, 6, 8, 10, 13, 16), restart=40, tol_star=1e-7):
    """Residual/error pairs from truncated block-Jacobi FGMRES solves of A x = b.
    b: CUDA complex128 tensor.  Returns (R, E) tensors [len(iterates), N]."""
    xs = torch.zeros_like(b)
    fb.fb_fgmres_solve(A, b, xs, pc=bj, tol=tol_star, restart=restart, maxit=3000, max_refine=8)
    R = torch.empty((len(iterates), b.numel()), dtype=b.dtype, device=b.device)
    E = torch.empty_like(R)
    ax = torch.empty_like(b)
    for q, j in enumerate(iterates):
        xj = torch.zeros_like(b)
        fb.fb_fgmres_solve(A, b, xj, pc=bj, tol=1e-14, restart=restart, maxit=int(j), max_refine=1)
        fb.fb_operator_apply(A, xj, ax)
        R[q] = b - ax
        E[q] = xs - xj
    torch.cuda.synchronize()
    return R, E


def krylov_inputs(A, pc, b, k=6):
    """Inputs the preconditioner meets inside a solve: the first k+1
    Arnoldi vectors of the solve of A x = b preconditioned by pc (residual
    objective only; returned with zero E rows)."""
    V = fb.fb_krylov_basis(A, pc, b, k)
    return V, torch.zeros_like(V)


def augment_noise(R, E, count, seed=0):
    """Appends `count` white-noise inputs (for the residual objective only;
    their E rows are zero and unused)."""
    g = torch.Generator(device=R.device)
    g.manual_seed(seed)
    Nz = torch.randn((count, R.shape[1]), dtype=R.dtype, device=R.device, generator=g)
    return torch.cat([R, Nz]), torch.cat([E, torch.zeros_like(Nz)])


def train(pc, R, E, steps=200, lr=1e-3, batch=8, seed=0, log_every=0, validate=None, every=20):
    """Adam on random mini-batches of the pairs.  With `validate` (a callable
    returning a score, lower is better, e.g. FGMRES iterations on a held-out
    right-hand side) the parameters with the best score, the initial ones
    included, are restored at the end.  Returns (loss history, validation log)."""
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    hist, vlog = [], []
    npairs = R.shape[0]
    best = None
    if validate is not None:
        best = (validate(), fb.fb_learned_params(pc))
        vlog.append((0, best[0]))
    for it in range(steps):
        idx = torch.randperm(npairs, generator=g)[:min(batch, npairs)].to(R.device)
        Rb = R.index_select(0, idx).contiguous()
        Eb = E.index_select(0, idx).contiguous()
        loss = fb.fb_learned_train_step(pc, Rb, Eb, lr)
        hist.append(loss)
        if log_every and it % log_every == 0:
            print(f"step {it} loss {loss:.4f}", flush=True)
        if validate is not None and ((it + 1) % every == 0 or it + 1 == steps):
            sc = validate()
            vlog.append((it + 1, sc))
            if sc < best[0]:
                best = (sc, fb.fb_learned_params(pc))
    if best is not None:
        fb.fb_learned_params(pc, best[1])
    return hist, vlog


def evaluate(pc, R, E):
    """Mean objective of the preconditioner on the pairs."""
    loss, _ = fb.fb_learned_loss_and_grad(pc, R.contiguous(), E.contiguous())
    return loss


def residual_error(A, pc, R):
    """Mean ||A P(r) - r|| / ||r|| over the rows of R: how far A P is from the
    identity on those inputs (what right-preconditioned GMRES sees)."""
    z = torch.empty_like(R[0])
    az = torch.empty_like(z)
    out = []
    for q in range(R.shape[0]):
        fb.fb_precond_apply(pc, R[q], z)
        fb.fb_operator_apply(A, z, az)
        out.append(((az - R[q]).norm() / R[q].norm()).item())
    return float(np.mean(out))
