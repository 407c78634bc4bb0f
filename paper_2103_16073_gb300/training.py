"""Training driver of the learned octree preconditioner.

Orchestration only: every step runs in the library (FGMRES solves, operator
applications, the network's forward/backward kernels and Adam).  Pairs
(r, e) come from the plain method's own solves: FGMRES with block Jacobi is
stopped after j iterations for several j, giving iterates x_j with
r_j = b - A x_j and e_j = x* - x_j, where x* is the converged solution, so
A e_j = r_j holds for the operator A the preconditioner will serve.
"""
from __future__ import annotations

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


def train(pc, R, E, steps=200, lr=1e-3, batch=8, seed=0, log_every=0):
    """Adam on random mini-batches of the pairs; returns the loss history."""
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    hist = []
    npairs = R.shape[0]
    for it in range(steps):
        idx = torch.randperm(npairs, generator=g)[:min(batch, npairs)].to(R.device)
        Rb = R.index_select(0, idx).contiguous()
        Eb = E.index_select(0, idx).contiguous()
        loss = fb.fb_learned_train_step(pc, Rb, Eb, lr)
        hist.append(loss)
        if log_every and it % log_every == 0:
            print(f"step {it} loss {loss:.4f}", flush=True)
    return hist


def evaluate(pc, R, E):
    """Mean relative squared error of the preconditioner on the pairs."""
    loss, _ = fb.fb_learned_loss_and_grad(pc, R.contiguous(), E.contiguous())
    return loss
