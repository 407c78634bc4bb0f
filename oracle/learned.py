"""FP64 reference of the learned octree preconditioner network (oracle,
test infrastructure).

The network refines block Jacobi, z = u + s N(F), u = BJ(v), s = rms(v), and
is applied as the variable right preconditioner flexible GMRES admits
(Sec. 3.1, Sec. 4).  Layout of the flat parameter vector (FP32 on the GPU,
FP64 here), weights W as [in x out] with Y = X W + b:
    W0[11x64] b0[64] | Wu_k[64x64] bu_k[64] (k=0..2) | Wd_k[128x64] bd_k[64]
    (k=0..2) | Wh[128x64] bh[64] | Wo[64x2] bo[2]
Forward (elements in tree order, SiLU activations):
    F = [Re v', Im v', Re u', Im u', n_x, n_y, n_z, 1, Re beta, Im beta, k delta_L],
        v' = conj(ph) v / s, u' = conj(ph) u / s, s = rms(v),
        ph = sum(v) / |sum(v)| (1 if zero), beta the element's admittance,
        k delta_L the wavenumber times the leaf box side (so one network can
        serve several frequencies and wall materials)
    H0 = silu(F W0 + b0);  G_L = leaf means of H0
    G_l = silu(mean over children of G_{l+1} Wu_k + bu_k),  l = L-1-k
    D_{L-3} = G_{L-3};  D_l = silu([G_l, D_{l-1}[parent]] Wd_k + bd_k),  l = L-2+k
    H1 = silu([H0, D_L[leaf]] Wh + bh);  O = H1 Wo + bo
    z = u + s ph (O_0 + i O_1)      (so z(a v) = a z(v) for complex a)
Objectives for a pair (r, e) with A e = r:
    error:     ||z(r) - e||^2 / ||e||^2
    residual:  ||A z(r) - r||^2 / ||r||^2   (what right-preconditioned GMRES
               sees: the residual the correction leaves)
``loss_grad`` returns the loss and the FP64 gradient by reverse-mode
differentiation written out layer by layer.  For the residual objective the
pull-back through A uses the adjoint passed in (the exact A^H gives the exact
gradient; ``approx_adjoint`` gives the stand-in a matrix-free code can apply).
"""
from __future__ import annotations

import numpy as np

HW, NF, DEPTH = 64, 11, 3


def layout():
    """Offsets of the named weight and bias blocks in the flat parameter
    vector (the layout above) and its total length."""
    sizes = [("W0", NF * HW), ("b0", HW)]
    for k in range(DEPTH):
        sizes += [(f"Wu{k}", HW * HW), (f"bu{k}", HW)]
    for k in range(DEPTH):
        sizes += [(f"Wd{k}", 2 * HW * HW), (f"bd{k}", HW)]
    sizes += [("Wh", 2 * HW * HW), ("bh", HW), ("Wo", HW * 2), ("bo", 2)]
    off, out = 0, {}
    for name, n in sizes:
        out[name] = (off, n)
        off += n
    return out, off


def unpack(theta):
    """The flat parameter vector as named FP64 arrays (weights [in x out])."""
    lay, _ = layout()
    shapes = {"W0": (NF, HW), "Wh": (2 * HW, HW), "Wo": (HW, 2)}
    for k in range(DEPTH):
        shapes[f"Wu{k}"] = (HW, HW)
        shapes[f"Wd{k}"] = (2 * HW, HW)
    P = {}
    for name, (o, n) in lay.items():
        a = np.asarray(theta[o:o + n], dtype=np.float64)
        P[name] = a.reshape(shapes[name]) if name in shapes else a
    return P


def silu(x):
    """SiLU activation x / (1 + e^{-x})."""
    return x / (1.0 + np.exp(-x))


def silu_grad(x):
    """Derivative of SiLU: s (1 + x (1 - s)), s = 1 / (1 + e^{-x})."""
    s = 1.0 / (1.0 + np.exp(-x))
    return s * (1.0 + x * (1.0 - s))


class TreeInfo:
    """What the network needs from the octree (tree order = elements sorted
    by leaf): leaf of each sorted position, leaf ranges, parents per level."""

    def __init__(self, tree):
        self.L = tree.L
        self.perm = tree.perm
        self.n = tree.perm.size
        self.leaf_start = np.append(tree.leaf_start, self.n)
        self.leaf_of = np.repeat(np.arange(len(tree.leaf_start)), tree.leaf_count)
        self.nbox = {l: len(tree.levels[l]) for l in range(tree.L + 1)}
        self.parent = {l: tree.parent_index(l) for l in range(1, tree.L + 1)}
        self.leaf_side = tree.delta(tree.L)


def _segmean(X, seg_id, nseg):
    out = np.zeros((nseg, X.shape[1]))
    np.add.at(out, seg_id, X)
    cnt = np.bincount(seg_id, minlength=nseg).astype(float)
    return out / np.maximum(cnt, 1)[:, None], cnt


def forward(theta, T, v, u, normals, beta=None, k=0.0):
    """z (element order) and a cache for the backward pass.  beta: admittance
    per element (zero when None); k: wavenumber."""
    P = unpack(theta)
    n, L = T.n, T.L
    depth = min(DEPTH, L)
    top = L - depth
    s = np.sqrt(np.mean(np.abs(v) ** 2))
    inv = 1.0 / s if s > 0 else 0.0
    tot = np.sum(v)
    ph = tot / abs(tot) if abs(tot) > 0 else 1.0 + 0j
    rot = np.conj(ph) * inv
    vp, up, nrm = v[T.perm] * rot, u[T.perm] * rot, normals[T.perm]
    b = np.zeros(n, np.complex128) if beta is None else np.broadcast_to(np.asarray(beta, np.complex128), (n,))[T.perm]
    F = np.column_stack([vp.real, vp.imag, up.real, up.imag, nrm, np.ones(n), b.real, b.imag,
                         np.full(n, k * T.leaf_side)])
    c = {"F": F, "s": s, "ph": ph}
    c["pre0"] = F @ P["W0"] + P["b0"]
    H0 = silu(c["pre0"])
    c["H0"] = H0
    G = {}
    G[L], c["leafcnt"] = _segmean(H0, T.leaf_of, T.nbox[L])
    c["preu"], c["Pm"], c["childcnt"] = {}, {}, {}
    for k, l in enumerate(range(L - 1, top - 1, -1)):
        Pm, cnt = _segmean(G[l + 1], T.parent[l + 1], T.nbox[l])
        c["Pm"][l], c["childcnt"][l] = Pm, cnt
        c["preu"][l] = Pm @ P[f"Wu{k}"] + P[f"bu{k}"]
        G[l] = silu(c["preu"][l])
    D = {top: G[top]}
    c["Cc"], c["pred"] = {}, {}
    for k, l in enumerate(range(top + 1, L + 1)):
        C = np.hstack([G[l], D[l - 1][T.parent[l]]])
        c["Cc"][l] = C
        c["pred"][l] = C @ P[f"Wd{k}"] + P[f"bd{k}"]
        D[l] = silu(c["pred"][l])
    E = np.hstack([H0, D[L][T.leaf_of]])
    c["E"] = E
    c["preh"] = E @ P["Wh"] + P["bh"]
    H1 = silu(c["preh"])
    c["H1"] = H1
    O = H1 @ P["Wo"] + P["bo"]
    zp = u[T.perm] + s * ph * (O[:, 0] + 1j * O[:, 1])
    z = np.empty(n, np.complex128)
    z[T.perm] = zp
    c.update(G=G, D=D, depth=depth, top=top)
    return z, c


def approx_adjoint(L, LP, area, beta, k):
    """Stand-in for A^H, A = I/2 + M - i k L diag(beta), built from the single-
    and adjoint-double-layer operators.  With one collocation point per flat
    element the far-field entries satisfy M_ij ~ L'_ji a_j / a_i and
    L_ij ~ L_ji a_j / a_i (the kernels are the same function of the centroid
    pair), so with D = diag(area)
        A^H ~ I/2 + D conj(L') D^-1 + i k conj(beta) D conj(L) D^-1,
    where conj(X) y = conj(X conj(y))."""
    def apply(w):
        y = np.conj(w / area)
        return 0.5 * w + area * np.conj(LP @ y) + 1j * k * np.conj(beta) * area * np.conj(L @ y)
    return apply


def loss_grad(theta, T, r, e, u, normals, objective="error", A=None, adjoint=None, beta=None, k=0.0):
    """(loss, gradient) for one pair; gradient in the flat layout.  The
    residual objective needs A (matrix) and adjoint (callable w -> ~A^H w)."""
    P = unpack(theta)
    z, c = forward(theta, T, r, u, normals, beta, k)
    L, top, depth = T.L, c["top"], c["depth"]
    if objective == "error":
        e2 = np.sum(np.abs(e) ** 2)
        d = z - e
        loss = np.sum(np.abs(d) ** 2) / e2
        dz = 2.0 * d / e2
    elif objective == "residual":
        r2 = np.sum(np.abs(r) ** 2)
        w = A @ z - r
        loss = np.sum(np.abs(w) ** 2) / r2
        dz = 2.0 * adjoint(w) / r2
    else:
        raise ValueError(objective)
    dzp = dz[T.perm] * np.conj(c["ph"])
    dO = c["s"] * np.column_stack([dzp.real, dzp.imag])
    g = {}
    g["Wo"] = c["H1"].T @ dO
    g["bo"] = dO.sum(0)
    dH1 = dO @ P["Wo"].T
    dph = dH1 * silu_grad(c["preh"])
    g["Wh"] = c["E"].T @ dph
    g["bh"] = dph.sum(0)
    dE = dph @ P["Wh"].T
    dH0 = dE[:, :HW].copy()
    dD = {l: np.zeros((T.nbox[l], HW)) for l in range(top, L + 1)}
    dG = {l: np.zeros((T.nbox[l], HW)) for l in range(top, L + 1)}
    np.add.at(dD[L], T.leaf_of, dE[:, HW:])
    for k, l in reversed(list(enumerate(range(top + 1, L + 1)))):
        dp = dD[l] * silu_grad(c["pred"][l])
        g[f"Wd{k}"] = c["Cc"][l].T @ dp
        g[f"bd{k}"] = dp.sum(0)
        dC = dp @ P[f"Wd{k}"].T
        dG[l] += dC[:, :HW]
        np.add.at(dD[l - 1], T.parent[l], dC[:, HW:])
    dG[top] += dD[top]
    for k, l in reversed(list(enumerate(range(L - 1, top - 1, -1)))):
        dp = dG[l] * silu_grad(c["preu"][l])
        g[f"Wu{k}"] = c["Pm"][l].T @ dp
        g[f"bu{k}"] = dp.sum(0)
        dPm = dp @ P[f"Wu{k}"].T
        dG[l + 1] += dPm[T.parent[l + 1]] / c["childcnt"][l][T.parent[l + 1]][:, None]
    dH0 += dG[L][T.leaf_of] / c["leafcnt"][T.leaf_of][:, None]
    dp0 = dH0 * silu_grad(c["pre0"])
    g["W0"] = c["F"].T @ dp0
    g["b0"] = dp0.sum(0)
    lay, total = layout()
    flat = np.zeros(total)
    for name, (o, nn) in lay.items():
        if name in g:
            flat[o:o + nn] = np.asarray(g[name]).ravel()
    return loss, flat


def block_jacobi(A_rows_fn, T, v):
    """u = BJ(v): per leaf, solve the leaf's self block of the system matrix.
    A_rows_fn(rows, cols) returns the dense block of A."""
    u = np.zeros_like(v)
    for b in range(len(T.leaf_start) - 1):
        idx = T.perm[T.leaf_start[b]:T.leaf_start[b + 1]]
        u[idx] = np.linalg.solve(A_rows_fn(idx, idx), v[idx])
    return u
