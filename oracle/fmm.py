"""A plain FMM matvec for the BEM operators (oracle, test infrastructure).

Sec. 3.3: near pairs (elements in touching leaves) use the stored entries of
the dense collocation matrix; all other pairs go through multipole and local
expansions (Eq. shft0) and the RCR translations (rotation, coaxial
translation, back-rotation) of Sec. 3.3.1:
    P2M -> M2M (up) -> M2L (V-lists, levels 2..L) -> L2L (down) -> L2P.
Far pairs use the same 3-point rule as the dense matrix, so the FMM
approximates exactly that matrix.

Truncation order per level (not in the paper, which defers it to another
reference): the excess-bandwidth rule
    p_l = max(p_min, ceil(k r_l + 1.8 d0^(2/3) (k r_l)^(1/3))),  r_l = sqrt(3)/2 delta_l.

Source model of column j (element T_j with area A_j, normal n_j, 3-point
rule points y_jq and weights w_q):
    L : monopole          ->  C_n^m += ik A_j sum_q w_q R_n^{-m}(y_jq - c) x_j
    M : dipole along n_j  ->  C_n^m += ik A_j sum_q w_q n_j.grad R_n^{-m}(y_jq - c) x_j
    A : dipole + monopole with strength -ik beta_j (Eq. dbem4)
Targets: L, M, A evaluate D_n^m R_n^m(x_i - c); L' evaluates n_i.grad of it.
"""
from __future__ import annotations

import math

import numpy as np

from . import bem, sph
from .octree import Octree


def order_rule(k, delta, d0=6.0, pmin=9):
    """Expansion order of a level with box side delta.  The paper gives no
    truncation rule (it cites its FMM reference); this is that reference's
    excess-bandwidth form p = ceil(k r + 1.8 d0^(2/3) (k r)^(1/3)), r = the
    half-diagonal sqrt(3)/2 delta, d0 the number of accurate digits, and at
    least pmin."""
    kr = k * math.sqrt(3.0) / 2.0 * delta
    p = math.ceil(kr + 1.8 * d0 ** (2.0 / 3.0) * kr ** (1.0 / 3.0))
    return max(int(pmin), int(p))


def _neg_m_index(p):
    out = []
    for n in range(p):
        for m in range(-n, n + 1):
            out.append(sph.idx(n, -m))
    return np.array(out)


def p2m_operator(mesh, k, beta, elems, c, p, kind):
    """W [p^2, len(elems)]: C = W @ x[elems] for a box centred at c."""
    el = mesh.el
    pts = mesh.q3[elems]                       # [e,3,3]
    rel = pts - c[None, None, :]
    neg = _neg_m_index(p)
    W = np.zeros((p * p, len(elems)), np.complex128)
    w3 = mesh.w3
    if kind in ("L", "A", "LP"):
        R = sph.regular(p, k, rel)[neg]        # [p^2, e, 3]
        mono = np.ones(len(elems), np.complex128)
        if kind == "A":
            mono = -1j * k * np.asarray(beta)[elems]
        W += np.sum(R * w3[None, None, :], axis=2) * mono[None, :]
    if kind in ("M", "A"):
        gR = sph.grad_regular(p, k, rel)[neg]  # [p^2, e, 3, 3]
        nd = np.sum(gR * el.normal[elems][None, :, None, :], axis=-1)
        W += np.sum(nd * w3[None, None, :], axis=2)
    return 1j * k * W * el.area[elems][None, :]


def l2p_operator(mesh, k, elems, c, p, kind):
    """V [len(elems), p^2]: y[elems] += V @ D for a leaf centred at c."""
    el = mesh.el
    rel = el.centroid[elems] - c[None, :]
    if kind == "LP":
        gR = sph.grad_regular(p, k, rel)       # [p^2, e, 3]
        return np.sum(gR * el.normal[elems][None, :, :], axis=-1).T
    return sph.regular(p, k, rel).T


def near_entries(mesh, k, beta, rows, cols, kind):
    """Near-field block of operator `kind` (L, M, LP or the system matrix A
    of Eq. dbem4) for collocation rows at the elements `rows` and element
    columns `cols`, with the singular and near-singular rules of the dense
    operator (Sec. 3.3: near interactions are computed directly)."""
    L, M, LP = bem.operator_rows(mesh, k, mesh.el.centroid[rows], mesh.el.normal[rows],
                                 rows, cols)
    if kind == "L":
        return L
    if kind == "M":
        return M
    if kind == "LP":
        return LP
    A = M - 1j * k * L * np.asarray(beta)[cols][None, :]
    for a, r in enumerate(rows):
        hit = np.nonzero(cols == r)[0]
        if hit.size:
            A[a, hit[0]] += 0.5
    return A


class FMM:
    """FMM approximation of one operator (kind in L, M, LP, A)."""

    def __init__(self, mesh, k, beta=None, kind="A", leaf_max=64, d0=6.0, pmin=9,
                 verts=None, level=None):
        self.mesh, self.k, self.kind = mesh, k, kind
        self.beta = np.zeros(mesh.n) if beta is None else np.asarray(beta)
        el = mesh.el
        vv = np.concatenate([el.v0, el.v1, el.v2]) if verts is None else verts
        self.tree = T = Octree(vv, el.centroid, mesh.rc, leaf_max, level)
        self.L = T.L
        self.p = {l: order_rule(k, T.delta(l), d0, pmin) for l in range(2, T.L + 1)}
        self.centers = {l: T.centers(l) for l in range(0, T.L + 1)}
        leaf_elems = [T.perm[s:s + c] for s, c in zip(T.leaf_start, T.leaf_count)]
        self.leaf_elems = leaf_elems
        pL = self.p[T.L]
        cL = self.centers[T.L]
        self.W = [p2m_operator(mesh, k, self.beta, e, cL[b], pL, kind) for b, e in enumerate(leaf_elems)]
        self.V = [l2p_operator(mesh, k, e, cL[b], pL, kind) for b, e in enumerate(leaf_elems)]
        U = T.ulist()
        self.U = U
        self.near = {}
        for t in range(len(leaf_elems)):
            srcs = U[U[:, 0] == t, 1]
            cols = np.concatenate([leaf_elems[s] for s in srcs])
            self.near[t] = (cols, near_entries(mesh, k, self.beta, leaf_elems[t], cols, kind))
        self._cache = {}
        self._rot = {}
        self._coax = {}
        self.vl = {l: T.vlist(l) for l in range(2, T.L + 1)}
        self.par = {l: T.parent_index(l) for l in range(1, T.L + 1)}

    def _T(self, lev_out, lev_in, offset, kind):
        """Translation matrix for an offset that is an integer multiple of
        half the finer box size; rotation blocks cached per direction and
        coaxial coefficients per (levels, kind, |t|)."""
        h = self.tree.delta(max(lev_out, lev_in)) / 2.0
        ioff = tuple(int(v) for v in np.round(np.asarray(offset) / h))
        key = (lev_out, lev_in, ioff, kind)
        if key not in self._cache:
            g = math.gcd(math.gcd(abs(ioff[0]), abs(ioff[1])), abs(ioff[2]))
            dkey = tuple(v // g for v in ioff)
            pmax = max(self.p.values())
            if dkey not in self._rot:
                self._rot[dkey] = sph.rotation_blocks(sph.rotation_to_z(np.array(dkey, float)), pmax)
            p_out, p_in = self.p[lev_out], self.p[lev_in]
            ckey = (lev_out, lev_in, kind, ioff[0] ** 2 + ioff[1] ** 2 + ioff[2] ** 2)
            if ckey not in self._coax:
                tau = float(np.linalg.norm(np.array(ioff, float))) * h
                self._coax[ckey] = sph.coaxial(max(p_out, p_in), self.k * tau, kind)
            self._cache[key] = sph.translation(np.array(ioff, float) * h, self.k, p_out, p_in,
                                               kind, rot=self._rot[dkey], coax=self._coax[ckey])
        return self._cache[key]

    def matvec(self, x):
        """y = (operator) x by the passes of Sec. 3.3: near field per leaf,
        P2M at the leaves, M2M upward, M2L over the interaction lists, L2L
        downward, L2P at the leaves."""
        x = np.asarray(x, np.complex128)
        T, L = self.tree, self.L
        y = np.zeros(self.mesh.n, np.complex128)
        for t, (cols, A) in self.near.items():
            y[self.leaf_elems[t]] += A @ x[cols]
        if L < 2:
            return y
        C = {L: np.stack([W @ x[e] for W, e in zip(self.W, self.leaf_elems)])}
        for lev in range(L - 1, 1, -1):
            pc = self.par[lev + 1]
            Cp = np.zeros((len(T.levels[lev]), self.p[lev] ** 2), np.complex128)
            for ch, par in enumerate(pc):
                off = self.centers[lev][par] - self.centers[lev + 1][ch]
                Cp[par] += self._T(lev, lev + 1, off, "RR") @ C[lev + 1][ch]
            C[lev] = Cp
        D = {}
        for lev in range(2, L + 1):
            Dl = np.zeros((len(T.levels[lev]), self.p[lev] ** 2), np.complex128)
            for t, s in self.vl[lev]:
                off = self.centers[lev][t] - self.centers[lev][s]
                Dl[t] += self._T(lev, lev, off, "SR") @ C[lev][s]
            if lev > 2:
                for ch, par in enumerate(self.par[lev]):
                    off = self.centers[lev][ch] - self.centers[lev - 1][par]
                    Dl[ch] += self._T(lev, lev - 1, off, "RR") @ D[lev - 1][par]
            D[lev] = Dl
        for b, e in enumerate(self.leaf_elems):
            y[e] += self.V[b] @ D[L][b]
        return y
