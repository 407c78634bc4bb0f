"""Pin: the oracle FMM (P2M, M2M, M2L, L2L, L2P with the RCR translations)
reproduces the dense collocation operators to the accuracy its truncation
allows; the per-leaf P2M operator reproduces the far field of its elements."""
import numpy as np
import pytest

from oracle import bem, fmm, sph
from paper_2103_16073_gb300 import workloads as W


@pytest.fixture(scope="module")
def small():
    wl = W.shoebox_workload("t", 3.0, 2.4, 2.0, (12, 10, 8), 250.0, 0.2, (0.7, 0.6, 0.5), 4, 0)
    mesh = bem.Mesh(wl.verts, wl.tris)
    L, M, LP = bem.dense_operators(mesh, wl.k)
    return wl, mesh, dict(L=L, M=M, LP=LP, A=bem.system_matrix(L, M, wl.k, wl.beta))


@pytest.mark.parametrize("kind", ["A", "L", "M", "LP"])
def test_fmm_matches_dense(small, kind):
    wl, mesh, mats = small
    F = fmm.FMM(mesh, wl.k, wl.beta, kind=kind, d0=6, pmin=12)
    assert F.L >= 2
    rng = np.random.default_rng(0)
    x = rng.standard_normal(mesh.n) + 1j * rng.standard_normal(mesh.n)
    y = F.matvec(x)
    yd = mats[kind] @ x
    assert np.linalg.norm(y - yd) / np.linalg.norm(yd) < 1e-5


def test_p2m_far_field(small):
    """C = W x for one leaf; sum_nm C_n^m S_n^m(x - c) equals the 3-point-rule
    far-field sum of A's columns for that leaf at a far point."""
    wl, mesh, _ = small
    F = fmm.FMM(mesh, wl.k, wl.beta, kind="A", d0=6, pmin=12)
    b = 3
    e = F.leaf_elems[b]
    c = F.centers[F.L][b]
    p = F.p[F.L]
    W_ = fmm.p2m_operator(mesh, wl.k, wl.beta, e, c, p + 14, "A")
    rng = np.random.default_rng(1)
    x = rng.standard_normal(len(e)) + 1j * rng.standard_normal(len(e))
    xt = c + np.array([1.1, -0.9, 0.8])
    S = sph.singular(p + 14, wl.k, xt - c)
    val = S @ (W_ @ x)
    el = mesh.el
    g, dny, _ = bem._kernels(xt[None, None, :], mesh.q3[e], el.normal[e][:, None, :],
                             np.zeros((1, 1, 3)), wl.k, smooth=False)
    direct = np.sum(el.area[e] * np.sum(mesh.w3 * (dny - 1j * wl.k * wl.beta[e][:, None] * g), axis=1) * x)
    assert abs(val - direct) < 1e-10 * abs(direct)
