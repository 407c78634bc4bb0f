"""Pins for the FP64 reference of the learned preconditioner network: the
hand-written reverse pass against central finite differences, and the
initial state z = BJ(v) when the output layer is zero."""
import numpy as np

from oracle import bem, learned
from oracle.octree import Octree
from paper_2103_16073_gb300 import workloads as W


def _setup():
    v, t, _ = W.shoebox_mesh(1.0, 0.8, 0.6, 8, 6, 5)
    mesh = bem.Mesh(v, t)
    el = mesh.el
    tree = Octree(np.concatenate([el.v0, el.v1, el.v2]), el.centroid, mesh.rc, 8, level=3)
    T = learned.TreeInfo(tree)
    rng = np.random.default_rng(0)
    n = mesh.n
    r = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    e = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    u = 0.7 * r + 0.1j * r
    _, total = learned.layout()
    theta = rng.standard_normal(total) * 0.2
    return T, r, e, u, el.normal, theta


def test_gradient_matches_finite_differences():
    T, r, e, u, nrm, theta = _setup()
    assert T.L == 3
    loss, g = learned.loss_grad(theta, T, r, e, u, nrm)
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(6):
        d = rng.standard_normal(theta.size)
        lp, _ = learned.loss_grad(theta + h * d, T, r, e, u, nrm)
        lm, _ = learned.loss_grad(theta - h * d, T, r, e, u, nrm)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g @ d) < 1e-6 * max(1.0, abs(fd))
    # single-block directions too (weights of every layer are reached)
    lay, _ = learned.layout()
    for name in ("W0", "Wu0", "Wd2", "Wh", "Wo", "bo"):
        o, n = lay[name]
        d = np.zeros(theta.size)
        d[o + n // 3] = 1.0
        lp, _ = learned.loss_grad(theta + h * d, T, r, e, u, nrm)
        lm, _ = learned.loss_grad(theta - h * d, T, r, e, u, nrm)
        assert abs((lp - lm) / (2 * h) - g[o + n // 3]) < 1e-6 * max(1.0, abs(g[o + n // 3]))


def test_zero_output_layer_is_block_jacobi():
    T, r, e, u, nrm, theta = _setup()
    lay, _ = learned.layout()
    for name in ("Wo", "bo"):
        o, n = lay[name]
        theta[o:o + n] = 0.0
    z, _ = learned.forward(theta, T, r, u, nrm)
    assert np.max(np.abs(z - u)) == 0.0
