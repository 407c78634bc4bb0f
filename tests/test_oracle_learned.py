"""Pins for the FP64 reference of the learned preconditioner network: the
hand-written reverse pass against central finite differences, and the
initial state z = BJ(v) when the output layer is zero."""
import numpy as np

from oracle import bem, learned
from oracle.octree import Octree
from paper_2103_16073_gb300 import workloads as W

BETA, K = None, 0.0   # admittance and wavenumber features (set by _setup)


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
    global BETA, K
    BETA = rng.uniform(0.05, 0.5, n) + 1j * rng.uniform(-0.1, 0.1, n)
    K = 7.0
    return T, r, e, u, el.normal, theta


def test_gradient_matches_finite_differences():
    T, r, e, u, nrm, theta = _setup()
    assert T.L == 3
    loss, g = learned.loss_grad(theta, T, r, e, u, nrm, beta=BETA, k=K)
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(6):
        d = rng.standard_normal(theta.size)
        lp, _ = learned.loss_grad(theta + h * d, T, r, e, u, nrm, beta=BETA, k=K)
        lm, _ = learned.loss_grad(theta - h * d, T, r, e, u, nrm, beta=BETA, k=K)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g @ d) < 1e-6 * max(1.0, abs(fd))
    # single-block directions too (weights of every layer are reached)
    lay, _ = learned.layout()
    for name, j in (("W0", None), ("W0", 8 * 64 + 5), ("W0", 9 * 64 + 17), ("W0", 10 * 64 + 40), ("Wu0", None),
                    ("Wd2", None), ("Wh", None), ("Wo", None), ("bo", None)):
        o, n = lay[name]
        j = n // 3 if j is None else j
        d = np.zeros(theta.size)
        d[o + j] = 1.0
        lp, _ = learned.loss_grad(theta + h * d, T, r, e, u, nrm, beta=BETA, k=K)
        lm, _ = learned.loss_grad(theta - h * d, T, r, e, u, nrm, beta=BETA, k=K)
        assert abs((lp - lm) / (2 * h) - g[o + j]) < 1e-6 * max(1.0, abs(g[o + j]))


def test_zero_output_layer_is_block_jacobi():
    T, r, e, u, nrm, theta = _setup()
    lay, _ = learned.layout()
    for name in ("Wo", "bo"):
        o, n = lay[name]
        theta[o:o + n] = 0.0
    z, _ = learned.forward(theta, T, r, u, nrm, BETA, K)
    assert np.max(np.abs(z - u)) == 0.0


def test_complex_homogeneous():
    """The network's input normalisation (rms scale, phase of sum v) makes the
    map commute with complex scaling, as a linear preconditioner does."""
    T, r, e, u, nrm, theta = _setup()
    z, _ = learned.forward(theta, T, r, u, nrm, BETA, K)
    for a in (2.5, -1.0, 1j, 0.3 * np.exp(2.1j)):
        za, _ = learned.forward(theta, T, a * r, a * u, nrm, BETA, K)
        assert np.max(np.abs(za - a * z)) < 1e-12 * abs(a) * np.max(np.abs(z))
    # and the map is not linear (the network is not a fixed matrix)
    r2 = np.roll(r, 7)
    u2 = np.roll(u, 7)
    z2, _ = learned.forward(theta, T, r2, u2, nrm, BETA, K)
    z12, _ = learned.forward(theta, T, r + r2, u + u2, nrm, BETA, K)
    assert np.max(np.abs(z12 - z - z2)) > 1e-3 * np.max(np.abs(z))


def _dense_small():
    v, t, _ = W.shoebox_mesh(1.0, 0.8, 0.6, 8, 6, 5)
    mesh = bem.Mesh(v, t)
    k = 4.0
    beta = np.full(mesh.n, 0.2 + 0.05j)
    L, M, LP = bem.dense_operators(mesh, k)
    return mesh, k, beta, L, LP, bem.system_matrix(L, M, k, beta)


def test_residual_objective_exact_adjoint_gradient():
    """With the exact A^H the residual objective's reverse pass is the exact
    gradient: central differences agree, and the loss is its definition."""
    T, r, e, u, nrm, theta = _setup()
    mesh, k, beta, L, LP, A = _dense_small()
    assert mesh.n == r.size
    AH = A.conj().T
    adj = lambda w: AH @ w
    loss, g = learned.loss_grad(theta, T, r, e, u, nrm, "residual", A, adj, beta=BETA, k=K)
    z, _ = learned.forward(theta, T, r, u, nrm, BETA, K)
    assert abs(loss - np.linalg.norm(A @ z - r) ** 2 / np.linalg.norm(r) ** 2) < 1e-12 * loss
    rng = np.random.default_rng(3)
    h = 1e-6
    for _ in range(4):
        d = rng.standard_normal(theta.size)
        lp, _ = learned.loss_grad(theta + h * d, T, r, e, u, nrm, "residual", A, adj, beta=BETA, k=K)
        lm, _ = learned.loss_grad(theta - h * d, T, r, e, u, nrm, "residual", A, adj, beta=BETA, k=K)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g @ d) < 1e-6 * max(1.0, abs(fd))


def test_approximate_adjoint_is_close():
    """The matrix-free stand-in for A^H (single- and adjoint-double-layer with
    area scaling) is within a few percent of the exact adjoint, and its
    surrogate gradient points downhill (positive inner product with the exact
    gradient)."""
    T, r, e, u, nrm, theta = _setup()
    mesh, k, beta, L, LP, A = _dense_small()
    adj = learned.approx_adjoint(L, LP, mesh.el.area, beta, k)
    rng = np.random.default_rng(2)
    w = rng.standard_normal(mesh.n) + 1j * rng.standard_normal(mesh.n)
    ex = A.conj().T @ w
    assert np.linalg.norm(adj(w) - ex) / np.linalg.norm(ex) < 0.1
    _, g_ex = learned.loss_grad(theta, T, r, e, u, nrm, "residual", A, lambda x: A.conj().T @ x, beta=BETA, k=K)
    _, g_ap = learned.loss_grad(theta, T, r, e, u, nrm, "residual", A, adj, beta=BETA, k=K)
    assert g_ap @ g_ex > 0.9 * np.linalg.norm(g_ap) * np.linalg.norm(g_ex)


def test_trained_network_gain_on_held_out_sources():
    """What the trained network gains, in FP64 on a dense operator (956
    elements, 300 Hz, leaves of <= 32): trained with Adam on the residual
    objective (exact adjoint) over the preconditioner inputs of block-Jacobi
    FGMRES solves for 8 sources, it fits them (mean residual loss well below
    block Jacobi's) and FGMRES, which admits the changing preconditioner,
    still converges on 3 held-out sources within two iterations of block
    Jacobi, and in all no more than block Jacobi.  Measured: residual loss
    0.77 -> 0.35, iterations 25, 25, 24 -> 24, 24, 23 (at 700 Hz the same
    recipe gives 56, 54, 58 -> 55-56, 53, 56-57): halving the mean residual
    of the training inputs buys about one iteration."""
    import math
    from oracle.fgmres import fgmres
    v, t, _ = W.shoebox_mesh(1.3, 1.1, 0.9, 11, 9, 7)
    mesh = bem.Mesh(v, t)
    n, k = mesh.n, 2 * math.pi * 300.0 / 343.0
    beta = np.full(n, 0.05 + 0.0j)
    Lm, Mm, _ = bem.dense_operators(mesh, k)
    A = bem.system_matrix(Lm, Mm, k, beta)
    el = mesh.el
    T = learned.TreeInfo(Octree(np.concatenate([el.v0, el.v1, el.v2]), el.centroid, mesh.rc, 32))
    blocks = []
    for b in range(len(T.leaf_start) - 1):
        idx = T.perm[T.leaf_start[b]:T.leaf_start[b + 1]]
        blocks.append((idx, np.linalg.inv(A[np.ix_(idx, idx)])))

    def bj(x):
        u = np.zeros_like(x)
        for idx, Bi in blocks:
            u[idx] = Bi @ x[idx]
        return u

    rng = np.random.default_rng(5)
    sources = [np.array([0.2, 0.2, 0.2]) + rng.uniform(0, 1, 3) * np.array([0.9, 0.7, 0.5]) for _ in range(11)]
    rhs = [Lm @ bem.gamma_monopole(mesh, k, beta, xs) for xs in sources]

    def solve(b, pc, log=None):
        def p(x):
            if log is not None:
                log.append(x.copy())
            return pc(x)
        return fgmres(lambda x: A @ x, b, tol=1e-6, restart=40, precond=p)[1]["iters"]

    inputs = []
    for b in rhs[:8]:
        solve(b, bj, inputs)
    U = [bj(x) for x in inputs]
    lay, total = learned.layout()
    theta = rng.standard_normal(total) * 0.05
    for name in ("Wo", "bo"):
        o, nn = lay[name]
        theta[o:o + nn] = 0.0
    adj = lambda w: A.conj().T @ w
    m1, m2 = np.zeros(total), np.zeros(total)
    for it in range(1, 201):
        g = np.zeros(total)
        for q in rng.choice(len(inputs), 8, replace=False):
            g += learned.loss_grad(theta, T, inputs[q], None, U[q], el.normal, "residual", A, adj, beta, k)[1] / 8
        m1 = 0.9 * m1 + 0.1 * g
        m2 = 0.999 * m2 + 0.001 * g * g
        theta -= 1e-3 * (m1 / (1 - 0.9 ** it)) / (np.sqrt(m2 / (1 - 0.999 ** it)) + 1e-8)
    loss_bj = np.mean([np.linalg.norm(A @ u - x) ** 2 / np.linalg.norm(x) ** 2 for x, u in zip(inputs, U)])
    loss_net = np.mean([learned.loss_grad(theta, T, x, None, u, el.normal, "residual", A, adj, beta, k)[0]
                        for x, u in zip(inputs, U)])
    net = lambda x: learned.forward(theta, T, x, bj(x), el.normal, beta, k)[0]
    it_bj = [solve(b, bj) for b in rhs[8:]]
    it_net = [solve(b, net) for b in rhs[8:]]
    print(f"residual loss: block Jacobi {loss_bj:.3f}, trained network {loss_net:.3f}; "
          f"held-out FGMRES iterations: block Jacobi {it_bj}, network {it_net}")
    assert loss_net < 0.7 * loss_bj
    assert all(a <= b + 2 for a, b in zip(it_net, it_bj))
    assert sum(it_net) <= sum(it_bj)


def test_coarse_correction_reaches_the_slow_directions():
    """Where the network's iterations go (same 956-element shoebox, dense FP64
    operator): a Galerkin coarse correction on per-leaf constant and linear
    functions added to block Jacobi, z = u + P (P^H A P)^+ P^H (v - A u),
    u = BJ(v), cuts the FGMRES iterations several-fold (measured 24-25 -> 6
    at 300 Hz, 50-54 -> 10-11 at 700 Hz, restart 60), so the directions that set the
    iteration count are smooth at the leaf scale: a correction of that form,
    not a per-element one, is what shortens the solve."""
    import math
    from oracle.fgmres import fgmres
    v, t, _ = W.shoebox_mesh(1.3, 1.1, 0.9, 11, 9, 7)
    mesh = bem.Mesh(v, t)
    n, k = mesh.n, 2 * math.pi * 700.0 / 343.0
    beta = np.full(n, 0.05 + 0.0j)
    Lm, Mm, _ = bem.dense_operators(mesh, k)
    A = bem.system_matrix(Lm, Mm, k, beta)
    el = mesh.el
    T = learned.TreeInfo(Octree(np.concatenate([el.v0, el.v1, el.v2]), el.centroid, mesh.rc, 32))
    blocks, cols = [], []
    for b in range(len(T.leaf_start) - 1):
        idx = T.perm[T.leaf_start[b]:T.leaf_start[b + 1]]
        blocks.append((idx, np.linalg.inv(A[np.ix_(idx, idx)])))
        c = el.centroid[idx] - el.centroid[idx].mean(0)
        for f in (np.ones(len(idx)), c[:, 0], c[:, 1], c[:, 2]):
            col = np.zeros(n, np.complex128)
            col[idx] = f
            cols.append(col)
    P = np.array(cols).T
    Aci = np.linalg.pinv(P.conj().T @ A @ P, rcond=1e-12)

    def bj(x):
        u = np.zeros_like(x)
        for idx, Bi in blocks:
            u[idx] = Bi @ x[idx]
        return u

    def two_level(x):
        u = bj(x)
        return u + P @ (Aci @ (P.conj().T @ (x - A @ u)))

    rng = np.random.default_rng(5)
    its_bj, its_2 = [], []
    for _ in range(3):
        xs = np.array([0.2, 0.2, 0.2]) + rng.uniform(0, 1, 3) * np.array([0.9, 0.7, 0.5])
        b = Lm @ bem.gamma_monopole(mesh, k, beta, xs)
        its_bj.append(fgmres(lambda x: A @ x, b, tol=1e-6, restart=60, precond=bj)[1]["iters"])
        its_2.append(fgmres(lambda x: A @ x, b, tol=1e-6, restart=60, precond=two_level)[1]["iters"])
    print(f"700 Hz FGMRES iterations: block Jacobi {its_bj}, with the coarse correction {its_2}")
    assert all(3 * a <= b for a, b in zip(its_2, its_bj))
