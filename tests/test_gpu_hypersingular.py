"""Hypersingular operator M' (Eq. ibem3) on the GPU: the dense FP64 path
against the oracle's dense matrix (same entry rule), and the FMM (FP64 and
mixed) against it; the FMM tolerance is stated here: the kernel has
derivatives on both sides, so its truncation error is larger than L's."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16073_gb300 as fb
from _cases import oracle_mesh, rel, seeded_vector, workload


@functools.lru_cache(maxsize=None)
def oracle_mp(name):
    from oracle import hypersingular as hs
    return hs.dense_mp(oracle_mesh(name), workload(name).k)


@pytest.fixture(scope="module", params=["small", "ragged"])
def case(request):
    wl = workload(request.param)
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = fb.fb_tree_build(mesh, 64)
    yield request.param, wl, mesh, tree
    fb.fb_tree_destroy(tree)
    fb.fb_mesh_destroy(mesh)


def _apply(op, x):
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    fb.fb_operator_apply(op, xd, yd)
    return yd.cpu().numpy()


def test_dense_matches_oracle(case):
    name, wl, mesh, tree = case
    op = fb.fb_operator_create(mesh, None, wl.k, fb.FB_OP_MP, fb.FB_PREC_FP64_DENSE, 6.0, 12)
    try:
        MP = oracle_mp(name)
        for s in (1, 2):
            x = seeded_vector(wl.n, 900 + s)
            assert rel(_apply(op, x), MP @ x) < 1e-12
    finally:
        fb.fb_operator_destroy(op)


@pytest.mark.parametrize("pmin", [14, 16])
def test_fmm_matches_oracle(case, pmin):
    name, wl, mesh, tree = case
    MP = oracle_mp(name)
    x = seeded_vector(wl.n, 950)
    ref = MP @ x
    errs = {}
    for prec in (fb.FB_PREC_FP64_FMM, fb.FB_PREC_MIXED_FMM):
        op = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_MP, prec, 6.0, pmin)
        try:
            errs[prec] = rel(_apply(op, x), ref)
        finally:
            fb.fb_operator_destroy(op)
    print(name, "pmin", pmin, "FP64 FMM", errs[fb.FB_PREC_FP64_FMM], "mixed", errs[fb.FB_PREC_MIXED_FMM])
    tol = 1e-5
    assert errs[fb.FB_PREC_FP64_FMM] < tol
    assert errs[fb.FB_PREC_MIXED_FMM] < tol


def test_mixed_refuses_orders_beyond_fp32_range(case):
    """At p = 18 on the low-frequency small room the coaxial coefficients pass
    the FP32 range: the mixed operator is refused, the FP64 one works."""
    name, wl, mesh, tree = case
    if name != "small":
        pytest.skip("low-frequency case only")
    with pytest.raises(fb.FBError):
        fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_L, fb.FB_PREC_MIXED_FMM, 6.0, 18)
    op = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_L, fb.FB_PREC_FP64_FMM, 6.0, 18)
    fb.fb_operator_destroy(op)
