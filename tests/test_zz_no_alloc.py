"""fb_operator_apply_noalloc: the FMM matvec for callers that cannot allocate
device memory when they apply an operator (stream capture, real-time
callbacks, fixed memory arenas).  Its expansion scratch lives in the
library's static device buffer; its output must match fb_operator_apply on
consecutive calls (the buffer keeps the previous call's contents, which the
call must clear).  Collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16073_gb300 as fb
from _cases import rel, seeded_vector, workload


@pytest.fixture(scope="module")
def setup():
    wl = workload("small")
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = fb.fb_tree_build(mesh, 64)
    ops = {
        "mixed": fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 6.0, 12),
        "fp64": fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_FP64_FMM, 6.0, 12),
        "dense": fb.fb_operator_create(mesh, None, wl.k, fb.FB_OP_A, fb.FB_PREC_FP64_DENSE),
    }
    yield wl, ops
    for op in ops.values():
        fb.fb_operator_destroy(op)
    fb.fb_tree_destroy(tree)
    fb.fb_mesh_destroy(mesh)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("mixed", 1e-5)])
def test_noalloc_matches_apply_on_consecutive_calls(setup, prec, tol):
    wl, ops = setup
    op = ops[prec]
    for seed in (21, 22):   # two calls in a row, different inputs
        x = torch.tensor(seeded_vector(wl.n, seed), device="cuda")
        y_ref = torch.empty_like(x)
        y_new = torch.full_like(x, float("nan"))
        fb.fb_operator_apply(op, x, y_ref)
        fb.fb_operator_apply_noalloc(op, x, y_new)
        torch.cuda.synchronize()
        a, b = y_new.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert rel(a, b) < tol


def test_noalloc_rejects_dense_operator(setup):
    wl, ops = setup
    x = torch.zeros(wl.n, dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(fb.FBError) as e:
        fb.fb_operator_apply_noalloc(ops["dense"], x, y)
    assert e.value.code == 1
