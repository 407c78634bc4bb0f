"""fb_operator_apply_noalloc: the FMM matvec for callers that cannot allocate
device memory when they apply an operator (real-time audio callbacks that
must not block in the driver's allocator, hosts whose device memory is a
fixed arena).  Its expansion scratch lives in the library's static device
buffer; its output must match fb_operator_apply on consecutive calls (the
buffer keeps the previous call's contents, which the call must clear), a
call leaves the device's free memory unchanged, and an operator whose
expansions exceed the buffer is refused.  Collected last on purpose."""
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


def test_noalloc_call_leaves_free_device_memory_unchanged(setup):
    """After a first call on the device (which resolves the buffer's address),
    further calls allocate nothing: the driver's free-memory count and
    torch's allocator are the same before and after."""
    wl, ops = setup
    op = ops["mixed"]
    x = torch.tensor(seeded_vector(wl.n, 23), device="cuda")
    y = torch.empty_like(x)
    fb.fb_operator_apply_noalloc(op, x, y)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        fb.fb_operator_apply_noalloc(op, x, y)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_noalloc_refuses_expansions_beyond_the_buffer():
    """An FP64 operator whose expansions (2 x sum over levels of boxes x p^2
    complex128 values) exceed FB_NOALLOC_SCRATCH_BYTES = 32 MiB is refused
    with FB_ERR_ARG before any device work."""
    wl = workload("sub")
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = fb.fb_tree_build(mesh, 64)
    op = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_FP64_FMM, 6.0, 64)
    try:
        L, _, _, nb = fb.fb_tree_info(tree)
        _, _, p = fb.fb_operator_info(op)
        need = 2 * 16 * sum(int(nb[l]) * int(p[l]) ** 2 for l in range(2, L + 1))
        assert need > 32 << 20
        x = torch.zeros(wl.n, dtype=torch.complex128, device="cuda")
        y = torch.zeros_like(x)
        with pytest.raises(fb.FBError) as e:
            fb.fb_operator_apply_noalloc(op, x, y)
        assert e.value.code == 1
        assert "bytes of expansion scratch" in str(e.value)
    finally:
        fb.fb_operator_destroy(op)
        fb.fb_tree_destroy(tree)
        fb.fb_mesh_destroy(mesh)
