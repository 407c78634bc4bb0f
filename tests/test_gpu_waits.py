"""Failure detection of the bounded device waits, without a GPU fault or
hang: every mbarrier wait of the tensor-core translation kernel is a bounded
poll.  A test hook makes the kernel wait on a barrier that nothing signals;
the bound runs out, the kernel waits for the copies and tensor-core
operations it has already issued, releases its tensor memory, records an
error flag and returns.  The host reads FB_ERR_TIMEOUT from
fb_operator_status after a matvec and as the status of a solve, and the same
operator then computes the same product again (the context stays usable)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16073_gb300 as fb
from _cases import rel, seeded_vector, workload


def test_wait_timeout_is_reported_and_context_stays_usable():
    wl = workload("sub")
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = fb.fb_tree_build(mesh, 64)
    A = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 6.0, 12)
    try:
        fb.fb_operator_set_translation(A, fb.FB_TRANS_TENSOR)   # every M2L level on the tensor cores
        x = torch.tensor(seeded_vector(wl.n, 81), device="cuda")
        y0 = torch.empty_like(x)
        fb.fb_operator_apply(A, x, y0)
        fb.fb_operator_status(A)                                  # no wait ran out
        prev = fb.fb_set_device_wait_limit(1 << 12)
        try:
            fb.fb_test_stall_device_waits(True)
            y = torch.empty_like(x)
            fb.fb_operator_apply(A, x, y)                         # launches fine; the waits run out on the device
            with pytest.raises(fb.FBError) as e:
                fb.fb_operator_status(A)
            assert e.value.code == 6                              # FB_ERR_TIMEOUT
            fb.fb_operator_status(A)                              # the flag was cleared by the read
            b = torch.tensor(seeded_vector(wl.n, 82), device="cuda")
            xs = torch.zeros_like(b)
            with pytest.raises(fb.FBError) as e:
                fb.fb_fgmres_solve(A, b, xs, tol=1e-6, restart=5, maxit=5, max_refine=1)
            assert e.value.code == 6
        finally:
            fb.fb_test_stall_device_waits(False)
            fb.fb_set_device_wait_limit(prev)
        y1 = torch.empty_like(x)
        fb.fb_operator_apply(A, x, y1)
        fb.fb_operator_status(A)
        torch.cuda.synchronize()
        assert rel(y1.cpu().numpy(), y0.cpu().numpy()) < 1e-6
    finally:
        fb.fb_operator_destroy(A)
        fb.fb_tree_destroy(tree)
        fb.fb_mesh_destroy(mesh)


def test_staged_tensor_rotation_wait_timeout():
    """The same for the staged RCR passes whose rotations run on the tensor
    cores: a bounded wait of their pipeline runs out, the kernel drains its
    bulk copies, frees its tensor memory and flags the operator; the next
    matvec computes the same product."""
    wl = workload("sub")
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = fb.fb_tree_build(mesh, 64)
    A = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 6.0, 30)
    try:
        fb.fb_operator_set_forms(A, [4 | 8 | 16 | 32 | 1024 | 2048] * 13)   # rotations and coaxial step
        x = torch.tensor(seeded_vector(wl.n, 83), device="cuda")
        y0 = torch.empty_like(x)
        fb.fb_operator_apply(A, x, y0)
        fb.fb_operator_status(A)
        prev = fb.fb_set_device_wait_limit(1 << 12)
        try:
            fb.fb_test_stall_device_waits(True)
            y = torch.empty_like(x)
            fb.fb_operator_apply(A, x, y)
            with pytest.raises(fb.FBError) as e:
                fb.fb_operator_status(A)
            assert e.value.code == 6
        finally:
            fb.fb_test_stall_device_waits(False)
            fb.fb_set_device_wait_limit(prev)
        y1 = torch.empty_like(x)
        fb.fb_operator_apply(A, x, y1)
        fb.fb_operator_status(A)
        torch.cuda.synchronize()
        assert rel(y1.cpu().numpy(), y0.cpu().numpy()) < 1e-6
    finally:
        fb.fb_operator_destroy(A)
        fb.fb_tree_destroy(tree)
        fb.fb_mesh_destroy(mesh)
