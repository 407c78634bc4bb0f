"""Staged rotation - coaxial - rotation (Sec. 3.3): the translation passes of
large orders run as batched GEMMs over all box pairs of a level that share
a polar angle (rotations) or a translation distance (coaxial step).  They
compute the same sums as the per-pair tiles, whose translation matrices and
FP64 matvec the oracle pins entry by entry (test_gpu_fmm.py), so both forms
must agree to FP64 rounding on every level, for M2L, M2M and L2L, with equal
and unequal orders between levels and for several right-hand sides."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16073_gb300 as fb
from _cases import oracle_dense, rel, seeded_vector, workload

TILES = [0] * 13
STAGED = [4 | 8] * 13     # bit 2: M2L staged, bit 3: M2M/L2L staged


@pytest.fixture(scope="module")
def sub():
    wl = workload("sub")
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = fb.fb_tree_build(mesh, 64)
    yield wl, mesh, tree
    fb.fb_tree_destroy(tree)
    fb.fb_mesh_destroy(mesh)


def apply(op, X):
    Y = torch.empty_like(X)
    if X.dim() == 1:
        fb.fb_operator_apply(op, X, Y)
    else:
        fb.fb_operator_apply_multi(op, X, Y)
    torch.cuda.synchronize()
    return Y.cpu().numpy()


@pytest.mark.parametrize("pmin", [12, 30])
@pytest.mark.parametrize("kind", [fb.FB_OP_A, fb.FB_OP_LP])
def test_staged_equals_tiles_fp64(sub, pmin, kind):
    """pmin = 12: orders 26 / 17 / 12 / 12 on levels 2-5 (unequal orders
    across M2M and L2L); pmin = 30: order 30 everywhere."""
    wl, mesh, tree = sub
    op = fb.fb_operator_create(mesh, tree, wl.k, kind, fb.FB_PREC_FP64_FMM, 6.0, pmin)
    try:
        x = torch.tensor(seeded_vector(wl.n, 41), device="cuda")
        fb.fb_operator_set_forms(op, TILES)
        y_t = apply(op, x)
        fb.fb_operator_set_forms(op, STAGED)
        y_s = apply(op, x)
        assert rel(y_s, y_t) < 1e-12
        # the FMM itself: within the FP64 FMM tolerance of the dense operator
        D = oracle_dense("sub")
        ref = D["A"] @ seeded_vector(wl.n, 41) if kind == fb.FB_OP_A else D["LP"] @ seeded_vector(wl.n, 41)
        assert rel(y_s, ref) < 1e-5
    finally:
        fb.fb_operator_destroy(op)


def test_staged_mixed_and_several_rhs(sub):
    """Mixed precision (FP32 passes) against the FP64 form, and three
    right-hand sides in one call against three single calls."""
    wl, mesh, tree = sub
    A64 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_FP64_FMM, 6.0, 30)
    A32 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 6.0, 30)
    try:
        fb.fb_operator_set_forms(A32, STAGED)
        X = torch.tensor(np.stack([seeded_vector(wl.n, 50 + r) for r in range(3)]), device="cuda")
        Y64 = np.stack([apply(A64, X[r].contiguous()) for r in range(3)])
        Y32 = apply(A32, X)
        for r in range(3):
            assert rel(Y32[r], Y64[r]) < 1e-5
            assert rel(apply(A32, X[r].contiguous()), Y32[r]) < 1e-6
    finally:
        fb.fb_operator_destroy(A64)
        fb.fb_operator_destroy(A32)


def test_autotune_chooses_among_rcr_forms(sub):
    """The autotuner times tiles and staged passes (FP64: RCR forms only),
    reports both, and the installed choice computes the same product."""
    wl, mesh, tree = sub
    op = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_FP64_FMM, 6.0, 30)
    try:
        x = torch.tensor(seeded_vector(wl.n, 61), device="cuda")
        fb.fb_operator_set_forms(op, TILES)
        y0 = apply(op, x)
        tune = fb.fb_operator_autotune(op, 1)
        assert tune and all(v["m2l_staged"] is not None and v["m2l_rcr"] is not None for v in tune.values())
        assert all(v["m2l_tensor"] is None for v in tune.values())
        assert rel(apply(op, x), y0) < 1e-12
    finally:
        fb.fb_operator_destroy(op)


def test_autotuned_large_orders_match_dense():
    """Orders 116 / 66 (the coarse shoebox at 7.5 kHz): the per-pair working
    set of level 2 exceeds a CTA, so that level always runs staged; after the
    autotuner rebuilt the plans (both precisions) the matvec still matches
    the oracle's dense matrix."""
    wl = workload("high_order")
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = fb.fb_tree_build(mesh, 64)
    ops = []
    try:
        x = seeded_vector(wl.n, 71)
        ref = oracle_dense("high_order")["A"] @ x
        xd = torch.tensor(x, device="cuda")
        for prec, tol in ((fb.FB_PREC_FP64_FMM, 1e-5), (fb.FB_PREC_MIXED_FMM, 2e-5)):
            op = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, prec, 6.0, 12)
            ops.append(op)
            tune = fb.fb_operator_autotune(op, 1)
            assert tune[2]["m2l_rcr"] is None and tune[2]["m2l_staged_on"]
            assert rel(apply(op, xd), ref) < tol
            # a saved choice asking for tiles everywhere keeps level 2 staged
            fb.fb_operator_set_forms(op, TILES)
            assert rel(apply(op, xd), ref) < tol
    finally:
        for op in ops:
            fb.fb_operator_destroy(op)
        fb.fb_tree_destroy(tree)
        fb.fb_mesh_destroy(mesh)


STAGED_TC = [4 | 8 | 16 | 32] * 13   # bits 4/5: the staged rotations on the tensor cores
STAGED_TCC = [4 | 8 | 16 | 32 | 1024 | 2048] * 13   # bits 10/11: the coaxial step too


@pytest.mark.parametrize("pmin", [12, 30])
@pytest.mark.parametrize("kind", [fb.FB_OP_A, fb.FB_OP_LP])
def test_staged_tensor_rotations_match_fp64(sub, pmin, kind):
    """Rotation and coaxial passes as 3xTF32 tcgen05 GEMMs (every degree
    from 0 on, both folded parts, M2L, M2M and L2L): the mixed matvec
    matches the FP64 form within the mixed tolerance 1e-5 (measured 3.4e-6;
    the CUDA-core staged passes 2.8e-7: the tensor cores' products of the
    split operands drop the lo x lo term and read each lo part as TF32)."""
    wl, mesh, tree = sub
    A64 = fb.fb_operator_create(mesh, tree, wl.k, kind, fb.FB_PREC_FP64_FMM, 6.0, pmin)
    A32 = fb.fb_operator_create(mesh, tree, wl.k, kind, fb.FB_PREC_MIXED_FMM, 6.0, pmin)
    try:
        x = torch.tensor(seeded_vector(wl.n, 43), device="cuda")
        y64 = apply(A64, x)
        fb.fb_operator_set_forms(A32, STAGED)
        y_s = apply(A32, x)
        fb.fb_operator_set_forms(A32, STAGED_TC)
        y_tc = apply(A32, x)
        assert rel(y_tc, y64) < 1e-5
        assert rel(y_s, y64) < 1e-5
        fb.fb_operator_set_forms(A32, STAGED_TCC)
        y_tcc = apply(A32, x)
        assert rel(y_tcc, y64) < 1e-5
        fb.fb_operator_status(A32)   # no bounded wait ran out
    finally:
        fb.fb_operator_destroy(A64)
        fb.fb_operator_destroy(A32)


def test_staged_tensor_rotations_several_rhs(sub):
    wl, mesh, tree = sub
    A32 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 6.0, 30)
    try:
        fb.fb_operator_set_forms(A32, STAGED_TCC)
        X = torch.tensor(np.stack([seeded_vector(wl.n, 80 + r) for r in range(3)]), device="cuda")
        Y = apply(A32, X)
        for r in range(3):
            assert rel(apply(A32, X[r].contiguous()), Y[r]) < 1e-6
    finally:
        fb.fb_operator_destroy(A32)


def test_staged_tensor_rotations_rejected_where_undefined(sub):
    wl, mesh, tree = sub
    A64 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_FP64_FMM, 6.0, 12)
    A32 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 6.0, 12)
    try:
        with pytest.raises(fb.FBError):
            fb.fb_operator_set_forms(A64, STAGED_TC)      # FP64: no tensor-core form
        with pytest.raises(fb.FBError):
            fb.fb_operator_set_forms(A32, [16 | 32] * 13)  # bits 4/5 refine the staged bits
    finally:
        fb.fb_operator_destroy(A64)
        fb.fb_operator_destroy(A32)


def test_staged_tensor_rotations_large_orders_match_dense():
    """Orders 116 / 66 (degree blocks up to 116 columns, several degrees per
    tile below): mixed matvec with the tensor-core rotations against the
    oracle's dense matrix, and the autotuner's report of the form."""
    wl = workload("high_order")
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = fb.fb_tree_build(mesh, 64)
    op = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 6.0, 12)
    try:
        x = seeded_vector(wl.n, 73)
        ref = oracle_dense("high_order")["A"] @ x
        xd = torch.tensor(x, device="cuda")
        fb.fb_operator_set_forms(op, STAGED_TC)
        assert rel(apply(op, xd), ref) < 2e-5
        fb.fb_operator_set_forms(op, STAGED_TCC)
        assert rel(apply(op, xd), ref) < 2e-5
        tune = fb.fb_operator_autotune(op, 1)
        assert tune[2]["m2l_staged_tc"] is not None and tune[2]["m2l_staged"] is not None
        assert tune[2]["m2l_staged_tcc"] is not None
        assert rel(apply(op, xd), ref) < 2e-5
    finally:
        fb.fb_operator_destroy(op)
        fb.fb_tree_destroy(tree)
        fb.fb_mesh_destroy(mesh)


STAGED_DF = [4 | 8 | 64 | 128] * 13   # bits 6/7: the staged passes in double-FP32 (FP64 operators)


@pytest.mark.parametrize("pmin", [12, 30])
@pytest.mark.parametrize("kind", [fb.FB_OP_A, fb.FB_OP_LP])
def test_staged_double_float_matches_fp64_tiles(sub, pmin, kind):
    """Staged passes in double-FP32 arithmetic (48-bit significand) on an
    FP64 operator: M2L, M2M and L2L against the FP64 per-pair tiles, far
    inside the FMM's own truncation error."""
    wl, mesh, tree = sub
    op = fb.fb_operator_create(mesh, tree, wl.k, kind, fb.FB_PREC_FP64_FMM, 6.0, pmin)
    try:
        x = torch.tensor(seeded_vector(wl.n, 45), device="cuda")
        fb.fb_operator_set_forms(op, TILES)
        y_t = apply(op, x)
        fb.fb_operator_set_forms(op, STAGED_DF)
        y_d = apply(op, x)
        assert rel(y_d, y_t) < 1e-11
        X = torch.tensor(np.stack([seeded_vector(wl.n, 90 + r) for r in range(3)]), device="cuda")
        Y = apply(op, X)
        for r in range(3):
            assert rel(apply(op, X[r].contiguous()), Y[r]) < 1e-13
    finally:
        fb.fb_operator_destroy(op)


def test_staged_double_float_rejected_where_undefined(sub):
    wl, mesh, tree = sub
    A32 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 6.0, 12)
    A64 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_FP64_FMM, 6.0, 12)
    try:
        with pytest.raises(fb.FBError):
            fb.fb_operator_set_forms(A32, STAGED_DF)        # double-FP32 forms are for FP64 operators
        with pytest.raises(fb.FBError):
            fb.fb_operator_set_forms(A64, [64 | 128] * 13)  # bits 6/7 refine the staged bits
    finally:
        fb.fb_operator_destroy(A32)
        fb.fb_operator_destroy(A64)


def test_staged_double_float_large_orders():
    """Orders 116 / 66: double-FP32 staged passes against the FP64 staged
    passes and the oracle's dense matrix."""
    wl = workload("high_order")
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = fb.fb_tree_build(mesh, 64)
    op = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_FP64_FMM, 6.0, 12)
    try:
        x = seeded_vector(wl.n, 75)
        ref = oracle_dense("high_order")["A"] @ x
        xd = torch.tensor(x, device="cuda")
        fb.fb_operator_set_forms(op, STAGED)
        y_s = apply(op, xd)
        fb.fb_operator_set_forms(op, STAGED_DF)
        y_d = apply(op, xd)
        assert rel(y_d, y_s) < 1e-11
        assert rel(y_d, ref) < 1e-5
        passes = fb.fb_operator_staged_pass_times(op)
        assert passes[2]["form"] == "df" and all(passes[2][k] > 0 for k in ("prep", "rot", "coax", "back"))
        A32 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 6.0, 12)
        try:
            fb.fb_operator_set_forms(A32, STAGED_TC)
            apply(A32, xd)
            p32 = fb.fb_operator_staged_pass_times(A32)
            assert p32[2]["form"] == "tensor_rot" and p32[2]["prep"] < 0    # no separate pre-pass
            assert all(p32[2][k] > 0 for k in ("rot", "coax", "back"))
        finally:
            fb.fb_operator_destroy(A32)
    finally:
        fb.fb_operator_destroy(op)
        fb.fb_tree_destroy(tree)
        fb.fb_mesh_destroy(mesh)


TILES_DF = [256 | 512] * 13   # bits 8/9: per-pair tiles in double-FP32 (FP64 operators)


@pytest.mark.parametrize("pmin", [12, 30])
def test_tiles_double_float_match_fp64_tiles(sub, pmin):
    """Per-pair RCR tiles in double-FP32 arithmetic: M2L, M2M and L2L against
    the FP64 tiles, one and several right-hand sides; levels whose tiles do
    not fit run staged in double-FP32."""
    wl, mesh, tree = sub
    op = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_FP64_FMM, 6.0, pmin)
    try:
        x = torch.tensor(seeded_vector(wl.n, 47), device="cuda")
        fb.fb_operator_set_forms(op, TILES)
        y_t = apply(op, x)
        fb.fb_operator_set_forms(op, TILES_DF)
        y_d = apply(op, x)
        assert rel(y_d, y_t) < 1e-11
        X = torch.tensor(np.stack([seeded_vector(wl.n, 95 + r) for r in range(3)]), device="cuda")
        Y = apply(op, X)
        for r in range(3):
            assert rel(apply(op, X[r].contiguous()), Y[r]) < 1e-13
        with pytest.raises(fb.FBError):
            fb.fb_operator_set_forms(op, [4 | 256] * 13)   # tiles and staged at once
    finally:
        fb.fb_operator_destroy(op)


def test_autotune_fp64_reports_double_float_forms(sub):
    wl, mesh, tree = sub
    op = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_FP64_FMM, 6.0, 30)
    try:
        x = torch.tensor(seeded_vector(wl.n, 62), device="cuda")
        fb.fb_operator_set_forms(op, TILES)
        y0 = apply(op, x)
        tune = fb.fb_operator_autotune(op, 1)
        assert all(v["m2l_tiles_df"] is not None and v["m2l_staged_df"] is not None for v in tune.values())
        assert all(v["m2l_staged_tc"] is None for v in tune.values())
        assert rel(apply(op, x), y0) < 1e-11
    finally:
        fb.fb_operator_destroy(op)
