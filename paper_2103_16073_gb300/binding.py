"""Python binding of libfmmbem (include/fmmbem.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays
and torch tensors to the plain pointers and sizes of the C ABI and raises
``FBError`` with the library's message when a call fails.  There is no CPU
fallback: importing this module builds (if needed) and loads the shared
library, and fails loudly if that is impossible.  The package imports it on
the first use of one of its names (``fb_*``, ``FB_*``, ``lib``, ...).

Array conventions: complex vectors are complex128 (interleaved re/im doubles).
A torch tensor on a CUDA device is passed as a device pointer on the current
torch stream; numpy arrays (or CPU tensors) are passed as host memory, which
the library copies in and out.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

__all__ = [
    "FBError", "lib", "FB_OP_L", "FB_OP_M", "FB_OP_LP", "FB_OP_A", "FB_OP_MP", "FB_PREC_FP64_DENSE",
    "FB_PREC_FP64_FMM", "FB_PREC_MIXED_FMM", "FB_PC_NONE", "FB_PC_BLOCK_JACOBI",
    "fb_version", "fb_mesh_create", "fb_mesh_set_admittance", "fb_mesh_info", "fb_mesh_geometry",
    "fb_mesh_destroy", "fb_tree_build", "fb_tree_info", "fb_tree_export", "fb_tree_destroy",
    "fb_operator_create", "fb_operator_apply", "fb_operator_info", "fb_operator_export",
    "fb_operator_destroy", "fb_gamma_monopole", "fb_precond_create", "fb_precond_destroy",
    "fb_precond_apply", "fb_fgmres_solve", "fb_eval_field", "fb_operator_apply_timed", "fb_kernel_launches",
    "fb_operator_apply_noalloc", "fb_operator_set_translation", "fb_measure_alu_peaks",
    "fb_precond_create_learned", "fb_learned_params", "fb_learned_set_objective",
    "fb_precond_create_inner", "FB_PC_INNER", "FB_PC_LEARNED", "fb_krylov_basis",
    "FB_LOSS_ERROR", "FB_LOSS_RESIDUAL", "fb_learned_loss_and_grad", "fb_learned_train_step",
    "fb_operator_apply_multi", "fb_fgmres_solve_multi", "FB_MAX_RHS", "FB_TUNE_TIMES", "fb_operator_autotune", "fb_operator_set_forms", "fb_batch_solve", "fb_operator_use_graphs", "fb_precond_use_graphs",
    "SolverOpts", "SolveInfo",
]

FB_OK = 0
FB_OP_L, FB_OP_M, FB_OP_LP, FB_OP_A, FB_OP_MP, FB_OP_IBEM, FB_OP_DBEM5 = 0, 1, 2, 3, 4, 5, 6
FB_PREC_FP64_DENSE, FB_PREC_FP64_FMM, FB_PREC_MIXED_FMM = 0, 1, 2
FB_MEM_HOST, FB_MEM_DEVICE = 0, 1
FB_PC_NONE, FB_PC_BLOCK_JACOBI = 0, 1
STATUS_NAMES = {0: "FB_OK", 1: "FB_ERR_ARG", 2: "FB_ERR_CUDA", 3: "FB_ERR_NOCONV",
                4: "FB_ERR_BREAKDOWN", 5: "FB_ERR_NAN", 6: "FB_ERR_TIMEOUT", 7: "FB_ERR_OOM",
                8: "FB_ERR_STATE"}


class FBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class SolverOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("restart", C.c_int), ("maxit", C.c_int),
                ("max_refine", C.c_int), ("inner_tol", C.c_double), ("true_op", C.c_void_p)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("refinements", C.c_int), ("true_matvecs", C.c_int),
                ("est_relres", C.c_double), ("true_relres", C.c_double), ("status", C.c_int),
                ("pc_fallbacks", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def _load():
    path = _build.build()
    if not os.path.exists(path):
        raise ImportError("libfmmbem.so is missing and could not be built")
    L = C.CDLL(path)
    vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
    pvp = C.POINTER(C.c_void_p)
    sigs = {
        "fb_version": (C.c_char_p, []),
        "fb_last_error": (i32, [C.c_char_p, C.c_size_t]),
        "fb_mesh_create": (i32, [vp, i64, vp, i64, vp, pvp]),
        "fb_mesh_set_admittance": (i32, [vp, vp, i32, vp]),
        "fb_mesh_info": (i32, [vp, C.POINTER(i64), C.POINTER(dbl), C.POINTER(dbl)]),
        "fb_mesh_geometry": (i32, [vp, vp, vp]),
        "fb_mesh_destroy": (None, [vp]),
        "fb_tree_build": (i32, [vp, i32, vp, pvp]),
        "fb_tree_info": (i32, [vp, C.POINTER(i32), vp, C.POINTER(dbl), vp]),
        "fb_tree_export": (i32, [vp, i32, i32, vp, C.POINTER(i64)]),
        "fb_tree_destroy": (None, [vp]),
        "fb_operator_create": (i32, [vp, vp, dbl, i32, i32, dbl, i32, vp, pvp]),
        "fb_operator_apply": (i32, [vp, vp, vp, i32, vp]),
        "fb_operator_info": (i32, [vp, C.POINTER(i64), C.POINTER(i32), vp]),
        "fb_operator_export": (i32, [vp, i32, i32, i64, vp, C.POINTER(i64)]),
        "fb_operator_destroy": (None, [vp]),
        "fb_gamma_monopole": (i32, [vp, dbl, vp, vp, i32, vp]),
        "fb_precond_create": (i32, [vp, i32, vp, pvp]),
        "fb_precond_destroy": (None, [vp]),
        "fb_precond_apply": (i32, [vp, vp, vp, i32, vp]),
        "fb_fgmres_solve": (i32, [vp, vp, vp, vp, C.POINTER(SolverOpts), C.POINTER(SolveInfo), i32, vp]),
        "fb_eval_field": (i32, [vp, dbl, vp, vp, vp, vp, i64, vp, i32, vp]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()


def _check(st):
    if st != FB_OK:
        buf = C.create_string_buffer(1024)
        lib.fb_last_error(buf, 1024)
        raise FBError(st, buf.value.decode(errors="replace"))


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return C.c_void_p(0)


def _is_cuda_tensor(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def _ptr(a, dtype=None):
    """(pointer, memspace, keepalive) for a numpy array or torch tensor."""
    if _is_cuda_tensor(a):
        if not a.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        return C.c_void_p(a.data_ptr()), FB_MEM_DEVICE, a
    if hasattr(a, "numpy"):
        a = a.detach().cpu().numpy()
    arr = np.ascontiguousarray(a, dtype=dtype)
    return C.c_void_p(arr.ctypes.data), FB_MEM_HOST, arr


def _cuda_ptr(t, name):
    """Device pointer of a contiguous CUDA tensor (the caller keeps it alive)."""
    if not _is_cuda_tensor(t):
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _same_space(*ms):
    if len(set(ms)) != 1:
        raise ValueError("all vector arguments must be host arrays or all device tensors")
    return ms[0]


def fb_version() -> str:
    return lib.fb_version().decode()


def fb_mesh_create(verts, tris, stream=None):
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    out = C.c_void_p()
    _check(lib.fb_mesh_create(v.ctypes.data, v.shape[0], t.ctypes.data, t.shape[0], _stream(stream),
                              C.byref(out)))
    return out


def fb_mesh_set_admittance(mesh, beta, stream=None):
    p, ms, keep = _ptr(beta, np.complex128)
    _check(lib.fb_mesh_set_admittance(mesh, p, ms, _stream(stream)))


def fb_mesh_info(mesh):
    n, rc, me = C.c_int64(), C.c_double(), C.c_double()
    _check(lib.fb_mesh_info(mesh, C.byref(n), C.byref(rc), C.byref(me)))
    return n.value, rc.value, me.value


def fb_mesh_geometry(mesh):
    n = fb_mesh_info(mesh)[0]
    c = np.empty((n, 3))
    nn = np.empty((n, 3))
    _check(lib.fb_mesh_geometry(mesh, c.ctypes.data, nn.ctypes.data))
    return c, nn


def fb_mesh_destroy(mesh):
    lib.fb_mesh_destroy(mesh)


def fb_tree_build(mesh, leaf_max=64, stream=None):
    out = C.c_void_p()
    _check(lib.fb_tree_build(mesh, int(leaf_max), _stream(stream), C.byref(out)))
    return out


def fb_tree_info(tree):
    L = C.c_int()
    org = np.zeros(3)
    side = C.c_double()
    nb = np.zeros(16, np.int64)
    _check(lib.fb_tree_info(tree, C.byref(L), org.ctypes.data, C.byref(side), nb.ctypes.data))
    return L.value, org, side.value, nb[:L.value + 1].copy()


def fb_tree_export(tree, which, level=0):
    cnt = C.c_int64()
    _check(lib.fb_tree_export(tree, which, level, None, C.byref(cnt)))
    width = 2 if which in (3, 4) else 1
    out = np.zeros(max(cnt.value * width, 1), np.int64)
    _check(lib.fb_tree_export(tree, which, level, out.ctypes.data, C.byref(cnt)))
    out = out[:cnt.value * width]
    return out.reshape(-1, 2) if width == 2 else out


def fb_tree_destroy(tree):
    lib.fb_tree_destroy(tree)


lib.fb_operator_create_like.restype = C.c_int
lib.fb_operator_create_like.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]


def fb_operator_create_like(donor, precision, d0=6.0, pmin=12, stream=None):
    """An FMM operator of the donor's mesh, tree, k and kind at another
    precision / order rule; the near-field entries are copied from an FP64
    FMM donor instead of being integrated again."""
    out = C.c_void_p()
    _check(lib.fb_operator_create_like(donor, int(precision), float(d0), int(pmin), _stream(stream), C.byref(out)))
    return out


def fb_operator_create(mesh, tree, k, kind, precision, d0=6.0, pmin=12, stream=None):
    out = C.c_void_p()
    _check(lib.fb_operator_create(mesh, tree, float(k), int(kind), int(precision), float(d0), int(pmin),
                                  _stream(stream), C.byref(out)))
    return out


def fb_operator_apply(op, x, y, stream=None):
    px, mx, kx = _ptr(x, np.complex128)
    if not _is_cuda_tensor(y) and not isinstance(y, np.ndarray):
        raise ValueError("y must be a numpy array or a CUDA tensor")
    py, my, ky = _ptr(y, np.complex128)
    _check(lib.fb_operator_apply(op, px, py, _same_space(mx, my), _stream(stream)))
    if my == FB_MEM_HOST and ky is not y:
        y[...] = ky
    return y


def fb_operator_info(op):
    n, L = C.c_int64(), C.c_int()
    p = np.zeros(16, np.int32)
    _check(lib.fb_operator_info(op, C.byref(n), C.byref(L), p.ctypes.data))
    return n.value, L.value, p[:L.value + 1].copy()


def fb_operator_export(op, which, level=0, index=0):
    cnt = C.c_int64()
    _check(lib.fb_operator_export(op, which, level, index, None, C.byref(cnt)))
    out = np.zeros(max(cnt.value, 1), np.complex128)
    _check(lib.fb_operator_export(op, which, level, index, out.ctypes.data, C.byref(cnt)))
    return out[:cnt.value]


def fb_operator_destroy(op):
    lib.fb_operator_destroy(op)


def fb_gamma_monopole(mesh, k, src, out, stream=None):
    s = np.ascontiguousarray(src, dtype=np.float64)
    po, mo, ko = _ptr(out, np.complex128)
    _check(lib.fb_gamma_monopole(mesh, float(k), s.ctypes.data, po, mo, _stream(stream)))
    if mo == FB_MEM_HOST and ko is not out:
        out[...] = ko
    return out


def fb_precond_create(op, kind=FB_PC_BLOCK_JACOBI, stream=None):
    out = C.c_void_p()
    _check(lib.fb_precond_create(op, int(kind), _stream(stream), C.byref(out)))
    return out if out.value else None


def fb_precond_destroy(pc):
    lib.fb_precond_destroy(pc)


def fb_precond_apply(pc, x, y, stream=None):
    px, mx, kx = _ptr(x, np.complex128)
    if not _is_cuda_tensor(y) and not isinstance(y, np.ndarray):
        raise ValueError("y must be a numpy array or a CUDA tensor")
    py, my, ky = _ptr(y, np.complex128)
    _check(lib.fb_precond_apply(pc, px, py, _same_space(mx, my), _stream(stream)))
    if my == FB_MEM_HOST and ky is not y:
        y[...] = ky
    return y


def fb_fgmres_solve(A, b, x, pc=None, tol=1e-8, restart=40, maxit=2000, max_refine=3, inner_tol=0.0,
                    true_op=None, stream=None, raise_on_noconv=False):
    pb, mb, kb = _ptr(b, np.complex128)
    if not _is_cuda_tensor(x) and not isinstance(x, np.ndarray):
        raise ValueError("x must be a numpy array or a CUDA tensor")
    px, mx, kx = _ptr(x, np.complex128)
    opts = SolverOpts(float(tol), int(restart), int(maxit), int(max_refine), float(inner_tol),
                      true_op.value if true_op is not None else None)
    info = SolveInfo()
    st = lib.fb_fgmres_solve(A, pc, pb, px, C.byref(opts), C.byref(info), _same_space(mb, mx),
                             _stream(stream))
    if st not in (FB_OK, 3, 5) or (raise_on_noconv and st != FB_OK):
        _check(st)
    if mx == FB_MEM_HOST and kx is not x:
        x[...] = kx
    return info.as_dict()


def fb_eval_field(mesh, k, psi_sc, gamma, rcv, out, src=None, stream=None):
    pp, m1, k1 = _ptr(psi_sc, np.complex128)
    pg, m2, k2 = _ptr(gamma, np.complex128)
    pr, m3, k3 = _ptr(rcv, np.float64)
    po, m4, k4 = _ptr(out, np.complex128)
    s = None if src is None else np.ascontiguousarray(src, dtype=np.float64)
    nr = (rcv.shape[0])
    _check(lib.fb_eval_field(mesh, float(k), pp, pg, None if s is None else s.ctypes.data, pr, nr, po,
                             _same_space(m1, m2, m3, m4), _stream(stream)))
    if m4 == FB_MEM_HOST and k4 is not out:
        out[...] = k4
    return out


lib.fb_operator_apply_timed.restype = C.c_int
lib.fb_operator_apply_timed.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
lib.fb_kernel_launches.restype = C.c_longlong
lib.fb_kernel_launches.argtypes = []
PHASES = ("p2m", "m2m", "m2l_tc", "m2l", "l2l", "near_l2p", "total")


def fb_operator_apply_timed(op, x, y, stream=None):
    """y = Op x on CUDA tensors; returns per-phase CUDA-event times (ms)."""
    ms = np.zeros(7)
    _check(lib.fb_operator_apply_timed(op, _cuda_ptr(x, "x"), _cuda_ptr(y, "y"), _stream(stream), ms.ctypes.data))
    return dict(zip(PHASES, ms.tolist()))


def fb_kernel_launches() -> int:
    return int(lib.fb_kernel_launches())


lib.fb_operator_apply_noalloc.restype = C.c_int
lib.fb_operator_apply_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
NOALLOC_SCRATCH_BYTES = 32 << 20


def fb_operator_apply_noalloc(op, x, y, stream=None):
    """y = Op x (FMM operators, CUDA tensors) with the expansion scratch in the
    library's static device buffer: no device allocation in the call."""
    if not (_is_cuda_tensor(x) and _is_cuda_tensor(y)):
        raise ValueError("fb_operator_apply_noalloc needs CUDA tensors")
    if not (x.is_contiguous() and y.is_contiguous()):
        raise ValueError("device tensors must be contiguous")
    _check(lib.fb_operator_apply_noalloc(op, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                         _stream(stream)))
    return y


FB_MAX_RHS = 64
FB_TUNE_TIMES = 14   # autotuner timings per level
lib.fb_operator_apply_multi.restype = C.c_int
lib.fb_operator_apply_multi.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]
lib.fb_fgmres_solve_multi.restype = C.c_int
lib.fb_fgmres_solve_multi.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                      C.POINTER(SolverOpts), C.POINTER(SolveInfo), C.c_int, C.c_void_p]


def _nrhs(a):
    if a.ndim != 2:
        raise ValueError("multi-RHS arrays are [nrhs, N]")
    return int(a.shape[0])


def fb_operator_apply_multi(op, X, Y, stream=None):
    """Y[r] = Op X[r] for every row r of the [nrhs, N] complex arrays."""
    R = _nrhs(X)
    px, mx, kx = _ptr(X, np.complex128)
    py, my, ky = _ptr(Y, np.complex128)
    _check(lib.fb_operator_apply_multi(op, px, py, R, _same_space(mx, my), _stream(stream)))
    if my == FB_MEM_HOST and ky is not Y:
        Y[...] = ky
    return Y


def fb_fgmres_solve_multi(A, B, X, pc=None, tol=1e-8, restart=40, maxit=2000, max_refine=3, inner_tol=0.0,
                          true_op=None, stream=None):
    """Lockstep FGMRES for the rows of B ([nrhs, N]); returns one info dict per row."""
    R = _nrhs(B)
    pb, mb, kb = _ptr(B, np.complex128)
    px, mx, kx = _ptr(X, np.complex128)
    opts = SolverOpts(float(tol), int(restart), int(maxit), int(max_refine), float(inner_tol),
                      true_op.value if true_op is not None else None)
    infos = (SolveInfo * R)()
    st = lib.fb_fgmres_solve_multi(A, pc, pb, px, R, C.byref(opts), infos, _same_space(mb, mx), _stream(stream))
    if st not in (FB_OK, 3, 5):
        _check(st)
    if mx == FB_MEM_HOST and kx is not X:
        X[...] = kx
    return [i.as_dict() for i in infos]


lib.fb_operator_autotune.restype = C.c_int
lib.fb_operator_autotune.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]


def fb_operator_autotune(op, nrhs=1, stream=None):
    """Times the translation forms per level (RCR as per-pair tiles, RCR as
    staged GEMM passes, tensor-core composed GEMMs for mixed operators) and
    installs the fastest; returns {level: {"m2l_rcr", "m2l_tensor",
    "m2m_l2l_rcr", "m2m_l2l_tensor", "m2l_staged", "m2m_l2l_staged",
    "m2l_staged_tc", "m2m_l2l_staged_tc", "m2l_staged_df", "m2m_l2l_staged_df",
    "m2l_tiles_df", "m2m_l2l_tiles_df", "m2l_staged_tcc", "m2m_l2l_staged_tcc"
    (ms, None if not a candidate),
    "m2l_on_tensor", "m2m_l2l_on_tensor", "m2l_staged_on", "m2m_l2l_staged_on",
    "m2l_staged_tc_on", "m2m_l2l_staged_tc_on", "m2l_staged_df_on",
    "m2m_l2l_staged_df_on", "m2l_tiles_df_on", "m2m_l2l_tiles_df_on",
    "m2l_staged_tcc_on", "m2m_l2l_staged_tcc_on", "choice"}}."""
    nt = FB_TUNE_TIMES
    times = np.full(nt * 13, -1.0)
    choice = np.zeros(13, np.int32)
    _check(lib.fb_operator_autotune(op, int(nrhs), _stream(stream), times.ctypes.data, choice.ctypes.data))
    out = {}
    for l in range(13):
        t = times[nt * l:nt * l + nt]
        if np.all(t < 0):
            continue
        f = lambda v: None if v < 0 else round(float(v), 4)
        out[l] = {"m2l_rcr": f(t[0]), "m2l_tensor": f(t[1]), "m2m_l2l_rcr": f(t[2]), "m2m_l2l_tensor": f(t[3]),
                  "m2l_staged": f(t[4]), "m2m_l2l_staged": f(t[5]), "m2l_staged_tc": f(t[6]),
                  "m2m_l2l_staged_tc": f(t[7]), "m2l_staged_df": f(t[8]), "m2m_l2l_staged_df": f(t[9]),
                  "m2l_tiles_df": f(t[10]), "m2m_l2l_tiles_df": f(t[11]), "m2l_staged_tcc": f(t[12]),
                  "m2m_l2l_staged_tcc": f(t[13]),
                  "m2l_on_tensor": bool(choice[l] & 1), "m2m_l2l_on_tensor": bool(choice[l] & 2),
                  "m2l_staged_on": bool(choice[l] & 4), "m2m_l2l_staged_on": bool(choice[l] & 8),
                  "m2l_staged_tc_on": bool(choice[l] & 16), "m2m_l2l_staged_tc_on": bool(choice[l] & 32),
                  "m2l_staged_df_on": bool(choice[l] & 64), "m2m_l2l_staged_df_on": bool(choice[l] & 128),
                  "m2l_tiles_df_on": bool(choice[l] & 256), "m2m_l2l_tiles_df_on": bool(choice[l] & 512),
                  "m2l_staged_tcc_on": bool(choice[l] & 1024), "m2m_l2l_staged_tcc_on": bool(choice[l] & 2048),
                  "choice": int(choice[l])}
    return out


class BatchJob(C.Structure):
    _fields_ = [("mesh", C.c_void_p), ("tree", C.c_void_p), ("k", C.c_double), ("nsrc", C.c_int),
                ("src", C.c_void_p), ("x", C.c_void_p), ("info", C.POINTER(SolveInfo)),
                ("setup_ms", C.c_double), ("solve_ms", C.c_double), ("status", C.c_int), ("order", C.c_int)]


class BatchOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("restart", C.c_int), ("maxit", C.c_int), ("d0", C.c_double),
                ("pmin", C.c_int), ("autotune", C.c_int), ("max_rhs", C.c_int), ("fp64_judge", C.c_int),
                ("lookahead", C.c_int), ("inner_iters", C.c_int), ("inner_d0", C.c_double), ("inner_pmin", C.c_int)]


lib.fb_batch_solve.restype = C.c_int
lib.fb_batch_solve.argtypes = [C.POINTER(BatchJob), C.c_int, C.POINTER(BatchOpts)]


def fb_batch_solve(jobs, tol=1e-4, restart=40, maxit=3000, d0=6.0, pmin=12, autotune=True, max_rhs=8,
                   fp64_judge=True, lookahead=True, inner_iters=0, inner_d0=0.5, inner_pmin=2):
    """jobs: list of dicts {mesh, tree, k, src [nsrc,3], x (CUDA complex128 [nsrc,N])}.
    Returns one dict per job: {status, setup_ms, solve_ms, order, infos}."""
    arr = (BatchJob * len(jobs))()
    keep = []
    for i, j in enumerate(jobs):
        src = np.ascontiguousarray(j["src"], dtype=np.float64).reshape(-1, 3)
        x = j["x"]
        if not _is_cuda_tensor(x) or not x.is_contiguous() or x.shape[0] != src.shape[0]:
            raise ValueError("x must be a contiguous CUDA tensor [nsrc, N]")
        infos = (SolveInfo * src.shape[0])()
        keep += [src, infos]
        arr[i] = BatchJob(j["mesh"].value if hasattr(j["mesh"], "value") else j["mesh"],
                          j["tree"].value if hasattr(j["tree"], "value") else j["tree"], float(j["k"]),
                          src.shape[0], src.ctypes.data, x.data_ptr(), infos, 0.0, 0.0, 0, -1)
    o = BatchOpts(float(tol), int(restart), int(maxit), float(d0), int(pmin), int(bool(autotune)), int(max_rhs),
                  int(bool(fp64_judge)), int(bool(lookahead)), int(inner_iters), float(inner_d0), int(inner_pmin))
    st = lib.fb_batch_solve(arr, len(jobs), C.byref(o))
    if st not in (FB_OK, 3, 5):
        _check(st)
    out = []
    for i in range(len(jobs)):
        infos = keep[2 * i + 1]
        out.append({"status": arr[i].status, "setup_ms": arr[i].setup_ms, "solve_ms": arr[i].solve_ms,
                    "order": arr[i].order, "infos": [q.as_dict() for q in infos]})
    return out


lib.fb_operator_use_graphs.restype = C.c_int
lib.fb_operator_use_graphs.argtypes = [C.c_void_p, C.c_int]
lib.fb_precond_use_graphs.restype = C.c_int
lib.fb_precond_use_graphs.argtypes = [C.c_void_p, C.c_int]


def fb_operator_use_graphs(op, enable=True):
    _check(lib.fb_operator_use_graphs(op, int(bool(enable))))


def fb_precond_use_graphs(pc, enable=True):
    _check(lib.fb_precond_use_graphs(pc, int(bool(enable))))


lib.fb_operator_set_forms.restype = C.c_int
lib.fb_operator_set_forms.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]


# form bits of a level's choice, in the order of the library's bit numbers 0..11
_FORM_FLAGS = ("m2l_on_tensor", "m2m_l2l_on_tensor", "m2l_staged_on", "m2m_l2l_staged_on",
               "m2l_staged_tc_on", "m2m_l2l_staged_tc_on", "m2l_staged_df_on", "m2m_l2l_staged_df_on",
               "m2l_tiles_df_on", "m2m_l2l_tiles_df_on", "m2l_staged_tcc_on", "m2m_l2l_staged_tcc_on")


def _forms_choice(forms):
    """The 13 per-level choice ints of fb_operator_set_forms from a dict as
    fb_operator_autotune returns (its "choice", else the "..._on" flags) or
    from a sequence of ints."""
    ch = np.zeros(13, np.int32)
    if isinstance(forms, dict):
        for l, v in forms.items():
            if "choice" in v:
                ch[int(l)] = int(v["choice"])
            else:
                ch[int(l)] = sum(1 << b for b, name in enumerate(_FORM_FLAGS) if v.get(name))
    else:
        ch[:len(forms)] = np.asarray(forms, np.int32)
    return ch


def fb_operator_set_forms(op, forms, stream=None):
    """Installs per-level translation forms: forms is the dict
    fb_operator_autotune returns (or one with the same "..._on" flags) or a
    sequence of up to 13 choice ints (bits 0-11 as in include/fmmbem.h)."""
    ch = _forms_choice(forms)
    _check(lib.fb_operator_set_forms(op, ch.ctypes.data, _stream(stream)))


FB_TRANS_AUTO, FB_TRANS_COMPOSED, FB_TRANS_RCR, FB_TRANS_TENSOR = 0, 1, 2, 3
lib.fb_operator_set_translation.restype = C.c_int
lib.fb_operator_set_translation.argtypes = [C.c_void_p, C.c_int]


def fb_operator_set_translation(op, method):
    _check(lib.fb_operator_set_translation(op, int(method)))


lib.fb_measure_alu_peaks.restype = C.c_int
lib.fb_measure_alu_peaks.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]


def fb_measure_alu_peaks(stream=None):
    """Measured (FP32, FP64) FMA throughput of the current device in TFLOP/s."""
    a, b = C.c_double(), C.c_double()
    _check(lib.fb_measure_alu_peaks(C.byref(a), C.byref(b), _stream(stream)))
    return a.value, b.value


FB_PC_LEARNED = 2
FB_PC_INNER = 3
lib.fb_precond_create_inner.restype = C.c_int
lib.fb_precond_create_inner.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                        C.POINTER(C.c_void_p)]


lib.fb_krylov_basis.restype = C.c_int
lib.fb_krylov_basis.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]


def fb_krylov_basis(A, pc, b, k, stream=None):
    """First k+1 Arnoldi vectors (CUDA complex128 [k+1, N]) of the right-
    preconditioned Krylov space of A from b (CUDA complex128 [N])."""
    import torch
    pb = _cuda_ptr(b, "b")
    V = torch.empty((int(k) + 1, b.numel()), dtype=b.dtype, device=b.device)
    _check(lib.fb_krylov_basis(A, pc, pb, int(k), C.c_void_p(V.data_ptr()), _stream(stream)))
    return V


def fb_precond_create_inner(op, inner_op, inner_pc=None, iters=4, stream=None):
    """Inner-outer preconditioner: `iters` GMRES steps on inner_op (right-
    preconditioned by inner_pc) per application."""
    out = C.c_void_p()
    _check(lib.fb_precond_create_inner(op, inner_op, inner_pc, int(iters), _stream(stream), C.byref(out)))
    return out
lib.fb_precond_create_learned.restype = C.c_int
lib.fb_precond_create_learned.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.POINTER(C.c_void_p)]
lib.fb_learned_params.restype = C.c_int
lib.fb_learned_params.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)]
lib.fb_learned_loss_and_grad.restype = C.c_int
lib.fb_learned_loss_and_grad.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_double),
                                         C.c_void_p, C.c_void_p]
lib.fb_learned_train_step.restype = C.c_int
lib.fb_learned_train_step.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                                      C.POINTER(C.c_double), C.c_void_p]


FB_LOSS_ERROR, FB_LOSS_RESIDUAL = 0, 1
lib.fb_learned_set_objective.restype = C.c_int
lib.fb_learned_set_objective.argtypes = [C.c_void_p, C.c_int]


def fb_learned_set_objective(pc, objective):
    _check(lib.fb_learned_set_objective(pc, int(objective)))


def fb_precond_create_learned(op, base, seed=2103_16073, stream=None):
    out = C.c_void_p()
    _check(lib.fb_precond_create_learned(op, base, int(seed), _stream(stream), C.byref(out)))
    return out


def fb_learned_params(pc, new=None):
    """Returns the FP32 parameters; replaces them first if `new` is given."""
    cnt = C.c_int64(0)
    if new is not None:
        arr = np.ascontiguousarray(new, dtype=np.float32)
        cnt.value = arr.size
        _check(lib.fb_learned_params(pc, None, arr.ctypes.data, C.byref(cnt)))
    _check(lib.fb_learned_params(pc, None, None, C.byref(cnt)))
    out = np.zeros(cnt.value, np.float32)
    _check(lib.fb_learned_params(pc, out.ctypes.data, None, C.byref(cnt)))
    return out


def fb_learned_loss_and_grad(pc, R, E, stream=None):
    """R, E: CUDA complex128 tensors [npairs, N].  Returns (loss, grad)."""
    pr, pe = _cuda_ptr(R, "R"), _cuda_ptr(E, "E")
    cnt = C.c_int64(0)
    _check(lib.fb_learned_params(pc, None, None, C.byref(cnt)))
    grad = np.zeros(cnt.value, np.float32)
    loss = C.c_double()
    _check(lib.fb_learned_loss_and_grad(pc, pr, pe, R.shape[0], C.byref(loss), grad.ctypes.data, _stream(stream)))
    return loss.value, grad


def fb_learned_train_step(pc, R, E, lr, stream=None):
    pr, pe = _cuda_ptr(R, "R"), _cuda_ptr(E, "E")
    loss = C.c_double()
    _check(lib.fb_learned_train_step(pc, pr, pe, R.shape[0], float(lr), C.byref(loss), _stream(stream)))
    return loss.value


lib.fb_mesh_set_admittance_plus.restype = C.c_int
lib.fb_mesh_set_admittance_plus.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
lib.fb_ibem_gammas_monopole.restype = C.c_int
lib.fb_ibem_gammas_monopole.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
lib.fb_ibem_rhs.restype = C.c_int
lib.fb_ibem_rhs.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
lib.fb_ibem_field.restype = C.c_int
lib.fb_ibem_field.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                              C.c_void_p]


def fb_mesh_set_admittance_plus(mesh, beta, stream=None):
    """Admittance of the + side (the side the normal points to) for the
    indirect system FB_OP_IBEM."""
    p, ms, keep = _ptr(beta, np.complex128)
    _check(lib.fb_mesh_set_admittance_plus(mesh, p, ms, _stream(stream)))


def fb_ibem_gammas_monopole(op, src, stream=None):
    """(gamma+, gamma-) of Eq. (ibem4) for a monopole at src: CUDA complex128
    tensors of N values each (op: an FB_OP_IBEM operator)."""
    import torch
    n = fb_operator_info(op)[0] // 2
    gp = torch.empty(n, dtype=torch.complex128, device="cuda")
    gm = torch.empty_like(gp)
    s = np.ascontiguousarray(src, dtype=np.float64)
    _check(lib.fb_ibem_gammas_monopole(op, s.ctypes.data, C.c_void_p(gp.data_ptr()), C.c_void_p(gm.data_ptr()),
                                       _stream(stream)))
    return gp, gm


def fb_ibem_rhs(op, gamma_p, gamma_m, stream=None):
    """Right-hand side of Eq. (ibem5) (CUDA complex128, 2N) from gamma+/-."""
    import torch
    b = torch.empty(2 * gamma_p.numel(), dtype=torch.complex128, device="cuda")
    _check(lib.fb_ibem_rhs(op, _cuda_ptr(gamma_p, "gamma_p"), _cuda_ptr(gamma_m, "gamma_m"), C.c_void_p(b.data_ptr()),
                           _stream(stream)))
    return b


def fb_ibem_field(op, x, gamma_p, gamma_m, rcv, stream=None):
    """Scattered field L[sigma] + M[mu] (Eq. ibem1) of a solution x (2N) at
    receivers rcv (CUDA float64 [nr, 3]); returns CUDA complex128 [nr]."""
    import torch
    out = torch.empty(rcv.shape[0], dtype=torch.complex128, device="cuda")
    _check(lib.fb_ibem_field(op, _cuda_ptr(x, "x"), _cuda_ptr(gamma_p, "gamma_p"), _cuda_ptr(gamma_m, "gamma_m"),
                             _cuda_ptr(rcv, "rcv"), int(rcv.shape[0]), C.c_void_p(out.data_ptr()), _stream(stream)))
    return out


lib.fb_dbem5_rhs.restype = C.c_int
lib.fb_dbem5_rhs.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
lib.fb_dbem5_psi.restype = C.c_int
lib.fb_dbem5_psi.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]


def fb_dbem5_rhs(op, gamma, stream=None):
    """Right-hand side of Eq. (dbem5) (CUDA complex128, N) from gamma."""
    import torch
    b = torch.empty_like(gamma)
    _check(lib.fb_dbem5_rhs(op, _cuda_ptr(gamma, "gamma"), C.c_void_p(b.data_ptr()), _stream(stream)))
    return b


def fb_dbem5_psi(op, q, gamma, stream=None):
    """psi_sc from the Eq. (dbem5) solution q = d psi_sc/dn."""
    import torch
    psi = torch.empty_like(q)
    _check(lib.fb_dbem5_psi(op, _cuda_ptr(q, "q"), _cuda_ptr(gamma, "gamma"), C.c_void_p(psi.data_ptr()),
                            _stream(stream)))
    return psi


lib.fb_image_field.restype = C.c_int
lib.fb_image_field.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_int, C.c_void_p,
                               C.c_int64, C.c_void_p, C.c_void_p]
lib.fb_pulse_synthesis.restype = C.c_int
lib.fb_pulse_synthesis.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_double, C.c_int,
                                   C.c_double, C.c_void_p, C.c_void_p]


def fb_image_field(room, src, R_walls, k, rcv, a_th=1e-7, stream=None):
    """Image-source field (Eq. an2) at receivers rcv (CUDA float64 [nr, 3])
    for wavenumbers k; returns CUDA complex128 [nf, nr]."""
    import torch
    room = np.ascontiguousarray(room, dtype=np.float64)
    src = np.ascontiguousarray(src, dtype=np.float64)
    Rw = np.ascontiguousarray(np.broadcast_to(np.asarray(R_walls, dtype=np.complex128), (6,)))
    kk = np.ascontiguousarray(np.atleast_1d(k), dtype=np.float64)
    out = torch.empty((kk.size, rcv.shape[0]), dtype=torch.complex128, device="cuda")
    _check(lib.fb_image_field(room.ctypes.data, src.ctypes.data, Rw.ctypes.data, float(a_th), kk.ctypes.data,
                              int(kk.size), _cuda_ptr(rcv, "rcv"), int(rcv.shape[0]), C.c_void_p(out.data_ptr()),
                              _stream(stream)))
    return out


def fb_pulse_synthesis(psi, freqs, df, dt, nt, pulse_dt, stream=None):
    """Time response (CUDA float64 [nt, nr]) to the pulse of Eq. (an3) from
    psi (CUDA complex128 [nf, nr]) at frequencies freqs (spacing df)."""
    import torch
    f = np.ascontiguousarray(freqs, dtype=np.float64)
    out = torch.empty((int(nt), psi.shape[1]), dtype=torch.float64, device="cuda")
    _check(lib.fb_pulse_synthesis(_cuda_ptr(psi, "psi"), f.ctypes.data, int(f.size), int(psi.shape[1]), float(df),
                                  float(dt), int(nt), float(pulse_dt), C.c_void_p(out.data_ptr()), _stream(stream)))
    return out


lib.fb_batch_partition.restype = C.c_int
lib.fb_batch_partition.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]


def fb_batch_partition(costs, nranks):
    """Owner rank of every job (largest cost first to the least loaded rank)
    and the resulting load per rank (host only, no GPU)."""
    c = np.ascontiguousarray(costs, dtype=np.float64)
    owner = np.zeros(c.shape[0], np.int32)
    load = np.zeros(int(nranks), np.float64)
    _check(lib.fb_batch_partition(c.ctypes.data, c.shape[0], int(nranks), owner.ctypes.data, load.ctypes.data))
    return owner, load


lib.fb_operator_status.restype = C.c_int
lib.fb_operator_status.argtypes = [C.c_void_p, C.c_void_p]
lib.fb_set_device_wait_limit.restype = C.c_int
lib.fb_set_device_wait_limit.argtypes = [C.c_longlong, C.POINTER(C.c_longlong)]
lib.fb_test_stall_device_waits.restype = C.c_int
lib.fb_test_stall_device_waits.argtypes = [C.c_int]


lib.fb_operator_set_near_bf16.restype = C.c_int
lib.fb_operator_set_near_bf16.argtypes = [C.c_void_p, C.c_int, C.c_void_p]


def fb_operator_set_near_bf16(op, enable=True, stream=None):
    """Near-field entries of a mixed operator as BF16 pairs (for low-accuracy
    inner operators) or back to FP32."""
    _check(lib.fb_operator_set_near_bf16(op, 1 if enable else 0, _stream(stream)))


lib.fb_operator_staged_pass_times.restype = C.c_int
lib.fb_operator_staged_pass_times.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]


def fb_operator_staged_pass_times(op, stream=None):
    """{level: {"prep", "rot", "coax", "back" (device ms of each staged M2L
    pass alone), "form" ("cuda", "tensor_rot", "tensor_rot_coax" or "df")}} for the operator's
    staged levels; overwrites its expansion buffers."""
    ms = np.full(4 * 13, -1.0)
    tc = np.zeros(13, np.int32)
    _check(lib.fb_operator_staged_pass_times(op, _stream(stream), ms.ctypes.data, tc.ctypes.data))
    out = {}
    for l in range(13):
        t = ms[4 * l:4 * l + 4]
        if np.all(t < 0):
            continue
        out[l] = {"prep": float(t[0]), "rot": float(t[1]), "coax": float(t[2]), "back": float(t[3]),
                  "form": {1: "cuda", 2: "tensor_rot", 3: "df", 5: "tensor_rot_coax"}.get(int(tc[l]), "none")}
    return out


def fb_operator_status(op, stream=None):
    """FB_OK, or raises FBError(FB_ERR_TIMEOUT) if a bounded device wait of the
    operator's kernels ran out since the last check (the flag is cleared)."""
    _check(lib.fb_operator_status(op, _stream(stream)))


def fb_set_device_wait_limit(limit):
    """Polls per bounded device wait (library-wide); returns the previous value."""
    prev = C.c_longlong()
    _check(lib.fb_set_device_wait_limit(int(limit), C.byref(prev)))
    return prev.value


def fb_test_stall_device_waits(enable):
    """Test hook: tensor-core kernels first wait on a barrier nothing signals."""
    _check(lib.fb_test_stall_device_waits(int(bool(enable))))
