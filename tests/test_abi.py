"""The C-ABI library builds, loads and exports every symbol its header
declares (no GPU needed: nothing here launches device work)."""
import os
import re

import paper_2103_16073_gb300 as fb

HEADER = os.path.join(os.path.dirname(__file__), "..", "include", "fmmbem.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^FB_API\s+[\w\s\*]+?\b(fb_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_api():
    names = declared_symbols()
    assert len(names) >= 20
    for must in ("fb_mesh_create", "fb_tree_build", "fb_operator_create", "fb_operator_apply",
                 "fb_fgmres_solve", "fb_eval_field", "fb_precond_create"):
        assert must in names


def test_library_exports_every_declared_symbol():
    for name in declared_symbols():
        assert hasattr(fb.lib, name), name


def test_version_and_error_buffer():
    assert "sm_103a" in fb.fb_version()
    import ctypes
    buf = ctypes.create_string_buffer(64)
    fb.lib.fb_last_error(buf, 64)


def test_argument_errors_are_reported_without_device_work():
    import numpy as np
    import pytest
    with pytest.raises(fb.FBError) as e:
        fb.fb_mesh_create(np.zeros((3, 3)), np.array([[0, 1, 5]]))   # index out of range
    assert e.value.code == 1


def test_new_entry_points_validate_arguments_on_the_host():
    """Argument checks of the broadband, indirect and dbem5 entry points run
    before any device work and report FB_ERR_ARG."""
    import ctypes as C
    import numpy as np
    lib = fb.lib
    room = np.array([8.0, 6.0, 3.0])
    outside = np.array([9.0, 2.0, 1.0])
    Rw = np.zeros(12)
    k = np.array([1.0])
    dummy = C.c_void_p(16)
    # source outside the room, no wavenumbers, non-positive threshold
    assert lib.fb_image_field(room.ctypes.data, outside.ctypes.data, Rw.ctypes.data, 1e-7, k.ctypes.data, 1,
                              dummy, 1, dummy, None) == 1
    src = np.array([3.0, 2.0, 1.0])
    assert lib.fb_image_field(room.ctypes.data, src.ctypes.data, Rw.ctypes.data, 1e-7, k.ctypes.data, 0,
                              dummy, 1, dummy, None) == 1
    assert lib.fb_image_field(room.ctypes.data, src.ctypes.data, Rw.ctypes.data, 0.0, k.ctypes.data, 1,
                              dummy, 1, dummy, None) == 1
    f = np.array([10.0])
    assert lib.fb_pulse_synthesis(dummy, f.ctypes.data, 1, 1, 0.0, 1e-3, 8, 1e-3, dummy, None) == 1   # df = 0
    assert lib.fb_pulse_synthesis(dummy, f.ctypes.data, 1, 1, 10.0, 1e-3, 0, 1e-3, dummy, None) == 1  # nt = 0
    # NULL handles
    assert lib.fb_ibem_rhs(None, dummy, dummy, dummy, None) == 1
    assert lib.fb_ibem_field(None, dummy, dummy, dummy, dummy, 1, dummy, None) == 1
    assert lib.fb_dbem5_rhs(None, dummy, dummy, None) == 1
    assert lib.fb_dbem5_psi(None, dummy, dummy, dummy, None) == 1
    assert lib.fb_krylov_basis(None, None, dummy, 3, dummy, None) == 1


def test_image_field_refuses_excessive_image_orders():
    """|R| = 0.999 with a_th = 1e-7 would need thousands of image orders per
    axis: refused on the host before any allocation."""
    import ctypes as C
    import numpy as np
    room = np.array([8.0, 6.0, 3.0])
    src = np.array([3.0, 2.0, 1.0])
    Rw = np.array([0.999, 0.0] * 6)
    k = np.array([1.0])
    dummy = C.c_void_p(16)
    assert fb.lib.fb_image_field(room.ctypes.data, src.ctypes.data, Rw.ctypes.data, 1e-7, k.ctypes.data, 1,
                                 dummy, 1, dummy, None) == 1


def test_input_generators_do_not_map_the_library():
    """The seeded input generators (shared with the oracle side) import
    without loading libfmmbem.so: the package loads its binding only on the
    first use of a binding name."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import paper_2103_16073_gb300 as P\n"
            "from paper_2103_16073_gb300 import workloads\n"
            "import oracle.bem\n"
            "assert 'paper_2103_16073_gb300.binding' not in sys.modules\n"
            "maps = open('/proc/self/maps').read()\n"
            "assert 'libfmmbem' not in maps\n"
            "P.FB_OP_A\n"
            "assert 'libfmmbem' in open('/proc/self/maps').read()\n" % root)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_operator_entry_points_refuse_null_handles_on_the_host():
    """The operator-level entry points (translation forms, autotuner, graphs,
    timing, no-allocation matvec, BF16 near field, sibling operators) report
    FB_ERR_ARG for a NULL handle or pointer before any device work."""
    import ctypes as C
    import numpy as np
    lib = fb.lib
    ms = np.zeros(64)
    ch = np.zeros(16, np.int32)
    out = C.c_void_p()
    cnt = C.c_int64()
    assert lib.fb_operator_create_like(None, fb.FB_PREC_MIXED_FMM, 6.0, 12, None, C.byref(out)) == 1
    assert lib.fb_operator_apply_noalloc(None, ms.ctypes.data, ms.ctypes.data, None) == 1
    assert lib.fb_operator_apply_timed(None, ms.ctypes.data, ms.ctypes.data, None, ms.ctypes.data) == 1
    assert lib.fb_operator_set_near_bf16(None, 1, None) == 1
    assert lib.fb_operator_staged_pass_times(None, None, ms.ctypes.data, ch.ctypes.data) == 1
    assert lib.fb_operator_autotune(None, 1, None, None, None) == 1
    assert lib.fb_operator_set_forms(None, ch.ctypes.data, None) == 1
    assert lib.fb_operator_set_translation(None, 0) == 1
    assert lib.fb_operator_use_graphs(None, 1) == 1
    assert lib.fb_precond_use_graphs(None, 1) == 1
    assert lib.fb_operator_status(None, None) == 1
    assert lib.fb_operator_export(None, 7, 0, 0, None, C.byref(cnt)) == 1
    assert lib.fb_operator_info(None, None, None, None) == 1


def test_device_wait_limit_is_a_host_setting():
    """fb_set_device_wait_limit refuses limits below 1 and returns the
    previous limit (a host-side value the tensor-core launches read)."""
    import ctypes as C
    lib = fb.lib
    prev = C.c_longlong()
    assert lib.fb_set_device_wait_limit(0, C.byref(prev)) == 1
    assert lib.fb_set_device_wait_limit(-5, None) == 1
    assert lib.fb_set_device_wait_limit(12345, C.byref(prev)) == 0
    old = prev.value
    assert old >= 1
    try:
        back = C.c_longlong()
        assert lib.fb_set_device_wait_limit(old, C.byref(back)) == 0
        assert back.value == 12345
    finally:
        lib.fb_set_device_wait_limit(old, None)


def test_empty_and_degenerate_meshes_are_refused_on_the_host():
    """No triangles, fewer than three vertices, or a negative vertex index:
    FB_ERR_ARG before any allocation."""
    import numpy as np
    import pytest
    v = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0]])
    for verts, tris in ((v, np.zeros((0, 3), np.int32)),
                        (v[:2], np.array([[0, 1, 1]])),
                        (v, np.array([[0, -1, 2]]))):
        with pytest.raises(fb.FBError) as e:
            fb.fb_mesh_create(verts, tris)
        assert e.value.code == 1


def test_forms_dict_round_trips_every_form_bit():
    """fb_operator_set_forms accepts the autotuner's dict: its "choice" ints,
    or all twelve "..._on" flags when no "choice" is given, or a list."""
    import numpy as np
    from paper_2103_16073_gb300 import binding
    tuned = {2: {"choice": 1044}, 5: {"choice": 3132}}
    assert list(binding._forms_choice(tuned)[[2, 5]]) == [1044, 3132]
    for bit, name in enumerate(binding._FORM_FLAGS):
        assert binding._forms_choice({3: {name: True}})[3] == 1 << bit
    flags = {4: {"m2l_staged_tc_on": True, "m2m_l2l_staged_tcc_on": True, "m2l_on_tensor": False}}
    assert binding._forms_choice(flags)[4] == 16 | 2048
    assert list(binding._forms_choice([0, 0, 20])[:4]) == [0, 0, 20, 0]
    assert binding._forms_choice([]).shape == (13,) and not np.any(binding._forms_choice([]))


def test_binding_constants_match_the_header():
    """Every FB_* integer constant the binding defines equals the header's
    #define of the same name (operator kinds, precisions, memory spaces,
    preconditioners, translation methods, limits, losses)."""
    import re
    from paper_2103_16073_gb300 import binding
    text = open(HEADER).read()
    defs = {}
    for name, val, sh in re.findall(r"^#define\s+(FB_[A-Z0-9_]+)\s+\(?(\d+)u?\s*(?:<<\s*(\d+))?", text,
                                    flags=re.M):
        defs[name] = int(val) << (int(sh) if sh else 0)
    checked = 0
    for name in dir(binding):
        if name.startswith("FB_") and isinstance(getattr(binding, name), int) and name in defs:
            assert getattr(binding, name) == defs[name], name
            checked += 1
    assert checked >= 20
    assert binding.NOALLOC_SCRATCH_BYTES == defs["FB_NOALLOC_SCRATCH_BYTES"]
    assert "FB_MAX_RHS" in defs and "FB_TUNE_TIMES" in defs


def test_device_pointer_marshalling_refuses_host_and_strided_tensors():
    """Entry points that take device pointers refuse a host array and a
    non-contiguous device tensor instead of passing a wrong layout."""
    import numpy as np
    import pytest
    from paper_2103_16073_gb300 import binding

    class FakeDevice:
        is_cuda = True

        def __init__(self, contiguous):
            self._c = contiguous

        def is_contiguous(self):
            return self._c

        def data_ptr(self):
            return 4096

    assert binding._cuda_ptr(FakeDevice(True), "x").value == 4096
    with pytest.raises(ValueError, match="contiguous"):
        binding._cuda_ptr(FakeDevice(False), "x")
    with pytest.raises(ValueError, match="CUDA"):
        binding._cuda_ptr(np.zeros(4, np.complex128), "x")
    with pytest.raises(ValueError, match="contiguous"):
        binding._ptr(FakeDevice(False))
