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
