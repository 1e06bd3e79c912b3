"""The C-ABI library builds, loads and exports every entry point include/feasm.h declares.

No compute call is made (no GPU needed): loading libfeasm.so does not touch the device.
"""
from __future__ import annotations

import ctypes
import os
import re

import pytest

from paper_1305_3122_gb300 import build, feasm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "feasm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fe_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("fe_mesh_create", "fe_pattern_build", "fe_assemble_mass", "fe_assemble_wmass",
                 "fe_assemble_stiff", "fe_assemble_elas", "fe_adjoint_stiff_wmass", "fe_batch_create",
                 "fe_batch_assemble_stiff_mass"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    assert sorted(feasm.SIGNATURES) == _declared()


def test_status_strings_without_gpu(libpath):
    L = feasm.lib()
    assert L.fe_status_string(0) == b"FE_OK"
    assert L.fe_status_string(5) == b"FE_ERR_BUFFER_TOO_SMALL"
    assert L.fe_status_string(9) == b"FE_ERR_LIMIT"


def test_null_arguments_rejected_on_host(libpath):
    """Argument checks happen on the host before any CUDA call."""
    L = feasm.lib()
    assert L.fe_mesh_create(3, 1, None, None, 0, None, None) == 1          # out is null
    h = ctypes.c_void_p()
    assert L.fe_mesh_create(-1, 1, None, None, 0, None, ctypes.byref(h)) == 1
    assert L.fe_pattern_build(None, 1, 0, None, ctypes.byref(h)) == 1
    assert L.fe_assemble_mass(None, None, 0, None, 0, None) == 1
    assert b"null" in L.fe_last_error()
