"""The C-ABI library loads and exports every entry point include/cprrtc.h declares; the
ctypes struct layouts match the header. No compute calls: this runs without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2505_06791_gb300 import build, capi


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    declared = capi.header_symbols()
    assert len(declared) >= 12
    L = C.CDLL(libpath)
    for name in declared:
        assert hasattr(L, name), name
    # the binding wires every declared function
    assert set(declared) <= set(capi._SIGS)


def test_struct_layouts_match_header():
    assert capi.JOINT_DT.itemsize == 56
    assert capi.SPHERE_DT.itemsize == 40
    assert capi.OBS_SPHERE_DT.itemsize == 32
    assert capi.OBS_BOX_DT.itemsize == 120
    assert capi.OBS_CAPSULE_DT.itemsize == 56
    # int, 7 doubles, int (padded to 8), 2 doubles
    assert C.sizeof(capi.cprrtc_constraint) == 88
    # field order mirrors the header's struct declarations
    hdr = open(capi.HEADER).read()
    body = hdr[:hdr.index("} cprrtc_constraint;")]
    body = re.sub(r"/\*.*?\*/", "", body[body.rindex("typedef struct {"):], flags=re.S)
    names = re.findall(r"(\w+);", body)
    assert names == ["type", "target", "tol_task", "c_sm", "tau_floor", "tol_sm", "alpha",
                     "lambda", "max_iters", "line_y", "yaw"]


def test_null_context_is_rejected(libpath):
    L = capi.lib()
    assert L.cprrtc_set_timing(None, 1) == capi.E_INVALID_ARG
    assert L.cprrtc_destroy(None) == capi.OK
    assert L.cprrtc_create(None, 0, None) == capi.E_INVALID_ARG


def test_binding_refuses_to_run_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(capi, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(capi, "_lib", None)
    with pytest.raises(ImportError):
        capi.lib()


def test_oracle_is_not_imported_by_the_package():
    pkg = os.path.dirname(capi.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(root, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "cprrtc_oracle" not in text, f


def test_oracle_shares_nothing_with_the_cuda_library():
    """The oracle's sources include only the C library and its own header, and its Python
    loader imports nothing from the package (not even the input generators)."""
    root = os.path.join(os.path.dirname(os.path.dirname(capi.__file__)), "oracle")
    for f in os.listdir(root):
        if not f.endswith((".c", ".h", ".py")):
            continue
        text = open(os.path.join(root, f)).read()
        for inc in re.findall(r'#include\s*[<"]([^>"]+)[>"]', text):
            assert inc in ("cprrtc_oracle.h", "math.h", "pthread.h", "stdlib.h", "string.h",
                           "stdint.h"), (f, inc)
        assert "paper_2505_06791_gb300" not in text and "cprrtc.h" not in text, f
        assert "csrc" not in text, f
