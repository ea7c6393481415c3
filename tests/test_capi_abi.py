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
    # launch shapes of the uneven batch: four int arrays, one entry per problem class
    assert C.sizeof(capi.cprrtc_tuning) == 4 * capi.BATCH_CLASSES * 4
    body = hdr[:hdr.index("} cprrtc_tuning;")]
    body = re.sub(r"/\*.*?\*/", "", body[body.rindex("typedef struct {"):], flags=re.S)
    names = re.findall(r"int (\w+)\[CPRRTC_BATCH_CLASSES\];", body)
    assert names == [f[0] for f in capi.cprrtc_tuning._fields_]
    assert int(re.search(r"#define CPRRTC_BATCH_CLASSES (\d+)", hdr).group(1)) == capi.BATCH_CLASSES


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


def test_codes_agree_across_header_kernels_oracle_and_generators():
    """The constraint, status and error codes are written down separately in the public
    header, the kernels' device types, the oracle's header, the Python binding and the input
    generators (the oracle shares no code with the library): they must agree."""
    from paper_2505_06791_gb300 import synth as S

    root = os.path.dirname(os.path.dirname(capi.__file__))
    hdr = open(capi.HEADER).read()
    dev = open(os.path.join(os.path.dirname(capi.__file__), "csrc", "device_types.cuh")).read()
    orc = open(os.path.join(root, "oracle", "cprrtc_oracle.h")).read()

    def define(name):
        return int(re.search(r"#define\s+" + name + r"\s+\(?(-?\d+)\)?", hdr).group(1))

    def enum(text, name):
        return int(re.search(r"\b" + name + r"\s*=\s*(\d+)", text).group(1))

    cons = [("NONE", "kConsNone", "ORC_NONE", S.C_NONE),
            ("ROLL_PITCH", "kConsRollPitch", "ORC_ROLL_PITCH", S.C_ROLL_PITCH),
            ("Z_PLANE", "kConsZPlane", "ORC_Z_PLANE", S.C_Z_PLANE),
            ("LINE", "kConsLine", "ORC_LINE", S.C_LINE),
            ("ORIENT_PLANE", "kConsOrientPlane", "ORC_ORIENT_PLANE", S.C_ORIENT_PLANE),
            ("ORIENT_LINE", "kConsOrientLine", "ORC_ORIENT_LINE", S.C_ORIENT_LINE)]
    for h, d, o, s in cons:
        v = define("CPRRTC_CONSTRAINT_" + h)
        assert v == enum(dev, d) == enum(orc, o) == s, h
    status = [("VALID", "kValid", "ORC_VALID", capi.MOTION_VALID),
              ("PROJ_FAIL", "kProjFail", "ORC_PROJ_FAIL", capi.MOTION_PROJ_FAIL),
              ("COLLISION", "kCollision", "ORC_COLLISION", capi.MOTION_COLLISION)]
    for h, d, o, p in status:
        assert define("CPRRTC_MOTION_" + h) == enum(dev, d) == enum(orc, o) == p, h
    for name in ("INVALID_ARG", "NOT_CONFIGURED", "CUDA", "OOM", "CAPACITY", "TIMEOUT",
                 "UNSUPPORTED"):
        assert define("CPRRTC_E_" + name) == getattr(capi, "E_" + name), name
    assert define("CPRRTC_OK") == capi.OK == 0
    assert define("CPRRTC_MLP_BF16") == capi.MLP_BF16 == 0
    assert define("CPRRTC_MLP_FP32") == capi.MLP_FP32 == 1
    assert define("CPRRTC_MAX_DOF") == int(re.search(r"kMaxDof = (\d+)", dev).group(1)) == \
        int(re.search(r"ORC_MAX_DOF (\d+)", orc).group(1))
    assert define("CPRRTC_MAX_W") == int(re.search(r"kMaxW = (\d+)", dev).group(1)) == \
        int(re.search(r"ORC_MAX_W (\d+)", orc).group(1))
