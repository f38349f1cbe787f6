"""The C-ABI library loads without a GPU and exports every symbol of include/ffe.h."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1412_8754_gb300 import ffe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ffe.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^FFE_API\s+[\w\s\*]+?\b(ffe_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def built():
    from paper_1412_8754_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ffe_create", "ffe_destroy", "ffe_omega", "ffe_minimize", "ffe_phase_scan",
                     "ffe_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(ffe_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_symbol(built):
    assert sorted(ffe.exported_symbols()) == declared_functions()
    L = ffe.lib()  # loads without a GPU (static CUDA runtime)
    for n in declared_functions():
        assert hasattr(L, n)


def test_status_strings_without_gpu(built):
    L = ffe.lib()
    assert L.ffe_status_string(0) == b"ok"
    assert L.ffe_status_string(1) == b"invalid argument"
    assert L.ffe_last_error(None) == b""


def test_create_rejects_bad_model_before_device_work(built):
    import ctypes

    L = ffe.lib()
    h = ctypes.c_void_p()
    bad = ffe.ffe_model(ffe.FFE_MODEL_RAGHU2, ffe.FFE_FP32C, -1, 1.3, -0.85, -0.85, 1.54, -2.0, 1.0)
    assert L.ffe_create(ctypes.byref(bad), ctypes.byref(h)) == ffe.FFE_EINVAL
    bad2 = ffe.ffe_model(7, ffe.FFE_FP32C, -1, 1.3, -0.85, -0.85, 1.54, 2.0, 1.0)
    assert L.ffe_create(ctypes.byref(bad2), ctypes.byref(h)) == ffe.FFE_EUNSUPPORTED
    assert L.ffe_create(None, ctypes.byref(h)) == ffe.FFE_EINVAL
    assert not h.value


def test_null_context_is_rejected(built):
    L = ffe.lib()
    assert L.ffe_omega(None, None, 0, None, None, None) == ffe.FFE_EINVAL
    L.ffe_destroy(None)  # NULL-safe


def test_invalid_arguments_are_rejected_before_any_device_work(built):
    L = ffe.lib()
    om = np.zeros(4)
    y = np.zeros(4, dtype=np.float32)
    # no context, empty lines, bad N: FFE_EINVAL (1) without touching a GPU
    assert L.ffe_surrogate_targets(None, om.ctypes.data_as(ctypes.c_void_p), 1, 4, 8,
                                   y.ctypes.data_as(ctypes.c_void_p)) == 1
