"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports every
symbol that include/helm.h declares (no compute call: there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "helm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:helm_status|void|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2405_12380_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return build.LIB


def test_header_declares_the_boundary():
    names = _declared()
    for need in ("helm_create", "helm_apply", "helm_relax", "don_correct", "helm_solve", "don_load",
                 "helm_destroy"):
        assert need in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_2405_12380_gb300 import _lib
    assert set(_declared()) == set(_lib.SIGNATURES)


def test_no_gpu_means_no_device(libpath):
    """Without a GPU, helm_create reports HELM_NO_DEVICE instead of computing on the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2405_12380_gb300 import _lib
    L = _lib.lib()
    h = ctypes.c_void_p()
    mask = (ctypes.c_uint8 * 27)(*([1] * 27))
    st = L.helm_create(3, 3, 1.0, 0, 0.5, ctypes.cast(mask, ctypes.c_void_p), None, 0, ctypes.byref(h))
    assert st == _lib.HELM_NO_DEVICE


def test_checked_build_exports_the_same_boundary():
    """The bounds-checked variant (-DHELM_CHECKED) builds and exports every declared
    symbol as well."""
    from paper_2405_12380_gb300 import build
    if not os.path.exists(build.LIB_CHECKED):
        build.build(checked=True)
    lib = ctypes.CDLL(build.LIB_CHECKED)
    for name in _declared():
        assert hasattr(lib, name), name


def test_argument_checks_need_no_device(libpath):
    """Entry points reject bad arguments before touching the GPU: the concurrent solve
    (negative count, null handles; an empty batch is a no-op) and the convolution layer
    (a kernel larger than the padded input, a zero stride)."""
    from paper_2405_12380_gb300 import _lib
    L = _lib.lib()
    assert L.helm_solve_concurrent(-1, None, None, None, None, None, 0) == _lib.HELM_BAD_ARG
    assert L.helm_solve_concurrent(2, None, None, None, None, None, 0) == _lib.HELM_BAD_ARG
    assert L.helm_solve_concurrent(0, None, None, None, None, None, 0) == _lib.HELM_OK
    buf = (ctypes.c_float * 64)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    assert L.nn_conv3d(1, 1, 2, 1, 1, 0, p, p, None, p, None) == _lib.HELM_BAD_ARG
    assert L.nn_conv3d(1, 1, 8, 1, 0, 0, p, p, None, p, None) == _lib.HELM_BAD_ARG
    assert L.nn_conv3d_backward(1, 1, 8, 1, 1, 3, p, p, p, p, p, p, None) == _lib.HELM_BAD_ARG
