"""helm_residual_noalloc: the residual entry point for callers that cannot
allocate device memory (no handle, scratch in a fixed device array).

Checked through the C ABI against helm_residual, the handle-based entry point,
on two calls in a row (the second call reuses the scratch the first one left)."""
import ctypes

import numpy as np
import pytest

from tests.gpu_common import need_gpu, problem_for, rel, small_scene, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,n", [(2, 45), (3, 37)])
def test_noalloc_residual_matches_handle_residual(dim, n):
    need_gpu()
    from paper_2405_12380_gb300 import _lib as L
    lib = L.lib()
    s = small_scene(dim, n)
    P = problem_for(s)
    stream = torch.cuda.current_stream().cuda_stream
    mask = to_dev(s["mask"])
    for call in range(2):
        x = s["rng"].standard_normal(n ** dim) + 1j * s["rng"].standard_normal(n ** dim)
        f, xd = to_dev(s["b"]), to_dev(x)
        for conj in (0, 1):
            r_ref, n_ref = P.residual(f, xd, conj=conj)
            r = torch.empty_like(xd)
            nrm = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
            st = lib.helm_residual_noalloc(dim, n, s["k0"], s["cells"], 0.5, ctypes.c_void_p(mask.data_ptr()),
                                           None, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(xd.data_ptr()),
                                           ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(nrm.data_ptr()),
                                           conj, ctypes.c_void_p(stream))
            assert st == 0, L.STATUS_NAMES.get(st, st)
            torch.cuda.synchronize()
            assert rel(r.cpu().numpy(), r_ref.cpu().numpy()) <= 1e-13
            assert abs(nrm.item() - n_ref.item()) <= 1e-13 * n_ref.item()


def test_noalloc_rejects_oversized_and_unmasked():
    need_gpu()
    from paper_2405_12380_gb300 import _lib as L
    lib = L.lib()
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    # 3D n = 700: more operator blocks than scratch entries -> rejected before any launch
    st = lib.helm_residual_noalloc(3, 700, 5.0, 8, 0.5, p, None, p, p, p, p, 0, None)
    assert st == L.HELM_SCRATCH_TOO_SMALL
    s = small_scene(2, 33)
    m = s["mask"].copy(); m[5] = 0                       # hole in the outer ring
    md = to_dev(m)
    f = to_dev(s["b"]); r = torch.empty_like(f); nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = lib.helm_residual_noalloc(2, 33, 9.0, 4, 0.5, ctypes.c_void_p(md.data_ptr()), None,
                                   ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                   ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(nrm.data_ptr()), 0, None)
    assert st == L.HELM_BAD_ARG
