"""The bounds-checked build (libhelm_checked.so, -DHELM_CHECKED): the hot kernels of
both precisions run through it on grids that exercise the tile edges (odd and even
3D n, 2D), with results equal to the normal build's and no index out of range
recorded.  The checked library runs in a child process (HELM_LIBRARY=checked) so
that each process loads one libhelm."""
import json
import os
import subprocess
import sys

import pytest

from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import ctypes as C, json, sys
import numpy as np, torch
sys.path.insert(0, %(root)r)
import scenes
from tests.gpu_common import problem_for, small_scene, to_dev
import paper_2405_12380_gb300 as hm
from paper_2405_12380_gb300 import _lib
out = {}
for dim, n, prec, method, relax in [(3, 36, "mixed", "bicgstab", "rbgs"), (3, 37, "mixed", "bicgstab", "rbgs"),
                                    (3, 36, "fp64", "bicgstab", "rbgs"), (3, 21, "fp64", "fgmres", "jacobi"),
                                    (2, 45, "fp64", "bicgstab", "rbgs"), (3, 38, "mixed", "fgmres", "ssor")]:
    s = small_scene(dim, n)
    P = problem_for(s, precision=prec)
    layers = scenes.glorot_mlp(np.random.default_rng(3), [dim, 32, 32, 16])
    P.don_load(layers, 16, tau=1e-3)
    x, st = P.solve(to_dev(s["b"]), None, hm.opts(method, relax, 2, omega=1.1, tol=1e-6, maxit=60))
    xr = P.relax(relax if relax != "jacobi" else "rbgs", to_dev(s["b"], torch.complex64),
                 to_dev(s["b"], torch.complex64), sweeps=2, omega=1.2)
    out[f"{dim}-{n}-{prec}-{method}-{relax}"] = [x.cpu().numpy().tolist()[:64], st["iters"],
                                                 xr.cpu().numpy().tolist()[:64]]
    P.close()
chk, first = C.c_int(0), C.c_ulonglong(0)
rc = _lib.lib().helm_checked_status(C.byref(chk), C.byref(first))
out["checked"] = [rc, chk.value, first.value]
print("RESULT " + json.dumps(out, default=lambda z: [z.real, z.imag]))
"""


def _run(checked):
    env = dict(os.environ)
    if checked:
        env["HELM_LIBRARY"] = "checked"
    else:
        env.pop("HELM_LIBRARY", None)
    r = subprocess.run([sys.executable, "-c", CHILD % {"root": ROOT}], env=env, capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_checked_build_records_nothing_and_matches_normal_build():
    need_gpu()
    if not os.path.exists(os.path.join(ROOT, "paper_2405_12380_gb300", "libhelm_checked.so")):
        pytest.fail("libhelm_checked.so not built (__graft_entry__.build builds it)")
    a = _run(False)
    b = _run(True)
    assert b["checked"] == [0, 1, 0], b["checked"]          # checked build, no violation recorded
    assert a["checked"][:2] == [0, 0], a["checked"]
    for key in a:
        if key == "checked":
            continue
        xa, ia, ra = a[key]
        xb, ib, rb = b[key]
        assert ia == ib, (key, ia, ib)
        assert xa == xb, key                                 # same arithmetic, bit for bit
        assert ra == rb, key
