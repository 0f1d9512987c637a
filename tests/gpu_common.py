"""Shared helpers of the GPU parity tests: small seeded scenes, the oracle side and
the CUDA side built from the same inputs."""
import numpy as np
import pytest

import scenes
from oracle import assemble

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_12380_gb300 import build
    import os
    if not os.path.exists(build.LIB):
        build.build()


def small_scene(dim, n, k0=9.0, cells=4, box=None, seed=0, g_nonzero=False):
    rng = np.random.default_rng(seed)
    if box is None:
        w = max(2, n // 5)
        box = scenes.centred_box_nodes(n, w)
    mask = (scenes.ring_mask(dim, n) | scenes.box_mask(dim, n, *box)).reshape(-1).astype(np.uint8)
    N = n ** dim
    src = np.where(mask == 0, rng.standard_normal(N) + 1j * rng.standard_normal(N), 0)
    g = np.where(mask == 1, rng.standard_normal(N) + 1j * rng.standard_normal(N), 0) if g_nonzero else np.zeros(N, complex)
    k2 = assemble.k2_field(dim, n, k0, cells, 0.5)
    A = assemble.assemble(dim, n, k2, mask)
    b = assemble.rhs(dim, n, mask, src, g)
    return dict(dim=dim, n=n, k0=k0, cells=cells, mask=mask, src=src, g=g, A=A, b=b, rng=rng)


def problem_for(s, precision="fp64", k2=None):
    import paper_2405_12380_gb300 as hm
    return hm.Problem(s["dim"], s["n"], s["k0"], s["mask"], layer_cells=s["cells"], layer_strength=0.5,
                      k2=k2, precision=precision)


def to_dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t if dtype is None else t.to(dtype)


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
