"""Status codes of the failure paths, each made on the host without faulting the GPU:

* HELM_TIMEOUT: every grid barrier of the cooperative red-black cycle is told to
  wait for one block more than the launch has (helm_set_wait_limit), with a small
  poll limit, so each bounded wait runs out; the solve returns HELM_TIMEOUT within
  milliseconds and the next solve on the same handle matches the oracle again.
* HELM_BREAKDOWN: a crafted system with two fluid nodes and a zero diagonal,
  A = [[0, 16], [16, 0]] (h = 1/4, k^2 = 6/h^2 given as a stored field), and
  f = (1, i): <r0, A r0> = 16 i - 16 i = 0 exactly, so BiCGStab's first alpha
  divides by zero.
* HELM_SINGULAR_COARSE: on the same system a one-column trunk T(x) = x - 1/2
  vanishes at the second fluid node, so Q = e_1 and A_c = Q^T A Q = A_11 = 0.
* HELM_OUT_OF_MEMORY: a trunk basis of 256 columns on 540^3 nodes needs a 322 GB
  trunk matrix, more than the device holds; the allocation fails cleanly.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import scenes
from oracle import assemble
from tests.gpu_common import need_gpu, problem_for, rel, small_scene, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _two_node_problem(precision="fp64"):
    import paper_2405_12380_gb300 as hm
    n = 5
    mask = np.ones((n, n, n), np.uint8)          # [k, j, i]
    mask[1, 1, 1] = 0                            # node (i, j, k) = (1, 1, 1), x = 1/4
    mask[1, 1, 2] = 0                            # node (2, 1, 1), x = 1/2
    mask = mask.reshape(-1)
    hinv2 = 16.0                                 # h = 1/4 exactly
    k2 = np.full(n ** 3, 6.0 * hinv2 + 0j)       # k^2 - 6 h^-2 = 0 on the fluid nodes
    P = hm.Problem(3, n, np.sqrt(6.0 * hinv2), mask, layer_cells=0, layer_strength=0.0, k2=to_dev(k2),
                   precision=precision)
    l1, l2 = 1 + n * (1 + n * 1), 2 + n * (1 + n * 1)
    f = np.zeros(n ** 3, complex)
    f[l1], f[l2] = 1.0, 1j
    return P, f, (l1, l2)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bicgstab_breakdown_on_crafted_system(precision):
    import paper_2405_12380_gb300 as hm
    P, f, _ = _two_node_problem(precision)
    x, st = P.solve(to_dev(f), None, hm.opts("bicgstab", "none", 0, correction="none", tol=1e-10, maxit=50))
    assert st["status_name"] == "breakdown", st["status_name"]
    assert st["iters"] <= 2


def test_singular_coarse_operator():
    import paper_2405_12380_gb300 as hm
    P, f, _ = _two_node_problem()
    layers = [(np.array([[1.0, 0.0, 0.0]]), np.array([-0.5]))]     # T(x) = x - 1/2
    with pytest.raises(hm.HelmError) as e:
        P.don_load(layers, 1, tau=0.0)
    assert e.value.status == 7, e.value                                # HELM_SINGULAR_COARSE


@pytest.mark.parametrize("precision", ["fp64"])
def test_barrier_timeout_returns_timeout_and_handle_recovers(precision):
    """The double-float cooperative cycle of FP64 handles inside BiCGStab, and the
    same handle's preconditioner call (helm_precond).  (The complex64 cycle of
    mixed handles has no grid-wide wait: its sweeps are separate launches.)"""
    import paper_2405_12380_gb300 as hm
    import time
    s = small_scene(3, 25)
    P = problem_for(s, precision=precision)
    layers = scenes.glorot_mlp(np.random.default_rng(5), [3, 32, 32, 24])
    P.don_load(layers, 24, tau=1e-6)
    o = hm.opts("bicgstab", "rbgs", 3, tol=1e-10, maxit=4000)
    f = to_dev(s["b"])
    P.set_wait_limit(2000, 1)             # every barrier waits for one block that never comes
    t0 = time.perf_counter()
    x, st = P.solve(f, None, o)
    dt = time.perf_counter() - t0
    assert st["status_name"] == "timeout", st["status_name"]
    assert dt < 5.0, dt
    # the preconditioner call alone reports it too
    with pytest.raises(hm.HelmError) as e:
        P.precond(f, o)
    assert e.value.status == 11
    # back to normal waits: the barrier state was reset, the solve converges to the LU solution
    P.set_wait_limit(1 << 20, 0)
    x, st = P.solve(f, None, hm.opts("bicgstab", "rbgs", 3, tol=1e-10 if precision == "fp64" else 1e-6,
                                     maxit=4000))
    assert st["status"] == 0, st["status_name"]
    u = spla.spsolve(s["A"].tocsc(), s["b"])
    assert rel(x.cpu().numpy(), u) < (1e-7 if precision == "fp64" else 1e-3)


def test_out_of_memory_is_a_status():
    import paper_2405_12380_gb300 as hm
    n = 540
    mask = scenes.ring_mask(3, n).reshape(-1).astype(np.uint8)
    P = hm.Problem(3, n, 16.0, mask, layer_cells=8, layer_strength=0.5)
    layers = scenes.glorot_mlp(np.random.default_rng(0), [3, 256])
    with pytest.raises(hm.HelmError) as e:
        P.don_load(layers, 256, tau=1e-6)
    assert e.value.status == 9, e.value                                # HELM_OUT_OF_MEMORY
    # the handle is still usable
    x = torch.zeros(P.N, dtype=torch.complex128, device="cuda")
    y = P.apply(x)
    assert float(y.abs().max()) == 0.0
    P.close()
    torch.cuda.empty_cache()
