"""The tcgen05 BF16 GEMM (nn_gemm_bf16) against the oracle: the reference is the
FP64 product of the operands rounded to BF16 by the oracle's own rounding
(oracle/tb.py bf16_round, pinned against torch.bfloat16), so the only difference
left is the FP32 accumulation order: |C - ref| <= 4 K 2^-24 (|A_bf| |B_bf|) + a
tiny absolute term, element by element.  Shapes cover one tile, ragged edges in M,
N and K, several K steps (the four-stage ring wraps), all four transpose cases and
alpha / beta; the kernel's wait flag must stay clear."""
import ctypes as C

import numpy as np
import pytest

from oracle.tb import bf16_round
from tests.gpu_common import need_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("ta,tb,M,N,K", [(0, 0, 128, 128, 64), (0, 1, 200, 130, 100), (1, 0, 77, 300, 1000),
                                         (1, 1, 256, 256, 576), (0, 1, 1000, 96, 40), (0, 0, 5, 7, 3)])
def test_gemm_bf16_matches_rounded_oracle(ta, tb, M, N, K):
    from paper_2405_12380_gb300 import _lib as L
    rng = np.random.default_rng(M * 7 + N + K)
    A = rng.standard_normal((K, M) if ta else (M, K)).astype(np.float32)
    B = rng.standard_normal((N, K) if tb else (K, N)).astype(np.float32)
    C0 = rng.standard_normal((M, N)).astype(np.float32)
    opA = bf16_round((A.T if ta else A).astype(np.float64))
    opB = bf16_round((B.T if tb else B).astype(np.float64))
    for alpha, beta in ((1.0, 0.0), (0.7, -1.3)):
        ref = alpha * (opA @ opB) + beta * C0.astype(np.float64)
        bound = 4 * K * 2.0 ** -24 * abs(alpha) * (np.abs(opA) @ np.abs(opB)) + 2e-6 * abs(beta) * np.abs(C0) + 1e-30
        Ad, Bd, Cd = to_dev(A), to_dev(B), to_dev(C0)
        st = L.lib().nn_gemm_bf16(ta, tb, M, N, K, alpha, C.c_void_p(Ad.data_ptr()), A.shape[1],
                                  C.c_void_p(Bd.data_ptr()), B.shape[1], beta, C.c_void_p(Cd.data_ptr()), N, None)
        assert st == 0
        torch.cuda.synchronize()
        err = np.abs(Cd.cpu().numpy().astype(np.float64) - ref)
        assert np.all(err <= bound), (float(err.max()), float((err / bound).max()))
        flag = C.c_int(-1)
        assert L.lib().nn_gemm_bf16_status(C.byref(flag)) == 0 and flag.value == 0
