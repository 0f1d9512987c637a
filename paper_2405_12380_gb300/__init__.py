"""GB300-native meta-solvers for the complex Helmholtz equation (arXiv 2405.12380).

The compute path is libhelm.so (hand-written CUDA for sm_103a behind the C ABI of
include/helm.h); this package only marshals torch tensors into that ABI.
"""
from .helm import Batch, Problem, SolveOpts, HelmError, opts, solve_concurrent  # noqa: F401
