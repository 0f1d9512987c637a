"""FP64 CPU oracle for the Helmholtz meta-solvers -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct NumPy/SciPy restatement of what the CUDA path
computes, written from the paper (arXiv 2405.12380) and the textbook methods it
names.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg may import it.  It shares no code with the CUDA path and imports
nothing from the package; its inputs come from ``scenes`` (data only).

Modules:
  assemble  -- absorbing-layer k^2, sparse complex A, lifted right-hand side (Eq. 1, FD reading)
  relax     -- damped Jacobi, red-black Gauss-Seidel (Sec. 3.1.1, Eq. 2)
  tb        -- trunk MLP, trunk-basis coarse space M2 = P (R A P)^-1 R (App. C), hybrid cycle (Eq. 3)
  krylov    -- FGMRES(m) with CGS2 + complex Givens, right-preconditioned BiCGStab,
               relaxation meta-solver (hybrid Richardson)
  mlp       -- DeepONet branch/trunk MLP forward/backward, relative-L2 loss, Adam (App. B)
  cnn       -- 3D convolution layers of the CNN branch, forward and gradients (App. B)
  bvp, mg   -- the Sommerfeld / Neumann boundary rows (Eq. 1), the multigrid V-cycle (Sec. 4.3)
  adjoint   -- receiver sampling, adjoint solve and k^2 gradient

Parity status: every function is pinned by tests/test_oracle_*.py against closed
forms, library special cases, invariants or brute force.  The paper's own
iteration counts (FEM, GRF wavenumber, trained weights) are *parity unpinned*:
they cannot be reproduced from the paper's text.
"""
