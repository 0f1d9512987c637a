/*
 * helm.h -- C ABI of libhelm: GB300 (sm_103a) meta-solvers for the discretised
 * complex Helmholtz equation with an absorbing layer and a sound-soft scatterer
 * (arXiv 2405.12380, "Fast meta-solvers for 3D complex-shape scatterers using
 * neural operators trained on a non-scattering problem").
 *
 * Problem (Eq. 1, finite-difference reading): on n^d nodes of [0,1]^d,
 * d in {2,3}, h = 1/(n-1), flat index l = i + n*(j + n*k) (x fastest),
 *   fluid rows   (A x)_l = h^-2 sum_{fluid nbr m} x_m + (k_l^2 - 2d h^-2) x_l
 *   masked rows  (A x)_l = x_l                  (Dirichlet: scatterer + outer ring)
 *   k_l^2 = k0^2 (1 + i*s*eta_l^2), eta_l = max_a max(0, L - dist_a)/L,
 *   dist_a = min(i_a, n-1-i_a)     (absorbing layer of L cells, strength s)
 * unless a per-node complex k^2 field is supplied.  A is complex symmetric, so
 * A^H = conj(A); every operator entry point takes a `conj` flag for the adjoint.
 *
 * Conventions
 *  - Every call returns helm_status (0 = HELM_OK).  helm_last_error() gives a
 *    message for the last failing call on a handle.  No call asserts or traps.
 *  - Arrays marked [dev] are device pointers owned by the caller; [host] are
 *    host pointers.  Complex data is interleaved (re, im): complex128 = 2 doubles,
 *    complex64 = 2 floats.  Vectors have N = n^d entries.
 *  - Calls are asynchronous on the handle's stream (helm_set_stream), except
 *    don_load, helm_precond, helm_solve and helm_solve_host, which synchronise
 *    (the last two return statistics).
 *  - The handle owns its workspace (trunk basis, coarse operator, Krylov
 *    vectors) and frees it in helm_destroy.  It copies the mask and k^2 field.
 *  - No CPU fallback: without an sm_103a device helm_create returns HELM_NO_DEVICE.
 */
#ifndef HELM_H
#define HELM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct helm_handle helm_handle;

typedef enum {
    HELM_OK = 0,
    HELM_BAD_ARG = 1,          /* argument out of range, wrong dtype, null pointer */
    HELM_NO_DEVICE = 2,        /* no sm_103a GPU visible */
    HELM_CUDA_ERROR = 3,       /* a CUDA runtime call failed */
    HELM_NOT_CONVERGED = 4,    /* maxit reached above tol */
    HELM_DIVERGED = 5,         /* residual > 1e8 * initial, or NaN/Inf */
    HELM_BREAKDOWN = 6,        /* BiCGStab rho or omega = 0, (t,t) = 0 */
    HELM_SINGULAR_COARSE = 7,  /* zero pivot in the coarse operator A_c */
    HELM_NOT_READY = 8,        /* correction requested before don_load */
    HELM_OUT_OF_MEMORY = 9,
    HELM_SCRATCH_TOO_SMALL = 10, /* problem exceeds the fixed scratch of helm_residual_noalloc */
    HELM_TIMEOUT = 11          /* a bounded in-kernel wait (grid barrier) gave up */
} helm_status;

/* dtype of the vectors passed to a call */
enum { HELM_C128 = 0, HELM_C64 = 1 };
/* precision mode of a handle: FP64 (see helm_precond for the double-float parts),
 * or complex64 preconditioner (stencil, relaxation, projection with a BF16-rounded
 * Q) inside the FP64 outer method (FGMRES: Arnoldi, Hessenberg/Givens; BiCGStab:
 * vectors and recurrences; the true residual in FP64 for both). */
enum { HELM_FP64 = 0, HELM_MIXED = 1 };
/* relaxation kinds (Sec. 3.1.1: M = diag(A) -> Jacobi, lower triangle -> Gauss-Seidel,
 * SOR and SSOR; Gauss-Seidel-type sweeps in red-black order).  HELM_MG (Sec. 4.3):
 * a geometric multigrid V-cycle with damped-Jacobi smoothing (helm_mg_setup). */
enum { HELM_RELAX_NONE = 0, HELM_JACOBI = 1, HELM_RBGS = 2, HELM_SOR = 3, HELM_SSOR = 4, HELM_MG = 5 };
/* second-stage correction M2 (Eq. 3): none, trunk-basis Galerkin (App. C) */
enum { HELM_CORR_NONE = 0, HELM_CORR_TB = 1, HELM_CORR_NONLINEAR = 2 };
/* outer methods */
enum { HELM_METHOD_RELAX = 0, HELM_METHOD_FGMRES = 1, HELM_METHOD_BICGSTAB = 2 };
/* trunk activations on hidden layers: tanh, or Leaky ReLU (App. B's trunk; slope
 * 0.01 for negative arguments) */
enum { HELM_ACT_TANH = 0, HELM_ACT_LEAKY_RELU = 1 };

/* Options of one solve.  `relax`, `n_r`, `omega` and `correction` define the
 * hybrid cycle M (Eq. 3): n_r relaxation sweeps from zero, then M2 on the new
 * residual.  METHOD_RELAX runs that cycle as a Richardson iteration on A u = f
 * (relaxation meta-solver); FGMRES/BICGSTAB use it as a right preconditioner
 * (Krylov meta-solver).  Convergence: ||f - A x||_2 <= tol ||f||_2, true residual
 * in FP64.  `restart` is m of FGMRES(m) (1..64).  `maxit` counts Arnoldi
 * steps / BiCGStab iterations / relaxation cycles.  conj = 1 solves with
 * conj(A) = A^H (adjoint), using the conjugated preconditioner. */
typedef struct {
    int method;
    int relax;
    int n_r;
    double omega;
    int correction;
    double tol;
    int restart;
    int maxit;
    int conj;
} helm_solve_opts;

typedef struct {
    int status;          /* helm_status of the solve */
    int iters;           /* Arnoldi steps / BiCGStab iterations / cycles */
    int cycles;          /* FGMRES restarts, BiCGStab restarts */
    int precond_applies;
    int matvecs;
    double rel_res;      /* final true relative residual ||f - A x|| / ||f|| */
    double ms;           /* device time of the solve (CUDA events) */
    long long launches;  /* kernels launched by the solve */
    int n_restrict;      /* trunk-basis restrictions (fused residual + Q^T r) */
    int n_prolong;       /* trunk-basis prolongations (z += Q y) */
    double restrict_ms;  /* summed CUDA-event time of the restriction kernels (profiling on) */
    double prolong_ms;   /* summed CUDA-event time of the prolongation kernels (profiling on) */
    int n_sweep;         /* relaxation launches that read neighbours: half-sweeps, or whole
                            red-black cycles of the cooperative double-float path
                            (FP64 handles, profiling on) */
    int n_apply;         /* operator applications of the BiCGStab loop (profiling on) */
    double sweep_ms;     /* their summed CUDA-event time */
    double apply_ms;     /* their summed CUDA-event time */
} helm_stats;

/* Create a problem handle.  Eq. 1 on n^dim nodes (dim 2 or 3, 3 <= n <= 2048,
 * n^dim < 2^31), wavenumber k0, absorbing layer of `layer_cells` cells with
 * strength s (Im k^2 ramps to s*k0^2).  mask [dev] N bytes, 1 = Dirichlet node;
 * the outer node ring must be masked (HELM_BAD_ARG otherwise, checked on device).
 * k2 [dev] N complex128 or NULL: when given it is the full k^2 of every fluid
 * node and the layer formula is not applied.  precision: HELM_FP64 or
 * HELM_MIXED.  The handle keeps its own copies of mask and k2. */
helm_status helm_create(int dim, int n, double k0, int layer_cells, double layer_strength,
                        const uint8_t* mask, const double* k2, int precision,
                        helm_handle** out);
/* The paper's own boundary-value problem (Eq. 1): no absorbing layer and no
 * Dirichlet ring; every outer-boundary node is an unknown whose row comes from
 * eliminating the ghost node of a central difference -- first-order Sommerfeld
 * condition du/dn - i k0 u = 0 on every face, except, with neumann_top, the top
 * face (y = 1 in 2D, z = 1 in 3D) where du/dn = g (incoming wave, data g passed to
 * helm_rhs).  A row of a node on b faces is scaled by 2^-b, which keeps A complex
 * symmetric: fluid neighbours couple with weight h^-2 2^-|F(l) and F(m)| (F the set
 * of faces a node lies on), and the diagonal is 2^-b (k^2 - 2d h^-2 + 2 i k0 a / h)
 * with a the node's Sommerfeld faces.  mask [dev] N bytes, 1 = Dirichlet (the
 * scatterer; the outer ring is NOT masked); k2 [dev] N complex128 or NULL (k0^2).
 * helm_rhs on such a handle gives b_l = g_l on masked nodes and, on fluid nodes,
 * 2^-b (src_l - (2/h) g_l [l on the Neumann face]) minus the weighted Dirichlet
 * values of masked neighbours.  FP64 handles; the trunk-basis, relaxation and
 * Krylov calls work as on helm_create handles (through the generic kernels);
 * helm_layer_k2, helm_set_k2, helm_k2_gradient and helm_mg_setup return
 * HELM_BAD_ARG. */
helm_status helm_create_bvp(int dim, int n, double k0, const uint8_t* mask, const double* k2, int neumann_top,
                            helm_handle** out);
helm_status helm_destroy(helm_handle* h);
/* stream: a cudaStream_t (NULL = legacy default stream). */
helm_status helm_set_stream(helm_handle* h, void* stream);
const char* helm_last_error(const helm_handle* h);

/* Bounds-checked build (the library compiled with -DHELM_CHECKED, which replaces a
 * sanitizer here): its kernels check the indices of their vector, table and basis
 * accesses, and an index out of range is recorded (the source line << 8 | the
 * translation unit's id + 1, first one only) and replaced by 0 instead of being
 * used; nothing traps.  Synchronises the device, then sets *checked = 1 in a
 * checked build (0 otherwise) and *first to the first recorded violation since the
 * previous call (0: none), and clears the records. */
helm_status helm_checked_status(int* checked, unsigned long long* first);
/* on = 1: bracket every trunk-basis restriction and prolongation, every
 * relaxation launch and every BiCGStab operator application with CUDA events on
 * the handle's stream and report their counts and summed times in helm_stats
 * (the event records lengthen the solve a little). */
helm_status helm_set_profiling(helm_handle* h, int on);
/* Bounded waits of the cooperative red-black cycle (one launch whose phases are
 * separated by grid barriers, one block per SM, co-residency checked by an
 * occupancy query before the launch): a block polls the barrier at most `polls`
 * times (> 0; default 2^20, about a second) before it gives up, records the
 * timeout and goes on; the call then returns HELM_TIMEOUT and resets the barrier.
 * extra_arrivals > 0 makes every barrier wait for that many blocks more than the
 * launch has, so that each wait runs out: host-side fault injection for tests of
 * the timeout path (0 for normal use).  helm_precond synchronises and checks too. */
helm_status helm_set_wait_limit(helm_handle* h, unsigned polls, unsigned extra_arrivals);

/* Reliable updates of the complex64 BiCGStab of HELM_MIXED handles (Sleijpen and
 * van der Vorst's reliable updating of the residual): the FP32 increment is folded
 * into the FP64 iterate and the residual recomputed in FP64 when the recursive
 * residual falls below delta times its largest value since the last update
 * (default 0.1); a recursive residual above runaway times the last true residual
 * (default 1e3) drops the increment and restarts; guard > 0 tries each fold first
 * and takes the increment back out (and restarts) when the true residual would
 * exceed guard times the best true residual so far (default 0: no guard).  After
 * four such restarts (runaways or rejected folds) the solve continues, for the rest
 * of maxit, as the FP64 BiCGStab with the same complex64 cycle from the FP64 iterate
 * (the statistics add both parts).  A solve that ends unconverged keeps its last
 * increment only if the true residual stays within 100x of the best one seen.
 * HELM_BAD_ARG unless 0 < delta < 1, runaway > 1, guard >= 0. */
helm_status helm_set_reliable(helm_handle* h, double delta, double runaway, double guard);

/* Multigrid hierarchy for HELM_MG (Sec. 4.3, DeepONet-MG-Krylov): `levels` grids in
 * all (1..8), each coarser one by vertex coarsening n -> (n + 1) / 2 (so n must
 * stay odd and >= 5 down to the coarsest), coarse node I at fine node 2I; the mask
 * and k^2 of a coarse node are those of fine node 2I, and the operator is the
 * stencil of Eq. 1 with the coarse h.  Restriction: full weighting (the transpose
 * of (bi/tri)linear interpolation over 2^d); prolongation: (bi/tri)linear
 * interpolation, added on unmasked fine nodes.  The V-cycle (HELM_MG with
 * opts.n_r = m, opts.omega the Jacobi damping): smoother from zero, coarse-grid
 * correction, smoother; the smoother is m damped-Jacobi sweeps, the trunk-basis
 * correction, m sweeps (the 2-1-2 strategy for m = 2) on the finest level when
 * opts.correction = HELM_CORR_TB, else 2 m + 1 sweeps; the coarsest level only
 * smooths from zero.  The cycle is linear, so it preconditions FGMRES and
 * BiCGStab.  FP64 handles; synchronises. */
helm_status helm_mg_setup(helm_handle* h, int levels);

/* Grid query: N, h. */
helm_status helm_info(const helm_handle* h, long long* N, double* hstep);

/* k2_out [dev] N complex128 = k0^2 * scale_l * (1 + i*s*eta_l^2) with the
 * layer profile of the handle; scale [dev] N doubles or NULL (= 1). */
helm_status helm_layer_k2(helm_handle* h, const double* scale, double* k2_out);

/* Right-hand side with the Dirichlet data moved across (App. D): b_l = g_l on
 * masked nodes, b_l = src_l - h^-2 sum_{masked nbr m} g_m on fluid nodes.
 * src, g, b [dev] complex128. */
helm_status helm_rhs(helm_handle* h, const double* src, const double* g, double* b);

/* y = A x (conj = 0) or conj(A) x (conj = 1).  x, y [dev], dtype HELM_C128 or
 * HELM_C64, must not overlap. */
helm_status helm_apply(helm_handle* h, const void* x, void* y, int conj, int dtype);

/* r = f - A x; if norm2 [dev] is not NULL, *norm2 = ||r||_2^2 (FP64). */
helm_status helm_residual(helm_handle* h, const void* f, const void* x, void* r,
                          double* norm2, int conj, int dtype);

/* `sweeps` relaxation sweeps on A x = f in place (Eq. 2):
 * HELM_JACOBI: x <- x + omega D^-1 (f - A x), D = diag(A) (1 on masked rows);
 * HELM_RBGS:   red ((i+j+k) even) then black half-sweeps, x_l <- x_l + D_l^-1 (f - A x)_l
 *              with the latest neighbours (omega unused). */
helm_status helm_relax(helm_handle* h, int kind, double omega, int sweeps, const void* f,
                       void* x, int conj, int dtype);

/* Load the trunk network and build the trunk-basis coarse space (App. C):
 * T_lj = trunk(x_l)_j (Eq. 6) for j < p, zero rows on masked nodes; natural-order
 * selection keeps column j when its part orthogonal to the columns already kept
 * exceeds tau * ||T_j|| (tau = 0 keeps every nonzero column); Q orthonormal with
 * span(Q) = span(selected columns); A_c = Q^T A Q (complex, k x k); A_c^-1 by
 * Gauss-Jordan with partial pivoting.
 * weights [host] FP64: per layer W (row-major out x in) then bias; widths[0] = dim,
 * widths[n_layers] >= p; act (HELM_ACT_TANH or HELM_ACT_LEAKY_RELU) on hidden layers
 * only.  p <= 256.
 * Synchronises.  Returns HELM_SINGULAR_COARSE on a zero pivot. */
helm_status don_load(helm_handle* h, const double* weights, const int* widths, int n_layers,
                     int act, int p, double tau);
/* k = number of kept columns; kept_idx [host] (p ints) or NULL. */
helm_status don_info(const helm_handle* h, int* k, int* kept_idx);
/* Copy Q (N x k FP64, row-major: k contiguous per node) into q_out [dev]. */
helm_status don_get_q(const helm_handle* h, double* q_out);
/* Copy A_c^-1 (k x k complex128, row-major) into out [dev]. */
helm_status don_get_ainv(const helm_handle* h, double* out);

/* Load the branch network of the trained DeepONet (App. B): widths[0] = 2N (input
 * [Re r, Im r] / ||r||, real parts first), widths[n_layers] = 2p (p of don_load:
 * real-part coefficients first), ReLU on hidden layers, hidden widths <= 4096.
 * weights [host] FP32: per layer W (row-major out x in) then bias.  Needs
 * don_load first (the raw trunk matrix T, masked rows zero, is kept in FP32). */
helm_status don_load_branch(helm_handle* h, const float* weights, const int* widths, int n_layers);

/* z += M2 r.  HELM_CORR_TB: M2 = Q A_c^-1 Q^T (App. C, linear).
 * HELM_CORR_NONLINEAR: M2 r = s (T b_re + i T b_im), b = Branch([Re r, Im r]/s),
 * s = ||r|| (DeepONet inference on the residual, Eq. 3; positively homogeneous;
 * FP32 network).  r, z [dev] HELM_C128. */
helm_status don_correct(helm_handle* h, int mode, const void* r, void* z, int conj, int dtype);

/* z = M(r), the hybrid cycle of `opts` (Eq. 3).  r, z [dev] HELM_C128.
 * On an FP64 handle with a tabulated k^2, the red-black Gauss-Seidel cycle with
 * the trunk-basis correction runs in double-float arithmetic (value = hi + lo,
 * two FP32 numbers, 48-bit significand) on the FP32 pipes, the residual of the
 * correction on the red rows only (it vanishes on the black rows after the black
 * half-sweep); z agrees with the FP64 evaluation to about 1e-14 relative. */
helm_status helm_precond(helm_handle* h, const helm_solve_opts* opts, const void* r, void* z);

/* Solve A x = f (conj(A) x = f if opts->conj).  f [dev] complex128, x [dev]
 * complex128: initial guess in, solution out.  Masked entries of x are set to
 * f on entry (x_l = g_l).  res_hist [host] or NULL: relative true residual
 * after every restart/cycle, up to hist_len values (FGMRES: per Arnoldi step,
 * Givens estimate).  Synchronises; stats [host] may be NULL.  The stopping test
 * and the final rel_res use the FP64 residual.  BiCGStab with the double-float
 * cycle (see helm_precond) applies A to the cycle's double-float output and
 * rounds to FP64 once; its Krylov vectors, dots and recurrences are FP64.
 * HELM_TIMEOUT reports a bounded in-kernel wait of the cooperative red-black
 * cycle that gave up (never expected with the default limit; see
 * helm_set_wait_limit); the barrier state is reset, so the next call starts clean. */
helm_status helm_solve(helm_handle* h, const helm_solve_opts* opts, const void* f, void* x,
                       helm_stats* stats, double* res_hist, int hist_len);

/* As helm_solve with f and x in host memory [host] (pinned or pageable): the
 * copies to and from the device are part of the call. */
helm_status helm_solve_host(helm_handle* h, const helm_solve_opts* opts, const double* f,
                            double* x, helm_stats* stats, double* res_hist, int hist_len);

/* ---- adjoint method (receiver-misfit loss, gradient w.r.t. the per-node k^2) ----
 * Receivers sample u by trilinear interpolation of the 8 nodes of the grid cell
 * that contains them (3D handles).  For a real loss L(u) with G = dL/dRe u +
 * i dL/dIm u, the adjoint conj(A) lambda = G (A^H = conj(A), helm_solve with
 * conj = 1) gives dL/dRe k^2_l + i dL/dIm k^2_l = -lambda_l conj(u_l) on fluid
 * nodes and 0 on Dirichlet nodes, because dA/dk^2_l = e_l e_l^T on fluid rows. */

/* idx [dev] 8*nrec ints and w [dev] 8*nrec doubles: corner nodes and trilinear
 * weights of the receivers xyz [dev] (nrec x 3 doubles, coordinates in [0,1]^3). */
helm_status helm_receivers_setup(helm_handle* h, int nrec, const double* xyz, int* idx, double* w);
/* out[r] = sum_q w[8r+q] u[idx[8r+q]]  (out [dev] nrec complex128). */
helm_status helm_receivers_sample(helm_handle* h, int nrec, const int* idx, const double* w,
                                  const double* u, double* out);
/* b = S^T e: b [dev] N complex128 is overwritten (zero except at receiver corners). */
helm_status helm_receivers_adjoint(helm_handle* h, int nrec, const int* idx, const double* w,
                                   const double* e, double* b);
/* grad [dev] N complex128 = -lambda conj(u) on fluid nodes, 0 on masked nodes. */
helm_status helm_k2_gradient(helm_handle* h, const double* lambda, const double* u, double* grad);
/* Replace the k^2 field (k2 [dev] N complex128, copied).  If a trunk basis is
 * loaded, the coarse operator A_c = Q^T A Q and its inverse are rebuilt for the
 * new operator (Q depends only on the trunk and the mask).  Synchronises. */
helm_status helm_set_k2(helm_handle* h, const double* k2);

/* ---- dense layers for DeepONet training (App. B), FP32, row-major, on `stream` ----
 * nn_gemm: C = alpha op(A) op(B) + beta C; op(A) is M x K (A stored K x M when
 * transA), op(B) is K x N (B stored N x K when transB).
 * nn_bias_act: X = act(X + bias) in place, act 0 = none, 1 = ReLU, 2 = tanh, 3 = Leaky
 *   ReLU (slope 0.01) (bias may be NULL).
 * nn_act_backward: dX *= act'(Y), Y the activation output.
 * nn_bias_grad: db[c] = sum_r dY[r][c].
 * nn_adam: Adam with bias correction, step t >= 1.
 * nn_rel_l2: per-sample ||pred - target||^2 / ||target||^2 over P2 values and the
 *   gradient of the batch mean with respect to pred.
 * nn_gather: dst[r][c] = src[row_idx[r]][col_idx[c]] (NULL index = identity). */
/* 3D convolution layer of the CNN branch (App. B: 3 x 3 x 3 kernels), FP32, layout
 * [batch][channel][z][y][x], W [Co][Ci][3][3][3]:
 *   Y[b][o][z][y][x] = bias[o] + sum_{i, kz, ky, kx} W[o][i][kz][ky][kx]
 *                      X[b][i][z s + kz - pad][y s + ky - pad][x s + kx - pad]
 * (zeros outside X), Y [dev] B x Co x Do^3 with Do = (D + 2 pad - 3) / s + 1; bias may be
 * NULL.  nn_conv3d_backward writes, for the given dY, dX (B x Ci x D^3), dW and db (Co)
 * of sum(dY * Y); any of the three may be NULL.  Every value is summed in a fixed
 * order (no atomics).  stride >= 1, 0 <= pad <= 2; HELM_BAD_ARG otherwise. */
helm_status nn_conv3d(int B, int Ci, int D, int Co, int stride, int pad, const float* X, const float* W,
                      const float* bias, float* Y, void* stream);
helm_status nn_conv3d_backward(int B, int Ci, int D, int Co, int stride, int pad, const float* X, const float* W,
                               const float* dY, float* dX, float* dW, float* db, void* stream);
helm_status nn_gemm(int transA, int transB, int M, int N, int K, float alpha, const float* A, int lda,
                    const float* B, int ldb, float beta, float* C, int ldc, void* stream);
helm_status nn_bias_act(int rows, int cols, float* X, const float* bias, int act, void* stream);
helm_status nn_act_backward(long long n, float* dX, const float* Y, int act, void* stream);
helm_status nn_bias_grad(int rows, int cols, const float* dY, float* db, void* stream);
helm_status nn_adam(long long n, float* p, const float* g, float* m, float* v, float lr, float beta1,
                    float beta2, float eps, int t, void* stream);
helm_status nn_rel_l2(int B, int P2, const float* pred, const float* target, float* dpred, float* loss,
                      void* stream);
helm_status nn_gather(int rows, int cols, const float* src, long long lds, const int* row_idx,
                      const int* col_idx, float* dst, void* stream);

/* The same product on the tensor cores (tcgen05, sm_103a): op(A) and op(B) are
 * rounded to BF16 (nearest even) and multiplied with FP32 accumulation, C = alpha
 * op(A) op(B) + beta C in FP32 (dense layers of the DeepONet in mixed-precision
 * training, App. B).  Uses a per-device BF16 workspace grown on demand (held until
 * exit).  Asynchronous on `stream`; every wait inside the kernel is bounded, and a
 * wait that ran out (never expected) is reported, and cleared, by
 * nn_gemm_bf16_status (*timed_out = 1; the results since then are invalid). */
helm_status nn_gemm_bf16(int transA, int transB, int M, int N, int K, float alpha, const float* A, int lda,
                         const float* B, int ldb, float beta, float* C, int ldc, void* stream);
helm_status nn_gemm_bf16_status(int* timed_out);

/* ---- batched solves (many independent problems, one launch per phase) ----
 * The problems are existing HELM_MIXED handles with a loaded trunk basis; their
 * vectors are packed one after another and every phase of FGMRES runs as one
 * persistent launch over a queue of tiles (tile_rows consecutive nodes of one
 * problem) for all problems at once, with per-problem reductions, Givens
 * rotations, convergence and Krylov dimensions.  Preconditioner: complex64
 * damped Jacobi or red-black GS (n_r sweeps, or none) + trunk-basis correction
 * with each problem's BF16 basis; Arnoldi, Hessenberg, Givens and the true
 * residual in FP64.  The handles must outlive the batch; it uses the stream of hs[0]. */
typedef struct helm_batch helm_batch;
helm_status helm_batch_create(int nprob, helm_handle** hs, helm_batch** out);
helm_status helm_batch_destroy(helm_batch* b);
/* Tile length (multiple of 32, 32..8192 nodes) and persistent grid size. */
helm_status helm_batch_set_tile(helm_batch* b, int tile_rows, int grid);
/* FGMRES(opts->restart) on every problem: f[i], x[i] [dev] complex128 of problem i
 * (x: initial guess in, solution out); stats [host] nprob entries or NULL.
 * Returns HELM_OK when every problem converged, else the last failing status. */
helm_status helm_batch_solve(helm_batch* b, const helm_solve_opts* opts, const double* const* f,
                             double* const* x, helm_stats* stats);

/* Many independent solves at once, each stopping at its own convergence: problem i
 * is solved exactly as helm_solve(hs[i], opts, f[i], x[i], &stats[i], NULL, 0) would
 * (same kernels, same result bit for bit), but on a private non-blocking stream per
 * problem, ordered after that handle's stream, from a pool of min(nprob, threads)
 * host threads (threads <= 0: one per problem), so that the GPU overlaps the
 * problems' launches instead of running one problem after another, and no problem
 * waits for the slowest one (unlike helm_batch_solve's lockstep).  The handles must be
 * distinct HELM_MIXED handles (the complex64 cycles launch no grid-wide barriers, so
 * any number of them may share the GPU); each keeps its own stream setting, restored
 * before return.  f[i], x[i] [dev] complex128 as in helm_solve; stats [host] nprob
 * entries or NULL.  Synchronous.  Returns HELM_OK when every problem converged, else
 * the status of the first problem (by index) that did not; HELM_BAD_ARG for null or
 * repeated handles or an FP64 handle. */
helm_status helm_solve_concurrent(int nprob, helm_handle** hs, const helm_solve_opts* opts, const double* const* f,
                                  double* const* x, helm_stats* stats, int threads);

/* Residual without allocation (no counterpart in the paper: an interface for
 * callers that cannot allocate device memory -- code running inside a memory
 * pool or arena it does not own, plugins whose host forbids cudaMalloc, code
 * that must not touch the allocator).  Computes r = f - A x (conj(A) if conj)
 * and *norm2 = ||r||_2^2 in FP64 exactly like helm_residual, but needs no
 * handle: the operator is described by the arguments of helm_create (mask [dev]
 * N bytes with the outer ring masked, k2 [dev] complex128 field or NULL), and
 * f, x, r [dev] complex128, norm2 [dev] one double are the caller's.
 *  - Scratch: a file-scope device array of 65536 doubles (512 KiB) that every
 *    GPU loading the library holds until the process exits.  Problems whose
 *    operator grid has more than 65536 thread blocks (3D n > 640) are rejected
 *    with HELM_SCRATCH_TOO_SMALL.
 *  - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 *  - The first call on a device looks up the array's device address (once per
 *    device, with that device current).
 *  - Synchronises `stream` (a cudaStream_t, NULL = legacy default) once to check
 *    that the outer ring is masked (HELM_BAD_ARG otherwise), so no call can be
 *    made while that stream is being captured into a CUDA graph.
 *  - Every call shares the scratch array and the ring-check flag beside it (both
 *    keep the last call's contents): calls that overlap on the GPU (other
 *    streams, other host threads) race on both. */
helm_status helm_residual_noalloc(int dim, int n, double k0, int layer_cells, double layer_strength,
                                  const uint8_t* mask, const double* k2, const double* f,
                                  const double* x, double* r, double* norm2, int conj, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HELM_H */
