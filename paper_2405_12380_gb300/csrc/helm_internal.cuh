// Internal declarations shared by the libhelm translation units.
//
// Data layout in HBM
//   vectors       N complex, interleaved (double2 / float2), flat index i + n(j + n k)
//   mask          N uint8 (1 = Dirichlet: outer ring + scatterer)
//   Q             k x N pairs (hi, lo) of FP32 (= the FP64 basis to ~2^-48), column-major:
//                 basis vector j is Q[j*N .. j*N+N) (node-major copies exist only during setup)
//   A_c^-1        k x k complex128, row-major
//   Krylov basis  V: (m+1) x N complex128, Z: m x N complex128, one vector after another
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/helm.h"

namespace helm {

// ------------------------------------------------ bounds-checked build (HELM_CHECKED)
// Compiled with -DHELM_CHECKED, HCHK(i, n) checks 0 <= i < n before an access: an
// index out of range is recorded in a device word of the translation unit (the
// first one wins: its source line and the unit's id) and replaced by 0, so the
// access stays inside the buffer and nothing traps.  helm_checked_status reads and
// clears the words of every unit.  In the normal build HCHK(i, n) is just i.
std::vector<unsigned long long (*)()>& checked_units();
#ifdef HELM_CHECKED
#ifndef HELM_TU_ID
#define HELM_TU_ID 0
#endif
static __device__ unsigned long long g_helm_oob = 0ull;
__device__ __forceinline__ long long helm_chk(long long i, long long n, int line) {
    if ((unsigned long long)i >= (unsigned long long)n) {
        atomicCAS(&g_helm_oob, 0ull, ((unsigned long long)line << 8) | (unsigned long long)(HELM_TU_ID + 1));
        return 0;
    }
    return i;
}
#define HCHK(i, n) (::helm::helm_chk((long long)(i), (long long)(n), __LINE__))
static unsigned long long checked_take_unit() {
    unsigned long long v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_helm_oob, sizeof(v)) != cudaSuccess) return 0;
    cudaMemcpyToSymbol(g_helm_oob, &z, sizeof(z));
    return v;
}
struct CheckedUnitRegistration {
    explicit CheckedUnitRegistration(unsigned long long (*take)()) { checked_units().push_back(take); }
};
static CheckedUnitRegistration checked_unit_registration(&checked_take_unit);
#else
#define HCHK(i, n) (i)
#endif

// NVTX range for the phases of a call (setup, solve, preconditioner, Arnoldi step);
// free when no profiler is attached
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int kMaxLayerCells = 64;
constexpr int kMaxP = 256;          // trunk basis functions
constexpr int kMaxRestart = 64;     // FGMRES(m)
constexpr int kRedBlocks = 304;     // blocks of the fixed-grid reductions (2 per SM)
constexpr int kFinThreads = 1024;

// ------------------------------------------------------------ complex helpers
template <typename R> struct CT;
template <> struct CT<double> { using T = double2; };
template <> struct CT<float> { using T = float2; };

__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ float2 cscale(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// ------------------------------------------------------ operator description
// Everything a stencil kernel needs, passed by value.  The absorbing layer is
// tabulated by the layer index m = max_a max(0, L - dist_a) in 0..L, so k^2 and
// the inverse diagonal of a fluid node are table lookups (no per-node FP64
// division); with a stored k^2 field the per-node arrays are used instead.
template <typename R>
struct Op {
    using C = typename CT<R>::T;
    int dim, n, L;
    long long N;
    R hinv2;                 // h^-2
    R dre;                   // k0^2 - 2 d h^-2 (real part of the diagonal, layer form)
    const uint8_t* mask;
    const uint8_t* lidx;     // per-node layer index m (flat-index kernels; avoids index division)
    const uint8_t* nbm;      // per-node neighbour code: bit q = neighbour q fluid, 0x80 = masked node
    const C* k2;             // stored k^2 field or nullptr
    const C* invd;           // per-node 1/diag for the stored field, or nullptr
    // Sommerfeld / Neumann outer boundary (helm_create_bvp) or nullptr: per node
    // (number of boundary faces b << 4) | (bit a: the node lies on a face normal to
    // axis a); the row is scaled by 2^-b and a neighbour across axis a weighs
    // 2^-(b - [node on an axis-a face]) (symmetric scaling of the ghost-point rows)
    const uint8_t* face;
    R im[kMaxLayerCells + 1];        // Im k^2 by layer index
    C invd_tab[kMaxLayerCells + 1];  // 1/(diag) by layer index (fluid nodes)
};

// Double-float (FP32 pair, hi + lo) copies of the operator constants, for the
// red-black Gauss-Seidel cycle of FP64 handles that runs on the FP32 pipes
struct DfTab {
    float2 hinv2;                            // h^-2
    float2 dre;                              // real part of the tabulated diagonal
    float2 im[kMaxLayerCells + 1];           // Im k^2 by layer index
    float4 invd[kMaxLayerCells + 1];         // 1/diag by layer index: (re hi, re lo, im hi, im lo)
};

// device scalar slots of the Krylov drivers (double2 each, in helm_handle::sc)
enum { S_RHO = 0, S_RHO_OLD, S_ALPHA, S_OMEGA, S_BETA, S_SN2, S_RN2, S_FLAGS, S_TS, S_TT,
       S_BETA2, S_WN2, S_EST, S_BN2, S_STOP, S_TOLS, S_NSLOTS };
// S_FLAGS.x = 1: ||s|| met the tolerance this iteration; S_FLAGS.y = 1: breakdown
// S_TOLS.x: the absolute tolerance tol ||f|| of the complex64 BiCGStab (set per solve,
// so that its captured iteration does not depend on the solve)
// S_STOP.x = 1: the BiCGStab iteration that set it ended the loop (converged, broke
// down or diverged); later x/r updates are no-ops until the next reset

// ------------------------------------------------------------ kernel launchers
// stencil.cu
// returns the number of per-block partial sums written to `partials` (when given)
template <typename R>
int launch_apply(const Op<R>& op, const typename CT<R>::T* x, const typename CT<R>::T* f,
                 typename CT<R>::T* y, double* partials, int conj, bool resid, cudaStream_t s);
template <typename R>
void launch_jacobi(const Op<R>& op, double omega, const typename CT<R>::T* f,
                   const typename CT<R>::T* xin, typename CT<R>::T* xout, int conj, bool xzero,
                   cudaStream_t s);
// omega: 1 = Gauss-Seidel; otherwise SOR (each node moves by omega times its GS step)
template <typename R>
void launch_rbgs_half(const Op<R>& op, int colour, const typename CT<R>::T* f, typename CT<R>::T* x,
                      int conj, bool xzero, cudaStream_t s, double omega = 1.0);
// one full red-black sweep, colour c0 on every node then colour 1 - c0, from xin
// (nullptr: from zero) into xout (a different buffer) in one launch; returns false
// without launching where the fused kernel does not apply (2D, odd n, n > 256,
// outer-boundary rows, unaligned vectors)
bool launch_rbgs_sweep32(const Op<float>& op, int c0, const float2* f, const float2* xin, float2* xout, int conj,
                         double omega, cudaStream_t s);
bool rbgs_sweep32_ok(const Op<float>& op, const void* f, const void* x, const void* tmp);
// r_red[q] = (f - A x) at the red node of pair q (the pair layout: 3D, n even; the
// red rows in the order of the red-row basis copy), zero on masked nodes; false
// without launching where the pair layout does not apply
bool launch_red_residual32(const Op<float>& op, const float2* f, const float2* x, float2* r_red, int conj,
                           cudaStream_t s);
// complex64 y = A x with the partial sums of a BiCGStab reduction in the epilogue
// (mode 1: <w, y> with w = rhat, for alpha; mode 2: <y, w> and <y, y> with w = s,
// for omega), 2 or 3 floats per block in parts (the block count is at most
// apply_grid_blocks); nothing is written once S_STOP is set.  Returns the number of blocks, or 0 without
// launching where the pair kernels do not apply.
int launch_apply32_bicg(const Op<float>& op, int mode, const float2* x, float2* y, const float2* w, int conj,
                        const double2* sc, float* parts, cudaStream_t s);
int apply_grid_blocks(int dim, int n);
int bicg_grid_blocks(int dim, int n);
void launch_rhs(const Op<double>& op, const double2* src, const double2* g, double2* b, cudaStream_t s);
void launch_layer_k2(const Op<double>& op, double k0, double strength, const double* scale,
                     double2* k2, cudaStream_t s);
void launch_invd_field(const Op<double>& op, double2* invd, cudaStream_t s);
void launch_check_ring(const Op<double>& op, int* bad, cudaStream_t s);
void launch_layer_index(const Op<double>& op, uint8_t* lidx, cudaStream_t s);
void launch_nbr_code(const Op<double>& op, uint8_t* code, cudaStream_t s);
// outer-boundary problem: face bytes (see Op::face), the effective k^2 field that
// makes diag_of return the scaled boundary diagonal, and the right-hand side
void launch_face_code(const Op<double>& op, uint8_t* face, cudaStream_t s);
void launch_bvp_k2(const Op<double>& op, const double2* k2phys, double k0, int neumann_top, double2* k2eff,
                   cudaStream_t s);
void launch_rhs_bvp(const Op<double>& op, const double2* src, const double2* g, int neumann_top, double2* b,
                    cudaStream_t s);
// BiCGStab fused kernels (reduction + scalar update in the last block; counter zero between uses)
void launch_apply_bicg(const Op<double>& op, int mode, const double2* x, double2* y, const double2* w, int conj,
                       double2* sc, double* parts, unsigned* counter, cudaStream_t s);
void launch_bicg_s_fused(const double2* r, const double2* v, double2* sv, double2* sc, long long N, double* parts,
                         unsigned* counter, double tol_abs, cudaStream_t s);
// x/r update; its last block also decides S_STOP from ||r|| / bnorm <= tol, a
// breakdown flag or a non-finite residual (the host's test, evaluated identically)
void launch_bicg_xr_fused(double2* x, double2* r, const double2* phat, const double2* shat, const double2* sv,
                          const double2* t, const double2* rhat, double2* sc, long long N, double* parts,
                          unsigned* counter, double tol, double bnorm, cudaStream_t s);

// bicg32.cu: complex64 BiCGStab with reliable updates (HELM_MIXED handles); each
// reduction finishes in the last block of its kernel (parts: 3 doubles per block)
int bicg32_blocks();
void launch_b32_update_p(const float2* r, const float2* v, float2* p, const double2* sc, long long N, cudaStream_t s);
void launch_b32_alpha(const float2* rhat, const float2* v, double2* sc, long long N, double* parts, unsigned* counter,
                      cudaStream_t s);
void launch_b32_s(const float2* r, const float2* v, float2* sv, double2* sc, long long N, double* parts,
                  unsigned* counter, cudaStream_t s);
void launch_b32_set_tol(double2* sc, double tol_abs, cudaStream_t s);
// k32_s / k32_xr taking alpha / omega from the partial sums of launch_apply32_bicg
// (na, no blocks): every block sums them in the same fixed order, block 0 stores the
// scalar and its flags
void launch_b32_s_dot(const float2* r, const float2* v, float2* sv, double2* sc, long long N, double* parts,
                      unsigned* counter, const float* aparts, int na, cudaStream_t s);
void launch_b32_xr_dot(float2* xl, float2* r, const float2* phat, const float2* shat, const float2* sv,
                       const float2* t, const float2* rhat, double2* sc, long long N, double* parts, unsigned* counter,
                       const float* oparts, int no, cudaStream_t s);
void launch_b32_omega(const float2* t, const float2* sv, double2* sc, long long N, double* parts, unsigned* counter,
                      cudaStream_t s);
void launch_b32_xr(float2* xl, float2* r, const float2* phat, const float2* shat, const float2* sv, const float2* t,
                   const float2* rhat, double2* sc, long long N, double* parts, unsigned* counter, cudaStream_t s);
// mode 0: x += xl, xl = 0; 1: xl = 0; 2: x += xl (xl kept); 3: x -= xl, xl = 0
void launch_b32_fold(double2* x, float2* xl, long long N, cudaStream_t s, int mode = 0);
void launch_b32_replace(const double2* r64, float2* r, float2* rhat, float2* p, float2* v, int restart, double2* sc,
                        long long N, double* parts, unsigned* counter, cudaStream_t s);

// blas.cu
// partial reductions over a fixed grid of kRedBlocks blocks
void launch_dot(const double2* a, const double2* b, long long N, double2* partials, cudaStream_t s);
void launch_norm2(const double2* a, long long N, double* partials, cudaStream_t s);
void launch_sum_real(const double* partials, int nparts, double* out, cudaStream_t s);
// BiCGStab pieces (scalars live in device memory, see blas.cu)
void launch_bicg_update_p(const double2* r, const double2* v, double2* p, const double2* sc, long long N,
                          cudaStream_t s);
void launch_bicg_scalar(int recipe, const double* partials, int nparts, double2* sc, double tol_abs,
                        cudaStream_t s);
// FGMRES pieces
void launch_mdot(const double2* V, int nv, const double2* w, long long N, double2* partials,
                 cudaStream_t s);
void launch_mupdate(const double2* V, int nv, const double2* coef, double sign, double2* w, long long N,
                    double* norm_partials, cudaStream_t s);
void launch_mdot_finalize(const double2* partials, int nparts, int nv, double2* out, int accumulate,
                          double2* copy, cudaStream_t s);
void launch_scale_vec(const double2* w, double2* v, const double* norm2, long long N, cudaStream_t s);
void launch_givens(double2* H, int ldh, int j, double* cs, double2* sn, double2* g, const double* wnorm2,
                   double* est, cudaStream_t s);
void launch_hsolve(const double2* H, int ldh, int k, const double2* g, double2* y, cudaStream_t s);
void launch_init_g(double2* g, int m1, const double* beta2, cudaStream_t s);
void launch_set_masked(double2* x, const double2* f, const uint8_t* mask, long long N, cudaStream_t s);
void launch_cvt_f64_to_f32(const double2* a, float2* b, long long N, cudaStream_t s);
void launch_cvt_f32_to_f64(const float2* a, double2* b, long long N, cudaStream_t s);
void launch_mupdate32(const float2* V, int nv, const double2* coef, double sign, double2* w, long long N,
                      cudaStream_t s);

// tb.cu
void launch_trunk_eval(const Op<double>& op, const double* dW, const int* widths, int n_layers, int p, int act,
                       double* T, int ldt, cudaStream_t s);
void launch_gram(const double* A, int lda, int p, const double* B, int ldb, int q, long long N,
                 double* partials, double* out, cudaStream_t s);
void launch_select_chol(const double* G, int p, int ldg, double tau, double* W, double* R, int* kept,
                        int* nkept, int* flag, cudaStream_t s);
void launch_tri_inverse(const double* R, int k, int ldr, double* Rinv, cudaStream_t s);
void launch_gather_times_upper(const double* T, int ldt, const int* kept, int k, const double* Rinv, int ldr,
                               double* Q, int ldq, long long N, cudaStream_t s);
void launch_apply_columns(const Op<double>& op, const double* Q, int ldq, int k, double* W, int ldw,
                          cudaStream_t s);
void launch_gauss_jordan(const double* C, int ldc, int k, double2* Ainv, double2* work, int* flag,
                         cudaStream_t s);
void launch_coarse_apply(const double2* partials, int nblk, int k, const double2* Ainv, int conj, double2* y,
                         double2* cbuf, cudaStream_t s);
// FP64 projection on FP32 pipes: Q as (hi, lo) FP32 pairs, column-major k x N
// (N rows: the projection also runs on the compact red rows, N = ceil(N / 2))
int project_blocks(long long N);
// column stride of a column-major basis with `rows` rows: a multiple of 64 entries
// (512-byte aligned columns) with at least one zero padding entry
inline long long basis_ld(long long rows) { return (rows + 1 + 63) / 64 * 64; }
void launch_project_df(const float2* Q, long long ld, int k, const double2* r, long long N, double2* partials,
                       int nblk, cudaStream_t s);
void launch_prolong_df(const float2* Q, long long ld, int k, const double2* y, double2* z, long long N,
                       cudaStream_t s);
void launch_split_basis(double* A, int ld, int k, float2* B, long long ldb, long long N, cudaStream_t s);
void launch_cm_pair_to_rm(const float2* B, long long ldb, int k, double* A, long long N, cudaStream_t s);
// Q_red (k x ceil(N / 2)): the red rows of Q, row m = the red node of pair (2m, 2m + 1)
void launch_red_rows(const float2* Q, long long ldq, int k, long long N, int n, float2* Qr, long long ldr,
                     cudaStream_t s);
// double-float red-black Gauss-Seidel (stencil.cu): fs = f as FP32 pairs and the
// first (red) half-sweep from x = 0; later half-sweeps; the red-row residual
// written as FP32 pairs (one entry per node pair)
void launch_rbgs_df_first(const Op<double>& op, const DfTab& t, const double2* f, float4* fs, float4* xs, int conj,
                          cudaStream_t s);
void launch_rbgs_df(const Op<double>& op, const DfTab& t, int colour, const float4* fs, float4* xs, int conj,
                    cudaStream_t s);
void launch_residual_red_df(const Op<double>& op, const DfTab& t, const float4* fs, const float4* xs, float4* r_red,
                            int conj, cudaStream_t s);
// the same cycle (first half-sweep, n_r sweeps, red residual) as one cooperative
// launch with grid barriers; bar2 = two zeroed counters, *err set if a barrier
// wait times out.  Returns cudaErrorNotSupported where cooperative launch is not
// available (the caller then uses the kernels above).
// pre = 1: the cycle's input is the BiCGStab update p = f + beta (w - omega v),
// written to w; pre = 2: s = f - alpha v written to w, ||s||^2 into the BiCGStab
// scalars (parts: one double per block); pre = 0: f itself (v, w, sc, parts unused)
int cycle_df_blocks(long long N);
cudaError_t launch_cycle_df(const Op<double>& op, const DfTab& t, int pre, const double2* f, const double2* v,
                            double2* w, double2* sc, double* parts, double tol_abs, float4* fs, float4* xs,
                            float4* r_red, int n_r, int conj, unsigned* bar2, int* err, unsigned spin_limit,
                            unsigned extra_arrivals, cudaStream_t s);
// projection of a residual given as FP32 pairs (float4 per complex entry, N rows)
void launch_project_df_split(const float2* Q, long long ld, int k, const float4* r, long long N, double2* partials,
                             int nblk, cudaStream_t s);
// z = base + Q y with base given as FP32 pairs (float4 per complex entry); zdf
// (optional) receives z as FP32 pairs too
void launch_prolong_df_base(const float2* Q, long long ld, int k, const double2* y, const float4* base, double2* z,
                            float4* zdf, long long N, cudaStream_t s);
// k_apply_bicg for an x given as FP32 pairs: y = A x in double-float, y in FP64
void launch_apply_bicg_df(const Op<double>& op, const DfTab& t, int mode, const float4* x, double2* y,
                          const double2* w, int conj, double2* sc, double* parts, unsigned* counter, cudaStream_t s);
// r_red[m] = (v - A z) at the red node of pair m (stencil.cu)
void launch_residual_red(const Op<double>& op, const double2* z, const double2* v, double2* r_red, int conj,
                         cudaStream_t s);
// nonlinear DeepONet correction: raw trunk matrix in FP32 (p x N), branch in FP32
void launch_rm_to_cm_f32(const double* A, int ld, int p, float* B, long long N, cudaStream_t s);
void launch_nl_pack(const double2* r, const double* s2, float* x, long long N, cudaStream_t s);
void launch_nl_prolong(const float* T, int p, const float* b, const double* s2, double2* z, long long N,
                       cudaStream_t s);
// mixed precision: BF16 basis (column-major k columns of stride basis_ld(N), zero
// padding), complex64 vectors, FP32 accumulation
void launch_round_bf16(double* A, int ld, int k, long long N, cudaStream_t s);
void launch_rm_to_cm_bf16(const double* A, int ld, int k, void* B, long long ldb, long long N, cudaStream_t s);
void launch_restrict32(const Op<float>& op, const void* Q, long long ldq, int k, const float2* v, const float2* z,
                       int conj, float2* partials, int nblk, cudaStream_t s);
void launch_coarse_apply32(const float2* partials, int nblk, int k, const double2* Ainv, int conj, float2* y,
                           double2* cbuf, cudaStream_t s);
void launch_prolong32(const void* Q, long long ldq, int k, const float2* y, float2* z, long long N, cudaStream_t s);
// the red rows of the BF16 basis (k x ceil(N / 2), stride basis_ld(ceil(N / 2)))
void launch_red_rows_bf16(const void* Q, long long ldq, int k, long long N, int n, void* Qr, long long ldr,
                          cudaStream_t s);
// c = Q_red^T (v - A z) over the red rows (the residual after a red-black sweep that
// ends with the black half-sweep); returns the number of block partials written
int restrict32_red_blocks(long long N);
// c partials = Q_red^T r_red from a stored red-row residual (M = red rows): returns
// the number of partial rows written (restrict32_rr_ranges(N))
int restrict32_rr_ranges(long long N);
int launch_restrict32_rr(const void* Qr, long long ldr, int k, const float2* r_red, long long M, float2* partials,
                         long long N, cudaStream_t s);
int launch_restrict32_red(const Op<float>& op, const void* Qr, long long ldr, int k, const float2* v,
                          const float2* z, int conj, float2* partials, cudaStream_t s);
int restrict_blocks(long long N);

// mg.cu: grid transfers of the multigrid V-cycle (n_f = 2 n_c - 1, coarse node I at fine 2I)
void launch_inject_mask(int dim, int nf, const uint8_t* fine, uint8_t* coarse, cudaStream_t s);
void launch_inject_c128(int dim, int nf, const double2* fine, double2* coarse, cudaStream_t s);
template <typename R>
void launch_restrict_fw(int dim, int nf, const typename CT<R>::T* rf, const uint8_t* mask_c, typename CT<R>::T* rc,
                        cudaStream_t s);
template <typename R>
void launch_prolong_add(int dim, int nf, const typename CT<R>::T* zc, const uint8_t* mask_f, typename CT<R>::T* zf,
                        cudaStream_t s);

// adjoint.cu
void launch_receivers_setup(int n, int nrec, const double* xyz, int* idx, double* w, cudaStream_t s);
void launch_receivers_sample(int nrec, const int* idx, const double* w, const double2* u, double2* out,
                             cudaStream_t s);
void launch_receivers_adjoint(int nrec, const int* idx, const double* w, const double2* e, double2* b,
                              cudaStream_t s);
void launch_k2_gradient(long long N, const uint8_t* mask, const double2* lam, const double2* u, double2* g,
                        cudaStream_t s);

// ------------------------------------------------------------------- handle
}  // namespace helm

struct helm_handle {
    int dim = 0, n = 0, L = 0, precision = 0;
    long long N = 0;
    double k0 = 0, strength = 0, h = 0, hinv2 = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    helm::Op<double> op64{};
    helm::Op<float> op32{};
    helm::DfTab dft{};
    uint8_t* mask = nullptr;
    uint8_t* lidx = nullptr;
    uint8_t* nbm = nullptr;
    uint8_t* face = nullptr;        // outer-boundary problem (helm_create_bvp): face bytes
    int bvp = 0, neumann_top = 0;
    double2* k2 = nullptr;
    double2* invd = nullptr;
    float2* k2f = nullptr;
    float2* invdf = nullptr;
    // scratch for reductions and device scalars
    double* red = nullptr;          // partial sums (size max(apply blocks, kRedBlocks) * 8 doubles)
    long long red_len = 0;
    double2* sc = nullptr;          // device scalars (BiCGStab/FGMRES)
    double* hpin = nullptr;         // pinned host mirror for status polling
    double* hring = nullptr;        // two pinned snapshots of the scalars (lagged BiCGStab polling)
    cudaEvent_t evring[2] = {nullptr, nullptr};
    int* dflag = nullptr;           // device int flags
    unsigned* counter = nullptr;    // block counter of the fused reductions (zero between kernels)
    double* fparts = nullptr;       // partials of the fused reductions
    // general temporaries (N complex128 each)
    std::vector<double2*> tmp;
    // trunk basis
    int p = 0, k = 0, ldq = 0;
    std::vector<int> kept;
    float2* Q = nullptr;            // FP32 pairs, k x N
    float2* Qr = nullptr;           // its red rows, k x ceil(N / 2)
    double2* Ainv = nullptr;
    double2* coarse_partials = nullptr;
    void* Qbf = nullptr;            // BF16 basis (MIXED handles), column-major k x basis_ld(N)
    void* Qbr = nullptr;            // its red rows, k x basis_ld(ceil(N / 2))
    float2* partials32 = nullptr;
    float2* y32 = nullptr;
    float2* Z32 = nullptr;          // FGMRES preconditioned vectors in complex64 (MIXED)
    int m32_alloc = 0;
    // nonlinear correction (trained branch)
    float* Traw = nullptr;          // p x N FP32, masked rows zero
    float* bw = nullptr;            // branch weights (per layer W row-major out x in, then bias)
    std::vector<int> bwidths;
    float* nl_x = nullptr;          // 2N
    float* nl_h0 = nullptr;         // hidden activations
    float* nl_h1 = nullptr;
    double2* cbuf = nullptr;
    double2* ybuf = nullptr;
    // Krylov workspace
    int m_alloc = 0;
    double2* V = nullptr;
    double2* Z = nullptr;
    double2* Hm = nullptr;
    double* cs = nullptr;
    double2* sn = nullptr;
    double2* g = nullptr;
    double2* y = nullptr;
    double2* hpart = nullptr;
    // mixed precision buffers
    std::vector<float2*> tmp32;
    std::vector<float2*> b32;       // complex64 BiCGStab vectors (MIXED handles)
    double* b32parts = nullptr;     // their reduction partials
    float* a32parts = nullptr;      // partials of the operator launches with a fused reduction
    // one iteration of the complex64 BiCGStab captured as a CUDA graph (replayed per
    // iteration; rebuilt when the cycle's options change, dropped when the basis,
    // the k^2 field or a workspace buffer changes)
    cudaGraphExec_t g32 = nullptr;
    long long g32_launches = 0;
    int g32_key[5] = {0, 0, 0, 0, 0};
    double g32_omega = 0.0;
    cudaStream_t cap_stream = nullptr;
    // multigrid hierarchy (helm_mg_setup): the coarser levels as handles of their own
    std::vector<helm_handle*> mg;
    int mg_levels = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // launch accounting and per-kernel event timing (helm_set_profiling)
    int profile = 0;
    long long launches = 0;
    // bounded waits of the cooperative cycle's grid barriers: polls before a wait
    // gives up, and arrivals added to the barrier target (0; > 0 injects a timeout)
    unsigned bar_spin = 1u << 20;
    unsigned bar_extra = 0;
    // reliable updates of the complex64 BiCGStab (helm_set_reliable)
    double rel_delta = 0.1, rel_runaway = 1e3, rel_guard = 0.0;
    // phases: 0 restriction, 1 prolongation, 2 relaxation half-sweeps that read
    // neighbours, 3 operator applications of the Krylov loop
    std::vector<cudaEvent_t> evpool[4];
    int evn[4] = {0, 0, 0, 0};
};
