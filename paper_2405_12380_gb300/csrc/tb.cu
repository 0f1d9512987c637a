// Trunk-basis (TB) coarse space and correction (App. C, Eq. 6).
//
// Setup (once per don_load):
//   T_lj = trunk(x_l)_j                     k_trunk      (FP64 SIMT, activations in smem)
//   G = T^T T                               k_gram       (split-K tiles + fixed-order sum)
//   natural-order selection + Cholesky      k_select_chol (one CTA, right-looking, drop test)
//   Q1 = T_S R^-1, then CholQR2 pass        k_tri_inverse, k_gather_upper
//   W = A Q (real columns -> complex)       k_apply_columns
//   A_c = Q^T W, A_c^-1 by Gauss-Jordan     k_gram, k_gauss_jordan (one CTA, partial pivoting)
// Per application (z += Q A_c^-1 Q^T (v - A z)), Q column-major (k x N) as FP32 pairs,
// plus a compact copy Q_red (k x M, M = ceil(N / 2)) of its red rows (i + j + k
// even), row m holding the red node of the node pair (2m, 2m + 1):
//   k_apply        r = v - A z (FP64 stencil, stencil.cu) when the sweeps left a z;
//                  after a red-black Gauss-Seidel sweep r vanishes on the black
//                  rows and k_residual_red computes the red rows into a compact
//                  array (one entry per pair)
//   k_project_df   r tile split once into FP32 pairs in shared memory; warps own
//                  columns and keep FP32-pair sums in registers across tiles (one
//                  FP32-pair warp reduction per block); on Q_red with the compact
//                  r after red-black Gauss-Seidel (half the basis is read)
//   k_coarse_*     fixed-order sum of block partials, y = A_c^-1 c (FP64, one block per row)
//   k_prolong_df   z_l += sum_j Q_j[l] y_j in FP32-pair arithmetic, one thread per node
#include <cuda_bf16.h>

#include "helm_internal.cuh"

namespace helm {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int layer_index(int i, int n, int L) {
    int d = min(i, n - 1 - i);
    return max(0, L - d);
}

// ------------------------------------------------------------ trunk network
constexpr int TR_NB = 16;        // nodes per block
constexpr int TR_T = 256;        // threads = max width

// dW: per layer, W^T (in x out, row-major) then bias (out); act: HELM_ACT_TANH or
// HELM_ACT_LEAKY_RELU on the hidden layers (slope kLeakySlope for negative arguments)
constexpr double kLeakySlope = 0.01;
__global__ void __launch_bounds__(TR_T) k_trunk(Op<double> op, const double* __restrict__ dW, int4 w03, int4 w47,
                                                int n_layers, int p, double* __restrict__ T, int ldt, int act) {
    extern __shared__ double sm[];
    double* a_in = sm;                       // [TR_NB][TR_T]
    double* a_out = sm + TR_NB * TR_T;       // [TR_NB][TR_T]
    const int widths[8] = {w03.x, w03.y, w03.z, w03.w, w47.x, w47.y, w47.z, w47.w};
    const long long node0 = (long long)blockIdx.x * TR_NB;
    const double h = 1.0 / (op.n - 1);
    // coordinates of the block's nodes
    for (int t = threadIdx.x; t < TR_NB * op.dim; t += TR_T) {
        int nb = t / op.dim, ax = t % op.dim;
        long long l = node0 + nb;
        double c = 0;
        if (l < op.N) {
            long long q = l;
            for (int a = 0; a < ax; ++a) q /= op.n;
            c = (double)(q % op.n) * h;
        }
        a_in[nb * TR_T + ax] = c;
    }
    __syncthreads();
    const double* W = dW;
    for (int layer = 0; layer < n_layers; ++layer) {
        const int win = widths[layer], wout = widths[layer + 1];
        const double* Wt = W;                 // win x wout
        const double* b = W + (long long)win * wout;
        const int o = threadIdx.x;
        if (o < wout) {
            double acc[TR_NB];
            const double bo = b[o];
#pragma unroll
            for (int nb = 0; nb < TR_NB; ++nb) acc[nb] = 0.0;
            for (int i = 0; i < win; ++i) {
                const double w = Wt[(long long)i * wout + o];
#pragma unroll
                for (int nb = 0; nb < TR_NB; ++nb) acc[nb] = fma(a_in[nb * TR_T + i], w, acc[nb]);
            }
            const bool last = layer == n_layers - 1;
#pragma unroll
            for (int nb = 0; nb < TR_NB; ++nb) {
                double v = acc[nb] + bo;
                a_out[nb * TR_T + o] = last ? v : (act == HELM_ACT_TANH ? tanh(v) : (v > 0.0 ? v : kLeakySlope * v));
            }
        }
        __syncthreads();
        double* tmp = a_in;
        a_in = a_out;
        a_out = tmp;
        W = b + wout;
        __syncthreads();
    }
    // a_in holds the output layer
    for (int t = threadIdx.x; t < TR_NB * ldt; t += TR_T) {
        int nb = t / ldt, j = t % ldt;
        long long l = node0 + nb;
        if (l >= op.N) continue;
        double v = (j < p && !op.mask[l]) ? a_in[nb * TR_T + j] : 0.0;
        T[l * ldt + j] = v;
    }
}

// ------------------------------------------------------------------- Gram
// C = A^T B over N rows; A: N x p (lda), B: N x q (ldb); 64 x 64 output tile per
// block, 4 x 4 per thread, split over row slices (blockIdx.z); partials then summed.
constexpr int GT = 64, GR = 32;

__global__ void __launch_bounds__(256) k_gram(const double* __restrict__ A, int lda, int p,
                                              const double* __restrict__ B, int ldb, int q, long long N,
                                              long long rows_per_split, double* __restrict__ partials) {
    __shared__ double As[GR][GT + 1];
    __shared__ double Bs[GR][GT + 1];
    const int ti = threadIdx.x / 16, tj = threadIdx.x % 16;   // 16 x 16 threads, 4 x 4 each
    const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
    const long long r0 = (long long)blockIdx.z * rows_per_split;
    const long long r1 = min(N, r0 + rows_per_split);
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = 0.0;
    for (long long rb = r0; rb < r1; rb += GR) {
        for (int t = threadIdx.x; t < GR * GT; t += 256) {
            int rr = t / GT, cc = t % GT;
            long long row = rb + rr;
            bool ok = row < r1;
            As[rr][cc] = (ok && i0 + cc < p) ? A[row * lda + i0 + cc] : 0.0;
            Bs[rr][cc] = (ok && j0 + cc < q) ? B[row * ldb + j0 + cc] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < GR; ++rr) {
            double av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[rr][ti + 16 * a];
#pragma unroll
            for (int c = 0; c < 4; ++c) bv[c] = Bs[rr][tj + 16 * c];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][c] = fma(av[a], bv[c], acc[a][c]);
        }
        __syncthreads();
    }
    double* P = partials + (long long)blockIdx.z * p * q;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int i = i0 + ti + 16 * a, j = j0 + tj + 16 * c;
            if (i < p && j < q) P[(long long)i * q + j] = acc[a][c];
        }
}

__global__ void k_gram_sum(const double* __restrict__ partials, int nsplit, long long pq, double* __restrict__ out) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < pq; e += (long long)gridDim.x * blockDim.x) {
        double s = 0;
        for (int z = 0; z < nsplit; ++z) s += partials[(long long)z * pq + e];
        out[e] = s;
    }
}

// ------------------------------------------- natural-order Cholesky with drop
// G (p x p, ldg) symmetric.  Right-looking: at step j the trailing block holds the
// Schur complement of the kept columns.  Column j is kept when its Schur diagonal
// d_j > tau^2 G_jj (and d_j > 0).  Output: compact upper R (k x k, ld p), kept[0..k).
// flag = 1 when no column is kept.
__global__ void __launch_bounds__(1024) k_select_chol(const double* __restrict__ G, int p, int ldg, double tau,
                                                      double* __restrict__ W, double* __restrict__ R,
                                                      int* __restrict__ kept, int* __restrict__ nkept, int* flag) {
    __shared__ int s_keep;
    __shared__ double s_rjj;
    __shared__ int s_k;
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) W[e] = G[(e / p) * (long long)ldg + e % p];
    if (threadIdx.x == 0) s_k = 0;
    __syncthreads();
    for (int j = 0; j < p; ++j) {
        if (threadIdx.x == 0) {
            const double g = G[(long long)j * ldg + j];
            const double d = W[j * p + j];
            const int keep = (g > 0.0) && (d > 0.0) && (d > tau * tau * g);
            s_keep = keep;
            s_rjj = keep ? sqrt(d) : 0.0;
        }
        __syncthreads();
        if (s_keep) {
            const double rjj = s_rjj;
            // row j of R (uncompacted) over the trailing columns b >= j
            for (int b = j + threadIdx.x; b < p; b += blockDim.x) W[j * p + b] = (b == j) ? rjj : W[j * p + b] / rjj;
            __syncthreads();
            const int m = p - j - 1;
            for (long long e = threadIdx.x; e < (long long)m * m; e += blockDim.x) {
                int a = j + 1 + (int)(e / m), b = j + 1 + (int)(e % m);
                if (b < a) continue;
                W[a * p + b] -= W[j * p + a] * W[j * p + b];
            }
            if (threadIdx.x == 0) {
                kept[s_k] = j;
                s_k = s_k + 1;
            }
        }
        __syncthreads();
    }
    const int k = s_k;
    // compact R: R[a][b] = W[kept[a]][kept[b]] for a <= b
    for (long long e = threadIdx.x; e < (long long)k * k; e += blockDim.x) {
        int a = (int)(e / k), b = (int)(e % k);
        R[(long long)a * p + b] = (b >= a) ? W[kept[a] * p + kept[b]] : 0.0;
    }
    if (threadIdx.x == 0) {
        *nkept = k;
        if (k == 0) *flag = 1;
    }
}

// inverse of an upper-triangular k x k matrix (ld ldr); one thread per column
__global__ void k_tri_inverse(const double* __restrict__ R, int k, int ldr, double* __restrict__ Rinv) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= k) return;
    // solve R x = e_c by back substitution; x_a = 0 for a > c
    for (int a = k - 1; a > c; --a) Rinv[(long long)a * ldr + c] = 0.0;
    for (int a = c; a >= 0; --a) {
        double s = (a == c) ? 1.0 : 0.0;
        for (int b = a + 1; b <= c; ++b) s -= R[(long long)a * ldr + b] * Rinv[(long long)b * ldr + c];
        Rinv[(long long)a * ldr + c] = s / R[(long long)a * ldr + a];
    }
}

// Q[l][c] = sum_{a <= c} T[l][kept[a]] Rinv[a][c]  (kept == nullptr: identity)
constexpr int GU_NB = 16;
__global__ void __launch_bounds__(256) k_gather_upper(const double* __restrict__ T, int ldt,
                                                      const int* __restrict__ kept, int k,
                                                      const double* __restrict__ Rinv, int ldr,
                                                      double* __restrict__ Q, int ldq, long long N) {
    extern __shared__ double ts[];     // [GU_NB][k]
    const long long l0 = (long long)blockIdx.x * GU_NB;
    for (int t = threadIdx.x; t < GU_NB * k; t += blockDim.x) {
        int nb = t / k, a = t % k;
        long long l = l0 + nb;
        ts[t] = l < N ? T[l * ldt + (kept ? kept[a] : a)] : 0.0;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < ldq; c += blockDim.x) {
        double acc[GU_NB];
#pragma unroll
        for (int nb = 0; nb < GU_NB; ++nb) acc[nb] = 0.0;
        if (c < k) {
            for (int a = 0; a <= c; ++a) {
                const double r = Rinv[(long long)a * ldr + c];
#pragma unroll
                for (int nb = 0; nb < GU_NB; ++nb) acc[nb] = fma(ts[nb * k + a], r, acc[nb]);
            }
        }
#pragma unroll
        for (int nb = 0; nb < GU_NB; ++nb) {
            long long l = l0 + nb;
            if (l < N) Q[l * ldq + c] = acc[nb];
        }
    }
}

// W[l][2c], W[l][2c+1] = Re, Im of (A q_c)_l for the real columns q_c of Q
__global__ void __launch_bounds__(256) k_apply_columns(Op<double> op, const double* __restrict__ Q, int ldq, int k,
                                                       double* __restrict__ W, int ldw) {
    const long long total = op.N * (long long)k;
    const long long sy = op.n, sz = (long long)op.n * op.n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long l = e / k;
        const int c = (int)(e % k);
        double re = 0, im = 0;
        if (!op.mask[l]) {
            double s = 0;
            if (op.face) {
                // Sommerfeld / Neumann outer boundary: neighbour code of the handle and
                // the symmetric face weights (see Op::face)
                const unsigned code = op.nbm[l], fc = op.face[l];
                const int nb = (int)(fc >> 4);
                const double wx = ldexp(1.0, -(nb - (int)(fc & 1u))), wy = ldexp(1.0, -(nb - (int)((fc >> 1) & 1u)));
                const double wz = ldexp(1.0, -(nb - (int)((fc >> 2) & 1u)));
                if (code & 1u) s += wx * Q[(l - 1) * ldq + c];
                if (code & 2u) s += wx * Q[(l + 1) * ldq + c];
                if (code & 4u) s += wy * Q[(l - sy) * ldq + c];
                if (code & 8u) s += wy * Q[(l + sy) * ldq + c];
                if (op.dim == 3) {
                    if (code & 16u) s += wz * Q[(l - sz) * ldq + c];
                    if (code & 32u) s += wz * Q[(l + sz) * ldq + c];
                }
            } else {
                if (!op.mask[l - 1]) s += Q[(l - 1) * ldq + c];
                if (!op.mask[l + 1]) s += Q[(l + 1) * ldq + c];
                if (!op.mask[l - sy]) s += Q[(l - sy) * ldq + c];
                if (!op.mask[l + sy]) s += Q[(l + sy) * ldq + c];
                if (op.dim == 3) {
                    if (!op.mask[l - sz]) s += Q[(l - sz) * ldq + c];
                    if (!op.mask[l + sz]) s += Q[(l + sz) * ldq + c];
                }
            }
            double dre, dim_;
            if (op.k2) {
                double2 kk2 = op.k2[l];
                dre = kk2.x - 2.0 * op.dim * op.hinv2;
                dim_ = kk2.y;
            } else {
                dre = op.dre;
                dim_ = op.im[op.lidx[l]];
            }
            const double qv = Q[l * ldq + c];
            re = op.hinv2 * s + dre * qv;
            im = dim_ * qv;
        }
        W[l * ldw + 2 * c] = re;
        W[l * ldw + 2 * c + 1] = im;
    }
}

// Gauss-Jordan with partial pivoting on the complex k x k matrix
// A_c[i][c] = C[i][2c] + i C[i][2c+1]; one CTA; work: k x 2k complex.
__global__ void __launch_bounds__(1024) k_gauss_jordan(const double* __restrict__ C, int ldc, int k,
                                                       double2* __restrict__ Ainv, double2* __restrict__ Wk,
                                                       int* flag) {
    __shared__ int s_piv;
    __shared__ double s_val[32];
    __shared__ int s_idx[32];
    const int w2 = 2 * k;
    for (long long e = threadIdx.x; e < (long long)k * w2; e += blockDim.x) {
        int i = (int)(e / w2), c = (int)(e % w2);
        Wk[e] = c < k ? make_double2(C[(long long)i * ldc + 2 * c], C[(long long)i * ldc + 2 * c + 1])
                      : make_double2(c - k == i ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = 0; j < k; ++j) {
        // pivot: largest |a_ij| for i >= j (ties -> smallest index)
        double best = -1;
        int bi = j;
        for (int i = j + threadIdx.x; i < k; i += blockDim.x) {
            double v = hypot(Wk[(long long)i * w2 + j].x, Wk[(long long)i * w2 + j].y);
            if (v > best) { best = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            double ov = __shfl_xor_sync(0xffffffffu, best, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { s_val[warp] = best; s_idx[warp] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double bv = s_val[0];
            int bix = s_idx[0];
            for (int q = 1; q < nw; ++q)
                if (s_val[q] > bv || (s_val[q] == bv && s_idx[q] < bix)) { bv = s_val[q]; bix = s_idx[q]; }
            s_piv = bv > 0 ? bix : -1;
            if (bv <= 0) *flag = 2;
        }
        __syncthreads();
        const int piv = s_piv;
        if (piv < 0) return;
        if (piv != j) {
            for (int c = threadIdx.x; c < w2; c += blockDim.x) {
                double2 t = Wk[(long long)j * w2 + c];
                Wk[(long long)j * w2 + c] = Wk[(long long)piv * w2 + c];
                Wk[(long long)piv * w2 + c] = t;
            }
        }
        __syncthreads();
        const double2 pv = Wk[(long long)j * w2 + j];
        const double2 ipv = cdiv(make_double2(1, 0), pv);
        __syncthreads();
        for (int c = threadIdx.x; c < w2; c += blockDim.x) Wk[(long long)j * w2 + c] = cmul(Wk[(long long)j * w2 + c], ipv);
        __syncthreads();
        for (long long e = threadIdx.x; e < (long long)k * w2; e += blockDim.x) {
            int i = (int)(e / w2), c = (int)(e % w2);
            if (i == j || c < j) continue;
            double2 f = Wk[(long long)i * w2 + j];
            if (c == j) continue;
            Wk[e] = csub(Wk[e], cmul(f, Wk[(long long)j * w2 + c]));
        }
        __syncthreads();
        for (int i = threadIdx.x; i < k; i += blockDim.x)
            if (i != j) Wk[(long long)i * w2 + j] = make_double2(0, 0);
        __syncthreads();
    }
    for (long long e = threadIdx.x; e < (long long)k * k; e += blockDim.x) {
        int i = (int)(e / k), c = (int)(e % k);
        Ainv[e] = Wk[(long long)i * w2 + k + c];
    }
}

// ---------------------------------------------------------- per application
// Q is column-major here: basis vector j occupies Q[j*N .. j*N + N).
constexpr int RS_T = 256;        // threads per restriction block
constexpr int RS_TILE = 256;     // rows per tile (one residual per thread)

// ---------------------------------------------- FP32-pair (df64) projection
// GB300 issues FP32 FMAs 64x faster than FP64 ones, so the FP64 restriction and
// prolongation keep Q as pairs (hi, lo) of FP32 numbers with Q = hi + lo to ~2^-48
// and run the products and sums in FP32-pair arithmetic: a product is formed
// exactly as p + e (e from an FMA), the cross terms hi*lo are added to e, and the
// running sum is kept as an unevaluated pair with an exact two-sum.  Only the
// operand r (or y) is split once per node (or once per block), and the result is
// converted back to FP64 once per sum.

__device__ __forceinline__ void split_f64(double x, float& hi, float& lo) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
}

// (sh, sl) += (ah + al) * (bh + bl), dropping al*bl (~2^-48 relative)
__device__ __forceinline__ void pair_fma(float& sh, float& sl, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float s = sh + p;
    const float bb = s - sh;
    const float err = (sh - (s - bb)) + (p - bb);
    sh = s;
    sl += err + e;
}

// (sh, sl) summed over the warp in FP32-pair arithmetic (exact two-sums); the
// result is valid in every lane
__device__ __forceinline__ void pair_warp_sum(float& sh, float& sl) {
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, sh, o);
        const float ol = __shfl_xor_sync(0xffffffffu, sl, o);
        const float s = sh + oh;
        const float bb = s - sh;
        const float err = (sh - (s - bb)) + (oh - bb);
        sh = s;
        sl = sl + ol + err;
    }
}

constexpr int PJ_T = 512;        // threads per projection block (16 warps), two blocks per SM
constexpr int PJ_TILE = 512;     // rows per tile (one per thread)

// partials[b][j] = sum over the rows of block b of Q_j[l] r_l (r given in FP64, or
// SPLIT: already as FP32 pairs, one float4 per complex entry)
template <int KPW, bool SPLIT>
__global__ void __launch_bounds__(PJ_T, 2) k_project_df(const float2* __restrict__ Q, long long ld, int k,
                                                     const void* __restrict__ rv_, long long N,
                                                     double2* __restrict__ partials, long long rows_per_block) {
    __shared__ float4 rs[PJ_TILE];       // (re hi, re lo, im hi, im lo)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = PJ_T / 32;
    constexpr int RPL = PJ_TILE / 32;
    const long long r0 = (long long)blockIdx.x * rows_per_block;
    const long long r1 = min(N, r0 + rows_per_block);
    float acc[KPW][4];
#pragma unroll
    for (int c = 0; c < KPW; ++c) acc[c][0] = acc[c][1] = acc[c][2] = acc[c][3] = 0.f;
    for (long long t0 = r0; t0 < r1; t0 += PJ_TILE) {
        const long long l = t0 + threadIdx.x;
        float4 rp = make_float4(0.f, 0.f, 0.f, 0.f);
        if (SPLIT) {
            if (l < r1) rp = static_cast<const float4*>(rv_)[l];
        } else {
            const double2 rv = l < r1 ? static_cast<const double2*>(rv_)[l] : make_double2(0, 0);
            split_f64(rv.x, rp.x, rp.y);
            split_f64(rv.y, rp.z, rp.w);
        }
        __syncthreads();
        rs[threadIdx.x] = rp;
        __syncthreads();
        const int rows = (int)min((long long)PJ_TILE, r1 - t0);
#pragma unroll
        for (int c = 0; c < KPW; ++c) {
            const int j = warp + NW * c;
            if (j < k) {
                const float2* Qj = Q + (long long)j * ld + t0;
                float a0 = acc[c][0], a1 = acc[c][1], a2 = acc[c][2], a3 = acc[c][3];
                // all loads of the column issued before use (rows past the end of the
                // block read nothing and meet r = 0 in shared memory)
                float2 qv[RPL];
#pragma unroll
                for (int u = 0; u < RPL; ++u)
                    qv[u] = (lane + 32 * u < rows) ? __ldg(Qj + lane + 32 * u) : make_float2(0.f, 0.f);
#pragma unroll
                for (int u = 0; u < RPL; ++u) {
                    const float4 rr = rs[lane + 32 * u];
                    pair_fma(a0, a1, qv[u].x, qv[u].y, rr.x, rr.y);
                    pair_fma(a2, a3, qv[u].x, qv[u].y, rr.z, rr.w);
                }
                acc[c][0] = a0; acc[c][1] = a1; acc[c][2] = a2; acc[c][3] = a3;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < KPW; ++c) {
        const int j = warp + NW * c;
        pair_warp_sum(acc[c][0], acc[c][1]);
        pair_warp_sum(acc[c][2], acc[c][3]);
        if (lane == 0 && j < k)
            partials[(long long)blockIdx.x * k + j] =
                make_double2((double)acc[c][0] + (double)acc[c][1], (double)acc[c][2] + (double)acc[c][3]);
    }
}

// c_j = fixed-order sum of the block partials, one block per column
__global__ void __launch_bounds__(64) k_coarse_reduce(const double2* __restrict__ partials, int nblk, int k,
                                                      double2* __restrict__ c) {
    __shared__ double2 red[2];
    const int j = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double sx = 0, sy = 0;
    for (int b = threadIdx.x; b < nblk; b += 64) {
        const double2 q = partials[(long long)b * k + j];
        sx += q.x;
        sy += q.y;
    }
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if (lane == 0) red[w] = make_double2(sx, sy);
    __syncthreads();
    if (threadIdx.x == 0) c[j] = make_double2(red[0].x + red[1].x, red[0].y + red[1].y);
}

// y_i = sum_j A_c^-1[i][j] c_j (conj: conj(A_c^-1)), one block per row
__global__ void __launch_bounds__(64) k_coarse_gemv(const double2* __restrict__ Ainv, int k, int conj,
                                                    const double2* __restrict__ c, double2* __restrict__ y) {
    __shared__ double2 red[2];
    const int i = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double sx = 0, sy = 0;
    for (int j = threadIdx.x; j < k; j += 64) {
        double2 a = Ainv[(long long)i * k + j];
        if (conj) a.y = -a.y;
        const double2 cj = c[j];
        sx += a.x * cj.x - a.y * cj.y;
        sy += a.x * cj.y + a.y * cj.x;
    }
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if (lane == 0) red[w] = make_double2(sx, sy);
    __syncthreads();
    if (threadIdx.x == 0) y[i] = make_double2(red[0].x + red[1].x, red[0].y + red[1].y);
}

// complex64 partials of the BF16-basis restriction: c_j = sum over blocks (FP64, fixed
// order), one block per column; then y (complex64) = A_c^-1 c, one block per row --
// spread over k SMs like the FP64 pair above
// c_j = sum of the nblk partial rows (FP32 partials): one block per column, a
// strided FP32 sum per thread, an FP32 butterfly per warp, the warps in order
// (FP64 adds and shuffles run at a small fraction of the FP32 rate on this GPU)
__global__ void __launch_bounds__(256) k_coarse32_reduce(const float2* __restrict__ partials, int nblk, int k,
                                                         double2* __restrict__ c) {
    __shared__ float2 red[8];
    const int j = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float sx = 0.f, sy = 0.f;
    for (int b = threadIdx.x; b < nblk; b += 256) {
        const float2 q = partials[(long long)b * k + j];
        sx += q.x;
        sy += q.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) red[w] = make_float2(sx, sy);
    __syncthreads();
    if (threadIdx.x == 0) {
        float tx = 0.f, ty = 0.f;
        for (int q = 0; q < 8; ++q) {
            tx += red[q].x;
            ty += red[q].y;
        }
        c[j] = make_double2(tx, ty);
    }
}

__global__ void __launch_bounds__(64) k_coarse32_gemv(const double2* __restrict__ Ainv, int k, int conj,
                                                      const double2* __restrict__ c, float2* __restrict__ y) {
    __shared__ double2 red[2];
    const int i = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double sx = 0, sy = 0;
    for (int j = threadIdx.x; j < k; j += 64) {
        double2 a = Ainv[(long long)i * k + j];
        if (conj) a.y = -a.y;
        const double2 cj = c[j];
        sx += a.x * cj.x - a.y * cj.y;
        sy += a.x * cj.y + a.y * cj.x;
    }
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if (lane == 0) red[w] = make_double2(sx, sy);
    __syncthreads();
    if (threadIdx.x == 0) y[i] = make_float2((float)(red[0].x + red[1].x), (float)(red[0].y + red[1].y));
}

// z_l += sum_j Q_j[l] y_j in FP32-pair arithmetic, one thread per node
// BASE: z_l = base_l + sum_j Q_j[l] y_j with base given as FP32 pairs
template <bool BASE>
// (and, given zdf, also the sum as FP32 pairs)
__global__ void __launch_bounds__(256) k_prolong_df(const float2* __restrict__ Q, long long ld, int k,
                                                    const double2* __restrict__ y, double2* __restrict__ z,
                                                    const float4* __restrict__ base, float4* __restrict__ zdf,
                                                    long long N) {
    __shared__ float4 ys[kMaxP];
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        float4 t;
        split_f64(y[j].x, t.x, t.y);
        split_f64(y[j].y, t.z, t.w);
        ys[j] = t;
    }
    __syncthreads();
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < N; l += (long long)gridDim.x * blockDim.x) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        const float2* q = Q + l;
        int j = 0;
        for (; j + 8 <= k; j += 8) {
            float2 qv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) qv[u] = __ldg(q + (long long)(j + u) * ld);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float4 yy = ys[j + u];
                pair_fma(a0, a1, qv[u].x, qv[u].y, yy.x, yy.y);
                pair_fma(a2, a3, qv[u].x, qv[u].y, yy.z, yy.w);
            }
        }
        for (; j < k; ++j) {
            const float2 qv = q[(long long)j * ld];
            const float4 yy = ys[j];
            pair_fma(a0, a1, qv.x, qv.y, yy.x, yy.y);
            pair_fma(a2, a3, qv.x, qv.y, yy.z, yy.w);
        }
        if (BASE) {
            // (b + a) as a pair sum, then one conversion to FP64
            const float4 b = base[l];
            float s0 = b.x + a0, bb = s0 - b.x, e0 = (b.x - (s0 - bb)) + (a0 - bb) + (b.y + a1);
            float s1 = b.z + a2;
            bb = s1 - b.z;
            const float e1 = (b.z - (s1 - bb)) + (a2 - bb) + (b.w + a3);
            z[l] = make_double2((double)s0 + (double)e0, (double)s1 + (double)e1);
            if (zdf) {
                const float h0 = s0 + e0, h1 = s1 + e1;
                zdf[l] = make_float4(h0, e0 - (h0 - s0), h1, e1 - (h1 - s1));
            }
        } else {
            double2 zz = z[l];
            z[l] = make_double2(zz.x + ((double)a0 + (double)a1), zz.y + ((double)a2 + (double)a3));
        }
    }
}

// colour of node l of a grid with n nodes per side: (i + j + k) mod 2, 0 = red
__device__ __forceinline__ int node_colour(long long l, int n) {
    const unsigned ul = (unsigned)l, un = (unsigned)n;
    const unsigned r = ul / un;          // row index j + n k
    const unsigned kk = r / un;
    return (int)(((ul - r * un) + (r - kk * un) + kk) & 1u);
}

// Q_red[j][m] = Q[j][red node of pair m]; every pair (2m, 2m + 1) holds one red and
// one black node (rows of even length start on even l; for odd n the colour is the
// parity of l), and a last single node (odd N) is red
__global__ void k_red_rows(const float2* __restrict__ Q, long long ldq, int k, long long N, int n,
                           float2* __restrict__ Qr, long long ldr) {
    const long long M = (N + 1) / 2;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < M * k;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long j = idx / M, m = idx - j * M;
        const long long l = 2 * m + node_colour(2 * m, n);
        Qr[j * ldr + m] = Q[j * ldq + l];
    }
}

// FP64 row-major Q (N x ld) -> column-major pairs (k x N) of FP32 (hi, lo), and
// the row-major FP64 values replaced by hi + lo (the basis the kernels use)
__global__ void k_split_basis(double* __restrict__ A, int ld, int k, float2* __restrict__ B, long long ldb,
                              long long N) {
    __shared__ float2 tile[32][33];
    const long long l0 = (long long)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        long long l = l0 + r;
        int c = c0 + threadIdx.x;
        float2 v = make_float2(0.f, 0.f);
        if (l < N && c < k) {
            split_f64(A[l * ld + c], v.x, v.y);
            A[l * ld + c] = (double)v.x + (double)v.y;
        }
        tile[r][threadIdx.x] = v;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int c = c0 + r;
        long long l = l0 + threadIdx.x;
        if (c < k && l < N) B[(long long)c * ldb + l] = tile[threadIdx.x][r];
    }
}

__global__ void k_cm_pair_to_rm(const float2* __restrict__ B, long long ldb, int k, double* __restrict__ A,
                                long long N) {
    __shared__ double tile[32][33];
    const long long l0 = (long long)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int c = c0 + r;
        long long l = l0 + threadIdx.x;
        double v = 0.0;
        if (c < k && l < N) {
            const float2 q = B[(long long)c * ldb + l];
            v = (double)q.x + (double)q.y;
        }
        tile[r][threadIdx.x] = v;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        long long l = l0 + r;
        int c = c0 + threadIdx.x;
        if (l < N && c < k) A[l * k + c] = tile[threadIdx.x][r];
    }
}

// ------------------------------------------------ nonlinear DeepONet correction
// row-major FP64 T (N x ld, p used) -> column-major FP32 (p x N)
__global__ void k_rm_to_cm_f32(const double* __restrict__ A, int ld, int p, float* __restrict__ B, long long N) {
    __shared__ float tile[32][33];
    const long long l0 = (long long)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        long long l = l0 + r;
        int c = c0 + threadIdx.x;
        tile[r][threadIdx.x] = (l < N && c < p) ? (float)A[l * ld + c] : 0.0f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int c = c0 + r;
        long long l = l0 + threadIdx.x;
        if (c < p && l < N) B[(long long)c * N + l] = tile[threadIdx.x][r];
    }
}

// branch input [Re r, Im r] / s, s^2 read from the device (s = 0 -> zeros)
__global__ void k_nl_pack(const double2* __restrict__ r, const double* __restrict__ s2, float* __restrict__ x,
                          long long N) {
    const double s = sqrt(*s2);
    const double inv = s > 0 ? 1.0 / s : 0.0;
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < N; l += (long long)gridDim.x * blockDim.x) {
        const double2 v = r[l];
        x[l] = (float)(v.x * inv);
        x[N + l] = (float)(v.y * inv);
    }
}

// z_l += s (sum_j T_j[l] b_j + i sum_j T_j[l] b_{p+j})
__global__ void __launch_bounds__(256) k_nl_prolong(const float* __restrict__ T, int p, const float* __restrict__ b,
                                                    const double* __restrict__ s2, double2* __restrict__ z, long long N) {
    __shared__ float bs[2 * kMaxP];
    for (int j = threadIdx.x; j < 2 * p; j += blockDim.x) bs[j] = b[j];
    __syncthreads();
    const double s = sqrt(*s2);
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < N; l += (long long)gridDim.x * blockDim.x) {
        float re = 0.f, im = 0.f;
#pragma unroll 8
        for (int j = 0; j < p; ++j) {
            const float t = T[(long long)j * N + l];
            re = fmaf(t, bs[j], re);
            im = fmaf(t, bs[p + j], im);
        }
        double2 zz = z[l];
        z[l] = make_double2(zz.x + s * re, zz.y + s * im);
    }
}

// ------------------------------------------------- mixed precision (BF16 Q)
// Q rounded to BF16 (round to nearest even of the FP64 value via FP32).
__global__ void k_round_bf16(double* __restrict__ A, int ld, int k, long long N) {
    const long long total = N * (long long)ld;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        if ((int)(e % ld) < k) A[e] = (double)__bfloat162float(__float2bfloat16_rn((float)A[e]));
    }
}

// row-major FP64 (N x ld) -> column-major BF16 (k columns of stride ldb)
__global__ void k_rm_to_cm_bf16(const double* __restrict__ A, int ld, int k, __nv_bfloat16* __restrict__ B, long long ldb,
                                long long N) {
    __shared__ float tile[32][33];
    const long long l0 = (long long)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        long long l = l0 + r;
        int c = c0 + threadIdx.x;
        tile[r][threadIdx.x] = (l < N && c < k) ? (float)A[l * ld + c] : 0.0f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int c = c0 + r;
        long long l = l0 + threadIdx.x;
        if (c < k && l < N) B[(long long)c * ldb + l] = __float2bfloat16_rn(tile[threadIdx.x][r]);
    }
}

// complex64 restriction with a BF16 basis, FP32 accumulation: same structure as k_restrict
template <int KPW>
__global__ void __launch_bounds__(RS_T) k_restrict32(Op<float> op, const __nv_bfloat16* __restrict__ Q, long long ldq, int k,
                                                     const float2* __restrict__ v, const float2* __restrict__ z,
                                                     int conj, float2* __restrict__ partials,
                                                     long long rows_per_block) {
    __shared__ float2 rs[RS_TILE];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = RS_T / 32;
    const long long r0 = (long long)blockIdx.x * rows_per_block;
    const long long r1 = min(op.N, r0 + rows_per_block);
    const long long N = op.N;
    float2 acc[KPW];
#pragma unroll
    for (int c = 0; c < KPW; ++c) acc[c] = make_float2(0.f, 0.f);
    const long long sy = op.n, sz = (long long)op.n * op.n;
    for (long long t0 = r0; t0 < r1; t0 += RS_TILE) {
        const long long l = t0 + threadIdx.x;
        float2 r = make_float2(0.f, 0.f);
        if (l < r1 && !op.mask[l]) {
            r = v[l];
            if (z) {
                float2 s = make_float2(0.f, 0.f);
                const uint8_t* mk = op.mask;
                if (!mk[l - 1]) s = cadd(s, z[l - 1]);
                if (!mk[l + 1]) s = cadd(s, z[l + 1]);
                if (!mk[l - sy]) s = cadd(s, z[l - sy]);
                if (!mk[l + sy]) s = cadd(s, z[l + sy]);
                if (op.dim == 3) {
                    if (!mk[l - sz]) s = cadd(s, z[l - sz]);
                    if (!mk[l + sz]) s = cadd(s, z[l + sz]);
                }
                float2 d;
                if (op.k2) {
                    d = op.k2[l];
                    d.x -= 2.0f * op.dim * op.hinv2;
                } else {
                    d = make_float2(op.dre, op.im[op.lidx[l]]);
                }
                if (conj) d.y = -d.y;
                const float2 zc = z[l];
                r.x -= op.hinv2 * s.x + (d.x * zc.x - d.y * zc.y);
                r.y -= op.hinv2 * s.y + (d.x * zc.y + d.y * zc.x);
            }
        }
        __syncthreads();
        rs[threadIdx.x] = r;
        __syncthreads();
        const int rows = (int)min((long long)RS_TILE, r1 - t0);
#pragma unroll
        for (int c = 0; c < KPW; ++c) {
            const int j = warp + NW * c;
            if (j < k) {
                const __nv_bfloat16* Qj = Q + (long long)j * ldq + t0;
                float ax = acc[c].x, ay = acc[c].y;
                for (int q = lane; q < rows; q += 32) {
                    const float qv = __bfloat162float(Qj[q]);
                    const float2 rr = rs[q];
                    ax = fmaf(qv, rr.x, ax);
                    ay = fmaf(qv, rr.y, ay);
                }
                acc[c].x = ax;
                acc[c].y = ay;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < KPW; ++c) {
        const int j = warp + NW * c;
        float sx = acc[c].x, sy2 = acc[c].y;
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy2 += __shfl_xor_sync(0xffffffffu, sy2, o);
        }
        if (lane == 0 && j < k) partials[(long long)blockIdx.x * k + j] = make_float2(sx, sy2);
    }
}


__global__ void __launch_bounds__(256) k_prolong32(const __nv_bfloat16* __restrict__ Q, long long ldq, int k,
                                                   const float2* __restrict__ y, float2* __restrict__ z, long long N) {
    __shared__ float2 ys[kMaxP];
    for (int j = threadIdx.x; j < k; j += blockDim.x) ys[j] = y[j];
    __syncthreads();
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < N; l += (long long)gridDim.x * blockDim.x) {
        float sx = 0.f, sy = 0.f;
        const __nv_bfloat16* q = Q + l;
#pragma unroll 8
        for (int j = 0; j < k; ++j) {
            const float qv = __bfloat162float(q[(long long)j * ldq]);
            sx = fmaf(qv, ys[j].x, sx);
            sy = fmaf(qv, ys[j].y, sy);
        }
        float2 zz = z[l];
        z[l] = make_float2(zz.x + sx, zz.y + sy);
    }
}

// ---- the trunk-basis correction of the complex64 red-black cycle ---------------
// BF16 basis columns have a stride that is a multiple of 64 entries with zero
// padding, so that a thread reads eight consecutive rows of a column with one
// 16-byte load.  Eight BF16 values of a uint4, in memory order (BF16 is the top
// half of an FP32 number).
__device__ __forceinline__ void bf16x8(const uint4 u, float* q) {
    q[0] = __uint_as_float(u.x << 16); q[1] = __uint_as_float(u.x & 0xffff0000u);
    q[2] = __uint_as_float(u.y << 16); q[3] = __uint_as_float(u.y & 0xffff0000u);
    q[4] = __uint_as_float(u.z << 16); q[5] = __uint_as_float(u.z & 0xffff0000u);
    q[6] = __uint_as_float(u.w << 16); q[7] = __uint_as_float(u.w & 0xffff0000u);
}

// Qr[j][m] = Q[j][red node of pair m] (BF16; the red node of pair (2m, 2m + 1) is
// 2m + colour(2m); an odd N's last pair may name node N, a zero padding row)
__global__ void k_red_rows_bf16(const __nv_bfloat16* __restrict__ Q, long long ldq, int k, long long N, int n,
                                __nv_bfloat16* __restrict__ Qr, long long ldr) {
    const long long M = (N + 1) / 2;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < M * k;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long j = idx / M, m = idx - j * M;
        const long long l = 2 * m + node_colour(2 * m, n);
        Qr[j * ldr + m] = Q[j * ldq + l];
    }
}

// (v - A z) at the red node of pair m (complex64); zero on masked nodes and past N
__device__ __forceinline__ float2 red_residual32(const Op<float>& op, const float2* __restrict__ v,
                                                 const float2* __restrict__ z, long long m, int conj) {
    const long long l = 2 * m + node_colour(2 * m, op.n);
    if (l >= op.N) return make_float2(0.f, 0.f);
    const unsigned code = op.nbm[l];
    if (code & 0x80u) return make_float2(0.f, 0.f);
    const long long sy = op.n, sz = (long long)op.n * op.n;
    float2 s = make_float2(0.f, 0.f);
    if (code & 1u) s = cadd(s, z[HCHK(l - 1, op.N)]);
    if (code & 2u) s = cadd(s, z[HCHK(l + 1, op.N)]);
    if (code & 4u) s = cadd(s, z[HCHK(l - sy, op.N)]);
    if (code & 8u) s = cadd(s, z[HCHK(l + sy, op.N)]);
    if (op.dim == 3) {
        if (code & 16u) s = cadd(s, z[HCHK(l - sz, op.N)]);
        if (code & 32u) s = cadd(s, z[HCHK(l + sz, op.N)]);
    }
    float2 d;
    if (op.k2) {
        d = op.k2[l];
        d.x -= 2.0f * op.dim * op.hinv2;
    } else {
        d = make_float2(op.dre, op.im[op.lidx[l]]);
    }
    if (conj) d.y = -d.y;
    const float2 zc = z[l], vv = v[l];
    return make_float2(vv.x - (op.hinv2 * s.x + (d.x * zc.x - d.y * zc.y)),
                       vv.y - (op.hinv2 * s.y + (d.x * zc.y + d.y * zc.x)));
}

constexpr int RR_T = 256;     // threads of the red-row restriction
constexpr int RR_ROWS = 8;    // consecutive red rows per thread (one 16-byte basis load per column)
constexpr int RR_KC = 8;      // columns per chunk (registers)

// c = Q_red^T r with r = v - A z on the red rows (after a red-black sweep that ends
// with the black half-sweep the residual vanishes on black and masked rows).  A
// warp takes 32 x 8 consecutive red rows; per chunk of 8 columns each lane sums its
// 8 rows in FP32, the warp adds its lanes (fixed butterfly) and lane 0 adds the
// chunk into the warp's row of shared memory; at the end the block sums its warps
// in a fixed order into partials[block][j].  Deterministic.
__global__ void __launch_bounds__(RR_T, 4) k_restrict32_red(Op<float> op, const __nv_bfloat16* __restrict__ Qr,
                                                         long long ldr, int k, const float2* __restrict__ v,
                                                         const float2* __restrict__ z, int conj,
                                                         float2* __restrict__ partials, long long M) {
    constexpr int NW = RR_T / 32;
    constexpr int WROWS = 32 * RR_ROWS;            // red rows of one warp tile
    __shared__ float2 sacc[NW][kMaxP];
    // the warp tile's residuals, 8 rows per lane with one padding slot per lane
    __shared__ float2 rsm[NW][32 * (RR_ROWS + 1)];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = lane; j < k; j += 32) sacc[warp][j] = make_float2(0.f, 0.f);
    __syncwarp();
    const long long groups = (M + RR_ROWS - 1) / RR_ROWS;
    const long long wtiles = (groups + 31) / 32;
    for (long long wt = blockIdx.x * (long long)NW + warp; wt < wtiles; wt += (long long)gridDim.x * NW) {
        // residuals of the tile's rows computed with consecutive rows on consecutive
        // lanes (coalesced neighbour loads), then read back eight consecutive rows per lane
        const long long mt = wt * WROWS;
#pragma unroll
        for (int q = 0; q < RR_ROWS; ++q) {
            const int row = lane + 32 * q;
            const long long m = mt + row;
            rsm[warp][row + row / RR_ROWS] = (m < M) ? red_residual32(op, v, z, m, conj) : make_float2(0.f, 0.f);
        }
        __syncwarp();
        const long long m0 = mt + (long long)lane * RR_ROWS;
        float2 r[RR_ROWS];
#pragma unroll
        for (int q = 0; q < RR_ROWS; ++q) r[q] = rsm[warp][lane * (RR_ROWS + 1) + q];
        __syncwarp();
        for (int c0 = 0; c0 < k; c0 += RR_KC) {
            float ax[RR_KC], ay[RR_KC];
#pragma unroll
            for (int c = 0; c < RR_KC; ++c) {
                ax[c] = 0.f;
                ay[c] = 0.f;
                if (c0 + c < k && m0 < M) {
                    const uint4 u = __ldcs(reinterpret_cast<const uint4*>(Qr + (long long)(c0 + c) * ldr + m0));
                    float qv[8];
                    bf16x8(u, qv);
#pragma unroll
                    for (int q = 0; q < RR_ROWS; ++q) {
                        ax[c] = fmaf(qv[q], r[q].x, ax[c]);
                        ay[c] = fmaf(qv[q], r[q].y, ay[c]);
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < RR_KC; ++c)
                for (int o = 16; o > 0; o >>= 1) {
                    ax[c] += __shfl_xor_sync(0xffffffffu, ax[c], o);
                    ay[c] += __shfl_xor_sync(0xffffffffu, ay[c], o);
                }
            if (lane == 0)
#pragma unroll
                for (int c = 0; c < RR_KC; ++c)
                    if (c0 + c < k) {
                        sacc[warp][c0 + c].x += ax[c];
                        sacc[warp][c0 + c].y += ay[c];
                    }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += RR_T) {
        float2 t = make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < NW; ++w) t = cadd(t, sacc[w][j]);
        partials[(long long)blockIdx.x * k + j] = t;
    }
}

// c = Q_red^T r_red from a stored red-row residual: a tall-skinny product.  A warp
// owns RQ_COLS columns and one range of RQ_RANGE rows; per 256 rows each lane loads
// its 8 consecutive residual rows and then all its 16-byte basis pieces (one per
// column, issued together) before the FMAs, and keeps the complex sums in
// registers over the range; the lanes are added once at the end (fixed butterfly)
// and lane 0 writes partials[range][j].  Deterministic.
constexpr int RQ_COLS = 8;
constexpr int RQ_RANGE = 1024;
__global__ void __launch_bounds__(256) k_restrict32_rr(const __nv_bfloat16* __restrict__ Qr, long long ldr, int k,
                                                       const float2* __restrict__ r, long long M,
                                                       float2* __restrict__ partials, int S) {
    const int lane = threadIdx.x & 31;
    const int rg = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int c0 = blockIdx.y * RQ_COLS;
    if (rg >= S) return;
    const int nc = min(RQ_COLS, k - c0);
    float ax[RQ_COLS], ay[RQ_COLS];
#pragma unroll
    for (int c = 0; c < RQ_COLS; ++c) ax[c] = ay[c] = 0.f;
#pragma unroll 1
    for (int it = 0; it < RQ_RANGE / 256; ++it) {
        const long long m0 = (long long)rg * RQ_RANGE + it * 256 + lane * 8;
        if (m0 >= M) break;
        uint4 u[RQ_COLS];
#pragma unroll
        for (int c = 0; c < RQ_COLS; ++c)
            u[c] = c < nc ? __ldcs(reinterpret_cast<const uint4*>(
                                Qr + HCHK((long long)(c0 + c) * ldr + m0, (long long)k * ldr - 7)))
                          : make_uint4(0u, 0u, 0u, 0u);
        float2 rv[8];
        if (m0 + 8 <= M) {
            const float4* r4 = reinterpret_cast<const float4*>(r + HCHK(m0, M - 7));
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 t = r4[q];
                rv[2 * q] = make_float2(t.x, t.y);
                rv[2 * q + 1] = make_float2(t.z, t.w);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) rv[q] = (m0 + q < M) ? r[m0 + q] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int c = 0; c < RQ_COLS; ++c) {
            float qv[8];
            bf16x8(u[c], qv);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                ax[c] = fmaf(qv[q], rv[q].x, ax[c]);
                ay[c] = fmaf(qv[q], rv[q].y, ay[c]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < RQ_COLS; ++c)
        for (int o = 16; o > 0; o >>= 1) {
            ax[c] += __shfl_xor_sync(0xffffffffu, ax[c], o);
            ay[c] += __shfl_xor_sync(0xffffffffu, ay[c], o);
        }
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < RQ_COLS; ++c)
            if (c < nc) partials[(long long)rg * k + c0 + c] = make_float2(ax[c], ay[c]);
}

// z += Q y, eight consecutive rows per thread (16-byte basis loads, 64-byte z
// accesses); z must be 16-byte aligned
__global__ void __launch_bounds__(256) k_prolong32v(const __nv_bfloat16* __restrict__ Q, long long ldq, int k,
                                                    const float2* __restrict__ y, float2* __restrict__ z,
                                                    long long N) {
    __shared__ float2 ys[kMaxP];
    for (int j = threadIdx.x; j < k; j += blockDim.x) ys[j] = y[j];
    __syncthreads();
    const long long groups = (N + 7) / 8;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < groups;
         g += (long long)gridDim.x * blockDim.x) {
        const long long l0 = g * 8;
        float ax[8], ay[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            ax[q] = 0.f;
            ay[q] = 0.f;
        }
        const __nv_bfloat16* Qg = Q + l0;
#pragma unroll 8
        for (int j = 0; j < k; ++j) {
            const uint4 u =
                __ldcs(reinterpret_cast<const uint4*>(Q + HCHK((long long)j * ldq + l0, (long long)k * ldq - 7)));
            float qv[8];
            bf16x8(u, qv);
            const float2 yj = ys[j];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                ax[q] = fmaf(qv[q], yj.x, ax[q]);
                ay[q] = fmaf(qv[q], yj.y, ay[q]);
            }
        }
        if (l0 + 8 <= N) {
            float4* z4 = reinterpret_cast<float4*>(z + HCHK(l0, N - 7));
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float4 t = z4[q];
                t.x += ax[2 * q];
                t.y += ay[2 * q];
                t.z += ax[2 * q + 1];
                t.w += ay[2 * q + 1];
                z4[q] = t;
            }
        } else {
            for (int q = 0; q < 8; ++q)
                if (l0 + q < N) {
                    float2 t = z[l0 + q];
                    z[l0 + q] = make_float2(t.x + ax[q], t.y + ay[q]);
                }
        }
    }
}

}  // namespace

void launch_trunk_eval(const Op<double>& op, const double* dW, const int* widths, int n_layers, int p, int act,
                       double* T, int ldt, cudaStream_t s) {
    int w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i <= n_layers && i < 8; ++i) w[i] = widths[i];
    size_t smem = 2 * TR_NB * TR_T * sizeof(double);
    cudaFuncSetAttribute(k_trunk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    long long blocks = (op.N + TR_NB - 1) / TR_NB;
    k_trunk<<<(unsigned)blocks, TR_T, smem, s>>>(op, dW, make_int4(w[0], w[1], w[2], w[3]),
                                                 make_int4(w[4], w[5], w[6], w[7]), n_layers, p, T, ldt, act);
}

void launch_gram(const double* A, int lda, int p, const double* B, int ldb, int q, long long N, double* partials,
                 double* out, cudaStream_t s) {
    int gx = (p + GT - 1) / GT, gy = (q + GT - 1) / GT;
    int nsplit = (2 * 152 + gx * gy - 1) / (gx * gy);
    long long rows = (N + nsplit - 1) / nsplit;
    rows = ((rows + GR - 1) / GR) * GR;
    nsplit = (int)((N + rows - 1) / rows);
    k_gram<<<dim3(gx, gy, nsplit), 256, 0, s>>>(A, lda, p, B, ldb, q, N, rows, partials);
    long long pq = (long long)p * q;
    k_gram_sum<<<(unsigned)((pq + 255) / 256), 256, 0, s>>>(partials, nsplit, pq, out);
}

void launch_select_chol(const double* G, int p, int ldg, double tau, double* W, double* R, int* kept, int* nkept,
                        int* flag, cudaStream_t s) {
    k_select_chol<<<1, 1024, 0, s>>>(G, p, ldg, tau, W, R, kept, nkept, flag);
}

void launch_tri_inverse(const double* R, int k, int ldr, double* Rinv, cudaStream_t s) {
    k_tri_inverse<<<(k + 127) / 128, 128, 0, s>>>(R, k, ldr, Rinv);
}

void launch_gather_times_upper(const double* T, int ldt, const int* kept, int k, const double* Rinv, int ldr,
                               double* Q, int ldq, long long N, cudaStream_t s) {
    size_t smem = GU_NB * k * sizeof(double);
    cudaFuncSetAttribute(k_gather_upper, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_gather_upper<<<(unsigned)((N + GU_NB - 1) / GU_NB), 256, smem, s>>>(T, ldt, kept, k, Rinv, ldr, Q, ldq, N);
}

void launch_apply_columns(const Op<double>& op, const double* Q, int ldq, int k, double* W, int ldw,
                          cudaStream_t s) {
    k_apply_columns<<<4 * 152, 256, 0, s>>>(op, Q, ldq, k, W, ldw);
}

void launch_gauss_jordan(const double* C, int ldc, int k, double2* Ainv, double2* work, int* flag,
                         cudaStream_t s) {
    k_gauss_jordan<<<1, 1024, 0, s>>>(C, ldc, k, Ainv, work, flag);
}

int restrict_blocks(long long N) {
    long long b = (N + RS_TILE - 1) / RS_TILE;
    return (int)(b < 2 * 152 ? (b < 1 ? 1 : b) : 2 * 152);
}

void launch_coarse_apply(const double2* partials, int nblk, int k, const double2* Ainv, int conj, double2* y,
                         double2* cbuf, cudaStream_t s) {
    // two small launches spread over k SMs (FP64 is 2 FMA/clk per SM: one CTA would serialise)
    k_coarse_reduce<<<k, 64, 0, s>>>(partials, nblk, k, cbuf);
    k_coarse_gemv<<<k, 64, 0, s>>>(Ainv, k, conj, cbuf, y);
}


int project_blocks(long long N) {
    long long b = (N + PJ_TILE - 1) / PJ_TILE;
    return (int)(b < 2 * 152 ? (b < 1 ? 1 : b) : 2 * 152);
}

void launch_project_df(const float2* Q, long long ld, int k, const double2* r, long long N, double2* partials,
                       int nblk, cudaStream_t s) {
    long long rows = (N + nblk - 1) / nblk;
    const int kpw = (k + 15) / 16;
#define PJ_CASE(K) k_project_df<K, false><<<nblk, PJ_T, 0, s>>>(Q, ld, k, r, N, partials, rows)
    if (kpw <= 1) PJ_CASE(1);
    else if (kpw <= 2) PJ_CASE(2);
    else if (kpw <= 4) PJ_CASE(4);
    else if (kpw <= 8) PJ_CASE(8);
    else PJ_CASE(16);
#undef PJ_CASE
}

void launch_prolong_df(const float2* Q, long long ld, int k, const double2* y, double2* z, long long N,
                       cudaStream_t s) {
    long long b = (N + 255) / 256;
    k_prolong_df<false><<<(unsigned)(b < 8 * 152 ? b : 8 * 152), 256, 0, s>>>(Q, ld, k, y, z, nullptr, nullptr, N);
}

void launch_prolong_df_base(const float2* Q, long long ld, int k, const double2* y, const float4* base, double2* z,
                            float4* zdf, long long N, cudaStream_t s) {
    long long b = (N + 255) / 256;
    k_prolong_df<true><<<(unsigned)(b < 8 * 152 ? b : 8 * 152), 256, 0, s>>>(Q, ld, k, y, z, base, zdf, N);
}

void launch_project_df_split(const float2* Q, long long ld, int k, const float4* r, long long N, double2* partials,
                             int nblk, cudaStream_t s) {
    long long rows = (N + nblk - 1) / nblk;
    const int kpw = (k + 15) / 16;
#define PJ_CASE(K) k_project_df<K, true><<<nblk, PJ_T, 0, s>>>(Q, ld, k, r, N, partials, rows)
    if (kpw <= 1) PJ_CASE(1);
    else if (kpw <= 2) PJ_CASE(2);
    else if (kpw <= 4) PJ_CASE(4);
    else if (kpw <= 8) PJ_CASE(8);
    else PJ_CASE(16);
#undef PJ_CASE
}

void launch_red_rows(const float2* Q, long long ldq, int k, long long N, int n, float2* Qr, long long ldr,
                     cudaStream_t s) {
    k_red_rows<<<4 * 152, 256, 0, s>>>(Q, ldq, k, N, n, Qr, ldr);
}

void launch_split_basis(double* A, int ld, int k, float2* B, long long ldb, long long N, cudaStream_t s) {
    dim3 g((unsigned)((N + 31) / 32), (k + 31) / 32);
    k_split_basis<<<g, dim3(32, 8), 0, s>>>(A, ld, k, B, ldb, N);
}

void launch_cm_pair_to_rm(const float2* B, long long ldb, int k, double* A, long long N, cudaStream_t s) {
    dim3 g((unsigned)((N + 31) / 32), (k + 31) / 32);
    k_cm_pair_to_rm<<<g, dim3(32, 8), 0, s>>>(B, ldb, k, A, N);
}

void launch_rm_to_cm_f32(const double* A, int ld, int p, float* B, long long N, cudaStream_t s) {
    dim3 g((unsigned)((N + 31) / 32), (p + 31) / 32);
    k_rm_to_cm_f32<<<g, dim3(32, 8), 0, s>>>(A, ld, p, B, N);
}

void launch_nl_pack(const double2* r, const double* s2, float* x, long long N, cudaStream_t s) {
    long long b = (N + 255) / 256;
    k_nl_pack<<<(unsigned)(b < 8 * 152 ? b : 8 * 152), 256, 0, s>>>(r, s2, x, N);
}

void launch_nl_prolong(const float* T, int p, const float* b, const double* s2, double2* z, long long N,
                       cudaStream_t s) {
    long long nb = (N + 255) / 256;
    k_nl_prolong<<<(unsigned)(nb < 8 * 152 ? nb : 8 * 152), 256, 0, s>>>(T, p, b, s2, z, N);
}

void launch_round_bf16(double* A, int ld, int k, long long N, cudaStream_t s) {
    k_round_bf16<<<4 * 152, 256, 0, s>>>(A, ld, k, N);
}

void launch_rm_to_cm_bf16(const double* A, int ld, int k, void* B, long long ldb, long long N, cudaStream_t s) {
    dim3 g((unsigned)((N + 31) / 32), (k + 31) / 32);
    k_rm_to_cm_bf16<<<g, dim3(32, 8), 0, s>>>(A, ld, k, static_cast<__nv_bfloat16*>(B), ldb, N);
}

void launch_red_rows_bf16(const void* Q, long long ldq, int k, long long N, int n, void* Qr, long long ldr,
                          cudaStream_t s) {
    k_red_rows_bf16<<<4 * 152, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(Q), ldq, k, N, n,
                                            static_cast<__nv_bfloat16*>(Qr), ldr);
}

int restrict32_red_blocks(long long N) {
    const long long M = (N + 1) / 2;
    const long long wtiles = ((M + RR_ROWS - 1) / RR_ROWS + 31) / 32;
    const long long b = (wtiles + RR_T / 32 - 1) / (RR_T / 32);
    return (int)(b < 4 * 152 ? (b < 1 ? 1 : b) : 4 * 152);
}

int launch_restrict32_red(const Op<float>& op, const void* Qr, long long ldr, int k, const float2* v,
                          const float2* z, int conj, float2* partials, cudaStream_t s) {
    const int nb = restrict32_red_blocks(op.N);
    k_restrict32_red<<<nb, RR_T, 0, s>>>(op, static_cast<const __nv_bfloat16*>(Qr), ldr, k, v, z, conj, partials,
                                         (op.N + 1) / 2);
    return nb;
}

int restrict32_rr_ranges(long long N) {
    const long long M = (N + 1) / 2;
    return (int)std::max<long long>(1, (M + RQ_RANGE - 1) / RQ_RANGE);
}

int launch_restrict32_rr(const void* Qr, long long ldr, int k, const float2* r_red, long long M, float2* partials,
                         long long N, cudaStream_t s) {
    const int S = restrict32_rr_ranges(N);
    const dim3 g((S + 7) / 8, (k + RQ_COLS - 1) / RQ_COLS);
    k_restrict32_rr<<<g, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(Qr), ldr, k, r_red, M, partials, S);
    return S;
}

void launch_restrict32(const Op<float>& op, const void* Qv, long long ldq, int k, const float2* v, const float2* z,
                       int conj, float2* partials, int nblk, cudaStream_t s) {
    const __nv_bfloat16* Q = static_cast<const __nv_bfloat16*>(Qv);
    long long rows = (op.N + nblk - 1) / nblk;
    const int kpw = (k + 7) / 8;
#define RS_CASE(K) k_restrict32<K><<<nblk, RS_T, 0, s>>>(op, Q, ldq, k, v, z, conj, partials, rows)
    if (kpw <= 1) RS_CASE(1);
    else if (kpw <= 2) RS_CASE(2);
    else if (kpw <= 4) RS_CASE(4);
    else if (kpw <= 8) RS_CASE(8);
    else if (kpw <= 16) RS_CASE(16);
    else RS_CASE(32);
#undef RS_CASE
}

void launch_coarse_apply32(const float2* partials, int nblk, int k, const double2* Ainv, int conj, float2* y,
                           double2* cbuf, cudaStream_t s) {
    k_coarse32_reduce<<<k, 256, 0, s>>>(partials, nblk, k, cbuf);
    k_coarse32_gemv<<<k, 64, 0, s>>>(Ainv, k, conj, cbuf, y);
}

void launch_prolong32(const void* Q, long long ldq, int k, const float2* y, float2* z, long long N, cudaStream_t s) {
    const __nv_bfloat16* Qb = static_cast<const __nv_bfloat16*>(Q);
    if ((reinterpret_cast<uintptr_t>(z) & 15u) == 0 && (reinterpret_cast<uintptr_t>(Q) & 15u) == 0 && ldq % 8 == 0) {
        const long long b = ((N + 7) / 8 + 255) / 256;
        k_prolong32v<<<(unsigned)(b < 8 * 152 ? b : 8 * 152), 256, 0, s>>>(Qb, ldq, k, y, z, N);
        return;
    }
    long long b = (N + 255) / 256;
    k_prolong32<<<(unsigned)(b < 8 * 152 ? b : 8 * 152), 256, 0, s>>>(Qb, ldq, k, y, z, N);
}

}  // namespace helm
