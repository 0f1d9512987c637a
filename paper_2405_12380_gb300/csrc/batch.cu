// Batched DeepONet-FGMRES: many independent problems of different sizes solved
// together, one launch per phase over all of them.
//
// Vectors of all problems are packed one after another (problem b occupies
// [off_b, off_b + N_b)).  The work of a phase is a queue of tiles of TILE
// consecutive nodes of one problem; the kernels are persistent (a fixed grid
// walks the queue) and read the tile's problem from a device table.  Per-problem
// reductions are segmented: one partial per tile, summed in a fixed order per
// problem.  FGMRES runs in lockstep: every active problem takes Arnoldi step j
// at the same time, problems that converge (or hit maxit) drop out through an
// active mask, and each restarts with its own Krylov dimension.  Each Arnoldi step
// (about twenty kernels and two status copies) is captured once per solve as a
// CUDA graph on a private stream and replayed; the host reads the status between
// steps to update the active mask.
//
// Precision (the mixed form): complex64 hybrid cycle (damped Jacobi + trunk-basis
// correction with each problem's BF16 basis) and complex64 Arnoldi matvec inside
// an FP64 FGMRES (V, CGS2, Hessenberg, Givens, true residual in FP64).
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "bicg.cuh"
#include "helm_internal.cuh"

using namespace helm;

namespace {

constexpr int BT = 256;                 // threads per block
constexpr int kMaxLayer = kMaxLayerCells + 1;
// per-problem FP32 table block: Im k^2 (kTabPad floats) then 1/diag (kMaxLayer float2);
// kTabPad is even so that the float2 part is 8-byte aligned
constexpr int kTabPad = kMaxLayer + (kMaxLayer & 1);
constexpr int kTabF = kTabPad + 2 * kMaxLayer;

struct BProb {
    int dim, n, L, k;
    long long N, off;                   // nodes, offset in packed vectors
    int tile0, ntiles;                  // tiles of this problem in the queue
    double hinv2, dre;
    float hinv2f, dref;
    const uint8_t* mask;
    const uint8_t* lidx;
    const double* im;                   // Im k^2 by layer index (device, kMaxLayer)
    const float* imf;
    const float2* invdf;                // 1/diag by layer index, complex64 (device, kMaxLayer)
    const __nv_bfloat16* Qbf;           // k columns of stride ldq
    long long ldq;
    const double2* Ainv;                // k x k
    const double2* k2;                  // optional field (FP64) / k2f (FP32) and inverse diagonal
    const float2* k2f;
    const float2* invd_field;
};

struct Tile {
    int prob;
    int pad;
    long long first;                    // first node (local index)
};

__device__ __forceinline__ void node_ijk(const BProb& P, long long l, int& i, int& j, int& k) {
    const int li = (int)l;
    i = li % P.n;
    const int t = li / P.n;
    j = t % P.n;
    k = t / P.n;
}

// ------------------------------------------------------------- stencil pieces
__device__ __forceinline__ float2 b_nbr_sum32(const BProb& P, const float2* __restrict__ x, long long l) {
    const long long sy = P.n, sz = (long long)P.n * P.n;
    float2 s = make_float2(0.f, 0.f);
    const uint8_t* mk = P.mask;
    if (!mk[l - 1]) s = cadd(s, x[l - 1]);
    if (!mk[l + 1]) s = cadd(s, x[l + 1]);
    if (!mk[l - sy]) s = cadd(s, x[l - sy]);
    if (!mk[l + sy]) s = cadd(s, x[l + sy]);
    if (P.dim == 3) {
        if (!mk[l - sz]) s = cadd(s, x[l - sz]);
        if (!mk[l + sz]) s = cadd(s, x[l + sz]);
    }
    return s;
}

__device__ __forceinline__ float2 b_diag32(const BProb& P, long long l) {
    if (P.k2f) {
        float2 d = P.k2f[l];
        d.x -= 2.0f * P.dim * P.hinv2f;
        return d;
    }
    return make_float2(P.dref, P.imf[P.lidx[l]]);
}

__device__ __forceinline__ float2 b_invd32(const BProb& P, long long l) {
    return P.invd_field ? P.invd_field[l] : P.invdf[P.lidx[l]];
}

// y32 = A32 x32 (complex64), per tile
__global__ void __launch_bounds__(BT) kb_apply32(const BProb* __restrict__ probs, const Tile* __restrict__ tiles,
                                                 int ntiles, int tile_rows, const float2* __restrict__ x,
                                                 float2* __restrict__ y, const int* __restrict__ active) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        if (!active[T.prob]) continue;
        const BProb& P = probs[T.prob];
        const float2* xb = x + P.off;
        float2* yb = y + P.off;
        for (int r = threadIdx.x; r < tile_rows; r += BT) {
            const long long l = T.first + r;
            if (l >= P.N) break;
            const float2 xc = xb[l];
            float2 out;
            if (P.mask[l]) {
                out = xc;
            } else {
                const float2 s = b_nbr_sum32(P, xb, l);
                const float2 d = b_diag32(P, l);
                out.x = P.hinv2f * s.x + (d.x * xc.x - d.y * xc.y);
                out.y = P.hinv2f * s.y + (d.x * xc.y + d.y * xc.x);
            }
            yb[l] = out;
        }
    }
}

// damped Jacobi sweep in complex64 on A z = v: zout = (1-w) zin + w D^-1 (v - h^-2 sum nbrs);
// zin == nullptr: the sweep from zero (zout = w D^-1 v)
__global__ void __launch_bounds__(BT) kb_jacobi32(const BProb* __restrict__ probs, const Tile* __restrict__ tiles,
                                                  int ntiles, int tile_rows, float omega, const float2* __restrict__ v,
                                                  const float2* __restrict__ zin, float2* __restrict__ zout,
                                                  const int* __restrict__ active) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        if (!active[T.prob]) continue;
        const BProb& P = probs[T.prob];
        const float2* vb = v + P.off;
        const float2* zb = zin ? zin + P.off : nullptr;
        float2* ob = zout + P.off;
        for (int r = threadIdx.x; r < tile_rows; r += BT) {
            const long long l = T.first + r;
            if (l >= P.N) break;
            const float2 fl = vb[l];
            float2 out;
            if (P.mask[l]) {
                out = zb ? cadd(zb[l], cscale(omega, csub(fl, zb[l]))) : cscale(omega, fl);
            } else {
                const float2 id = b_invd32(P, l);
                if (!zb) {
                    out = cscale(omega, cmul(id, fl));
                } else {
                    const float2 s = b_nbr_sum32(P, zb, l);
                    const float2 g = make_float2(fl.x - P.hinv2f * s.x, fl.y - P.hinv2f * s.y);
                    const float2 tt = cmul(id, g);
                    out = make_float2((1.f - omega) * zb[l].x + omega * tt.x, (1.f - omega) * zb[l].y + omega * tt.y);
                }
            }
            ob[l] = out;
        }
    }
}

// red-black Gauss-Seidel half-sweep in complex64, in place: nodes of colour c get
// D^-1 (v - h^-2 sum of fluid neighbours) (masked: v); xzero: z starts at zero
__global__ void __launch_bounds__(BT) kb_rbgs32(const BProb* __restrict__ probs, const Tile* __restrict__ tiles,
                                                int ntiles, int tile_rows, int colour, int xzero,
                                                const float2* __restrict__ v, float2* __restrict__ z,
                                                const int* __restrict__ active) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        if (!active[T.prob]) continue;
        const BProb& P = probs[T.prob];
        const float2* vb = v + P.off;
        float2* zb = z + P.off;
        for (int r = threadIdx.x; r < tile_rows; r += BT) {
            const long long l = T.first + r;
            if (l >= P.N) break;
            int i, j, k;
            node_ijk(P, l, i, j, k);
            if (((i + j + (P.dim == 3 ? k : 0)) & 1) != colour) {
                if (xzero) zb[l] = make_float2(0.f, 0.f);
                continue;
            }
            const float2 fl = vb[l];
            float2 out;
            if (P.mask[l]) {
                out = fl;
            } else {
                const float2 id = b_invd32(P, l);
                if (xzero) {
                    out = cmul(id, fl);
                } else {
                    const float2 s = b_nbr_sum32(P, zb, l);
                    out = cmul(id, make_float2(fl.x - P.hinv2f * s.x, fl.y - P.hinv2f * s.y));
                }
            }
            zb[l] = out;
        }
    }
}

// r32 = v32 - A32 z32
__global__ void __launch_bounds__(BT) kb_resid32(const BProb* __restrict__ probs, const Tile* __restrict__ tiles,
                                                 int ntiles, int tile_rows, const float2* __restrict__ v,
                                                 const float2* __restrict__ z, float2* __restrict__ r,
                                                 const int* __restrict__ active) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        if (!active[T.prob]) continue;
        const BProb& P = probs[T.prob];
        const float2* zb = z + P.off;
        for (int rr = threadIdx.x; rr < tile_rows; rr += BT) {
            const long long l = T.first + rr;
            if (l >= P.N) break;
            const float2 zc = zb[l];
            float2 az;
            if (P.mask[l]) {
                az = zc;
            } else {
                const float2 s = b_nbr_sum32(P, zb, l);
                const float2 d = b_diag32(P, l);
                az.x = P.hinv2f * s.x + (d.x * zc.x - d.y * zc.y);
                az.y = P.hinv2f * s.y + (d.x * zc.y + d.y * zc.x);
            }
            r[P.off + l] = csub(v[P.off + l], az);
        }
    }
}

// FP64 residual r = f - A x with per-tile ||r||^2 partials (true residual)
__global__ void __launch_bounds__(BT) kb_resid64(const BProb* __restrict__ probs, const Tile* __restrict__ tiles,
                                                 int ntiles, int tile_rows, const double2* __restrict__ f,
                                                 const double2* __restrict__ x, double2* __restrict__ r,
                                                 double* __restrict__ partials, const int* __restrict__ active) {
    __shared__ double red[BT / 32];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        const BProb& P = probs[T.prob];
        double acc = 0;
        if (active[T.prob]) {
            const double2* xb = x + P.off;
            const long long sy = P.n, sz = (long long)P.n * P.n;
            for (int rr = threadIdx.x; rr < tile_rows; rr += BT) {
                const long long l = T.first + rr;
                if (l >= P.N) break;
                const double2 xc = xb[l];
                double2 ax;
                if (P.mask[l]) {
                    ax = xc;
                } else {
                    double2 s = make_double2(0, 0);
                    const uint8_t* mk = P.mask;
                    if (!mk[l - 1]) s = cadd(s, xb[l - 1]);
                    if (!mk[l + 1]) s = cadd(s, xb[l + 1]);
                    if (!mk[l - sy]) s = cadd(s, xb[l - sy]);
                    if (!mk[l + sy]) s = cadd(s, xb[l + sy]);
                    if (P.dim == 3) {
                        if (!mk[l - sz]) s = cadd(s, xb[l - sz]);
                        if (!mk[l + sz]) s = cadd(s, xb[l + sz]);
                    }
                    double2 d;
                    if (P.k2) {
                        d = P.k2[l];
                        d.x -= 2.0 * P.dim * P.hinv2;
                    } else {
                        d = make_double2(P.dre, P.im[P.lidx[l]]);
                    }
                    ax.x = P.hinv2 * s.x + (d.x * xc.x - d.y * xc.y);
                    ax.y = P.hinv2 * s.y + (d.x * xc.y + d.y * xc.x);
                }
                const double2 q = csub(f[P.off + l], ax);
                r[P.off + l] = q;
                acc += q.x * q.x + q.y * q.y;
            }
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0;
            for (int w = 0; w < BT / 32; ++w) s += red[w];
            partials[t] = s;
        }
    }
}

// ---------------------------------------------------- trunk-basis correction
// partials[t][j] = sum over the tile of Qbf_j[l] r_l (complex64, FP32 accumulation)
__global__ void __launch_bounds__(BT) kb_project32(const BProb* __restrict__ probs, const Tile* __restrict__ tiles,
                                                   int ntiles, int tile_rows, const float2* __restrict__ r,
                                                   float2* __restrict__ partials, int kmax,
                                                   const int* __restrict__ active) {
    extern __shared__ float2 rs[];      // tile_rows
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        if (!active[T.prob]) continue;
        const BProb& P = probs[T.prob];
        const int rows = (int)min((long long)tile_rows, P.N - T.first);
        __syncthreads();
        for (int q = threadIdx.x; q < rows; q += BT) rs[q] = P.mask[T.first + q] ? make_float2(0.f, 0.f) : r[P.off + T.first + q];
        __syncthreads();
        for (int j = warp; j < P.k; j += BT / 32) {
            const __nv_bfloat16* Qj = P.Qbf + (long long)j * P.ldq + T.first;
            float ax = 0.f, ay = 0.f;
            for (int q = lane; q < rows; q += 32) {
                const float qv = __bfloat162float(Qj[q]);
                ax = fmaf(qv, rs[q].x, ax);
                ay = fmaf(qv, rs[q].y, ay);
            }
            for (int o = 16; o > 0; o >>= 1) {
                ax += __shfl_xor_sync(0xffffffffu, ax, o);
                ay += __shfl_xor_sync(0xffffffffu, ay, o);
            }
            if (lane == 0) partials[(long long)t * kmax + j] = make_float2(ax, ay);
        }
    }
}

// per problem: c = sum of its tiles' partials (fixed order, FP64), y = A_c^-1 c
__global__ void kb_coarse(const BProb* __restrict__ probs, int nprob, const float2* __restrict__ partials, int kmax,
                          float2* __restrict__ y, const int* __restrict__ active) {
    __shared__ double2 c[kMaxP];
    const int b = blockIdx.x;
    if (b >= nprob || !active[b]) return;
    const BProb& P = probs[b];
    for (int j = threadIdx.x; j < P.k; j += blockDim.x) {
        double sx = 0, sy = 0;
        for (int t = 0; t < P.ntiles; ++t) {
            const float2 q = partials[(long long)(P.tile0 + t) * kmax + j];
            sx += q.x;
            sy += q.y;
        }
        c[j] = make_double2(sx, sy);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < P.k; i += blockDim.x) {
        double sx = 0, sy = 0;
        for (int j = 0; j < P.k; ++j) {
            const double2 a = P.Ainv[(long long)i * P.k + j];
            sx += a.x * c[j].x - a.y * c[j].y;
            sy += a.x * c[j].y + a.y * c[j].x;
        }
        y[(long long)b * kmax + i] = make_float2((float)sx, (float)sy);
    }
}

// z += Q y per tile
__global__ void __launch_bounds__(BT) kb_prolong32(const BProb* __restrict__ probs, const Tile* __restrict__ tiles,
                                                   int ntiles, int tile_rows, const float2* __restrict__ y, int kmax,
                                                   float2* __restrict__ z, const int* __restrict__ active) {
    __shared__ float2 ys[kMaxP];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        if (!active[T.prob]) continue;
        const BProb& P = probs[T.prob];
        __syncthreads();
        for (int j = threadIdx.x; j < P.k; j += BT) ys[j] = y[(long long)T.prob * kmax + j];
        __syncthreads();
        for (int rr = threadIdx.x; rr < tile_rows; rr += BT) {
            const long long l = T.first + rr;
            if (l >= P.N) break;
            float sx = 0.f, sy = 0.f;
            for (int j = 0; j < P.k; ++j) {
                const float qv = __bfloat162float(P.Qbf[(long long)j * P.ldq + l]);
                sx = fmaf(qv, ys[j].x, sx);
                sy = fmaf(qv, ys[j].y, sy);
            }
            float2 zz = z[P.off + l];
            z[P.off + l] = make_float2(zz.x + sx, zz.y + sy);
        }
    }
}

// ---------------------------------------------------------------- FGMRES
// partials[t][i] = sum over the tile of conj(V_i) w, i < nv (V: nv packed vectors)
__global__ void __launch_bounds__(BT) kb_mdot(const BProb* __restrict__ probs, const Tile* __restrict__ tiles,
                                              int ntiles, int tile_rows, const double2* __restrict__ V, long long NT,
                                              int nv, const double2* __restrict__ w, double2* __restrict__ partials,
                                              const int* __restrict__ active) {
    extern __shared__ double2 ws[];      // tile_rows
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        if (!active[T.prob]) continue;
        const BProb& P = probs[T.prob];
        const int rows = (int)min((long long)tile_rows, P.N - T.first);
        const long long base = P.off + T.first;
        __syncthreads();
        for (int q = threadIdx.x; q < rows; q += BT) ws[q] = w[base + q];
        __syncthreads();
        for (int i = warp; i < nv; i += BT / 32) {
            const double2* Vi = V + (long long)i * NT + base;
            double ax = 0, ay = 0;
            for (int q = lane; q < rows; q += 32) {
                const double2 u = Vi[q], bq = ws[q];
                ax += u.x * bq.x + u.y * bq.y;
                ay += u.x * bq.y - u.y * bq.x;
            }
            for (int o = 16; o > 0; o >>= 1) {
                ax += __shfl_xor_sync(0xffffffffu, ax, o);
                ay += __shfl_xor_sync(0xffffffffu, ay, o);
            }
            if (lane == 0) partials[(long long)t * (kMaxRestart + 1) + i] = make_double2(ax, ay);
        }
    }
}

// out[b][i] (+)= sum over problem b's tiles of partials[t][i]; copy[b][i] = the plain sum
__global__ void kb_mdot_fin(const BProb* __restrict__ probs, int nprob, const double2* __restrict__ partials, int nv,
                            double2* __restrict__ out, int ldo, int accumulate, double2* __restrict__ copy,
                            const int* __restrict__ active) {
    const int b = blockIdx.x;
    if (b >= nprob || !active[b]) return;
    const BProb& P = probs[b];
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        double sx = 0, sy = 0;
        for (int t = 0; t < P.ntiles; ++t) {
            const double2 q = partials[(long long)(P.tile0 + t) * (kMaxRestart + 1) + i];
            sx += q.x;
            sy += q.y;
        }
        const double2 s = make_double2(sx, sy);
        if (copy) copy[(long long)b * (kMaxRestart + 1) + i] = s;
        double2* o = out + (long long)b * ldo + i;
        *o = accumulate ? cadd(*o, s) : s;
    }
}

// w += sign sum_i V_i coef[b][i] per tile; optional per-tile ||w||^2 partials
__global__ void __launch_bounds__(BT) kb_mupdate(const BProb* __restrict__ probs, const Tile* __restrict__ tiles,
                                                 int ntiles, int tile_rows, const double2* __restrict__ V, long long NT,
                                                 int nv, const double2* __restrict__ coef, int ldc, double sign,
                                                 double2* __restrict__ w, double* __restrict__ partials,
                                                 const int* __restrict__ active) {
    __shared__ double2 c[kMaxRestart + 1];
    __shared__ double red[BT / 32];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        const BProb& P = probs[T.prob];
        double acc = 0;
        const bool act = active[T.prob];
        __syncthreads();
        if (act)
            for (int i = threadIdx.x; i < nv; i += BT) c[i] = cscale(sign, coef[(long long)T.prob * ldc + i]);
        __syncthreads();
        if (act) {
            for (int rr = threadIdx.x; rr < tile_rows; rr += BT) {
                const long long l = T.first + rr;
                if (l >= P.N) break;
                const long long g = P.off + l;
                double2 s = w[g];
                for (int i = 0; i < nv; ++i) {
                    const double2 v = V[(long long)i * NT + g];
                    s.x += c[i].x * v.x - c[i].y * v.y;
                    s.y += c[i].x * v.y + c[i].y * v.x;
                }
                w[g] = s;
                acc += s.x * s.x + s.y * s.y;
            }
        }
        if (partials) {
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
            __syncthreads();
            if (threadIdx.x == 0) {
                double s = 0;
                for (int q = 0; q < BT / 32; ++q) s += red[q];
                partials[t] = s;
            }
        }
    }
}

// x += Z32 y for problem-specific Krylov dimensions kdim[b]
__global__ void __launch_bounds__(BT) kb_update_x(const BProb* __restrict__ probs, const Tile* __restrict__ tiles,
                                                  int ntiles, int tile_rows, const float2* __restrict__ Z, long long NT,
                                                  const double2* __restrict__ y, const int* __restrict__ kdim,
                                                  double2* __restrict__ x) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        const BProb& P = probs[T.prob];
        const int kd = kdim[T.prob];
        if (kd == 0) continue;
        for (int rr = threadIdx.x; rr < tile_rows; rr += BT) {
            const long long l = T.first + rr;
            if (l >= P.N) break;
            const long long g = P.off + l;
            double2 s = x[g];
            for (int i = 0; i < kd; ++i) {
                const float2 zf = Z[(long long)i * NT + g];
                const double2 c = y[(long long)T.prob * (kMaxRestart + 1) + i];
                s.x += c.x * zf.x - c.y * zf.y;
                s.y += c.x * zf.y + c.y * zf.x;
            }
            x[g] = s;
        }
    }
}

// per problem sum of tile partials (fixed order) into out[b]
__global__ void kb_seg_sum(const BProb* __restrict__ probs, int nprob, const double* __restrict__ partials,
                           double* __restrict__ out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nprob) return;
    const BProb& P = probs[b];
    double s = 0;
    for (int t = 0; t < P.ntiles; ++t) s += partials[P.tile0 + t];
    out[b] = s;
}

// v = w / sqrt(norm2[b]) per tile (active problems with nonzero norm)
__global__ void __launch_bounds__(BT) kb_scale(const BProb* __restrict__ probs, const Tile* __restrict__ tiles,
                                               int ntiles, int tile_rows, const double2* __restrict__ w,
                                               double2* __restrict__ v, const double* __restrict__ norm2,
                                               const int* __restrict__ active) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        if (!active[T.prob]) continue;
        const BProb& P = probs[T.prob];
        const double nn = sqrt(norm2[T.prob]);
        if (nn == 0) continue;
        const double inv = 1.0 / nn;
        for (int rr = threadIdx.x; rr < tile_rows; rr += BT) {
            const long long l = T.first + rr;
            if (l >= P.N) break;
            v[P.off + l] = cscale(inv, w[P.off + l]);
        }
    }
}

// Givens step j for every active problem (one thread per problem)
__global__ void kb_givens(int nprob, double2* __restrict__ H, int ldh, int m, int j, double* __restrict__ cs,
                          double2* __restrict__ sn, double2* __restrict__ g, const double* __restrict__ wn2,
                          double* __restrict__ est, const int* __restrict__ active) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nprob || !active[b]) return;
    double2* col = H + (long long)b * ldh * m + (long long)j * ldh;
    double* csb = cs + (long long)b * m;
    double2* snb = sn + (long long)b * m;
    double2* gb = g + (long long)b * (m + 1);
    const double hn = sqrt(wn2[b]);
    col[j + 1] = make_double2(hn, 0);
    for (int i = 0; i < j; ++i) {
        const double2 a = col[i], bb = col[i + 1];
        col[i] = cadd(cscale(csb[i], a), cmul(snb[i], bb));
        col[i + 1] = csub(cscale(csb[i], bb), cmulc(snb[i], a));
    }
    const double2 a = col[j], bb = col[j + 1];
    double c;
    double2 s, r;
    const double ab = hypot(a.x, a.y), bbn = hypot(bb.x, bb.y);
    if (bbn == 0) {
        c = 1; s = make_double2(0, 0); r = a;
    } else if (ab == 0) {
        c = 0; s = make_double2(bb.x / bbn, -bb.y / bbn); r = make_double2(bbn, 0);
    } else {
        const double tt = sqrt(ab * ab + bbn * bbn);
        const double2 ph = make_double2(a.x / ab, a.y / ab);
        c = ab / tt;
        s = cscale(1.0 / tt, cmul(ph, make_double2(bb.x, -bb.y)));
        r = cscale(tt, ph);
    }
    csb[j] = c;
    snb[j] = s;
    col[j] = r;
    col[j + 1] = make_double2(0, 0);
    const double2 gj = gb[j];
    gb[j + 1] = cscale(-1.0, cmulc(s, gj));
    gb[j] = cscale(c, gj);
    est[b] = hypot(gb[j + 1].x, gb[j + 1].y);
}

// back substitution H y = g per problem with its Krylov dimension
__global__ void kb_hsolve(int nprob, const double2* __restrict__ H, int ldh, int m, const double2* __restrict__ g,
                          const int* __restrict__ kdim, double2* __restrict__ y) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nprob) return;
    const int k = kdim[b];
    const double2* Hb = H + (long long)b * ldh * m;
    const double2* gb = g + (long long)b * (m + 1);
    double2* yb = y + (long long)b * (kMaxRestart + 1);
    for (int i = k - 1; i >= 0; --i) {
        double2 s = gb[i];
        for (int q = i + 1; q < k; ++q) s = csub(s, cmul(Hb[(long long)q * ldh + i], yb[q]));
        yb[i] = cdiv(s, Hb[(long long)i * ldh + i]);
    }
}

// g[b] = (sqrt(beta2[b]), 0, ...), restart state
__global__ void kb_init_g(int nprob, int m, double2* __restrict__ g, const double* __restrict__ beta2,
                          const int* __restrict__ active) {
    const int b = blockIdx.x;
    if (b >= nprob || !active[b]) return;
    for (int i = threadIdx.x; i <= m; i += blockDim.x)
        g[(long long)b * (m + 1) + i] = make_double2(i == 0 ? sqrt(beta2[b]) : 0.0, 0);
}

// ------------------------------------------------- batched complex64 BiCGStab
// The BiCGStab of the single-problem mixed handles (complex64 vectors, operator
// and hybrid cycle; FP64 iterate with reliable updates) for all problems at once.
// Per-problem scalars are the slots of helm_internal.cuh at sc + b * S_NSLOTS; the
// control state of a problem is a BState; every decision (reliable update,
// convergence, restart after a breakdown, retirement) is taken on the device by
// the per-problem finishing kernels, which also keep the active mask, so one
// captured iteration is replayed without the host.
struct BState {
    double tol_abs;     // tol ||f_b||
    double bnorm;       // ||f_b||
    double maxrr;       // largest recursive ||r|| since the last reliable update
    double rel_res;     // last true relative residual
    int iters, maxit;
    double last_true;   // true ||r|| at the last reliable update
    int ru;             // 0; 1 reliable update; 2 update and restart (breakdown); 3 final update (maxit);
                        // 4 reset: the increment is dropped and the method restarts (runaway growth)
    int status;         // HELM_NOT_CONVERGED while running
    int since_start;    // iterations since the last (re)start
    int restarts;
};

// recipes of kb32_fin
enum { BF_ALPHA = 0, BF_SNORM, BF_OMEGA, BF_XR, BF_RU, BF_INIT };
// growth of the recursive residual over the last true one that counts as a runaway
constexpr double kRunaway = 1e3;

__device__ __forceinline__ double2* sc_of(double2* sc, int b) { return sc + (long long)b * S_NSLOTS; }
__device__ __forceinline__ bool b_skip(const double2* scb) { return scb[S_STOP].x != 0.0; }

// per tile: the vectors of a BiCGStab phase and its partials (up to 3 doubles per tile)
__device__ __forceinline__ void tile_reduce3(double a0, double a1, double a2, double* part, int t) {
    __shared__ double red[3][BT / 32];
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = a0;
        red[1][threadIdx.x >> 5] = a1;
        red[2][threadIdx.x >> 5] = a2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0, s1 = 0, s2 = 0;
        for (int w = 0; w < BT / 32; ++w) {
            s0 += red[0][w];
            s1 += red[1][w];
            s2 += red[2][w];
        }
        part[3 * (long long)t] = s0;
        part[3 * (long long)t + 1] = s1;
        part[3 * (long long)t + 2] = s2;
    }
}

// p = r + beta (p - omega v)
__global__ void __launch_bounds__(BT) kb32_p(const BProb* __restrict__ probs, const Tile* __restrict__ tiles, int ntiles,
                                             int tile_rows, const float2* __restrict__ r, const float2* __restrict__ v,
                                             float2* __restrict__ p, const double2* __restrict__ sc,
                                             const int* __restrict__ active) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        const double2* scb = sc + (long long)T.prob * S_NSLOTS;
        if (!active[T.prob] || b_skip(scb)) continue;
        const BProb& P = probs[T.prob];
        const float2 beta = make_float2((float)scb[S_BETA].x, (float)scb[S_BETA].y);
        const float2 om = make_float2((float)scb[S_OMEGA].x, (float)scb[S_OMEGA].y);
        for (int rr = threadIdx.x; rr < tile_rows; rr += BT) {
            const long long l = T.first + rr;
            if (l >= P.N) break;
            const long long g = P.off + l;
            p[g] = cadd(r[g], cmul(beta, csub(p[g], cmul(om, v[g]))));
        }
    }
}

// partials of <a, b> (conj(a) b) per tile
__global__ void __launch_bounds__(BT) kb32_dot(const BProb* __restrict__ probs, const Tile* __restrict__ tiles, int ntiles,
                                               int tile_rows, const float2* __restrict__ a, const float2* __restrict__ b,
                                               double* __restrict__ part, const double2* __restrict__ sc,
                                               const int* __restrict__ active) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        const double2* scb = sc + (long long)T.prob * S_NSLOTS;
        float re = 0.f, im = 0.f;
        if (active[T.prob] && !b_skip(scb)) {
            const BProb& P = probs[T.prob];
            for (int rr = threadIdx.x; rr < tile_rows; rr += BT) {
                const long long l = T.first + rr;
                if (l >= P.N) break;
                const float2 x = a[P.off + l], y = b[P.off + l];
                re = fmaf(x.x, y.x, fmaf(x.y, y.y, re));
                im = fmaf(x.x, y.y, fmaf(-x.y, y.x, im));
            }
        }
        tile_reduce3(re, im, 0.0, part, t);
    }
}

// s = r - alpha v, partials of ||s||^2
__global__ void __launch_bounds__(BT) kb32_s(const BProb* __restrict__ probs, const Tile* __restrict__ tiles, int ntiles,
                                             int tile_rows, const float2* __restrict__ r, const float2* __restrict__ v,
                                             float2* __restrict__ sv, double* __restrict__ part,
                                             const double2* __restrict__ sc, const int* __restrict__ active) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        const double2* scb = sc + (long long)T.prob * S_NSLOTS;
        float acc = 0.f;
        if (active[T.prob] && !b_skip(scb)) {
            const BProb& P = probs[T.prob];
            const float2 al = make_float2((float)scb[S_ALPHA].x, (float)scb[S_ALPHA].y);
            for (int rr = threadIdx.x; rr < tile_rows; rr += BT) {
                const long long l = T.first + rr;
                if (l >= P.N) break;
                const long long g = P.off + l;
                const float2 q = csub(r[g], cmul(al, v[g]));
                sv[g] = q;
                acc = fmaf(q.x, q.x, fmaf(q.y, q.y, acc));
            }
        }
        tile_reduce3(acc, 0.0, 0.0, part, t);
    }
}

// partials of <t, s> and <t, t>
__global__ void __launch_bounds__(BT) kb32_ts(const BProb* __restrict__ probs, const Tile* __restrict__ tiles, int ntiles,
                                              int tile_rows, const float2* __restrict__ tv, const float2* __restrict__ sv,
                                              double* __restrict__ part, const double2* __restrict__ sc,
                                              const int* __restrict__ active) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        const double2* scb = sc + (long long)T.prob * S_NSLOTS;
        float re = 0.f, im = 0.f, tt = 0.f;
        if (active[T.prob] && !b_skip(scb)) {
            const BProb& P = probs[T.prob];
            for (int rr = threadIdx.x; rr < tile_rows; rr += BT) {
                const long long l = T.first + rr;
                if (l >= P.N) break;
                const float2 x = tv[P.off + l], y = sv[P.off + l];
                re = fmaf(x.x, y.x, fmaf(x.y, y.y, re));
                im = fmaf(x.x, y.y, fmaf(-x.y, y.x, im));
                tt = fmaf(x.x, x.x, fmaf(x.y, x.y, tt));
            }
        }
        tile_reduce3(re, im, tt, part, t);
    }
}

// xl += alpha phat + omega shat; r = s - omega t; partials of ||r||^2 and <rhat, r>
__global__ void __launch_bounds__(BT) kb32_xr(const BProb* __restrict__ probs, const Tile* __restrict__ tiles, int ntiles,
                                              int tile_rows, float2* __restrict__ xl, float2* __restrict__ r,
                                              const float2* __restrict__ ph, const float2* __restrict__ sh,
                                              const float2* __restrict__ sv, const float2* __restrict__ tv,
                                              const float2* __restrict__ rh, double* __restrict__ part,
                                              const double2* __restrict__ sc, const int* __restrict__ active) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        const double2* scb = sc + (long long)T.prob * S_NSLOTS;
        float rn = 0.f, re = 0.f, im = 0.f;
        if (active[T.prob] && !b_skip(scb) && scb[S_FLAGS].y != 1.0) {
            const BProb& P = probs[T.prob];
            const float2 al = make_float2((float)scb[S_ALPHA].x, (float)scb[S_ALPHA].y);
            const float2 om = make_float2((float)scb[S_OMEGA].x, (float)scb[S_OMEGA].y);
            for (int rr = threadIdx.x; rr < tile_rows; rr += BT) {
                const long long l = T.first + rr;
                if (l >= P.N) break;
                const long long g = P.off + l;
                xl[g] = cadd(cadd(xl[g], cmul(al, ph[g])), cmul(om, sh[g]));
                const float2 q = csub(sv[g], cmul(om, tv[g]));
                r[g] = q;
                rn = fmaf(q.x, q.x, fmaf(q.y, q.y, rn));
                const float2 h = rh[g];
                re = fmaf(h.x, q.x, fmaf(h.y, q.y, re));
                im = fmaf(h.x, q.y, fmaf(-h.y, q.x, im));
            }
        }
        tile_reduce3(rn, re, im, part, t);
    }
}

// reliable update, first half, for problems with st.ru != 0: x += xl, xl = 0 (a reset,
// ru = 4, drops the increment: xl = 0 with x unchanged)
__global__ void __launch_bounds__(BT) kb32_fold(const BProb* __restrict__ probs, const Tile* __restrict__ tiles, int ntiles,
                                                int tile_rows, double2* __restrict__ x, float2* __restrict__ xl,
                                                const int* __restrict__ ruflag) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        if (!ruflag[T.prob]) continue;
        const BProb& P = probs[T.prob];
        for (int rr = threadIdx.x; rr < tile_rows; rr += BT) {
            const long long l = T.first + rr;
            if (l >= P.N) break;
            const long long g = P.off + l;
            const float2 d = xl[g];
            if (ruflag[T.prob] != 4) x[g] = make_double2(x[g].x + (double)d.x, x[g].y + (double)d.y);
            xl[g] = make_float2(0.f, 0.f);
        }
    }
}

// reliable update, second half: r = complex64(r64) (restart: rhat = r, p = v = 0);
// partials of <rhat, r>
__global__ void __launch_bounds__(BT) kb32_replace(const BProb* __restrict__ probs, const Tile* __restrict__ tiles,
                                                   int ntiles, int tile_rows, const double2* __restrict__ r64,
                                                   float2* __restrict__ r, float2* __restrict__ rh,
                                                   float2* __restrict__ p, float2* __restrict__ v,
                                                   double* __restrict__ part, const int* __restrict__ ruflag) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        const int ru = ruflag[T.prob];
        float re = 0.f, im = 0.f;
        if (ru) {
            const BProb& P = probs[T.prob];
            for (int rr = threadIdx.x; rr < tile_rows; rr += BT) {
                const long long l = T.first + rr;
                if (l >= P.N) break;
                const long long g = P.off + l;
                const float2 q = make_float2((float)r64[g].x, (float)r64[g].y);
                r[g] = q;
                float2 h;
                if (ru == 2 || ru == 4) {
                    rh[g] = q;
                    p[g] = make_float2(0.f, 0.f);
                    v[g] = make_float2(0.f, 0.f);
                    h = q;
                } else {
                    h = rh[g];
                }
                re = fmaf(h.x, q.x, fmaf(h.y, q.y, re));
                im = fmaf(h.x, q.y, fmaf(-h.y, q.x, im));
            }
        }
        tile_reduce3(re, im, 0.0, part, t);
    }
}

// One block per problem: the problem's tile partials summed in a fixed order, then
// the recurrence of `recipe` on its scalars and its control state.  `nrm` holds the
// true ||r||^2 of BF_RU / BF_INIT (from kb_resid64 + kb_seg_sum); ruflag mirrors
// BState.ru for the tile kernels and active the running problems.
__global__ void __launch_bounds__(64) kb32_fin(int recipe, const BProb* __restrict__ probs, int nprob,
                                               const double* __restrict__ part, double2* __restrict__ sc,
                                               BState* __restrict__ st, int* __restrict__ active,
                                               int* __restrict__ ruflag, const double* __restrict__ nrm, double delta) {
    const int b = blockIdx.x;
    if (b >= nprob) return;
    const BProb& P = probs[b];
    __shared__ double red[3][2];
    double a0 = 0, a1 = 0, a2 = 0;
    for (int q = threadIdx.x; q < P.ntiles; q += 64) {
        const long long t = P.tile0 + q;
        a0 += part[3 * t];
        a1 += part[3 * t + 1];
        a2 += part[3 * t + 2];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = a0;
        red[1][threadIdx.x >> 5] = a1;
        red[2][threadIdx.x >> 5] = a2;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double t0 = red[0][0] + red[0][1], t1 = red[1][0] + red[1][1], t2 = red[2][0] + red[2][1];
    double2* scb = sc + (long long)b * S_NSLOTS;
    BState& S = st[b];
    if (recipe == BF_INIT) {
        // initial true residual (x0 given): converged already, or a fresh start
        S.rel_res = S.bnorm > 0 ? sqrt(nrm[b]) / S.bnorm : 0.0;
        if (S.bnorm == 0 || sqrt(nrm[b]) <= S.tol_abs) {
            S.status = HELM_OK;
            active[b] = 0;
        } else {
            scb[S_RHO_OLD] = make_double2(1, 0);
            scb[S_ALPHA] = make_double2(1, 0);
            scb[S_OMEGA] = make_double2(1, 0);
            scb[S_FLAGS] = make_double2(0, 0);
            scb[S_STOP] = make_double2(0, 0);
            bicg_rho_beta(scb, make_double2(t0, t1), 1.0);
            S.maxrr = sqrt(nrm[b]);
            S.last_true = S.maxrr;
            S.since_start = 0;
        }
        ruflag[b] = 0;
        S.ru = 0;
        return;
    }
    if (recipe == BF_RU) {
        if (!S.ru) return;
        const double rt = sqrt(nrm[b]);
        S.rel_res = rt / S.bnorm;
        const int ru = S.ru;
        S.ru = 0;
        ruflag[b] = 0;
        if (rt <= S.tol_abs) {
            S.status = HELM_OK;
            active[b] = 0;
        } else if (!isfinite(rt)) {
            S.status = HELM_DIVERGED;
            active[b] = 0;
        } else if (ru == 3) {
            S.status = HELM_NOT_CONVERGED;
            active[b] = 0;
        } else if (ru == 2 && S.since_start <= 1) {
            S.status = HELM_BREAKDOWN;
            active[b] = 0;
        } else {
            if (ru == 2 || ru == 4) {
                scb[S_RHO_OLD] = make_double2(1, 0);
                scb[S_ALPHA] = make_double2(1, 0);
                scb[S_OMEGA] = make_double2(1, 0);
                S.since_start = 0;
                ++S.restarts;
            }
            scb[S_FLAGS] = make_double2(0, 0);
            scb[S_STOP] = make_double2(0, 0);
            bicg_rho_beta(scb, make_double2(t0, t1), 1.0);
            S.maxrr = rt;
            S.last_true = rt;
        }
        return;
    }
    if (!active[b] || b_skip(scb)) return;
    if (recipe == BF_ALPHA) {
        bicg_alpha(scb, make_double2(t0, t1));
    } else if (recipe == BF_SNORM) {
        bicg_snorm(scb, t0, S.tol_abs);
    } else if (recipe == BF_OMEGA) {
        bicg_omega(scb, make_double2(t0, t1), t2);
    } else {   // BF_XR
        const bool skip = scb[S_FLAGS].y == 1.0;
        if (!skip) {
            bicg_rnorm(scb, t0);
            bicg_rho_beta(scb, make_double2(t1, t2), 3.0);
        }
        ++S.iters;
        ++S.since_start;
        const double rn = sqrt(scb[S_RN2].x);
        const bool brk = scb[S_FLAGS].y != 0.0;
        if (brk || !isfinite(rn) || rn <= S.tol_abs) {
            scb[S_STOP].x = 1.0;
            S.ru = brk ? 2 : (!isfinite(rn) ? 4 : 1);
        } else if (rn > kRunaway * S.last_true) {
            // the complex64 recursion ran away: drop the increment, restart from x
            scb[S_STOP].x = 1.0;
            S.ru = 4;
        } else if (rn < delta * S.maxrr) {
            S.ru = 1;
        } else if (rn > S.maxrr) {
            S.maxrr = rn;
        }
        if (S.iters >= S.maxit && S.ru == 0) S.ru = 3;
        ruflag[b] = S.ru;
    }
}

__global__ void kb_cvt64to32(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < n; l += (long long)gridDim.x * blockDim.x)
        b[l] = make_float2((float)a[l].x, (float)a[l].y);
}
__global__ void kb_cvt32to64(const float2* __restrict__ a, double2* __restrict__ b, long long n) {
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < n; l += (long long)gridDim.x * blockDim.x)
        b[l] = make_double2(a[l].x, a[l].y);
}

}  // namespace

// ===================================================================== batch
struct helm_batch {
    int nprob = 0;
    long long NT = 0;
    int tile_rows = 1024;
    int ntiles = 0;
    int grid = 4 * 152;
    int kmax = 0;
    cudaStream_t stream = nullptr;
    std::vector<helm_handle*> hs;
    std::vector<BProb> hprobs;
    BProb* probs = nullptr;
    Tile* tiles = nullptr;
    double* tables = nullptr;           // per problem: im (kMaxLayer) doubles
    float* tablesf = nullptr;           // per problem: imf (kMaxLayer) + invdf (2 kMaxLayer)
    int* active = nullptr;
    int* kdim = nullptr;
    double2 *f = nullptr, *x = nullptr, *V = nullptr, *w = nullptr;
    float2 *v32 = nullptr, *z32tmp = nullptr, *r32 = nullptr, *Z32 = nullptr, *w32 = nullptr;
    float2 *pp32 = nullptr, *y32 = nullptr;
    double2 *hpart = nullptr, *H = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr, *h2 = nullptr;
    double *cs = nullptr, *tpart = nullptr, *nrm = nullptr, *est = nullptr, *hpin = nullptr;
    int m_alloc = 0;
    // batched complex64 BiCGStab: r, rhat, p, v, s, t, phat, shat, xl (complex64), the
    // FP64 residual, per-problem scalars and control states, tile partials (3 each)
    float2* b32 = nullptr;
    double2* r64 = nullptr;
    double2* bsc = nullptr;
    BState* bst = nullptr;
    BState* hbst = nullptr;             // pinned mirror
    int* ruflag = nullptr;
    double* part3 = nullptr;
    cudaStream_t cstream = nullptr;     // private non-blocking stream of the solves (graph capture)
    cudaEvent_t join = nullptr;
    std::string err;
};

namespace {

template <typename T>
helm_status balloc(helm_batch* B, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return HELM_OK;
    if (cudaMalloc((void**)p, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        B->err = "cudaMalloc failed";
        return HELM_OUT_OF_MEMORY;
    }
    return HELM_OK;
}

template <typename T>
void bfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

helm_status build_tiles(helm_batch* B) {
    std::vector<Tile> tl;
    for (int b = 0; b < B->nprob; ++b) {
        BProb& P = B->hprobs[b];
        P.tile0 = (int)tl.size();
        for (long long f0 = 0; f0 < P.N; f0 += B->tile_rows) tl.push_back(Tile{b, 0, f0});
        P.ntiles = (int)tl.size() - P.tile0;
    }
    B->ntiles = (int)tl.size();
    bfree(B->tiles);
    bfree(B->tpart);
    bfree(B->hpart);
    bfree(B->pp32);
    helm_status st;
    if ((st = balloc(B, &B->tiles, tl.size())) != HELM_OK) return st;
    if ((st = balloc(B, &B->tpart, tl.size())) != HELM_OK) return st;
    if ((st = balloc(B, &B->hpart, tl.size() * (kMaxRestart + 1))) != HELM_OK) return st;
    if ((st = balloc(B, &B->pp32, tl.size() * (size_t)std::max(1, B->kmax))) != HELM_OK) return st;
    cudaMemcpy(B->tiles, tl.data(), tl.size() * sizeof(Tile), cudaMemcpyHostToDevice);
    cudaMemcpy(B->probs, B->hprobs.data(), B->hprobs.size() * sizeof(BProb), cudaMemcpyHostToDevice);
    return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_CUDA_ERROR;
}

helm_status ensure_batch_krylov(helm_batch* B, int m) {
    if (B->m_alloc >= m) return HELM_OK;
    bfree(B->V); bfree(B->Z32); bfree(B->H); bfree(B->sn); bfree(B->g); bfree(B->cs); bfree(B->y); bfree(B->h2);
    helm_status st;
    const int P = B->nprob;
    if ((st = balloc(B, &B->V, (size_t)(m + 1) * B->NT)) != HELM_OK) return st;
    if ((st = balloc(B, &B->Z32, (size_t)m * B->NT)) != HELM_OK) return st;
    if ((st = balloc(B, &B->H, (size_t)P * (m + 1) * m)) != HELM_OK) return st;
    if ((st = balloc(B, &B->sn, (size_t)P * m)) != HELM_OK) return st;
    if ((st = balloc(B, &B->cs, (size_t)P * m)) != HELM_OK) return st;
    if ((st = balloc(B, &B->g, (size_t)P * (m + 1))) != HELM_OK) return st;
    if ((st = balloc(B, &B->y, (size_t)P * (kMaxRestart + 1))) != HELM_OK) return st;
    if ((st = balloc(B, &B->h2, (size_t)P * (kMaxRestart + 1))) != HELM_OK) return st;
    B->m_alloc = m;
    return HELM_OK;
}

// ---------------------------------------------- batched complex64 BiCGStab
constexpr double kBatchReliableDelta = 0.1;

helm_status ensure_batch_b32(helm_batch* B) {
    if (B->b32) return HELM_OK;
    helm_status st;
    const int P = B->nprob;
    if ((st = balloc(B, &B->b32, (size_t)9 * B->NT)) != HELM_OK) return st;
    if ((st = balloc(B, &B->r64, (size_t)B->NT)) != HELM_OK) return st;
    if ((st = balloc(B, &B->bsc, (size_t)P * S_NSLOTS)) != HELM_OK) return st;
    if ((st = balloc(B, &B->bst, (size_t)P)) != HELM_OK) return st;
    if ((st = balloc(B, &B->ruflag, (size_t)P)) != HELM_OK) return st;
    if (cudaMallocHost((void**)&B->hbst, sizeof(BState) * P) != cudaSuccess) return HELM_OUT_OF_MEMORY;
    return HELM_OK;
}

// the hybrid cycle z = M(v) of every active problem (complex64, each problem's BF16 basis)
void batch_precond32(helm_batch* B, const helm_solve_opts* o, const float2* v, float2* z, cudaStream_t s,
                     long long& launches) {
    const int G = B->grid, NTL = B->ntiles, TR = B->tile_rows, P = B->nprob;
    const int nr = o->relax == HELM_RELAX_NONE ? 0 : o->n_r;
    if (nr == 0) {
        cudaMemsetAsync(z, 0, sizeof(float2) * B->NT, s);
    } else if (o->relax == HELM_RBGS) {
        for (int q = 0; q < nr; ++q) {
            kb_rbgs32<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, 0, q == 0, v, z, B->active);
            kb_rbgs32<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, 1, 0, v, z, B->active);
        }
        launches += 2 * nr;
    } else {
        float2* a = (nr % 2 == 1) ? z : B->z32tmp;
        float2* bb = (nr % 2 == 1) ? B->z32tmp : z;
        kb_jacobi32<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, (float)o->omega, v, nullptr, a, B->active);
        for (int q = 1; q < nr; ++q) {
            kb_jacobi32<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, (float)o->omega, v, a, bb, B->active);
            std::swap(a, bb);
        }
        launches += nr;
    }
    if (o->correction == HELM_CORR_TB) {
        const size_t smem32 = (size_t)TR * sizeof(float2);
        kb_resid32<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, v, z, B->r32, B->active);
        kb_project32<<<G, BT, smem32, s>>>(B->probs, B->tiles, NTL, TR, B->r32, B->pp32, B->kmax, B->active);
        kb_coarse<<<P, 128, 0, s>>>(B->probs, P, B->pp32, B->kmax, B->y32, B->active);
        kb_prolong32<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, B->y32, B->kmax, z, B->active);
        launches += 4;
    }
}

// BiCGStab with the hybrid-cycle preconditioner on every problem at once, in lockstep
// (helm_batch_solve with HELM_METHOD_BICGSTAB): one iteration of all problems, with the
// per-problem reliable updates, is one captured CUDA graph; the host replays it and
// polls the problems' states a few iterations behind.
helm_status batch_bicgstab(helm_batch* B, const helm_solve_opts* o, const double* const* f, double* const* x,
                           helm_stats* stats) {
    if (o->conj || o->correction == HELM_CORR_NONLINEAR || (o->relax != HELM_RELAX_NONE && o->relax != HELM_JACOBI &&
                                                            o->relax != HELM_RBGS) || o->maxit < 0 || !(o->tol >= 0))
        return HELM_BAD_ARG;
    helm_status st0 = ensure_batch_b32(B);
    if (st0 != HELM_OK) return st0;
    if (!B->part3 && balloc(B, &B->part3, (size_t)3 * B->ntiles) != HELM_OK) return HELM_OUT_OF_MEMORY;
    if (!B->cstream) {
        if (cudaStreamCreateWithFlags(&B->cstream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->join, cudaEventDisableTiming) != cudaSuccess)
            return HELM_CUDA_ERROR;
    }
    cudaStream_t s = B->cstream;
    if (cudaEventRecord(B->join, B->stream) != cudaSuccess || cudaStreamWaitEvent(s, B->join, 0) != cudaSuccess)
        return HELM_CUDA_ERROR;
    const int P = B->nprob, G = B->grid, NTL = B->ntiles, TR = B->tile_rows;
    const long long NT = B->NT;
    float2 *r = B->b32, *rh = r + NT, *p = rh + NT, *v = p + NT, *sv = v + NT, *tv = sv + NT, *ph = tv + NT,
           *sh = ph + NT, *xl = sh + NT;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    for (int b = 0; b < P; ++b) {
        const BProb& pb = B->hprobs[b];
        cudaMemcpyAsync(B->f + pb.off, f[b], sizeof(double2) * pb.N, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(B->x + pb.off, x[b], sizeof(double2) * pb.N, cudaMemcpyDeviceToDevice, s);
        launch_set_masked(B->x + pb.off, B->f + pb.off, pb.mask, pb.N, s);
    }
    long long launches = 0;
    // ||f_b||: the residual of x = 0
    std::vector<int> ones(P, 1);
    cudaMemcpyAsync(B->active, ones.data(), sizeof(int) * P, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(B->w, 0, sizeof(double2) * NT, s);
    kb_resid64<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, B->f, B->w, B->r64, B->tpart, B->active);
    kb_seg_sum<<<(P + 127) / 128, 128, 0, s>>>(B->probs, P, B->tpart, B->nrm);
    cudaMemcpyAsync(B->hpin, B->nrm, sizeof(double) * P, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return HELM_CUDA_ERROR;
    for (int b = 0; b < P; ++b) {
        BState& S = B->hbst[b];
        S = BState{};
        S.bnorm = std::sqrt(B->hpin[b]);
        S.tol_abs = o->tol * S.bnorm;
        S.maxit = o->maxit;
        S.status = HELM_NOT_CONVERGED;
    }
    cudaMemcpyAsync(B->bst, B->hbst, sizeof(BState) * P, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(B->ruflag, 0, sizeof(int) * P, s);
    cudaMemsetAsync(B->bsc, 0, sizeof(double2) * P * S_NSLOTS, s);
    cudaMemsetAsync(xl, 0, sizeof(float2) * NT, s);
    // initial true residual, a fresh start everywhere (ruflag = 2 for the replace kernel)
    std::vector<int> twos(P, 2);
    kb_resid64<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, B->f, B->x, B->r64, B->tpart, B->active);
    kb_seg_sum<<<(P + 127) / 128, 128, 0, s>>>(B->probs, P, B->tpart, B->nrm);
    cudaMemcpyAsync(B->ruflag, twos.data(), sizeof(int) * P, cudaMemcpyHostToDevice, s);
    kb32_replace<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, B->r64, r, rh, p, v, B->part3, B->ruflag);
    kb32_fin<<<P, 64, 0, s>>>(BF_INIT, B->probs, P, B->part3, B->bsc, B->bst, B->active, B->ruflag, B->nrm,
                              kBatchReliableDelta);
    launches += 6;
    if (cudaStreamSynchronize(s) != cudaSuccess) return HELM_CUDA_ERROR;
    // one iteration of every active problem, with the reliable updates the iteration asks for
    auto enqueue = [&]() {
        kb32_p<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, r, v, p, B->bsc, B->active);
        batch_precond32(B, o, p, ph, s, launches);
        kb_apply32<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, ph, v, B->active);
        kb32_dot<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, rh, v, B->part3, B->bsc, B->active);
        kb32_fin<<<P, 64, 0, s>>>(BF_ALPHA, B->probs, P, B->part3, B->bsc, B->bst, B->active, B->ruflag, B->nrm,
                                  kBatchReliableDelta);
        kb32_s<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, r, v, sv, B->part3, B->bsc, B->active);
        kb32_fin<<<P, 64, 0, s>>>(BF_SNORM, B->probs, P, B->part3, B->bsc, B->bst, B->active, B->ruflag, B->nrm,
                                  kBatchReliableDelta);
        batch_precond32(B, o, sv, sh, s, launches);
        kb_apply32<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, sh, tv, B->active);
        kb32_ts<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, tv, sv, B->part3, B->bsc, B->active);
        kb32_fin<<<P, 64, 0, s>>>(BF_OMEGA, B->probs, P, B->part3, B->bsc, B->bst, B->active, B->ruflag, B->nrm,
                                  kBatchReliableDelta);
        kb32_xr<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, xl, r, ph, sh, sv, tv, rh, B->part3, B->bsc, B->active);
        kb32_fin<<<P, 64, 0, s>>>(BF_XR, B->probs, P, B->part3, B->bsc, B->bst, B->active, B->ruflag, B->nrm,
                                  kBatchReliableDelta);
        kb32_fold<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, B->x, xl, B->ruflag);
        kb_resid64<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, B->f, B->x, B->r64, B->tpart, B->ruflag);
        kb_seg_sum<<<(P + 127) / 128, 128, 0, s>>>(B->probs, P, B->tpart, B->nrm);
        kb32_replace<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, B->r64, r, rh, p, v, B->part3, B->ruflag);
        kb32_fin<<<P, 64, 0, s>>>(BF_RU, B->probs, P, B->part3, B->bsc, B->bst, B->active, B->ruflag, B->nrm,
                                  kBatchReliableDelta);
        launches += 17;
    };
    cudaGraphExec_t gexec = nullptr;
    const long long l0 = launches;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return HELM_CUDA_ERROR;
    enqueue();
    cudaGraph_t graph = nullptr;
    if (cudaStreamEndCapture(s, &graph) != cudaSuccess) return HELM_CUDA_ERROR;
    const cudaError_t ie = cudaGraphInstantiate(&gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return HELM_CUDA_ERROR;
    const long long per_iter = launches - l0;
    launches = l0;
    // replay in rounds of kRound iterations; the states of round i are read while
    // round i + 1 runs (a finished problem makes every later kernel skip its tiles)
    constexpr int kRound = 8;
    cudaEvent_t rev[2];
    cudaEventCreateWithFlags(&rev[0], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&rev[1], cudaEventDisableTiming);
    std::vector<BState> snap[2] = {std::vector<BState>(P), std::vector<BState>(P)};
    BState* stage = B->hbst;            // pinned staging of one snapshot
    int rounds = 0, pending = -1;
    bool done = false;
    cudaError_t err = cudaSuccess;
    const int max_rounds = o->maxit / kRound + 2;
    while (!done && rounds <= max_rounds) {
        for (int q = 0; q < kRound && err == cudaSuccess; ++q) {
            err = cudaGraphLaunch(gexec, s);
            launches += per_iter;
        }
        if (err != cudaSuccess) break;
        // wait for the previous round's snapshot before reusing the staging buffer
        if (pending >= 0) {
            if ((err = cudaEventSynchronize(rev[pending])) != cudaSuccess) break;
            std::memcpy(snap[pending].data(), stage, sizeof(BState) * P);
            done = true;
            for (int b = 0; b < P; ++b)
                if (snap[pending][b].status == HELM_NOT_CONVERGED && snap[pending][b].iters < o->maxit) done = false;
        }
        const int slot = rounds & 1;
        cudaMemcpyAsync(stage, B->bst, sizeof(BState) * P, cudaMemcpyDeviceToHost, s);
        cudaEventRecord(rev[slot], s);
        pending = slot;
        ++rounds;
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    cudaGraphExecDestroy(gexec);
    cudaEventDestroy(rev[0]);
    cudaEventDestroy(rev[1]);
    if (err != cudaSuccess) return HELM_CUDA_ERROR;
    // final states; problems still running (maxit reached mid-round) fold their increment
    std::memcpy(snap[0].data(), stage, sizeof(BState) * P);
    std::vector<int> still(P, 0);
    bool any = false;
    for (int b = 0; b < P; ++b)
        if (snap[0][b].status == HELM_NOT_CONVERGED) { still[b] = 1; any = true; }
    if (any) {
        cudaMemcpyAsync(B->ruflag, still.data(), sizeof(int) * P, cudaMemcpyHostToDevice, s);
        kb32_fold<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, B->x, xl, B->ruflag);
        kb_resid64<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, B->f, B->x, B->r64, B->tpart, B->ruflag);
        kb_seg_sum<<<(P + 127) / 128, 128, 0, s>>>(B->probs, P, B->tpart, B->nrm);
        cudaMemcpyAsync(B->hpin, B->nrm, sizeof(double) * P, cudaMemcpyDeviceToHost, s);
        launches += 3;
        if (cudaStreamSynchronize(s) != cudaSuccess) return HELM_CUDA_ERROR;
        for (int b = 0; b < P; ++b)
            if (still[b] && snap[0][b].bnorm > 0) snap[0][b].rel_res = std::sqrt(B->hpin[b]) / snap[0][b].bnorm;
    }
    for (int b = 0; b < P; ++b) {
        const BProb& pb = B->hprobs[b];
        cudaMemcpyAsync(x[b], B->x + pb.off, sizeof(double2) * pb.N, cudaMemcpyDeviceToDevice, s);
    }
    cudaEventRecord(e1, s);
    cudaEventRecord(B->join, s);
    cudaStreamWaitEvent(B->stream, B->join, 0);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int worst = HELM_OK;
    for (int b = 0; b < P; ++b) {
        const BState& S = snap[0][b];
        if (stats) {
            helm_stats& sb = stats[b];
            sb = helm_stats{};
            sb.status = S.status;
            sb.iters = S.iters;
            sb.cycles = S.restarts;
            sb.rel_res = S.rel_res;
            sb.ms = ms;
            sb.launches = launches;
            sb.precond_applies = 2 * S.iters;
            sb.matvecs = 2 * S.iters;
        }
        if (S.status != HELM_OK) worst = S.status;
    }
    if (cudaGetLastError() != cudaSuccess) return HELM_CUDA_ERROR;
    return (helm_status)worst;
}

}  // namespace

extern "C" {

helm_status helm_batch_create(int nprob, helm_handle** hs, helm_batch** out) {
    if (!out || nprob < 1 || !hs) return HELM_BAD_ARG;
    *out = nullptr;
    for (int b = 0; b < nprob; ++b) {
        helm_handle* h = hs[b];
        if (!h || h->precision != HELM_MIXED || !h->Qbf || !h->Ainv) return HELM_NOT_READY;
    }
    helm_batch* B = new helm_batch();
    B->nprob = nprob;
    B->hs.assign(hs, hs + nprob);
    B->stream = hs[0]->stream;
    helm_status st;
    auto bail = [&](helm_status s) {
        helm_batch_destroy(B);
        return s;
    };
    if ((st = balloc(B, &B->probs, nprob)) != HELM_OK) return bail(st);
    if ((st = balloc(B, &B->tables, (size_t)nprob * kMaxLayer)) != HELM_OK) return bail(st);
    if ((st = balloc(B, &B->tablesf, (size_t)nprob * kTabF)) != HELM_OK) return bail(st);
    std::vector<double> tab((size_t)nprob * kMaxLayer);
    std::vector<float> tabf((size_t)nprob * kTabF, 0.0f);
    long long off = 0;
    for (int b = 0; b < nprob; ++b) {
        helm_handle* h = hs[b];
        BProb P{};
        P.dim = h->dim; P.n = h->n; P.L = h->L; P.k = h->k;
        P.N = h->N; P.off = off;
        P.hinv2 = h->op64.hinv2; P.dre = h->op64.dre;
        P.hinv2f = h->op32.hinv2; P.dref = h->op32.dre;
        P.mask = h->mask; P.lidx = h->lidx;
        for (int q = 0; q < kMaxLayer; ++q) {
            tab[(size_t)b * kMaxLayer + q] = h->op64.im[q];
            tabf[(size_t)b * kTabF + q] = h->op32.im[q];
            tabf[(size_t)b * kTabF + kTabPad + 2 * q] = h->op32.invd_tab[q].x;
            tabf[(size_t)b * kTabF + kTabPad + 2 * q + 1] = h->op32.invd_tab[q].y;
        }
        P.im = B->tables + (size_t)b * kMaxLayer;
        P.imf = B->tablesf + (size_t)b * kTabF;
        P.invdf = reinterpret_cast<const float2*>(B->tablesf + (size_t)b * kTabF + kTabPad);
        P.Qbf = static_cast<const __nv_bfloat16*>(h->Qbf);
        P.ldq = basis_ld(h->N);
        P.Ainv = h->Ainv;
        P.k2 = h->k2; P.k2f = h->k2f; P.invd_field = h->invdf;
        B->hprobs.push_back(P);
        B->kmax = std::max(B->kmax, h->k);
        off += h->N;
    }
    B->NT = off;
    cudaMemcpy(B->tables, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(B->tablesf, tabf.data(), tabf.size() * sizeof(float), cudaMemcpyHostToDevice);
    const long long NT = B->NT;
    if ((st = balloc(B, &B->f, NT)) != HELM_OK || (st = balloc(B, &B->x, NT)) != HELM_OK ||
        (st = balloc(B, &B->w, NT)) != HELM_OK || (st = balloc(B, &B->v32, NT)) != HELM_OK ||
        (st = balloc(B, &B->z32tmp, NT)) != HELM_OK || (st = balloc(B, &B->r32, NT)) != HELM_OK ||
        (st = balloc(B, &B->w32, NT)) != HELM_OK || (st = balloc(B, &B->active, nprob)) != HELM_OK ||
        (st = balloc(B, &B->kdim, nprob)) != HELM_OK || (st = balloc(B, &B->nrm, 4 * nprob)) != HELM_OK ||
        (st = balloc(B, &B->est, nprob)) != HELM_OK || (st = balloc(B, &B->y32, (size_t)nprob * kMaxP)) != HELM_OK)
        return bail(st);
    if (cudaMallocHost((void**)&B->hpin, sizeof(double) * 4 * nprob) != cudaSuccess) return bail(HELM_OUT_OF_MEMORY);
    if ((st = build_tiles(B)) != HELM_OK) return bail(st);
    *out = B;
    return HELM_OK;
}

helm_status helm_batch_destroy(helm_batch* B) {
    if (!B) return HELM_BAD_ARG;
    bfree(B->probs); bfree(B->tiles); bfree(B->tables); bfree(B->tablesf); bfree(B->active); bfree(B->kdim);
    bfree(B->f); bfree(B->x); bfree(B->V); bfree(B->w); bfree(B->v32); bfree(B->z32tmp); bfree(B->r32);
    bfree(B->Z32); bfree(B->w32); bfree(B->pp32); bfree(B->y32); bfree(B->hpart); bfree(B->H); bfree(B->sn);
    bfree(B->g); bfree(B->y); bfree(B->h2); bfree(B->cs); bfree(B->tpart); bfree(B->nrm); bfree(B->est);
    bfree(B->b32); bfree(B->r64); bfree(B->bsc); bfree(B->bst); bfree(B->ruflag); bfree(B->part3);
    if (B->hbst) cudaFreeHost(B->hbst);
    if (B->hpin) cudaFreeHost(B->hpin);
    if (B->cstream) cudaStreamDestroy(B->cstream);
    if (B->join) cudaEventDestroy(B->join);
    delete B;
    return HELM_OK;
}

helm_status helm_batch_set_tile(helm_batch* B, int tile_rows, int grid) {
    if (!B || tile_rows < 32 || tile_rows > 8192 || (tile_rows % 32) != 0 || grid < 1) return HELM_BAD_ARG;
    B->tile_rows = tile_rows;
    B->grid = grid;
    return build_tiles(B);
}

helm_status helm_batch_solve(helm_batch* B, const helm_solve_opts* o, const double* const* f, double* const* x,
                             helm_stats* stats) {
    NvtxRange nvtx("helm_batch_solve");
    if (!B || !o || !f || !x) return HELM_BAD_ARG;
    if (o->method == HELM_METHOD_BICGSTAB) return batch_bicgstab(B, o, f, x, stats);
    if (o->method != HELM_METHOD_FGMRES || o->restart < 1 || o->restart > kMaxRestart || o->conj ||
        o->correction == HELM_CORR_NONLINEAR)
        return HELM_BAD_ARG;
    const int m = o->restart;
    helm_status st = ensure_batch_krylov(B, m);
    if (st != HELM_OK) return st;
    // the solve runs on a private non-blocking stream (stream capture is not allowed on
    // the legacy default stream), ordered after the caller's stream and joined back
    if (!B->cstream) {
        if (cudaStreamCreateWithFlags(&B->cstream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->join, cudaEventDisableTiming) != cudaSuccess)
            return HELM_CUDA_ERROR;
    }
    cudaStream_t s = B->cstream;
    if (cudaEventRecord(B->join, B->stream) != cudaSuccess || cudaStreamWaitEvent(s, B->join, 0) != cudaSuccess)
        return HELM_CUDA_ERROR;
    const int P = B->nprob;
    const long long NT = B->NT;
    const int TR = B->tile_rows, NTL = B->ntiles, G = B->grid;
    const size_t smem64 = (size_t)TR * sizeof(double2), smem32 = (size_t)TR * sizeof(float2);
    cudaFuncSetAttribute(kb_mdot, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64);
    cudaFuncSetAttribute(kb_project32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem32);
    const int ldh = m + 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    // pack inputs; masked entries of x are the Dirichlet values
    for (int b = 0; b < P; ++b) {
        const BProb& pb = B->hprobs[b];
        cudaMemcpyAsync(B->f + pb.off, f[b], sizeof(double2) * pb.N, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(B->x + pb.off, x[b], sizeof(double2) * pb.N, cudaMemcpyDeviceToDevice, s);
        launch_set_masked(B->x + pb.off, B->f + pb.off, pb.mask, pb.N, s);
    }
    std::vector<int> act(P, 1), iters(P, 0), status(P, HELM_NOT_CONVERGED), cycles(P, 0);
    std::vector<double> bnorm(P, 0.0), relres(P, 0.0);
    long long launches = 0;
    // ||f||^2 per problem: residual with x = 0 is f; use a zero vector through kb_resid64 on w
    cudaMemsetAsync(B->w, 0, sizeof(double2) * NT, s);
    cudaMemcpyAsync(B->active, act.data(), sizeof(int) * P, cudaMemcpyHostToDevice, s);
    kb_resid64<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, B->f, B->w, B->V, B->tpart, B->active);
    kb_seg_sum<<<(P + 127) / 128, 128, 0, s>>>(B->probs, P, B->tpart, B->nrm);
    cudaMemcpyAsync(B->hpin, B->nrm, sizeof(double) * P, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return HELM_CUDA_ERROR;
    launches += 2;
    for (int b = 0; b < P; ++b) bnorm[b] = std::sqrt(B->hpin[b]);
    const double omega = o->omega;
    const int nr = o->relax == HELM_RELAX_NONE ? 0 : o->n_r;
    const bool tb = o->correction == HELM_CORR_TB;
    struct Graphs {                      // instantiated Arnoldi steps, freed on every exit
        std::vector<cudaGraphExec_t> g;
        ~Graphs() {
            for (auto e : g)
                if (e) cudaGraphExecDestroy(e);
        }
    } graphs;
    graphs.g.assign(m, nullptr);
    std::vector<cudaGraphExec_t>& step_graph = graphs.g;
    // kernels of one Arnoldi step (counted as the capture counts them)
    const long long step_launches = (nr == 0 ? 0 : (o->relax == HELM_RBGS ? 2 * nr : nr)) + (tb ? 4 : 0) + 13;
    while (true) {
        // true residual and restart decisions
        cudaMemcpyAsync(B->active, act.data(), sizeof(int) * P, cudaMemcpyHostToDevice, s);
        kb_resid64<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, B->f, B->x, B->V, B->tpart, B->active);
        kb_seg_sum<<<(P + 127) / 128, 128, 0, s>>>(B->probs, P, B->tpart, B->nrm);
        cudaMemcpyAsync(B->hpin, B->nrm, sizeof(double) * P, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return HELM_CUDA_ERROR;
        launches += 2;
        int nact = 0;
        for (int b = 0; b < P; ++b) {
            if (!act[b]) continue;
            const double beta = std::sqrt(B->hpin[b]);
            relres[b] = bnorm[b] > 0 ? beta / bnorm[b] : 0.0;
            if (bnorm[b] == 0 || beta <= o->tol * bnorm[b]) { status[b] = HELM_OK; act[b] = 0; }
            else if (!std::isfinite(beta)) { status[b] = HELM_DIVERGED; act[b] = 0; }
            else if (iters[b] >= o->maxit) { status[b] = HELM_NOT_CONVERGED; act[b] = 0; }
            else { ++cycles[b]; ++nact; }
        }
        if (nact == 0) break;
        cudaMemcpyAsync(B->active, act.data(), sizeof(int) * P, cudaMemcpyHostToDevice, s);
        kb_init_g<<<P, 64, 0, s>>>(P, m, B->g, B->nrm, B->active);
        kb_scale<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, B->V, B->V, B->nrm, B->active);
        cudaMemsetAsync(B->H, 0, sizeof(double2) * P * (m + 1) * m, s);
        launches += 2;
        std::vector<int> kd(P, 0), cact = act;
        for (int j = 0; j < m; ++j) {
          // one Arnoldi step (preconditioner, operator, CGS2, Givens, the two status
          // copies) is captured once per solve as a CUDA graph and replayed
          if (!step_graph[j]) {
            if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return HELM_CUDA_ERROR;
            double2* Vj = B->V + (long long)j * NT;
            double2* w = B->V + (long long)(j + 1) * NT;
            float2* Zj = B->Z32 + (long long)j * NT;
            // z = M(v_j): complex64 damped Jacobi from zero, then the trunk-basis correction
            kb_cvt64to32<<<G, BT, 0, s>>>(Vj, B->v32, NT);
            if (nr == 0) {
                cudaMemsetAsync(Zj, 0, sizeof(float2) * NT, s);
            } else if (o->relax == HELM_RBGS) {
                for (int q = 0; q < nr; ++q) {
                    // the first red half-sweep from zero also clears the black nodes
                    kb_rbgs32<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, 0, q == 0, B->v32, Zj, B->active);
                    kb_rbgs32<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, 1, 0, B->v32, Zj, B->active);
                }
                launches += 2 * nr;
            } else {
                float2* a = (nr % 2 == 1) ? Zj : B->z32tmp;
                float2* bb = (nr % 2 == 1) ? B->z32tmp : Zj;
                kb_jacobi32<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, (float)omega, B->v32, nullptr, a, B->active);
                for (int q = 1; q < nr; ++q) {
                    kb_jacobi32<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, (float)omega, B->v32, a, bb, B->active);
                    std::swap(a, bb);
                }
                launches += nr;
            }
            if (tb) {
                kb_resid32<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, B->v32, Zj, B->r32, B->active);
                kb_project32<<<G, BT, smem32, s>>>(B->probs, B->tiles, NTL, TR, B->r32, B->pp32, B->kmax, B->active);
                kb_coarse<<<P, 128, 0, s>>>(B->probs, P, B->pp32, B->kmax, B->y32, B->active);
                kb_prolong32<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, B->y32, B->kmax, Zj, B->active);
                launches += 4;
            }
            // w = A32 z (complex64), widened for the FP64 Arnoldi
            kb_apply32<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, Zj, B->w32, B->active);
            kb_cvt32to64<<<G, BT, 0, s>>>(B->w32, w, NT);
            // CGS2
            kb_mdot<<<G, BT, smem64, s>>>(B->probs, B->tiles, NTL, TR, B->V, NT, j + 1, w, B->hpart, B->active);
            kb_mdot_fin<<<P, 64, 0, s>>>(B->probs, P, B->hpart, j + 1, B->H + (long long)j * ldh, ldh * m, 0, nullptr,
                                         B->active);
            kb_mupdate<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, B->V, NT, j + 1, B->H + (long long)j * ldh,
                                        ldh * m, -1.0, w, nullptr, B->active);
            kb_mdot<<<G, BT, smem64, s>>>(B->probs, B->tiles, NTL, TR, B->V, NT, j + 1, w, B->hpart, B->active);
            kb_mdot_fin<<<P, 64, 0, s>>>(B->probs, P, B->hpart, j + 1, B->H + (long long)j * ldh, ldh * m, 1, B->h2,
                                         B->active);
            kb_mupdate<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, B->V, NT, j + 1, B->h2, kMaxRestart + 1, -1.0, w,
                                        B->tpart, B->active);
            kb_seg_sum<<<(P + 127) / 128, 128, 0, s>>>(B->probs, P, B->tpart, B->nrm + P);
            kb_givens<<<(P + 63) / 64, 64, 0, s>>>(P, B->H, ldh, m, j, B->cs, B->sn, B->g, B->nrm + P, B->est, B->active);
            kb_scale<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, w, w, B->nrm + P, B->active);
            launches += 13;
            cudaMemcpyAsync(B->hpin, B->nrm + P, sizeof(double) * P, cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(B->hpin + P, B->est, sizeof(double) * P, cudaMemcpyDeviceToHost, s);
            cudaGraph_t gr = nullptr;
            if (cudaStreamEndCapture(s, &gr) != cudaSuccess) return HELM_CUDA_ERROR;
            const cudaError_t ie = cudaGraphInstantiate(&step_graph[j], gr, 0);
            cudaGraphDestroy(gr);
            if (ie != cudaSuccess) return HELM_CUDA_ERROR;
          } else {
            launches += step_launches;
          }
            if (cudaGraphLaunch(step_graph[j], s) != cudaSuccess) return HELM_CUDA_ERROR;
            if (cudaStreamSynchronize(s) != cudaSuccess) return HELM_CUDA_ERROR;
            int still = 0;
            for (int b = 0; b < P; ++b) {
                if (!cact[b]) continue;
                ++iters[b];
                kd[b] = j + 1;
                const double est = B->hpin[P + b] / bnorm[b];
                if (B->hpin[b] == 0.0 || !std::isfinite(est) || est <= o->tol || iters[b] >= o->maxit) cact[b] = 0;
                else ++still;
            }
            if (still == 0) break;
            cudaMemcpyAsync(B->active, cact.data(), sizeof(int) * P, cudaMemcpyHostToDevice, s);
        }
        // x += Z y with each problem's own Krylov dimension
        cudaMemcpyAsync(B->kdim, kd.data(), sizeof(int) * P, cudaMemcpyHostToDevice, s);
        kb_hsolve<<<(P + 63) / 64, 64, 0, s>>>(P, B->H, ldh, m, B->g, B->kdim, B->y);
        kb_update_x<<<G, BT, 0, s>>>(B->probs, B->tiles, NTL, TR, B->Z32, NT, B->y, B->kdim, B->x);
        launches += 2;
        if (cudaGetLastError() != cudaSuccess) return HELM_CUDA_ERROR;
    }
    for (int b = 0; b < P; ++b) {
        const BProb& pb = B->hprobs[b];
        cudaMemcpyAsync(x[b], B->x + pb.off, sizeof(double2) * pb.N, cudaMemcpyDeviceToDevice, s);
    }
    cudaEventRecord(e1, s);
    cudaEventRecord(B->join, s);
    cudaStreamWaitEvent(B->stream, B->join, 0);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int worst = HELM_OK;
    for (int b = 0; b < P; ++b) {
        if (stats) {
            helm_stats& sb = stats[b];
            sb = helm_stats{};
            sb.status = status[b];
            sb.iters = iters[b];
            sb.cycles = cycles[b];
            sb.rel_res = relres[b];
            sb.ms = ms;
            sb.launches = launches;
        }
        if (status[b] != HELM_OK) worst = status[b];
    }
    if (cudaGetLastError() != cudaSuccess) return HELM_CUDA_ERROR;
    return (helm_status)worst;
}

}  // extern "C"
