// Dense layers of the DeepONet (App. B): FP32 GEMM, bias + activation and their
// gradients, the relative-L2 loss of the DeepONet output, and Adam.
//
// Row-major matrices throughout.  The GEMM computes C = alpha op(A) op(B) + beta C
// with 64 x 64 output tiles, a 16-deep K slab in shared memory and a 4 x 4
// register tile per thread; long-K products are split over blockIdx.z and
// combined with atomic adds (training tolerates the summation order).
#include <cuda_runtime.h>

#include "helm_internal.cuh"

namespace {

constexpr int GBM = 64, GBN = 64, GBK = 16;

__global__ void __launch_bounds__(256) k_sgemm(int transA, int transB, int M, int N, int K, float alpha,
                                               const float* __restrict__ A, int lda, const float* __restrict__ B,
                                               int ldb, float* __restrict__ C, int ldc, int kslice, int atomic) {
    __shared__ float As[GBK][GBM + 4];
    __shared__ float Bs[GBK][GBN + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const int k0 = blockIdx.z * kslice;
    const int k1 = min(K, k0 + kslice);
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int kb = k0; kb < k1; kb += GBK) {
        // A tile: GBM x GBK (op(A)[m][k]); B tile: GBK x GBN (op(B)[k][n])
        for (int t = threadIdx.x; t < GBM * GBK; t += 256) {
            int mm, kk;
            if (transA) { mm = t % GBM; kk = t / GBM; }        // A stored K x M: contiguous in m
            else { kk = t % GBK; mm = t / GBK; }               // A stored M x K: contiguous in k
            const int gm = m0 + mm, gk = kb + kk;
            float v = 0.f;
            if (gm < M && gk < k1) v = transA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
            As[kk][mm] = v;
        }
        for (int t = threadIdx.x; t < GBK * GBN; t += 256) {
            int kk, nn;
            if (transB) { kk = t % GBK; nn = t / GBK; }        // B stored N x K: contiguous in k
            else { nn = t % GBN; kk = t / GBN; }               // B stored K x N: contiguous in n
            const int gk = kb + kk, gn = n0 + nn;
            float v = 0.f;
            if (gn < N && gk < k1) v = transB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
            if (gm < M && gn < N) {
                float* c = C + (long long)gm * ldc + gn;
                if (atomic) atomicAdd(c, alpha * acc[i][j]);
                else *c += alpha * acc[i][j];
            }
        }
}

__global__ void k_scale_matrix(int M, int N, float beta, float* __restrict__ C, int ldc) {
    const long long total = (long long)M * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        float* c = C + (e / N) * ldc + e % N;
        *c = beta == 0.f ? 0.f : beta * *c;
    }
}

// X[r][c] = act(X[r][c] + bias[c]); act: 0 none, 1 ReLU, 2 tanh, 3 Leaky ReLU (slope 0.01)
__global__ void k_bias_act(int rows, int cols, float* __restrict__ X, const float* __restrict__ bias, int act) {
    const long long total = (long long)rows * cols;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        float v = X[e] + (bias ? bias[e % cols] : 0.f);
        if (act == 1) v = fmaxf(v, 0.f);
        else if (act == 2) v = tanhf(v);
        else if (act == 3) v = v > 0.f ? v : 0.01f * v;
        X[e] = v;
    }
}

// dX *= act'(Y), Y the activation output
__global__ void k_act_backward(long long n, float* __restrict__ dX, const float* __restrict__ Y, int act) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float y = Y[e];
        if (act == 1) dX[e] = y > 0.f ? dX[e] : 0.f;
        else if (act == 2) dX[e] *= (1.f - y * y);
        else if (act == 3) dX[e] = y > 0.f ? dX[e] : 0.01f * dX[e];   // the output keeps the input's sign
    }
}

// db[c] = sum_r dY[r][c]
__global__ void k_bias_grad(int rows, int cols, const float* __restrict__ dY, float* __restrict__ db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += dY[(long long)r * cols + c];
    db[c] = s;
}

// Adam (Kingma & Ba) with bias correction
__global__ void k_adam(long long n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float gi = g[e];
        const float mi = b1 * m[e] + (1.f - b1) * gi;
        const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
        m[e] = mi;
        v[e] = vi;
        p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Relative-L2 loss of the DeepONet output on sampled nodes.
// pred, target: B x (2P) with the real parts in columns [0, P) and the imaginary
// parts in [P, 2P).  loss[b] = ||pred_b - target_b||^2 / ||target_b||^2;
// dpred = d(mean_b loss[b]) / d pred.  One block per sample.
__global__ void k_rel_l2(int Bn, int P2, const float* __restrict__ pred, const float* __restrict__ target,
                         float* __restrict__ dpred, float* __restrict__ loss) {
    __shared__ float s_num[32], s_den[32];
    const int b = blockIdx.x;
    const float* pr = pred + (long long)b * P2;
    const float* tg = target + (long long)b * P2;
    float num = 0.f, den = 0.f;
    for (int e = threadIdx.x; e < P2; e += blockDim.x) {
        const float d = pr[e] - tg[e];
        num += d * d;
        den += tg[e] * tg[e];
    }
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { s_num[w] = num; s_den[w] = den; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f, c = 0.f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a += s_num[q]; c += s_den[q]; }
        s_num[0] = a;
        s_den[0] = c;
        loss[b] = a / c;
    }
    __syncthreads();
    const float scale = 2.f / (s_den[0] * Bn);
    for (int e = threadIdx.x; e < P2; e += blockDim.x) dpred[(long long)b * P2 + e] = scale * (pr[e] - tg[e]);
}

// dst[r][c] = src[ri[r]][ci[c]] (ri, ci may be null: identity)
__global__ void k_gather(int rows, int cols, const float* __restrict__ src, long long lds, const int* __restrict__ ri,
                         const int* __restrict__ ci, float* __restrict__ dst) {
    const long long total = (long long)rows * cols;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), c = (int)(e % cols);
        const long long sr = ri ? ri[r] : r;
        const long long sc = ci ? ci[c] : c;
        dst[e] = src[sr * lds + sc];
    }
}

int grid_for(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 8 * 152 ? (b < 1 ? 1 : b) : 8 * 152);
}

// ---- 3D convolution of the CNN branch (App. B): 3 x 3 x 3 kernels, stride s, zero
// padding pad, layout [batch][channel][z][y][x], W[out][in][kz][ky][kx].  Every output
// value is summed by one thread (inputs, then kz, ky, kx) or one block (fixed tree),
// so the results do not depend on scheduling.
constexpr int CK = 3;

__device__ __forceinline__ long long vox(int D, int z, int y, int x) { return ((long long)z * D + y) * D + x; }

// Y[b][o][.] = bias[o] + sum_{i,k} W[o][i][k] X[b][i][. s + k - pad]
__global__ void k_conv3d(int B, int Ci, int D, int Co, int Do, int stride, int pad, const float* __restrict__ X,
                         const float* __restrict__ W, const float* __restrict__ bias, float* __restrict__ Y) {
    const long long V = (long long)Do * Do * Do, total = (long long)B * Co * V;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long v = e % V;
        const int o = (int)((e / V) % Co), b = (int)(e / (V * Co));
        const int ox = (int)(v % Do), oy = (int)((v / Do) % Do), oz = (int)(v / ((long long)Do * Do));
        float acc = 0.f;
        for (int i = 0; i < Ci; ++i) {
            const float* xi = X + ((long long)b * Ci + i) * D * D * D;
            const float* wi = W + ((long long)o * Ci + i) * CK * CK * CK;
            for (int kz = 0; kz < CK; ++kz) {
                const int z = oz * stride + kz - pad;
                if (z < 0 || z >= D) continue;
                for (int ky = 0; ky < CK; ++ky) {
                    const int y = oy * stride + ky - pad;
                    if (y < 0 || y >= D) continue;
                    for (int kx = 0; kx < CK; ++kx) {
                        const int x = ox * stride + kx - pad;
                        if (x < 0 || x >= D) continue;
                        acc = fmaf(wi[(kz * CK + ky) * CK + kx], xi[vox(D, z, y, x)], acc);
                    }
                }
            }
        }
        Y[e] = acc + (bias ? bias[o] : 0.f);
    }
}

// dX[b][i][p] = sum_{o,k} W[o][i][k] dY[b][o][q] over the outputs q that read p with offset k
__global__ void k_conv3d_dx(int B, int Ci, int D, int Co, int Do, int stride, int pad, const float* __restrict__ W,
                            const float* __restrict__ dY, float* __restrict__ dX) {
    const long long V = (long long)D * D * D, total = (long long)B * Ci * V, Vo = (long long)Do * Do * Do;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long v = e % V;
        const int i = (int)((e / V) % Ci), b = (int)(e / (V * Ci));
        const int x = (int)(v % D), y = (int)((v / D) % D), z = (int)(v / ((long long)D * D));
        float acc = 0.f;
        for (int o = 0; o < Co; ++o) {
            const float* dyo = dY + ((long long)b * Co + o) * Vo;
            const float* wo = W + ((long long)o * Ci + i) * CK * CK * CK;
            for (int kz = 0; kz < CK; ++kz) {
                const int tz = z + pad - kz;
                if (tz < 0 || tz % stride) continue;
                const int oz = tz / stride;
                if (oz >= Do) continue;
                for (int ky = 0; ky < CK; ++ky) {
                    const int ty = y + pad - ky;
                    if (ty < 0 || ty % stride) continue;
                    const int oy = ty / stride;
                    if (oy >= Do) continue;
                    for (int kx = 0; kx < CK; ++kx) {
                        const int tx = x + pad - kx;
                        if (tx < 0 || tx % stride) continue;
                        const int ox = tx / stride;
                        if (ox >= Do) continue;
                        acc = fmaf(wo[(kz * CK + ky) * CK + kx], dyo[vox(Do, oz, oy, ox)], acc);
                    }
                }
            }
        }
        dX[e] = acc;
    }
}

// one block per weight (o, i, k) (and per bias o when i == Ci): the sum over the batch
// and the outputs of dY X at the offset, in a fixed order (strided per thread, then a
// shared-memory tree)
__global__ void __launch_bounds__(256) k_conv3d_dw(int B, int Ci, int D, int Co, int Do, int stride, int pad,
                                                   const float* __restrict__ X, const float* __restrict__ dY,
                                                   float* __restrict__ dW, float* __restrict__ db) {
    __shared__ float red[256];
    const int wid = blockIdx.x;                          // o * (Ci * 27 + 1) + i * 27 + k, k = 27: bias
    const int per = Ci * CK * CK * CK + 1;
    const int o = wid / per, r = wid % per;
    const bool is_bias = r == per - 1;
    const int i = is_bias ? 0 : r / (CK * CK * CK), k = is_bias ? 0 : r % (CK * CK * CK);
    const int kz = k / (CK * CK), ky = (k / CK) % CK, kx = k % CK;
    const long long Vo = (long long)Do * Do * Do, total = (long long)B * Vo;
    float acc = 0.f;
    for (long long e = threadIdx.x; e < total; e += blockDim.x) {
        const int b = (int)(e / Vo);
        const long long v = e % Vo;
        const float g = dY[((long long)b * Co + o) * Vo + v];
        if (is_bias) {
            acc += g;
            continue;
        }
        const int ox = (int)(v % Do), oy = (int)((v / Do) % Do), oz = (int)(v / ((long long)Do * Do));
        const int z = oz * stride + kz - pad, y = oy * stride + ky - pad, x = ox * stride + kx - pad;
        if (z < 0 || z >= D || y < 0 || y >= D || x < 0 || x >= D) continue;
        acc = fmaf(g, X[((long long)b * Ci + i) * D * D * D + vox(D, z, y, x)], acc);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (is_bias) {
            if (db) db[o] = red[0];
        } else if (dW) {
            dW[((long long)o * Ci + i) * CK * CK * CK + k] = red[0];
        }
    }
}

}  // namespace

extern "C" {

helm_status nn_gemm(int transA, int transB, int M, int N, int K, float alpha, const float* A, int lda, const float* B,
                    int ldb, float beta, float* C, int ldc, void* stream) {
    if (M < 0 || N < 0 || K < 0 || !C || (K > 0 && (!A || !B))) return HELM_BAD_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (M == 0 || N == 0) return HELM_OK;
    if (beta != 1.f) k_scale_matrix<<<grid_for((long long)M * N), 256, 0, s>>>(M, N, beta, C, ldc);
    if (K == 0 || alpha == 0.f) return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_CUDA_ERROR;
    const int gx = (N + GBN - 1) / GBN, gy = (M + GBM - 1) / GBM;
    // split K until there are about two blocks per SM
    int splits = 1;
    while ((long long)gx * gy * splits < 2 * 152 && K / (splits * 2) >= 4 * GBK) splits *= 2;
    int kslice = (K + splits - 1) / splits;
    kslice = ((kslice + GBK - 1) / GBK) * GBK;
    splits = (K + kslice - 1) / kslice;
    k_sgemm<<<dim3(gx, gy, splits), 256, 0, s>>>(transA, transB, M, N, K, alpha, A, lda, B, ldb, C, ldc, kslice,
                                                 splits > 1);
    return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_CUDA_ERROR;
}

helm_status nn_bias_act(int rows, int cols, float* X, const float* bias, int act, void* stream) {
    if (rows < 0 || cols < 0 || !X || act < 0 || act > 3) return HELM_BAD_ARG;
    k_bias_act<<<grid_for((long long)rows * cols), 256, 0, static_cast<cudaStream_t>(stream)>>>(rows, cols, X, bias, act);
    return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_CUDA_ERROR;
}

helm_status nn_act_backward(long long n, float* dX, const float* Y, int act, void* stream) {
    if (n < 0 || !dX || !Y || act < 0 || act > 3) return HELM_BAD_ARG;
    k_act_backward<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, dX, Y, act);
    return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_CUDA_ERROR;
}

helm_status nn_bias_grad(int rows, int cols, const float* dY, float* db, void* stream) {
    if (rows < 0 || cols < 0 || !dY || !db) return HELM_BAD_ARG;
    k_bias_grad<<<(cols + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(rows, cols, dY, db);
    return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_CUDA_ERROR;
}

helm_status nn_adam(long long n, float* p, const float* g, float* m, float* v, float lr, float beta1, float beta2,
                    float eps, int t, void* stream) {
    if (n < 0 || !p || !g || !m || !v || t < 1) return HELM_BAD_ARG;
    const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
    k_adam<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, p, g, m, v, lr, beta1, beta2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_CUDA_ERROR;
}

helm_status nn_gather(int rows, int cols, const float* src, long long lds, const int* row_idx, const int* col_idx,
                      float* dst, void* stream) {
    if (rows < 0 || cols < 0 || !src || !dst) return HELM_BAD_ARG;
    k_gather<<<grid_for((long long)rows * cols), 256, 0, static_cast<cudaStream_t>(stream)>>>(rows, cols, src, lds, row_idx,
                                                                                             col_idx, dst);
    return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_CUDA_ERROR;
}

helm_status nn_rel_l2(int B, int P2, const float* pred, const float* target, float* dpred, float* loss, void* stream) {
    if (B < 1 || P2 < 1 || !pred || !target || !dpred || !loss) return HELM_BAD_ARG;
    k_rel_l2<<<B, 256, 0, static_cast<cudaStream_t>(stream)>>>(B, P2, pred, target, dpred, loss);
    return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_CUDA_ERROR;
}

helm_status nn_conv3d(int B, int Ci, int D, int Co, int stride, int pad, const float* X, const float* W,
                      const float* bias, float* Y, void* stream) {
    if (B < 1 || Ci < 1 || Co < 1 || D < 1 || stride < 1 || pad < 0 || pad > 2 || !X || !W || !Y) return HELM_BAD_ARG;
    const int Do = (D + 2 * pad - CK) / stride + 1;
    if (D + 2 * pad < CK || Do < 1) return HELM_BAD_ARG;
    k_conv3d<<<grid_for((long long)B * Co * Do * Do * Do), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        B, Ci, D, Co, Do, stride, pad, X, W, bias, Y);
    return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_CUDA_ERROR;
}

helm_status nn_conv3d_backward(int B, int Ci, int D, int Co, int stride, int pad, const float* X, const float* W,
                               const float* dY, float* dX, float* dW, float* db, void* stream) {
    if (B < 1 || Ci < 1 || Co < 1 || D < 1 || stride < 1 || pad < 0 || pad > 2 || !dY) return HELM_BAD_ARG;
    if ((dX && !W) || ((dW || db) && !X)) return HELM_BAD_ARG;
    const int Do = (D + 2 * pad - CK) / stride + 1;
    if (D + 2 * pad < CK || Do < 1) return HELM_BAD_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dX)
        k_conv3d_dx<<<grid_for((long long)B * Ci * D * D * D), 256, 0, s>>>(B, Ci, D, Co, Do, stride, pad, W, dY, dX);
    if (dW || db)
        k_conv3d_dw<<<Co * (Ci * CK * CK * CK + 1), 256, 0, s>>>(B, Ci, D, Co, Do, stride, pad, X, dY, dW, db);
    return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_CUDA_ERROR;
}

}  // extern "C"
