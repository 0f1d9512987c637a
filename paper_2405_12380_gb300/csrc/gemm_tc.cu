// BF16 GEMM with FP32 accumulation on the fifth-generation tensor cores (tcgen05),
// for the dense layers of the DeepONet (App. B): C = alpha op(A) op(B) + beta C with
// FP32 row-major operands, as nn_gemm, but with op(A) and op(B) rounded to BF16.
//
// Structure (one CTA per 128 x 128 tile of C, 64-deep K steps, a four-stage ring):
//  - the operands are first converted to BF16 "K-major" copies (op(A) as M x K rows,
//    op(B)^T as N x K rows), zero-padded to multiples of 128 rows and 64 columns so
//    that every TMA box lies inside the copy and starts on a 16-byte boundary;
//  - warp 0: one elected thread loads the A and B boxes of a stage with
//    cp.async.bulk.tensor (128-byte swizzle) onto the stage's "full" mbarrier;
//  - warp 1: one elected thread issues tcgen05.mma.kind::f16 (M = 128, N = 128,
//    K = 16 per instruction, four per stage) into a TMEM accumulator and commits
//    each stage to its "empty" mbarrier, the last one to the "done" mbarrier;
//  - warp 2 allocates and frees the 128 TMEM columns;
//  - warps 4-7 (one per quarter of the TMEM lanes) read the accumulator with
//    tcgen05.ld and write alpha D + beta C for the valid rows and columns.
// Every mbarrier wait is bounded: a wait that runs out records an error flag and the
// thread goes on (the result is then garbage but the launch ends); the host reads
// the flag with nn_gemm_bf16_status.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "helm_internal.cuh"

namespace helm {

namespace {

constexpr int TBM = 128, TBN = 128, TBK = 64, STAGES = 4;
constexpr int TC_THREADS = 256;
constexpr unsigned kStageBytes = (TBM + TBN) * TBK * 2;        // 32 KiB
constexpr unsigned kWaitLimit = 1u << 26;

__device__ int g_tc_error;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase of the given parity; false (and the error flag) on a timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity) {
    // after one timeout in the launch the other waits give up at once
    if (*reinterpret_cast<volatile int*>(&g_tc_error)) return false;
    for (unsigned it = 0; it < kWaitLimit; ++it)
        if (mbar_try(b, parity)) return true;
    atomicExch(&g_tc_error, 1);
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(su32(dst)), "l"(map), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups
// 1024 bytes apart (start address and offsets in units of 16 bytes)
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
    const uint64_t addr = (su32(p) & 0x3FFFFu) >> 4;
    return addr | (uint64_t(1) << 16) | (uint64_t(1024 >> 4) << 32) | (uint64_t(1) << 46) | (uint64_t(2) << 61);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_bf16_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N,
                   int Kp, float alpha, float beta, float* __restrict__ C, int ldc) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte alignment of the stage buffers (the swizzle atom)
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + STAGES * TBM * TBK * 2;
    __shared__ uint64_t full[STAGES], empty[STAGES], done;
    __shared__ uint32_t tmem_base;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
    const int nk = Kp / TBK;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"(TBN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // producer
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % STAGES;
            if (kb >= STAGES) mbar_wait(&empty[s], ((kb / STAGES) - 1) & 1);
            mbar_expect_tx(&full[s], kStageBytes);
            tma_load_2d(sA + s * TBM * TBK * 2, &mapA, kb * TBK, m0, &full[s]);
            tma_load_2d(sB + s * TBN * TBK * 2, &mapB, kb * TBK, n0, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16(TBM, TBN);
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % STAGES;
            mbar_wait(&full[s], (kb / STAGES) & 1);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t da = smem_desc(sA + s * TBM * TBK * 2), db = smem_desc(sB + s * TBN * TBK * 2);
#pragma unroll
            for (int k = 0; k < TBK / 16; ++k) {
                // K = 16 BF16 = 32 bytes further along the swizzled 128-byte rows
                const uint64_t koff = (uint64_t)((k * 32) >> 4);
                const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da + koff), "l"(db + koff), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             su32(&empty[s]))
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&done))
                     : "memory");
    } else if (warp >= 4) {
        // epilogue: warp 4 + q reads TMEM lanes 32 q .. 32 q + 31 (rows of the tile)
        const int q = warp - 4;
        mbar_wait(&done, 0);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int row = m0 + 32 * q + lane;
        for (int c0 = 0; c0 < TBN; c0 += 32) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
                  "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
                  "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                  "=r"(v[30]), "=r"(v[31])
                : "r"(taddr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
                float* Cr = C + (long long)row * ldc;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = n0 + c0 + j;
                    if (col < N) {
                        const float d = __uint_as_float(v[j]);
                        Cr[col] = beta == 0.f ? alpha * d : fmaf(alpha, d, beta * Cr[col]);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 2) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TBN) : "memory");
    }
}

// dst (rows_p x Kp, BF16, row-major, zero padding) from the FP32 operand: element
// (r, k) of op(X) is X[r * ld + k] (trans = 0) or X[k * ld + r] (trans = 1)
__global__ void k_to_bf16_kmajor(const float* __restrict__ X, int ld, int trans, int rows, int K,
                                 __nv_bfloat16* __restrict__ dst, int rows_p, int Kp) {
    const long long total = (long long)rows_p * Kp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / Kp), k = (int)(e - (long long)r * Kp);
        float v = 0.f;
        if (r < rows && k < K) v = trans ? X[(long long)k * ld + r] : X[(long long)r * ld + k];
        dst[e] = __float2bfloat16_rn(v);
    }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    });
    return fn;
}

bool make_map(CUtensorMap* map, const void* base, int rows_p, int Kp) {
    EncodeFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows_p};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    const cuuint32_t box[2] = {TBK, TBM};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// per-device workspace of the BF16 copies (grown on demand, held until exit)
struct Ws {
    void* p = nullptr;
    size_t bytes = 0;
};
std::mutex g_ws_mutex;
Ws g_ws[64];

}  // namespace

}  // namespace helm

using namespace helm;

extern "C" helm_status nn_gemm_bf16(int transA, int transB, int M, int N, int K, float alpha, const float* A, int lda,
                                    const float* B, int ldb, float beta, float* C, int ldc, void* stream) {
    if (M < 0 || N < 0 || K < 0 || !A || !B || !C || ldc < N) return HELM_BAD_ARG;
    if (M == 0 || N == 0) return HELM_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int Mp = (M + TBM - 1) / TBM * TBM, Np = (N + TBN - 1) / TBN * TBN;
    const int Kp = K == 0 ? TBK : (K + TBK - 1) / TBK * TBK;
    const size_t need = ((size_t)Mp + Np) * Kp * 2;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return HELM_NO_DEVICE;
    std::lock_guard<std::mutex> lock(g_ws_mutex);
    Ws& w = g_ws[dev];
    if (w.bytes < need) {
        if (w.p) {
            cudaStreamSynchronize(s);
            cudaFree(w.p);
        }
        w.p = nullptr;
        w.bytes = 0;
        if (cudaMalloc(&w.p, need) != cudaSuccess) {
            cudaGetLastError();
            return HELM_OUT_OF_MEMORY;
        }
        w.bytes = need;
    }
    __nv_bfloat16* Ab = static_cast<__nv_bfloat16*>(w.p);
    __nv_bfloat16* Bb = Ab + (size_t)Mp * Kp;
    k_to_bf16_kmajor<<<4 * 152, 256, 0, s>>>(A, lda, transA, M, K, Ab, Mp, Kp);
    // op(B) is K x N; its K-major copy holds op(B)^T (N x K): element (n, k) = op(B)(k, n)
    k_to_bf16_kmajor<<<4 * 152, 256, 0, s>>>(B, ldb, !transB, N, K, Bb, Np, Kp);
    CUtensorMap ma, mb;
    if (!make_map(&ma, Ab, Mp, Kp) || !make_map(&mb, Bb, Np, Kp)) return HELM_CUDA_ERROR;
    const size_t smem = (size_t)STAGES * kStageBytes + 1024;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_gemm_bf16_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return HELM_CUDA_ERROR;
        attr = true;
    }
    dim3 grid(Np / TBN, Mp / TBM);
    k_gemm_bf16_tc<<<grid, TC_THREADS, smem, s>>>(ma, mb, M, N, Kp, alpha, beta, C, ldc);
    return cudaGetLastError() == cudaSuccess ? HELM_OK : HELM_CUDA_ERROR;
}

extern "C" helm_status nn_gemm_bf16_status(int* timed_out) {
    if (!timed_out) return HELM_BAD_ARG;
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int)) != cudaSuccess) return HELM_CUDA_ERROR;
    *timed_out = v;
    if (v) {
        const int z = 0;
        if (cudaMemcpyToSymbol(g_tc_error, &z, sizeof(int)) != cudaSuccess) return HELM_CUDA_ERROR;
    }
    return HELM_OK;
}
