// Complex64 BiCGStab with reliable updates (the BiCGStab of HELM_MIXED handles).
//
// The Krylov vectors (r, rhat, p, v, s, t, phat, shat and the solution increment
// xl) are complex64; the operator and the hybrid-cycle preconditioner run in
// complex64 (BF16 trunk basis); the iterate x and the true residual f - A x are
// FP64.  Each reduction sums FP32 products over a thread's few entries, then in
// FP64 across threads and blocks in a fixed order, and the last block to finish
// applies the scalar recurrence (bicg.cuh), as in the FP64 kernels.
//
// Reliable updates (Sleijpen and van der Vorst, "Reliable updated residuals in
// hybrid Bi-CG methods", Computing 56, 1996): from time to time the host folds the
// increment into the FP64 iterate, x += xl, xl = 0, recomputes the true residual
// in FP64 and replaces the recursive residual by its complex64 rounding, keeping
// the search direction p; rho and beta are recomputed for the replaced residual.
//
// Every kernel here leaves its vectors and the scalars untouched once S_STOP is
// set (the loop ended on the recursive residual, a breakdown or a non-finite
// value), so that an iteration queued behind the one that stopped changes
// nothing but the preconditioner's and the operator's scratch outputs, which it
// recomputes to the same values.
#include "bicg.cuh"

namespace helm {

namespace {

constexpr int kB32Threads = kFusedThreads;   // 256

__device__ __forceinline__ bool stopped(const double2* sc) { return sc[S_STOP].x != 0.0; }

// block sum of a per-thread FP32 value: an FP32 butterfly within each warp, then the
// warps' sums in a fixed order; valid in thread 0.  (FP64 adds and shuffles run at a
// small fraction of the FP32 rate on this GPU; the per-thread sums are FP32 already.)
__device__ __forceinline__ double block_sum32(float v) {
    __shared__ float red[kB32Threads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x == 0)
        for (int q = 0; q < kB32Threads / 32; ++q) s += red[q];
    return (double)s;
}

// the sum of nparts FP32 partials of W values (stride W), taken by every block in
// the same fixed order (so every block gets the same value bit for bit) -- a strided
// sum per thread, a butterfly per warp, the warps in order -- and returned to all
// threads of the block
template <int W>
__device__ __forceinline__ void all_blocks_sum(const float* parts, int nparts, float* out) {
    __shared__ float red[W][kB32Threads / 32];
    __shared__ float res[W];
    float v[W];
#pragma unroll
    for (int q = 0; q < W; ++q) v[q] = 0.f;
    for (int b = threadIdx.x; b < nparts; b += kB32Threads)
#pragma unroll
        for (int q = 0; q < W; ++q) v[q] += __ldcg(parts + (long long)b * W + q);
#pragma unroll
    for (int q = 0; q < W; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int q = 0; q < W; ++q) red[q][threadIdx.x >> 5] = v[q];
    __syncthreads();
    if (threadIdx.x < W) {
        float t = 0.f;
        for (int w = 0; w < kB32Threads / 32; ++w) t += red[threadIdx.x][w];
        res[threadIdx.x] = t;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < W; ++q) out[q] = res[q];
}

// complex64 as float2; two entries per float4
__device__ __forceinline__ float2 lo(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi(float4 a) { return make_float2(a.z, a.w); }
__device__ __forceinline__ float4 pack(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 caddf(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csubf(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 tof(double2 a) { return make_float2((float)a.x, (float)a.y); }
// conj(a) b accumulated into (re, im)
__device__ __forceinline__ void cdotacc(float2 a, float2 b, float& re, float& im) {
    re = fmaf(a.x, b.x, fmaf(a.y, b.y, re));
    im = fmaf(a.x, b.y, fmaf(-a.y, b.x, im));
}
__device__ __forceinline__ void nrmacc(float2 a, float& s) { s = fmaf(a.x, a.x, fmaf(a.y, a.y, s)); }

// Grid-stride loop over entry pairs (2q, 2q + 1); an odd N's last entry is a
// pair whose second half is absent (loaded as zero, not stored).
template <typename F>
__device__ __forceinline__ void for_pairs(long long N, F&& body) {
    const long long P = (N + 1) / 2;
    const bool odd = (N & 1) != 0;
    for (long long q = blockIdx.x * (long long)kB32Threads + threadIdx.x; q < P;
         q += (long long)gridDim.x * kB32Threads)
        body(q, odd && q == P - 1);
}

__device__ __forceinline__ float4 ld2(const float2* a, long long q, bool half) {
    if (!half) return reinterpret_cast<const float4*>(a)[q];
    const float2 v = a[2 * q];
    return make_float4(v.x, v.y, 0.f, 0.f);
}
__device__ __forceinline__ void st2(float2* a, long long q, bool half, float4 v) {
    if (!half) reinterpret_cast<float4*>(a)[q] = v;
    else a[2 * q] = make_float2(v.x, v.y);
}

// p = r + beta (p - omega v)
__global__ void __launch_bounds__(kB32Threads) k32_update_p(const float2* __restrict__ r, const float2* __restrict__ v,
                                                            float2* __restrict__ p, const double2* sc, long long N) {
    if (stopped(sc)) return;
    __shared__ float2 s_beta, s_omega;                     // converted once per block
    if (threadIdx.x == 0) {
        s_beta = tof(sc[S_BETA]);
        s_omega = tof(sc[S_OMEGA]);
    }
    __syncthreads();
    const float2 beta = s_beta, omega = s_omega;
    for_pairs(N, [&](long long q, bool half) {
        const float4 rr = ld2(r, q, half), vv = ld2(v, q, half), pp = ld2(p, q, half);
        const float2 a = caddf(lo(rr), cmulf(beta, csubf(lo(pp), cmulf(omega, lo(vv)))));
        const float2 b = caddf(hi(rr), cmulf(beta, csubf(hi(pp), cmulf(omega, hi(vv)))));
        st2(p, q, half, pack(a, b));
    });
}

// alpha = rho / <rhat, v>
__global__ void __launch_bounds__(kB32Threads) k32_alpha(const float2* __restrict__ rhat, const float2* __restrict__ v,
                                                         double2* sc, long long N, double* parts, unsigned* counter) {
    if (stopped(sc)) return;
    float re = 0.f, im = 0.f;
    for_pairs(N, [&](long long q, bool half) {
        const float4 a = ld2(rhat, q, half), b = ld2(v, q, half);
        cdotacc(lo(a), lo(b), re, im);
        cdotacc(hi(a), hi(b), re, im);
    });
    const double sre = block_sum32(re), sim = block_sum32(im);
    if (threadIdx.x == 0) {
        parts[2 * blockIdx.x] = sre;
        parts[2 * blockIdx.x + 1] = sim;
    }
    if (last_block_done(counter, gridDim.x)) {
        double tot[2];
        sum_parts<2>(parts, gridDim.x, threadIdx.x, tot);
        if (threadIdx.x == 0) {
            bicg_alpha(sc, make_double2(tot[0], tot[1]));
            *counter = 0;
        }
    }
}

// s = r - alpha v, ||s||^2 (||s|| <= tol ||f||, slot S_TOLS: the iteration ends after x += alpha phat).
// DOT: alpha = rho / <rhat, v> from the operator's partial sums (aparts, na blocks),
// computed by every block (bicg_alpha's arithmetic), stored by block 0
template <bool DOT>
__global__ void __launch_bounds__(kB32Threads) k32_s(const float2* __restrict__ r, const float2* __restrict__ v,
                                                     float2* __restrict__ s, double2* sc, long long N, double* parts,
                                                     unsigned* counter, const float* aparts, int na) {
    if (stopped(sc)) return;
    // the scalar in one thread, shared with the block (FP64 division is slow here)
    __shared__ float2 s_alpha;
    if (DOT) {
        float d[2];
        all_blocks_sum<2>(aparts, na, d);
        if (threadIdx.x == 0) {
            const bool brk = d[0] == 0.f && d[1] == 0.f;
            const double2 a64 = brk ? make_double2(0.0, 0.0) : cdiv(sc[S_RHO], make_double2(d[0], d[1]));
            s_alpha = tof(a64);
            if (blockIdx.x == 0) {
                sc[S_ALPHA] = a64;
                if (brk) sc[S_FLAGS].y = 1;
            }
        }
    } else if (threadIdx.x == 0) {
        s_alpha = tof(sc[S_ALPHA]);
    }
    __syncthreads();
    const float2 alpha = s_alpha;
    float acc = 0.f;
    for_pairs(N, [&](long long q, bool half) {
        const float4 rr = ld2(r, q, half), vv = ld2(v, q, half);
        const float2 a = csubf(lo(rr), cmulf(alpha, lo(vv)));
        const float2 b = csubf(hi(rr), cmulf(alpha, hi(vv)));
        nrmacc(a, acc);
        nrmacc(b, acc);
        st2(s, q, half, pack(a, b));
    });
    const double t = block_sum32(acc);
    if (threadIdx.x == 0) parts[blockIdx.x] = t;
    if (last_block_done(counter, gridDim.x)) {
        double tot[1];
        sum_parts<1>(parts, gridDim.x, threadIdx.x, tot);
        if (threadIdx.x == 0) {
            bicg_snorm(sc, tot[0], sc[S_TOLS].x);
            *counter = 0;
        }
    }
}

// omega = <t, s> / <t, t>
__global__ void __launch_bounds__(kB32Threads) k32_omega(const float2* __restrict__ t, const float2* __restrict__ s,
                                                         double2* sc, long long N, double* parts, unsigned* counter) {
    if (stopped(sc)) return;
    float re = 0.f, im = 0.f, tt = 0.f;
    for_pairs(N, [&](long long q, bool half) {
        const float4 a = ld2(t, q, half), b = ld2(s, q, half);
        cdotacc(lo(a), lo(b), re, im);
        cdotacc(hi(a), hi(b), re, im);
        nrmacc(lo(a), tt);
        nrmacc(hi(a), tt);
    });
    const double a0 = block_sum32(re), a1 = block_sum32(im), a2 = block_sum32(tt);
    if (threadIdx.x == 0) {
        parts[3 * blockIdx.x] = a0;
        parts[3 * blockIdx.x + 1] = a1;
        parts[3 * blockIdx.x + 2] = a2;
    }
    if (last_block_done(counter, gridDim.x)) {
        double tot[3];
        sum_parts<3>(parts, gridDim.x, threadIdx.x, tot);
        if (threadIdx.x == 0) {
            bicg_omega(sc, make_double2(tot[0], tot[1]), tot[2]);
            *counter = 0;
        }
    }
}

// xl += alpha phat + omega shat; r = s - omega t; ||r||^2 and the next rho = <rhat, r>
// with beta; the last block sets S_STOP on ||r|| <= tol ||f|| (slot S_TOLS), a
// breakdown flag or a non-finite residual.  DOT: omega = <t, s> / <t, t> from the
// operator's partial sums (oparts, no blocks), computed by every block with
// bicg_omega's arithmetic and stored (with its flags) by block 0
template <bool DOT>
__global__ void __launch_bounds__(kB32Threads, 4) k32_xr(float2* __restrict__ xl, float2* __restrict__ r,
                                                      const float2* __restrict__ phat, const float2* __restrict__ shat,
                                                      const float2* __restrict__ s, const float2* __restrict__ t,
                                                      const float2* __restrict__ rhat, double2* sc, long long N,
                                                      double* parts, unsigned* counter, const float* oparts, int no) {
    // the scalars in one thread, shared with the block (FP64 division is slow here)
    __shared__ float2 s_alpha, s_omega;
    __shared__ int s_skip;
    float d[3] = {0.f, 0.f, 0.f};
    const bool stop = stopped(sc);
    if (DOT && !stop) all_blocks_sum<3>(oparts, no, d);
    if (threadIdx.x == 0) {
        bool skip = stop || sc[S_FLAGS].y == 1.0;
        double2 omega64 = sc[S_OMEGA];
        if (DOT && !stop) {
            const double2 ts = make_double2(d[0], d[1]);
            const double tt = d[2];
            double flag = 0.0;
            if (sc[S_FLAGS].x != 0) {
                omega64 = make_double2(0, 0);
            } else if (tt == 0) {
                flag = 1.0;
                omega64 = make_double2(0, 0);
            } else {
                omega64 = make_double2(ts.x / tt, ts.y / tt);
                if (omega64.x == 0 && omega64.y == 0) flag = 2.0;   // breakdown after this update
            }
            if (flag == 1.0) skip = true;
            if (blockIdx.x == 0) {
                sc[S_TS] = ts;
                sc[S_TT] = make_double2(tt, 0);
                sc[S_OMEGA] = omega64;
                if (flag != 0.0) sc[S_FLAGS].y = flag;
            }
        }
        s_alpha = tof(sc[S_ALPHA]);
        s_omega = tof(omega64);
        s_skip = skip ? 1 : 0;
    }
    __syncthreads();
    const bool skip = s_skip != 0;
    float rn = 0.f, re = 0.f, im = 0.f;
    if (!skip) {
        const float2 alpha = s_alpha, omega = s_omega;
        for_pairs(N, [&](long long q, bool half) {
            const float4 xx = ld2(xl, q, half), ph = ld2(phat, q, half), sh = ld2(shat, q, half);
            const float4 ss = ld2(s, q, half), tt = ld2(t, q, half), rh = ld2(rhat, q, half);
            const float2 xa = caddf(caddf(lo(xx), cmulf(alpha, lo(ph))), cmulf(omega, lo(sh)));
            const float2 xb = caddf(caddf(hi(xx), cmulf(alpha, hi(ph))), cmulf(omega, hi(sh)));
            st2(xl, q, half, pack(xa, xb));
            const float2 ra = csubf(lo(ss), cmulf(omega, lo(tt)));
            const float2 rb = csubf(hi(ss), cmulf(omega, hi(tt)));
            st2(r, q, half, pack(ra, rb));
            nrmacc(ra, rn);
            nrmacc(rb, rn);
            cdotacc(lo(rh), ra, re, im);
            cdotacc(hi(rh), rb, re, im);
        });
    }
    const double a0 = block_sum32(rn), a1 = block_sum32(re), a2 = block_sum32(im);
    if (threadIdx.x == 0) {
        parts[3 * blockIdx.x] = a0;
        parts[3 * blockIdx.x + 1] = a1;
        parts[3 * blockIdx.x + 2] = a2;
    }
    if (last_block_done(counter, gridDim.x)) {
        double tot[3];
        sum_parts<3>(parts, gridDim.x, threadIdx.x, tot);
        if (threadIdx.x == 0) {
            if (!skip) {
                bicg_rnorm(sc, tot[0]);
                bicg_rho_beta(sc, make_double2(tot[1], tot[2]), 3.0);
            }
            if (!stopped(sc)) {
                const double rn = sqrt(sc[S_RN2].x);
                if (sc[S_FLAGS].y != 0.0 || !isfinite(rn) || rn <= sc[S_TOLS].x) sc[S_STOP].x = 1.0;
            }
            *counter = 0;
        }
    }
}

// reliable update, first half: x += xl (FP64), xl = 0; drop = 1 discards the increment
// mode 0: x += xl, xl = 0 (fold); 1: xl = 0 (drop); 2: x += xl, xl kept (trial
// fold); 3: x -= xl, xl = 0 (undo a trial fold)
__global__ void __launch_bounds__(kB32Threads) k32_fold(double2* __restrict__ x, float2* __restrict__ xl, long long N,
                                                        int mode) {
    for (long long l = blockIdx.x * (long long)kB32Threads + threadIdx.x; l < N;
         l += (long long)gridDim.x * kB32Threads) {
        if (mode != 1) {
            const float2 d = xl[l];
            const double2 xv = x[l];
            x[l] = mode == 3 ? make_double2(xv.x - (double)d.x, xv.y - (double)d.y)
                             : make_double2(xv.x + (double)d.x, xv.y + (double)d.y);
        }
        if (mode != 2) xl[l] = make_float2(0.f, 0.f);
    }
}

// reliable update, second half: r = complex64(r64); with restart = 1 also rhat = r,
// p = v = 0 and the scalars reset (a fresh start); then rho = <rhat, r> and beta in
// the last block (flag 1 on rho = 0)
__global__ void __launch_bounds__(kB32Threads) k32_replace(const double2* __restrict__ r64, float2* __restrict__ r,
                                                           float2* __restrict__ rhat, float2* __restrict__ p,
                                                           float2* __restrict__ v, int restart, double2* sc,
                                                           long long N, double* parts, unsigned* counter) {
    float re = 0.f, im = 0.f;
    for (long long l = blockIdx.x * (long long)kB32Threads + threadIdx.x; l < N;
         l += (long long)gridDim.x * kB32Threads) {
        const float2 q = tof(r64[l]);
        r[l] = q;
        float2 h;
        if (restart) {
            rhat[l] = q;
            p[l] = make_float2(0.f, 0.f);
            v[l] = make_float2(0.f, 0.f);
            h = q;
        } else {
            h = rhat[l];
        }
        cdotacc(h, q, re, im);
    }
    const double a0 = block_sum32(re), a1 = block_sum32(im);
    if (threadIdx.x == 0) {
        parts[2 * blockIdx.x] = a0;
        parts[2 * blockIdx.x + 1] = a1;
    }
    if (last_block_done(counter, gridDim.x)) {
        double tot[2];
        sum_parts<2>(parts, gridDim.x, threadIdx.x, tot);
        if (threadIdx.x == 0) {
            if (restart) {
                sc[S_RHO_OLD] = make_double2(1, 0);
                sc[S_ALPHA] = make_double2(1, 0);
                sc[S_OMEGA] = make_double2(1, 0);
            }
            sc[S_FLAGS] = make_double2(0, 0);
            sc[S_STOP] = make_double2(0, 0);
            bicg_rho_beta(sc, make_double2(tot[0], tot[1]), 1.0);
            *counter = 0;
        }
    }
}

__global__ void k32_set_tol(double2* sc, double tol_abs) { sc[S_TOLS] = make_double2(tol_abs, 0.0); }

}  // namespace

int bicg32_blocks() {
    static int nb = 0;
    if (nb == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        nb = 4 * (sms > 0 ? sms : 152);
    }
    return nb;
}

void launch_b32_update_p(const float2* r, const float2* v, float2* p, const double2* sc, long long N, cudaStream_t s) {
    k32_update_p<<<bicg32_blocks(), kB32Threads, 0, s>>>(r, v, p, sc, N);
}
void launch_b32_alpha(const float2* rhat, const float2* v, double2* sc, long long N, double* parts, unsigned* counter,
                      cudaStream_t s) {
    k32_alpha<<<bicg32_blocks(), kB32Threads, 0, s>>>(rhat, v, sc, N, parts, counter);
}
void launch_b32_s(const float2* r, const float2* v, float2* sv, double2* sc, long long N, double* parts,
                  unsigned* counter, cudaStream_t s) {
    k32_s<false><<<bicg32_blocks(), kB32Threads, 0, s>>>(r, v, sv, sc, N, parts, counter, nullptr, 0);
}
void launch_b32_s_dot(const float2* r, const float2* v, float2* sv, double2* sc, long long N, double* parts,
                      unsigned* counter, const float* aparts, int na, cudaStream_t s) {
    k32_s<true><<<bicg32_blocks(), kB32Threads, 0, s>>>(r, v, sv, sc, N, parts, counter, aparts, na);
}
void launch_b32_set_tol(double2* sc, double tol_abs, cudaStream_t s) { k32_set_tol<<<1, 1, 0, s>>>(sc, tol_abs); }
void launch_b32_omega(const float2* t, const float2* sv, double2* sc, long long N, double* parts, unsigned* counter,
                      cudaStream_t s) {
    k32_omega<<<bicg32_blocks(), kB32Threads, 0, s>>>(t, sv, sc, N, parts, counter);
}
void launch_b32_xr(float2* xl, float2* r, const float2* phat, const float2* shat, const float2* sv, const float2* t,
                   const float2* rhat, double2* sc, long long N, double* parts, unsigned* counter, cudaStream_t s) {
    k32_xr<false><<<bicg32_blocks(), kB32Threads, 0, s>>>(xl, r, phat, shat, sv, t, rhat, sc, N, parts, counter,
                                                          nullptr, 0);
}
void launch_b32_xr_dot(float2* xl, float2* r, const float2* phat, const float2* shat, const float2* sv,
                       const float2* t, const float2* rhat, double2* sc, long long N, double* parts, unsigned* counter,
                       const float* oparts, int no, cudaStream_t s) {
    k32_xr<true><<<bicg32_blocks(), kB32Threads, 0, s>>>(xl, r, phat, shat, sv, t, rhat, sc, N, parts, counter,
                                                         oparts, no);
}
void launch_b32_fold(double2* x, float2* xl, long long N, cudaStream_t s, int mode) {
    k32_fold<<<bicg32_blocks(), kB32Threads, 0, s>>>(x, xl, N, mode);
}
void launch_b32_replace(const double2* r64, float2* r, float2* rhat, float2* p, float2* v, int restart, double2* sc,
                        long long N, double* parts, unsigned* counter, cudaStream_t s) {
    k32_replace<<<bicg32_blocks(), kB32Threads, 0, s>>>(r64, r, rhat, p, v, restart, sc, N, parts, counter);
}

}  // namespace helm
