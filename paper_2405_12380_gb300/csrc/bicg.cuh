// BiCGStab scalar recurrences and the "last block done" reduction pattern, shared
// by the fused vector kernels (blas.cu) and the fused operator kernels (stencil.cu).
//
// A fused kernel writes one partial per block, fences, and counts finished blocks
// with an atomic; the last block to finish sums all partials in a fixed order
// (deterministic) and applies the scalar recurrence, so a reduction and its scalar
// update cost no extra launch.
#pragma once

#include "helm_internal.cuh"

namespace helm {

constexpr int kFusedThreads = 256;

// true in exactly one block: the last one to finish writing its partials
__device__ __forceinline__ bool last_block_done(unsigned* counter, unsigned nblocks) {
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const unsigned t = atomicAdd(counter, 1u);
        s_last = (t == nblocks - 1);
    }
    __syncthreads();
    return s_last;
}

// fixed-order sum of nparts partials of W doubles (stride W) by a block of
// kFusedThreads threads (flat thread index tid); result valid in tid 0
template <int W>
__device__ __forceinline__ void sum_parts(const double* parts, int nparts, int tid, double* out) {
    __shared__ double red[W][kFusedThreads / 32];
    double v[W];
#pragma unroll
    for (int q = 0; q < W; ++q) v[q] = 0.0;
    for (int b = tid; b < nparts; b += kFusedThreads)
#pragma unroll
        for (int q = 0; q < W; ++q) v[q] += __ldcg(parts + (long long)b * W + q);
#pragma unroll
    for (int q = 0; q < W; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if ((tid & 31) == 0)
#pragma unroll
        for (int q = 0; q < W; ++q) red[q][tid >> 5] = v[q];
    __syncthreads();
    if (tid == 0)
#pragma unroll
        for (int q = 0; q < W; ++q) {
            double s = 0.0;
            for (int w = 0; w < kFusedThreads / 32; ++w) s += red[q][w];
            out[q] = s;
        }
}

// --- recurrences (one thread), slots S_* of helm_internal.cuh ----------------
// rho = <rhat, r>, beta = (rho / rho_old)(alpha / omega); flag value on rho == 0
__device__ __forceinline__ void bicg_rho_beta(double2* sc, double2 rho, double flag) {
    sc[S_RHO] = rho;
    if (rho.x == 0 && rho.y == 0) sc[S_FLAGS].y = flag;
    sc[S_BETA] = cmul(cdiv(rho, sc[S_RHO_OLD]), cdiv(sc[S_ALPHA], sc[S_OMEGA]));
    sc[S_FLAGS].x = 0;
}
// alpha = rho / <rhat, v>
__device__ __forceinline__ void bicg_alpha(double2* sc, double2 d) {
    if (d.x == 0 && d.y == 0) {
        sc[S_FLAGS].y = 1;
        sc[S_ALPHA] = make_double2(0, 0);
    } else {
        sc[S_ALPHA] = cdiv(sc[S_RHO], d);
    }
}
// ||s||^2; ||s|| <= tol_abs ends the iteration after x += alpha phat
__device__ __forceinline__ void bicg_snorm(double2* sc, double v, double tol_abs) {
    sc[S_SN2] = make_double2(v, 0);
    if (sqrt(v) <= tol_abs) sc[S_FLAGS].x = 1;
}
// omega = <t, s> / <t, t>
__device__ __forceinline__ void bicg_omega(double2* sc, double2 ts, double tt) {
    sc[S_TS] = ts;
    sc[S_TT] = make_double2(tt, 0);
    if (sc[S_FLAGS].x != 0) {
        sc[S_OMEGA] = make_double2(0, 0);
    } else if (tt == 0) {
        sc[S_FLAGS].y = 1;
        sc[S_OMEGA] = make_double2(0, 0);
    } else {
        const double2 om = make_double2(ts.x / tt, ts.y / tt);
        sc[S_OMEGA] = om;
        if (om.x == 0 && om.y == 0) sc[S_FLAGS].y = 2;   // breakdown after this update
    }
}
// ||r||^2 after the update; rho_old = rho unless the iteration ended early
__device__ __forceinline__ void bicg_rnorm(double2* sc, double v) {
    sc[S_RN2] = make_double2(v, 0);
    if (sc[S_FLAGS].x == 0) sc[S_RHO_OLD] = sc[S_RHO];
}

}  // namespace helm
