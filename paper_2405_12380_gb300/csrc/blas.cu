// Fused BLAS-1 and the scalar recurrences of BiCGStab and FGMRES.
//
// Reductions are deterministic: a fixed grid of kRedBlocks blocks writes one
// partial per block, and a single block sums the partials in a fixed order.
// Scalars (rho, alpha, omega, beta, norms, Hessenberg columns, Givens
// rotations) stay in device memory; the host only reads a status word.
#include "bicg.cuh"
#include "helm_internal.cuh"

namespace helm {

namespace {

constexpr int TB = 256;

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double2 warp_sum(double2 v) {
    v.x = warp_sum(v.x);
    v.y = warp_sum(v.y);
    return v;
}

// block-wide sum (TB threads); result valid in thread 0
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[TB / 32];
    v = warp_sum(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < TB / 32 ? red[lane] : 0.0;
        v = warp_sum(v);
    }
    return v;
}
__device__ __forceinline__ double2 block_sum(double2 v) {
    double a = block_sum(v.x);
    double b = block_sum(v.y);
    return make_double2(a, b);
}

__global__ void __launch_bounds__(TB) k_dot(const double2* __restrict__ a, const double2* __restrict__ b,
                                            long long N, double2* partials) {
    double2 acc = make_double2(0, 0);
    for (long long l = blockIdx.x * (long long)TB + threadIdx.x; l < N; l += (long long)gridDim.x * TB) {
        double2 u = a[l], v = b[l];
        acc.x += u.x * v.x + u.y * v.y;
        acc.y += u.x * v.y - u.y * v.x;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(TB) k_norm2(const double2* __restrict__ a, long long N, double* partials) {
    double acc = 0;
    for (long long l = blockIdx.x * (long long)TB + threadIdx.x; l < N; l += (long long)gridDim.x * TB) {
        double2 u = a[l];
        acc += u.x * u.x + u.y * u.y;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// fixed-order sum of partials by one block of kFinThreads threads
template <typename T>
__device__ __forceinline__ T fin_sum(const T* partials, int nparts);

__device__ __forceinline__ double fin_sum_d(const double* p, int nparts) {
    __shared__ double red[kFinThreads / 32];
    double v = 0;
    for (int i = threadIdx.x; i < nparts; i += kFinThreads) v += p[i];
    v = warp_sum(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = red[lane];
        v = warp_sum(v);
    }
    __syncthreads();
    return v;  // valid in thread 0
}

__device__ __forceinline__ double2 fin_sum_c(const double2* p, int nparts, int stride = 1, int offset = 0) {
    __shared__ double2 red[kFinThreads / 32];
    double2 v = make_double2(0, 0);
    for (int i = threadIdx.x; i < nparts; i += kFinThreads) {
        double2 q = p[(long long)i * stride + offset];
        v.x += q.x;
        v.y += q.y;
    }
    v = warp_sum(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = red[lane];
        v = warp_sum(v);
    }
    __syncthreads();
    return v;
}

__global__ void __launch_bounds__(kFinThreads) k_sum_real(const double* partials, int nparts, double* out) {
    double v = fin_sum_d(partials, nparts);
    if (threadIdx.x == 0) *out = v;
}
// ---------------------------------------------------------------- BiCGStab

__global__ void __launch_bounds__(TB) k_bicg_p(const double2* __restrict__ r, const double2* __restrict__ v,
                                               double2* __restrict__ p, const double2* __restrict__ sc, long long N) {
    const double2 beta = sc[S_BETA], omega = sc[S_OMEGA];
    for (long long l = blockIdx.x * (long long)TB + threadIdx.x; l < N; l += (long long)gridDim.x * TB) {
        double2 t = csub(p[l], cmul(omega, v[l]));
        p[l] = cadd(r[l], cmul(beta, t));
    }
}

// s = r - alpha v with ||s||^2, the scalar update in the last block
__global__ void __launch_bounds__(kFusedThreads) k_bicg_s_fused(const double2* __restrict__ r, const double2* __restrict__ v,
                                                                double2* __restrict__ s, double2* sc, long long N,
                                                                double* parts, unsigned* counter, double tol_abs) {
    const double2 alpha = sc[S_ALPHA];
    double acc = 0;
    for (long long l = blockIdx.x * (long long)kFusedThreads + threadIdx.x; l < N; l += (long long)gridDim.x * kFusedThreads) {
        const double2 q = csub(r[l], cmul(alpha, v[l]));
        s[l] = q;
        acc += q.x * q.x + q.y * q.y;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) parts[blockIdx.x] = acc;
    if (last_block_done(counter, gridDim.x)) {
        double tot[1];
        sum_parts<1>(parts, gridDim.x, threadIdx.x, tot);
        if (threadIdx.x == 0) {
            bicg_snorm(sc, tot[0], tol_abs);
            *counter = 0;
        }
    }
}

// x += alpha phat + omega shat; r = s - omega t; ||r||^2 and the next rho = <rhat, r>
// with beta, in the last block (breakdown flag 3: rho = 0 for the next iteration)
__global__ void __launch_bounds__(kFusedThreads) k_bicg_xr_fused(double2* __restrict__ x, double2* __restrict__ r,
                                                                 const double2* __restrict__ phat,
                                                                 const double2* __restrict__ shat,
                                                                 const double2* __restrict__ s,
                                                                 const double2* __restrict__ t,
                                                                 const double2* __restrict__ rhat, double2* sc,
                                                                 long long N, double* parts, unsigned* counter,
                                                                 double tol, double bnorm) {
    const double2 alpha = sc[S_ALPHA], omega = sc[S_OMEGA];
    const bool skip = sc[S_FLAGS].y == 1.0 || sc[S_STOP].x != 0.0;
    double rn = 0;
    double2 rho = make_double2(0, 0);
    for (long long l = blockIdx.x * (long long)kFusedThreads + threadIdx.x; l < N && !skip;
         l += (long long)gridDim.x * kFusedThreads) {
        double2 xv = cadd(x[l], cmul(alpha, phat[l]));
        xv = cadd(xv, cmul(omega, shat[l]));
        x[l] = xv;
        const double2 q = csub(s[l], cmul(omega, t[l]));
        r[l] = q;
        rn += q.x * q.x + q.y * q.y;
        const double2 h = rhat[l];
        rho.x += h.x * q.x + h.y * q.y;
        rho.y += h.x * q.y - h.y * q.x;
    }
    rn = block_sum(rn);
    rho = block_sum(rho);
    if (threadIdx.x == 0) {
        parts[3 * blockIdx.x + 0] = rn;
        parts[3 * blockIdx.x + 1] = rho.x;
        parts[3 * blockIdx.x + 2] = rho.y;
    }
    if (last_block_done(counter, gridDim.x)) {
        double tot[3];
        sum_parts<3>(parts, gridDim.x, threadIdx.x, tot);
        if (threadIdx.x == 0) {
            if (!skip) {
                bicg_rnorm(sc, tot[0]);
                bicg_rho_beta(sc, make_double2(tot[1], tot[2]), 3.0);
            }
            if (sc[S_STOP].x == 0.0) {
                const double res = sqrt(sc[S_RN2].x) / bnorm;
                if (sc[S_FLAGS].y != 0.0 || !isfinite(res) || res <= tol) sc[S_STOP].x = 1.0;
            }
            *counter = 0;
        }
    }
}

// recipes: 0 = rho & beta (complex partials), 1 = alpha, 2 = ||s||^2, 3 = omega, 4 = ||r||^2, 5 = reset
__global__ void __launch_bounds__(kFinThreads) k_bicg_scalar(int recipe, const double* partials, int nparts,
                                                             double2* sc, double tol_abs) {
    if (recipe == 0 || recipe == 1) {
        double2 d = fin_sum_c(reinterpret_cast<const double2*>(partials), nparts);
        if (threadIdx.x != 0) return;
        if (recipe == 0) {
            sc[S_RHO] = d;
            if (d.x == 0 && d.y == 0) sc[S_FLAGS].y = 1;
            double2 q = cmul(cdiv(d, sc[S_RHO_OLD]), cdiv(sc[S_ALPHA], sc[S_OMEGA]));
            sc[S_BETA] = q;
            sc[S_FLAGS].x = 0;
        } else {
            if (d.x == 0 && d.y == 0) {
                sc[S_FLAGS].y = 1;
                sc[S_ALPHA] = make_double2(0, 0);
            } else {
                sc[S_ALPHA] = cdiv(sc[S_RHO], d);
            }
        }
    } else if (recipe == 2 || recipe == 4) {
        double v = fin_sum_d(partials, nparts);
        if (threadIdx.x != 0) return;
        if (recipe == 2) {
            sc[S_SN2] = make_double2(v, 0);
            if (sqrt(v) <= tol_abs) sc[S_FLAGS].x = 1;
        } else {
            sc[S_RN2] = make_double2(v, 0);
            if (sc[S_FLAGS].x == 0) sc[S_RHO_OLD] = sc[S_RHO];
        }
    } else if (recipe == 3) {
        double2 ts = fin_sum_c(reinterpret_cast<const double2*>(partials), nparts, 2, 0);
        double2 tt = fin_sum_c(reinterpret_cast<const double2*>(partials), nparts, 2, 1);
        if (threadIdx.x != 0) return;
        sc[S_TS] = ts;
        sc[S_TT] = tt;
        if (sc[S_FLAGS].x != 0) {
            sc[S_OMEGA] = make_double2(0, 0);
        } else if (tt.x == 0) {
            sc[S_FLAGS].y = 1;
            sc[S_OMEGA] = make_double2(0, 0);
        } else {
            double2 om = make_double2(ts.x / tt.x, ts.y / tt.x);
            sc[S_OMEGA] = om;
            if (om.x == 0 && om.y == 0) sc[S_FLAGS].y = 2;   // breakdown after this update
        }
    } else if (recipe == 5) {
        if (threadIdx.x != 0) return;
        sc[S_RHO_OLD] = make_double2(1, 0);
        sc[S_ALPHA] = make_double2(1, 0);
        sc[S_OMEGA] = make_double2(1, 0);
        sc[S_FLAGS] = make_double2(0, 0);
        sc[S_STOP] = make_double2(0, 0);
    }
}

// ------------------------------------------------------------------ FGMRES
constexpr int MD_TILE = 512;

// partials[b * nv + i] = sum over this block's tiles of conj(V_i) . w
__global__ void __launch_bounds__(TB) k_mdot(const double2* __restrict__ V, int nv, const double2* __restrict__ w,
                                             long long N, double2* partials) {
    __shared__ double2 ws[MD_TILE];
    __shared__ double2 acc[kMaxRestart + 1];
    for (int i = threadIdx.x; i < nv; i += TB) acc[i] = make_double2(0, 0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long t0 = (long long)blockIdx.x * MD_TILE; t0 < N; t0 += (long long)gridDim.x * MD_TILE) {
        const int rows = (int)min((long long)MD_TILE, N - t0);
        __syncthreads();
        for (int r = threadIdx.x; r < rows; r += TB) ws[r] = w[t0 + r];
        __syncthreads();
        for (int i = warp; i < nv; i += TB / 32) {
            const double2* Vi = V + (long long)i * N + t0;
            double2 a = make_double2(0, 0);
            for (int r = lane; r < rows; r += 32) {
                double2 u = Vi[r], b = ws[r];
                a.x += u.x * b.x + u.y * b.y;
                a.y += u.x * b.y - u.y * b.x;
            }
            a = warp_sum(a);
            if (lane == 0) acc[i] = cadd(acc[i], a);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nv; i += TB) partials[(long long)blockIdx.x * nv + i] = acc[i];
}

// out[i] (+)= sum_b partials[b * nv + i]; one warp per vector, fixed order
__global__ void k_mdot_fin(const double2* __restrict__ partials, int nparts, int nv, double2* out, int accumulate,
                           double2* copy) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < nv; i += blockDim.x / 32) {
        double2 a = make_double2(0, 0);
        for (int b = lane; b < nparts; b += 32) a = cadd(a, partials[(long long)b * nv + i]);
        a = warp_sum(a);
        if (lane == 0) {
            if (copy) copy[i] = a;
            out[i] = accumulate ? cadd(out[i], a) : a;
        }
    }
}

// w += sign * sum_i V_i coef_i; optional ||w||^2 partials
__global__ void __launch_bounds__(TB) k_mupdate(const double2* __restrict__ V, int nv, const double2* __restrict__ coef,
                                                double sign, double2* __restrict__ w, long long N, double* partials) {
    __shared__ double2 c[kMaxRestart + 1];
    for (int i = threadIdx.x; i < nv; i += TB) c[i] = cscale(sign, coef[i]);
    __syncthreads();
    double acc = 0;
    for (long long l = blockIdx.x * (long long)TB + threadIdx.x; l < N; l += (long long)gridDim.x * TB) {
        double2 s = w[l];
        for (int i = 0; i < nv; ++i) {
            double2 v = V[(long long)i * N + l];
            s.x += c[i].x * v.x - c[i].y * v.y;
            s.y += c[i].x * v.y + c[i].y * v.x;
        }
        w[l] = s;
        acc += s.x * s.x + s.y * s.y;
    }
    if (partials) {
        acc = block_sum(acc);
        if (threadIdx.x == 0) partials[blockIdx.x] = acc;
    }
}

// w += sign * sum_i V_i coef_i with complex64 vectors V (FP64 accumulation)
__global__ void __launch_bounds__(TB) k_mupdate32(const float2* __restrict__ V, int nv, const double2* __restrict__ coef,
                                                  double sign, double2* __restrict__ w, long long N) {
    __shared__ double2 c[kMaxRestart + 1];
    for (int i = threadIdx.x; i < nv; i += TB) c[i] = cscale(sign, coef[i]);
    __syncthreads();
    for (long long l = blockIdx.x * (long long)TB + threadIdx.x; l < N; l += (long long)gridDim.x * TB) {
        double2 s = w[l];
        for (int i = 0; i < nv; ++i) {
            float2 vf = V[(long long)i * N + l];
            double2 v = make_double2(vf.x, vf.y);
            s.x += c[i].x * v.x - c[i].y * v.y;
            s.y += c[i].x * v.y + c[i].y * v.x;
        }
        w[l] = s;
    }
}

__global__ void __launch_bounds__(TB) k_scale_vec(const double2* __restrict__ w, double2* __restrict__ v,
                                                  const double* norm2, long long N) {
    const double nn = sqrt(*norm2);
    if (nn == 0) return;
    const double inv = 1.0 / nn;
    for (long long l = blockIdx.x * (long long)TB + threadIdx.x; l < N; l += (long long)gridDim.x * TB)
        v[l] = cscale(inv, w[l]);
}

// Givens step for column j of the Hessenberg matrix (column-major, ldh rows).
// H[0..j, j] holds h = V^H w; wnorm2 = ||w||^2 after orthogonalisation.
__global__ void k_givens(double2* H, int ldh, int j, double* cs, double2* sn, double2* g, const double* wnorm2,
                         double* est) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double2* col = H + (long long)j * ldh;
    const double hn = sqrt(*wnorm2);
    col[j + 1] = make_double2(hn, 0);
    for (int i = 0; i < j; ++i) {
        double2 a = col[i], b = col[i + 1];
        double2 s = sn[i];
        double c = cs[i];
        col[i] = cadd(cscale(c, a), cmul(s, b));
        col[i + 1] = csub(cscale(c, b), cmulc(s, a));
    }
    double2 a = col[j], b = col[j + 1];
    double c;
    double2 s, r;
    double ab = hypot(a.x, a.y), bb = hypot(b.x, b.y);
    if (bb == 0) {
        c = 1; s = make_double2(0, 0); r = a;
    } else if (ab == 0) {
        c = 0; s = make_double2(b.x / bb, -b.y / bb); r = make_double2(bb, 0);
    } else {
        double t = sqrt(ab * ab + bb * bb);
        double2 ph = make_double2(a.x / ab, a.y / ab);
        c = ab / t;
        s = cscale(1.0 / t, cmul(ph, make_double2(b.x, -b.y)));
        r = cscale(t, ph);
    }
    cs[j] = c;
    sn[j] = s;
    col[j] = r;
    col[j + 1] = make_double2(0, 0);
    double2 gj = g[j];
    g[j + 1] = cscale(-1.0, cmulc(s, gj));
    g[j] = cscale(c, gj);
    *est = hypot(g[j + 1].x, g[j + 1].y);
}

__global__ void k_hsolve(const double2* H, int ldh, int k, const double2* g, double2* y) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
        double2 s = g[i];
        for (int q = i + 1; q < k; ++q) s = csub(s, cmul(H[(long long)q * ldh + i], y[q]));
        y[i] = cdiv(s, H[(long long)i * ldh + i]);
    }
}

__global__ void k_init_g(double2* g, int m1, const double* beta2) {
    int i = threadIdx.x;
    if (i < m1) g[i] = make_double2(i == 0 ? sqrt(*beta2) : 0.0, 0);
}

__global__ void __launch_bounds__(TB) k_set_masked(double2* __restrict__ x, const double2* __restrict__ f,
                                                   const uint8_t* __restrict__ mask, long long N) {
    for (long long l = blockIdx.x * (long long)TB + threadIdx.x; l < N; l += (long long)gridDim.x * TB)
        if (mask[l]) x[l] = f[l];
}

__global__ void __launch_bounds__(TB) k_cvt64to32(const double2* __restrict__ a, float2* __restrict__ b, long long N) {
    for (long long l = blockIdx.x * (long long)TB + threadIdx.x; l < N; l += (long long)gridDim.x * TB)
        b[l] = make_float2((float)a[l].x, (float)a[l].y);
}
__global__ void __launch_bounds__(TB) k_cvt32to64(const float2* __restrict__ a, double2* __restrict__ b, long long N) {
    for (long long l = blockIdx.x * (long long)TB + threadIdx.x; l < N; l += (long long)gridDim.x * TB)
        b[l] = make_double2((double)a[l].x, (double)a[l].y);
}

int stream_blocks(long long N) {
    long long b = (N + TB - 1) / TB;
    return (int)(b < 4 * kRedBlocks ? (b < 1 ? 1 : b) : 4 * kRedBlocks);
}

}  // namespace

void launch_dot(const double2* a, const double2* b, long long N, double2* partials, cudaStream_t s) {
    k_dot<<<kRedBlocks, TB, 0, s>>>(a, b, N, partials);
}
void launch_norm2(const double2* a, long long N, double* partials, cudaStream_t s) {
    k_norm2<<<kRedBlocks, TB, 0, s>>>(a, N, partials);
}
void launch_sum_real(const double* partials, int nparts, double* out, cudaStream_t s) {
    k_sum_real<<<1, kFinThreads, 0, s>>>(partials, nparts, out);
}
void launch_bicg_update_p(const double2* r, const double2* v, double2* p, const double2* sc, long long N,
                          cudaStream_t s) {
    k_bicg_p<<<stream_blocks(N), TB, 0, s>>>(r, v, p, sc, N);
}
void launch_bicg_s_fused(const double2* r, const double2* v, double2* sv, double2* sc, long long N, double* parts,
                         unsigned* counter, double tol_abs, cudaStream_t s) {
    k_bicg_s_fused<<<kRedBlocks, kFusedThreads, 0, s>>>(r, v, sv, sc, N, parts, counter, tol_abs);
}
void launch_bicg_xr_fused(double2* x, double2* r, const double2* phat, const double2* shat, const double2* sv,
                          const double2* t, const double2* rhat, double2* sc, long long N, double* parts,
                          unsigned* counter, double tol, double bnorm, cudaStream_t s) {
    k_bicg_xr_fused<<<kRedBlocks, kFusedThreads, 0, s>>>(x, r, phat, shat, sv, t, rhat, sc, N, parts, counter, tol,
                                                         bnorm);
}
void launch_bicg_scalar(int recipe, const double* partials, int nparts, double2* sc, double tol_abs,
                        cudaStream_t s) {
    k_bicg_scalar<<<1, kFinThreads, 0, s>>>(recipe, partials, nparts, sc, tol_abs);
}
void launch_mdot(const double2* V, int nv, const double2* w, long long N, double2* partials, cudaStream_t s) {
    k_mdot<<<kRedBlocks, TB, 0, s>>>(V, nv, w, N, partials);
}
void launch_mupdate(const double2* V, int nv, const double2* coef, double sign, double2* w, long long N,
                    double* norm_partials, cudaStream_t s) {
    k_mupdate<<<norm_partials ? kRedBlocks : stream_blocks(N), TB, 0, s>>>(V, nv, coef, sign, w, N,
                                                                            norm_partials);
}
void launch_mdot_finalize(const double2* partials, int nparts, int nv, double2* out, int accumulate,
                          double2* copy, cudaStream_t s) {
    k_mdot_fin<<<1, 512, 0, s>>>(partials, nparts, nv, out, accumulate, copy);
}
void launch_mupdate32(const float2* V, int nv, const double2* coef, double sign, double2* w, long long N,
                      cudaStream_t s) {
    k_mupdate32<<<stream_blocks(N), TB, 0, s>>>(V, nv, coef, sign, w, N);
}
void launch_scale_vec(const double2* w, double2* v, const double* norm2, long long N, cudaStream_t s) {
    k_scale_vec<<<stream_blocks(N), TB, 0, s>>>(w, v, norm2, N);
}
void launch_givens(double2* H, int ldh, int j, double* cs, double2* sn, double2* g, const double* wnorm2,
                   double* est, cudaStream_t s) {
    k_givens<<<1, 32, 0, s>>>(H, ldh, j, cs, sn, g, wnorm2, est);
}
void launch_hsolve(const double2* H, int ldh, int k, const double2* g, double2* y, cudaStream_t s) {
    k_hsolve<<<1, 32, 0, s>>>(H, ldh, k, g, y);
}
void launch_init_g(double2* g, int m1, const double* beta2, cudaStream_t s) {
    k_init_g<<<1, 128, 0, s>>>(g, m1, beta2);
}
void launch_set_masked(double2* x, const double2* f, const uint8_t* mask, long long N, cudaStream_t s) {
    k_set_masked<<<stream_blocks(N), TB, 0, s>>>(x, f, mask, N);
}
void launch_cvt_f64_to_f32(const double2* a, float2* b, long long N, cudaStream_t s) {
    k_cvt64to32<<<stream_blocks(N), TB, 0, s>>>(a, b, N);
}
void launch_cvt_f32_to_f64(const float2* a, double2* b, long long N, cudaStream_t s) {
    k_cvt32to64<<<stream_blocks(N), TB, 0, s>>>(a, b, N);
}

}  // namespace helm
