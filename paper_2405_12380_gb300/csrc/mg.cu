// Grid transfers of the geometric multigrid V-cycle (Sec. 4.3, DeepONet-MG).
//
// Vertex-centred coarsening: coarse node I sits at fine node 2I (n_f = 2 n_c - 1).
// Restriction is full weighting, the transpose of (bi/tri)linear interpolation
// divided by 2^d: weights 1/4, 1/2, 1/4 along each axis.  Coarse right-hand sides
// are zero on masked coarse nodes (the outer ring of the coarse grid is masked, so
// the 3^d fine neighbours of every unmasked coarse node exist).  Prolongation adds
// the interpolated coarse correction on unmasked fine nodes only.
#include "helm_internal.cuh"

namespace helm {

namespace {

template <typename C> struct Zero;
template <> struct Zero<double2> { __device__ static double2 v() { return make_double2(0.0, 0.0); } };
template <> struct Zero<float2> { __device__ static float2 v() { return make_float2(0.f, 0.f); } };

__device__ __forceinline__ double2 axpy_c(double w, double2 a, double2 acc) {
    return make_double2(fma(w, a.x, acc.x), fma(w, a.y, acc.y));
}
__device__ __forceinline__ float2 axpy_c(float w, float2 a, float2 acc) {
    return make_float2(fmaf(w, a.x, acc.x), fmaf(w, a.y, acc.y));
}

template <typename T>
__global__ void k_inject(int dim, int nf, const T* __restrict__ fine, T* __restrict__ coarse) {
    const int nc = (nf + 1) / 2;
    const long long Nc = dim == 3 ? (long long)nc * nc * nc : (long long)nc * nc;
    for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < Nc;
         L += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(L % nc), J = (int)((L / nc) % nc), K = dim == 3 ? (int)(L / ((long long)nc * nc)) : 0;
        const long long l = 2LL * I + (long long)nf * (2LL * J + (long long)nf * 2LL * K);
        coarse[L] = fine[l];
    }
}

// r_c(I) = sum over the 3^d fine nodes 2I + delta of prod_a w(delta_a) r_f, w(0) = 1/2,
// w(+-1) = 1/4; zero on masked coarse nodes
template <typename R>
__global__ void k_restrict_fw(int dim, int nf, const typename CT<R>::T* __restrict__ rf,
                              const uint8_t* __restrict__ mask_c, typename CT<R>::T* __restrict__ rc) {
    using C = typename CT<R>::T;
    const int nc = (nf + 1) / 2;
    const long long Nc = dim == 3 ? (long long)nc * nc * nc : (long long)nc * nc;
    const R w1[3] = {(R)0.25, (R)0.5, (R)0.25};
    for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < Nc;
         L += (long long)gridDim.x * blockDim.x) {
        if (mask_c[L]) {
            rc[L] = Zero<C>::v();
            continue;
        }
        const int I = (int)(L % nc), J = (int)((L / nc) % nc), K = dim == 3 ? (int)(L / ((long long)nc * nc)) : 0;
        C acc = Zero<C>::v();
        const int kz0 = dim == 3 ? -1 : 0, kz1 = dim == 3 ? 1 : 0;
        for (int dz = kz0; dz <= kz1; ++dz) {
            const R wz = dim == 3 ? w1[dz + 1] : (R)1;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const long long l = (2LL * I + dx) + (long long)nf * ((2LL * J + dy) + (long long)nf * (2LL * K + dz));
                    acc = axpy_c(wz * w1[dy + 1] * w1[dx + 1], rf[l], acc);
                }
        }
        rc[L] = acc;
    }
}

// z_f += P z_c on unmasked fine nodes: along each axis an even index takes coarse
// node i/2 (weight 1), an odd one the two coarse nodes around it (1/2 each)
template <typename R>
__global__ void k_prolong_add(int dim, int nf, const typename CT<R>::T* __restrict__ zc,
                              const uint8_t* __restrict__ mask_f, typename CT<R>::T* __restrict__ zf) {
    using C = typename CT<R>::T;
    const int nc = (nf + 1) / 2;
    const long long Nf = dim == 3 ? (long long)nf * nf * nf : (long long)nf * nf;
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < Nf;
         l += (long long)gridDim.x * blockDim.x) {
        if (mask_f[l]) continue;
        const int i = (int)(l % nf), j = (int)((l / nf) % nf), k = dim == 3 ? (int)(l / ((long long)nf * nf)) : 0;
        int ci[3][2], nci[3];
        R cw[3][2];
        const int idx[3] = {i, j, k};
        for (int a = 0; a < 3; ++a) {
            if (a == 2 && dim == 2) {
                ci[a][0] = 0; cw[a][0] = (R)1; nci[a] = 1;
            } else if ((idx[a] & 1) == 0) {
                ci[a][0] = idx[a] >> 1; cw[a][0] = (R)1; nci[a] = 1;
            } else {
                ci[a][0] = idx[a] >> 1; ci[a][1] = (idx[a] >> 1) + 1;
                cw[a][0] = (R)0.5; cw[a][1] = (R)0.5; nci[a] = 2;
            }
        }
        C acc = Zero<C>::v();
        for (int c = 0; c < nci[2]; ++c)
            for (int b = 0; b < nci[1]; ++b)
                for (int a = 0; a < nci[0]; ++a) {
                    const long long L = ci[0][a] + (long long)nc * (ci[1][b] + (long long)nc * ci[2][c]);
                    acc = axpy_c(cw[0][a] * cw[1][b] * cw[2][c], zc[L], acc);
                }
        C out = zf[l];
        out.x += acc.x;
        out.y += acc.y;
        zf[l] = out;
    }
}

}  // namespace

void launch_inject_mask(int dim, int nf, const uint8_t* fine, uint8_t* coarse, cudaStream_t s) {
    k_inject<uint8_t><<<4 * 152, 256, 0, s>>>(dim, nf, fine, coarse);
}
void launch_inject_c128(int dim, int nf, const double2* fine, double2* coarse, cudaStream_t s) {
    k_inject<double2><<<4 * 152, 256, 0, s>>>(dim, nf, fine, coarse);
}
template <typename R>
void launch_restrict_fw(int dim, int nf, const typename CT<R>::T* rf, const uint8_t* mask_c, typename CT<R>::T* rc,
                        cudaStream_t s) {
    k_restrict_fw<R><<<4 * 152, 256, 0, s>>>(dim, nf, rf, mask_c, rc);
}
template <typename R>
void launch_prolong_add(int dim, int nf, const typename CT<R>::T* zc, const uint8_t* mask_f, typename CT<R>::T* zf,
                        cudaStream_t s) {
    k_prolong_add<R><<<4 * 152, 256, 0, s>>>(dim, nf, zc, mask_f, zf);
}
template void launch_restrict_fw<double>(int, int, const double2*, const uint8_t*, double2*, cudaStream_t);
template void launch_restrict_fw<float>(int, int, const float2*, const uint8_t*, float2*, cudaStream_t);
template void launch_prolong_add<double>(int, int, const double2*, const uint8_t*, double2*, cudaStream_t);
template void launch_prolong_add<float>(int, int, const float2*, const uint8_t*, float2*, cudaStream_t);

}  // namespace helm
