// Receiver sampling, its transpose and the k^2 gradient of the adjoint method.
//
// Receivers sample u by trilinear interpolation of the 8 nodes of their grid
// cell; the transpose scatters receiver values back onto those nodes.  With
// conj(A) lambda = S^T G (A^H = conj(A)), the gradient of a real loss with
// respect to the per-node complex k^2 is -lambda conj(u) on fluid nodes.
#include "helm_internal.cuh"

namespace helm {
namespace {

__global__ void k_receivers_setup(int n, int nrec, const double* __restrict__ xyz, int* __restrict__ idx,
                                  double* __restrict__ w) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrec) return;
    const double h = 1.0 / (n - 1);
    int c[3];
    double t[3];
    for (int a = 0; a < 3; ++a) {
        const double s = xyz[3 * r + a] / h;
        int ci = (int)floor(s);
        ci = min(ci, n - 2);
        ci = max(ci, 0);
        c[a] = ci;
        t[a] = s - ci;
    }
    int q = 0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                const double wx = dx ? t[0] : 1 - t[0];
                const double wy = dy ? t[1] : 1 - t[1];
                const double wz = dz ? t[2] : 1 - t[2];
                w[8 * r + q] = wx * wy * wz;
                idx[8 * r + q] = (c[0] + dx) + n * ((c[1] + dy) + n * (c[2] + dz));
                ++q;
            }
}

__global__ void k_receivers_sample(int nrec, const int* __restrict__ idx, const double* __restrict__ w,
                                   const double2* __restrict__ u, double2* __restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrec) return;
    double2 s = make_double2(0, 0);
    for (int q = 0; q < 8; ++q) {
        const double2 v = u[idx[8 * r + q]];
        s.x += w[8 * r + q] * v.x;
        s.y += w[8 * r + q] * v.y;
    }
    out[r] = s;
}

// b = S^T e on a zeroed b; one thread in a fixed order (deterministic)
__global__ void k_receivers_adjoint(int nrec, const int* __restrict__ idx, const double* __restrict__ w,
                                    const double2* __restrict__ e, double2* __restrict__ b) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int r = 0; r < nrec; ++r)
        for (int q = 0; q < 8; ++q) {
            const int l = idx[8 * r + q];
            b[l].x += w[8 * r + q] * e[r].x;
            b[l].y += w[8 * r + q] * e[r].y;
        }
}

__global__ void k_k2_gradient(long long N, const uint8_t* __restrict__ mask, const double2* __restrict__ lam,
                              const double2* __restrict__ u, double2* __restrict__ g) {
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < N; l += (long long)gridDim.x * blockDim.x) {
        if (mask[l]) {
            g[l] = make_double2(0, 0);
        } else {
            const double2 a = lam[l], c = u[l];
            // -lambda * conj(u)
            g[l] = make_double2(-(a.x * c.x + a.y * c.y), -(a.y * c.x - a.x * c.y));
        }
    }
}

}  // namespace

void launch_receivers_setup(int n, int nrec, const double* xyz, int* idx, double* w, cudaStream_t s) {
    k_receivers_setup<<<(nrec + 127) / 128, 128, 0, s>>>(n, nrec, xyz, idx, w);
}
void launch_receivers_sample(int nrec, const int* idx, const double* w, const double2* u, double2* out,
                             cudaStream_t s) {
    k_receivers_sample<<<(nrec + 127) / 128, 128, 0, s>>>(nrec, idx, w, u, out);
}
void launch_receivers_adjoint(int nrec, const int* idx, const double* w, const double2* e, double2* b,
                              cudaStream_t s) {
    k_receivers_adjoint<<<1, 32, 0, s>>>(nrec, idx, w, e, b);
}
void launch_k2_gradient(long long N, const uint8_t* mask, const double2* lam, const double2* u, double2* g,
                        cudaStream_t s) {
    k_k2_gradient<<<4 * 152, 256, 0, s>>>(N, mask, lam, u, g);
}

}  // namespace helm
