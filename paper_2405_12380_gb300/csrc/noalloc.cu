// Residual and residual norm without any device allocation.
//
// Some callers cannot allocate device memory: code that runs inside a memory
// pool or arena it does not own, plugins whose host forbids cudaMalloc (which
// also synchronises the device), and code that must not touch the allocator
// between CUDA graph captures.  helm_residual_noalloc serves them: it needs no
// handle (helm_create allocates) and takes its reduction scratch from a
// file-scope device array that every GPU loading this library holds until exit.
#include <cmath>
#include <mutex>

#include "helm_internal.cuh"

using namespace helm;

namespace {

// Block partials of ||r||^2 (one double per block of the operator grid) and the
// outer-ring check flag.  512 KiB + 256 B per device, for the process lifetime.
constexpr long long kScratchDoubles = 65536;
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];
static __device__ __align__(256) int g_noalloc_flag[64];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};
int* g_flag_ptr[kMaxDevices] = {nullptr};

// Device addresses of the static arrays for the current device (set up once per device).
helm_status scratch_for_current_device(double** scratch, int** flag) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return HELM_NO_DEVICE;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* s = nullptr;
        void* f = nullptr;
        if (cudaGetSymbolAddress(&s, g_noalloc_scratch) != cudaSuccess ||
            cudaGetSymbolAddress(&f, g_noalloc_flag) != cudaSuccess) {
            cudaGetLastError();
            return HELM_CUDA_ERROR;
        }
        g_scratch_ptr[dev] = static_cast<double*>(s);
        g_flag_ptr[dev] = static_cast<int*>(f);
    }
    *scratch = g_scratch_ptr[dev];
    *flag = g_flag_ptr[dev];
    return HELM_OK;
}

}  // namespace

extern "C" helm_status helm_residual_noalloc(int dim, int n, double k0, int layer_cells, double layer_strength,
                                             const uint8_t* mask, const double* k2, const double* f,
                                             const double* x, double* r, double* norm2, int conj, void* stream) {
    if ((dim != 2 && dim != 3) || n < 3 || layer_cells < 0 || layer_cells > kMaxLayerCells || !mask || !f || !x ||
        !r || !norm2 || !std::isfinite(k0) || !std::isfinite(layer_strength))
        return HELM_BAD_ARG;
    long long N = 1;
    for (int a = 0; a < dim; ++a) N *= n;
    if (N >= (1LL << 31) || n > 65535) return HELM_BAD_ARG;
    if ((long long)apply_grid_blocks(dim, n) > kScratchDoubles) return HELM_SCRATCH_TOO_SMALL;
    double* scratch = nullptr;
    int* flag = nullptr;
    helm_status st = scratch_for_current_device(&scratch, &flag);
    if (st != HELM_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // operator tables on the host (same formulas as helm_create)
    Op<double> op{};
    const double h = 1.0 / (n - 1);
    op.dim = dim;
    op.n = n;
    op.L = layer_cells;
    op.N = N;
    op.hinv2 = 1.0 / (h * h);
    op.dre = k0 * k0 - 2.0 * dim / (h * h);
    op.mask = mask;
    op.k2 = reinterpret_cast<const double2*>(k2);
    op.invd = nullptr;
    for (int m = 0; m <= kMaxLayerCells; ++m) {
        double eta = (layer_cells > 0 && m <= layer_cells) ? (double)m / (double)layer_cells : 0.0;
        op.im[m] = k0 * k0 * ((layer_strength * eta) * eta);
        op.invd_tab[m] = make_double2(0.0, 0.0);
    }
    // the stencil reads the neighbours of every fluid node: the outer ring must be masked
    if (cudaMemsetAsync(flag, 0, sizeof(int), s) != cudaSuccess) return HELM_CUDA_ERROR;
    launch_check_ring(op, flag, s);
    int bad = 0;
    if (cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return HELM_CUDA_ERROR;
    if (bad) return HELM_BAD_ARG;
    // every block writes its own partial, so the scratch needs no clearing
    const int nb = launch_apply<double>(op, reinterpret_cast<const double2*>(x), reinterpret_cast<const double2*>(f),
                                        reinterpret_cast<double2*>(r), scratch, conj, true, s);
    launch_sum_real(scratch, nb, norm2, s);
    if (cudaGetLastError() != cudaSuccess) return HELM_CUDA_ERROR;
    return HELM_OK;
}
