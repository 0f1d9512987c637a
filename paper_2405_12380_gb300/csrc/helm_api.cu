// C ABI of libhelm and the host drivers of the meta-solvers (Sec. 3.1).
//
// The drivers only launch kernels and read back a few status words from pinned
// memory; every vector operation, reduction and scalar recurrence runs on the
// device (stencil.cu, blas.cu, tb.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "helm_internal.cuh"

using namespace helm;

// the per-unit violation records of the bounds-checked build
std::vector<unsigned long long (*)()>& helm::checked_units() {
    static std::vector<unsigned long long (*)()> units;
    return units;
}

namespace {

helm_status fail(helm_handle* h, helm_status st, const std::string& msg) {
    if (h) h->err = msg;
    return st;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(h, HELM_CUDA_ERROR, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define CKL()                                                                                        \
    do {                                                                                             \
        cudaError_t e_ = cudaGetLastError();                                                         \
        if (e_ != cudaSuccess)                                                                       \
            return fail(h, HELM_CUDA_ERROR, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
    } while (0)

#define TRY(expr)                          \
    do {                                   \
        helm_status st_ = (expr);          \
        if (st_ != HELM_OK) return st_;    \
    } while (0)

template <typename T>
helm_status dalloc(helm_handle* h, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return HELM_OK;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(h, HELM_OUT_OF_MEMORY, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return HELM_OK;
}

template <typename T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

int round32(int k) { return ((k + 31) / 32) * 32; }

// drop the captured iterations (their kernels name buffers and operator tables that
// are about to change)
void drop_graphs(helm_handle* h) {
    if (h->g32) cudaGraphExecDestroy(h->g32);
    h->g32 = nullptr;
}

helm_status ensure_tmp(helm_handle* h, size_t count) {
    while (h->tmp.size() < count) {
        double2* p = nullptr;
        TRY(dalloc(h, &p, (size_t)h->N));
        h->tmp.push_back(p);
    }
    return HELM_OK;
}

helm_status ensure_tmp32(helm_handle* h, size_t count) {
    while (h->tmp32.size() < count) {
        float2* p = nullptr;
        TRY(dalloc(h, &p, (size_t)h->N));
        h->tmp32.push_back(p);
    }
    return HELM_OK;
}

double* scal(helm_handle* h, int slot) { return reinterpret_cast<double*>(h->sc + slot); }

bool red_black(int kind) { return kind == HELM_RBGS || kind == HELM_SOR || kind == HELM_SSOR; }


helm_status poll(helm_handle* h) {
    CK(cudaMemcpyAsync(h->hpin, h->sc, S_NSLOTS * sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return HELM_OK;
}
double hs(const helm_handle* h, int slot, int im = 0) { return h->hpin[2 * slot + im]; }
// a grid-barrier wait of the cooperative cycle gave up (flag 4 in S_FLAGS.y, read by poll)
bool barrier_timed_out(const helm_handle* h) { return hs(h, S_FLAGS, 1) == 4.0; }

// ||f - A x||^2 into slot (FP64)
helm_status residual_norm(helm_handle* h, const double2* f, const double2* x, double2* r, int conj, int slot) {
    const int nb = launch_apply<double>(h->op64, x, f, r, h->red, conj, true, h->stream);
    launch_sum_real(h->red, nb, scal(h, slot), h->stream);
    h->launches += 2;
    CKL();
    return HELM_OK;
}

helm_status norm2_into(helm_handle* h, const double2* a, int slot) {
    launch_norm2(a, h->N, h->red, h->stream);
    launch_sum_real(h->red, kRedBlocks, scal(h, slot), h->stream);
    h->launches += 2;
    CKL();
    return HELM_OK;
}

// event pair around one launch of phase ph (0 restrict, 1 prolong, 2 sweep, 3 operator)
void ev_mark(helm_handle* h, int ph, int end) {
    if (!h->profile) return;
    auto& pool = h->evpool[ph];
    const size_t need = 2 * (size_t)h->evn[ph] + 2;
    while (pool.size() < need) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        pool.push_back(e);
    }
    cudaEventRecord(pool[2 * h->evn[ph] + end], h->stream);
    if (end) ++h->evn[ph];
}

double ev_sum(helm_handle* h, int ph) {
    double t = 0;
    for (int q = 0; q < h->evn[ph]; ++q) {
        float ms = 0;
        cudaEventElapsedTime(&ms, h->evpool[ph][2 * q], h->evpool[ph][2 * q + 1]);
        t += ms;
    }
    return t;
}

// `sweeps` red-black sweeps in place (Eq. 2 with M = the lower triangle of the
// red-black ordered A): HELM_RBGS red then black half-sweeps; HELM_SOR the same with
// each node moved by omega times its Gauss-Seidel step; HELM_SSOR the forward sweep
// (red, black) then the backward one (black, red).  from_zero: x = 0 on entry (the
// first half-sweep reads no neighbours; its other colour must already be zero).
template <typename R>
void red_black_sweeps(helm_handle* h, const Op<R>& op, int kind, double omega, int sweeps,
                      const typename CT<R>::T* f, typename CT<R>::T* x, int conj, bool from_zero) {
    const double w = kind == HELM_RBGS ? 1.0 : omega;
    static const int fwd[2] = {0, 1}, sym[4] = {0, 1, 1, 0};
    const int* order = kind == HELM_SSOR ? sym : fwd;
    const int per = kind == HELM_SSOR ? 4 : 2;
    for (int q = 0; q < sweeps; ++q)
        for (int c = 0; c < per; ++c) {
            const bool first = from_zero && q == 0 && c == 0;
            if (!first) ev_mark(h, 2, 0);
            launch_rbgs_half<R>(op, order[c], f, x, conj, first, h->stream, w);
            if (!first) ev_mark(h, 2, 1);
        }
    h->launches += (long long)per * sweeps;
}

// complex64 Gauss-Seidel-type sweeps as fused full sweeps (one launch each, out of
// place): the launches alternate between x and tmp so that the last one writes x.
// SSOR is a forward sweep (colour 0 first) and a backward one (colour 1 first).
// From zero the first launch reads nothing; otherwise an odd launch count first
// copies x to tmp.  Returns false (nothing launched) where the fused kernel does
// not apply.
bool fused_sweeps32(helm_handle* h, int kind, double omega, int sweeps, const float2* f, float2* x, float2* tmp,
                    int conj, bool from_zero) {
    const double w = kind == HELM_RBGS ? 1.0 : omega;
    const int per = kind == HELM_SSOR ? 2 : 1;
    const int L = per * sweeps;
    if (L <= 0) return false;
    if (!rbgs_sweep32_ok(h->op32, f, x, tmp)) return false;
    const float2* in = from_zero ? nullptr : x;
    if (!from_zero && L % 2 == 1) {
        if (cudaMemcpyAsync(tmp, x, sizeof(float2) * h->N, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
            return false;
        in = tmp;
    }
    for (int i = 0; i < L; ++i) {
        float2* out = ((L - 1 - i) % 2 == 0) ? x : tmp;
        const int c0 = (kind == HELM_SSOR && i % 2 == 1) ? 1 : 0;
        ev_mark(h, 2, 0);
        launch_rbgs_sweep32(h->op32, c0, f, in, out, conj, w, h->stream);
        ev_mark(h, 2, 1);
        in = out;
    }
    h->launches += L;
    return true;
}

// z = n sweeps of the relaxation on A z = r from z = 0 (FP64)
helm_status relax_from_zero(helm_handle* h, int kind, double omega, int sweeps, const double2* r, double2* z,
                            int conj) {
    cudaStream_t s = h->stream;
    if (kind == HELM_RELAX_NONE || sweeps <= 0) {
        CK(cudaMemsetAsync(z, 0, sizeof(double2) * h->N, s));
        return HELM_OK;
    }
    if (kind == HELM_JACOBI) {
        TRY(ensure_tmp(h, 1));
        // sweep 1 from zero writes z; later sweeps ping-pong so that the last lands in z
        double2* a = (sweeps % 2 == 1) ? z : h->tmp[0];
        double2* b = (sweeps % 2 == 1) ? h->tmp[0] : z;
        launch_jacobi<double>(h->op64, omega, r, nullptr, a, conj, true, s);
        for (int q = 1; q < sweeps; ++q) {
            ev_mark(h, 2, 0);
            launch_jacobi<double>(h->op64, omega, r, a, b, conj, false, s);
            ev_mark(h, 2, 1);
            std::swap(a, b);
        }
        h->launches += sweeps;
        CKL();
        return HELM_OK;
    }
    if (red_black(kind)) {
        CK(cudaMemsetAsync(z, 0, sizeof(double2) * h->N, s));
        red_black_sweeps<double>(h, h->op64, kind, omega, sweeps, r, z, conj, true);
        CKL();
        return HELM_OK;
    }
    return fail(h, HELM_BAD_ARG, "unknown relaxation kind");
}

// z += Q A_c^-1 Q^T (v - A zres)   (zres may be null: plain restriction of v).
// black_zero: zres is the result of red-black Gauss-Seidel sweeps ending with the
// black half-sweep, so v - A zres vanishes on black and masked nodes (each black
// row was just solved exactly; masked rows hold x = v) and only the red rows are
// computed and projected.
helm_status tb_correct(helm_handle* h, const double2* v, const double2* zres, double2* z, int conj,
                       bool black_zero = false) {
    if (!h->Q) return fail(h, HELM_NOT_READY, "trunk basis not loaded (don_load)");
    const double2* r = v;
    const bool red_only = zres && black_zero;
    const long long rows = red_only ? (h->N + 1) / 2 : h->N;
    const int nblk = project_blocks(rows);
    if (zres) {
        // r = v - A zres (FP64 stencil), then the projection streams Q once
        TRY(ensure_tmp(h, 14));
        if (red_only) launch_residual_red(h->op64, zres, v, h->tmp[13], conj, h->stream);
        else launch_apply<double>(h->op64, zres, v, h->tmp[13], nullptr, conj, true, h->stream);
        h->launches += 1;
        r = h->tmp[13];
    }
    ev_mark(h, 0, 0);
    launch_project_df(red_only ? h->Qr : h->Q, red_only ? basis_ld((h->N + 1) / 2) : basis_ld(h->N), h->k, r, rows,
                      h->coarse_partials, nblk, h->stream);
    ev_mark(h, 0, 1);
    launch_coarse_apply(h->coarse_partials, nblk, h->k, h->Ainv, conj, h->ybuf, h->cbuf, h->stream);
    ev_mark(h, 1, 0);
    launch_prolong_df(h->Q, basis_ld(h->N), h->k, h->ybuf, z, h->N, h->stream);
    ev_mark(h, 1, 1);
    h->launches += 4;
    CKL();
    return HELM_OK;
}

// z += s (T b_re + i T b_im), b = Branch([Re v, Im v] / s), s = ||v|| (FP32 network)
helm_status nl_correct(helm_handle* h, const double2* v, double2* z) {
    if (!h->bw || !h->Traw) return fail(h, HELM_NOT_READY, "branch network not loaded (don_load_branch)");
    cudaStream_t s = h->stream;
    TRY(norm2_into(h, v, S_TS));
    double* s2 = scal(h, S_TS);
    launch_nl_pack(v, s2, h->nl_x, h->N, s);
    const float* in = h->nl_x;
    const float* W = h->bw;
    const int nl = (int)h->bwidths.size() - 1;
    float* bufs[2] = {h->nl_h0, h->nl_h1};
    for (int l = 0; l < nl; ++l) {
        const int win = h->bwidths[l], wout = h->bwidths[l + 1];
        float* out = bufs[l % 2];
        helm_status st = nn_gemm(0, 1, 1, wout, win, 1.0f, in, win, W, win, 0.0f, out, wout, s);
        if (st != HELM_OK) return fail(h, st, "branch layer");
        st = nn_bias_act(1, wout, out, W + (size_t)win * wout, l < nl - 1 ? 1 : 0, s);
        if (st != HELM_OK) return fail(h, st, "branch activation");
        W += (size_t)win * wout + wout;
        in = out;
    }
    launch_nl_prolong(h->Traw, h->p, in, s2, z, h->N, s);
    h->launches += 3 + 2 * nl + 2;
    CKL();
    return HELM_OK;
}

// complex64 hybrid cycle with the BF16 basis (MIXED handles): z32 = M(v32)
helm_status precond32(helm_handle* h, const helm_solve_opts* o, const float2* v, float2* z, int conj) {
    cudaStream_t s = h->stream;
    const bool no_relax = o->relax == HELM_RELAX_NONE || o->n_r <= 0;
    if (no_relax && o->correction == HELM_CORR_NONE) {
        CK(cudaMemcpyAsync(z, v, sizeof(float2) * h->N, cudaMemcpyDeviceToDevice, s));
        return HELM_OK;
    }
    if (no_relax) {
        CK(cudaMemsetAsync(z, 0, sizeof(float2) * h->N, s));
    } else if (o->relax == HELM_JACOBI) {
        TRY(ensure_tmp32(h, 4));
        float2* a = (o->n_r % 2 == 1) ? z : h->tmp32[3];
        float2* b = (o->n_r % 2 == 1) ? h->tmp32[3] : z;
        launch_jacobi<float>(h->op32, o->omega, v, nullptr, a, conj, true, s);
        for (int q = 1; q < o->n_r; ++q) {
            launch_jacobi<float>(h->op32, o->omega, v, a, b, conj, false, s);
            std::swap(a, b);
        }
        h->launches += o->n_r;
    } else {
        TRY(ensure_tmp32(h, 4));
        if (!fused_sweeps32(h, o->relax, o->omega, o->n_r, v, z, h->tmp32[3], conj, true)) {
            CK(cudaMemsetAsync(z, 0, sizeof(float2) * h->N, s));
            red_black_sweeps<float>(h, h->op32, o->relax, o->omega, o->n_r, v, z, conj, true);
        }
    }
    if (o->correction == HELM_CORR_TB) {
        if (!h->Qbf) return fail(h, HELM_NOT_READY, "trunk basis not loaded (don_load)");
        int nblk = restrict_blocks(h->N);
        ev_mark(h, 0, 0);
        // after the black half-sweep v - A z vanishes on black and masked rows: with
        // the pair layout the red rows' residual is stored compactly (in the sweep
        // buffer, free again) and projected by a plain tall-skinny product
        if (!no_relax && o->relax == HELM_RBGS && h->Qbr &&
            launch_red_residual32(h->op32, v, z, h->tmp32[3], conj, s)) {
            nblk = launch_restrict32_rr(h->Qbr, basis_ld((h->N + 1) / 2), h->k, h->tmp32[3], (h->N + 1) / 2,
                                        h->partials32, h->N, s);
            h->launches += 1;
        } else if (!no_relax && o->relax == HELM_RBGS && h->Qbr) {
            // after the black half-sweep v - A z vanishes on black and masked rows:
            // project the red rows only
            nblk = launch_restrict32_red(h->op32, h->Qbr, basis_ld((h->N + 1) / 2), h->k, v, z, conj,
                                         h->partials32, s);
        } else {
            launch_restrict32(h->op32, h->Qbf, basis_ld(h->N), h->k, v, no_relax ? nullptr : z, conj,
                              h->partials32, nblk, s);
        }
        ev_mark(h, 0, 1);
        launch_coarse_apply32(h->partials32, nblk, h->k, h->Ainv, conj, h->y32, h->cbuf, s);
        ev_mark(h, 1, 0);
        launch_prolong32(h->Qbf, basis_ld(h->N), h->k, h->y32, z, h->N, s);
        ev_mark(h, 1, 1);
        h->launches += 4;
    }
    CKL();
    return HELM_OK;
}

// The hybrid cycle with red-black Gauss-Seidel and the trunk-basis correction on an
// FP64 handle, with the sweeps in double-float arithmetic on the FP32 pipes:
// z = n_r sweeps on A z = r from z = 0, then z += Q A_c^-1 Q^T (r - A z), where the
// residual is formed on the red rows only (after the black half-sweep it vanishes on
// black and masked rows) and z is converted to FP64 once, inside the prolongation.
// pre (0, 1, 2) and pv, pw, tol_abs: see launch_cycle_df (the BiCGStab update of
// the preconditioner's input fused into the cycle; requires the cooperative cycle)
helm_status precond_rbgs_tb_df(helm_handle* h, const helm_solve_opts* o, const double2* r, double2* z, int conj,
                               int pre = 0, const double2* pv = nullptr, double2* pw = nullptr,
                               double tol_abs = 0.0, float4* zdf = nullptr) {
    if (!h->Q) return fail(h, HELM_NOT_READY, "trunk basis not loaded (don_load)");
    TRY(ensure_tmp(h, 16));
    cudaStream_t s = h->stream;
    float4* fs = reinterpret_cast<float4*>(h->tmp[14]);
    float4* xs = reinterpret_cast<float4*>(h->tmp[15]);
    float4* rr = reinterpret_cast<float4*>(h->tmp[13]);
    if (cycle_df_blocks(h->N) > 0) {
        // one cooperative launch for the whole red-black part and the red residual
        ev_mark(h, 2, 0);
        CK(launch_cycle_df(h->op64, h->dft, pre, r, pv, pw, h->sc, h->fparts, tol_abs, fs, xs, rr, o->n_r, conj,
                           h->counter + 2, h->dflag + 2, h->bar_spin, h->bar_extra, s));
        ev_mark(h, 2, 1);
        h->launches -= 2 * o->n_r;
    } else {
        if (pre != 0) return fail(h, HELM_BAD_ARG, "fused update needs the cooperative cycle");
        launch_rbgs_df_first(h->op64, h->dft, r, fs, xs, conj, s);
        for (int q = 0; q < o->n_r; ++q) {
            if (q > 0) {
                ev_mark(h, 2, 0);
                launch_rbgs_df(h->op64, h->dft, 0, fs, xs, conj, s);
                ev_mark(h, 2, 1);
            }
            ev_mark(h, 2, 0);
            launch_rbgs_df(h->op64, h->dft, 1, fs, xs, conj, s);
            ev_mark(h, 2, 1);
        }
        launch_residual_red_df(h->op64, h->dft, fs, xs, rr, conj, s);
    }
    const long long rows = (h->N + 1) / 2;
    const int nblk = project_blocks(rows);
    ev_mark(h, 0, 0);
    launch_project_df_split(h->Qr, basis_ld(rows), h->k, rr, rows, h->coarse_partials, nblk, s);
    ev_mark(h, 0, 1);
    launch_coarse_apply(h->coarse_partials, nblk, h->k, h->Ainv, conj, h->ybuf, h->cbuf, s);
    ev_mark(h, 1, 0);
    launch_prolong_df_base(h->Q, basis_ld(h->N), h->k, h->ybuf, xs, z, zdf, h->N, s);
    ev_mark(h, 1, 1);
    h->launches += 2 * o->n_r + 5;
    CKL();
    return HELM_OK;
}

// ---------------------------------------------------------------- multigrid
// `sweeps` damped-Jacobi sweeps on A z = r on handle H, z from zero if `zero`; the
// sweeps alternate between z and jt so that the last one lands in z
helm_status jacobi_sweeps(helm_handle* h, double omega, int sweeps, const double2* r, double2* z, double2* jt,
                          int conj, bool zero, cudaStream_t s) {
    if (sweeps <= 0) {
        if (zero) CK(cudaMemsetAsync(z, 0, sizeof(double2) * h->N, s));
        return HELM_OK;
    }
    double2* bufs[2] = {z, jt};
    int src = zero ? -1 : 0;
    for (int q = 0; q < sweeps; ++q) {
        const int dst = ((sweeps - 1 - q) % 2 == 0) ? 0 : 1;
        if (src == dst) {
            CK(cudaMemcpyAsync(bufs[1 - src], bufs[src], sizeof(double2) * h->N, cudaMemcpyDeviceToDevice, s));
            src = 1 - src;
        }
        launch_jacobi<double>(h->op64, omega, r, src < 0 ? nullptr : bufs[src], bufs[dst], conj, src < 0, s);
        src = dst;
    }
    CKL();
    return HELM_OK;
}

// z = V(r) on level `level` (handle H; level 0 is h itself), Sec. 4.3 DeepONet-MG:
// smoother from zero, coarse-grid correction z += P V_c(R (r - A z)) (zero on masked
// nodes), smoother again; the smoother is n_r damped-Jacobi sweeps, the trunk-basis
// correction, n_r sweeps (the 2-1-2 strategy for n_r = 2) on level 0 when the
// correction is the trunk basis, else 2 n_r + 1 sweeps; the coarsest level only
// smooths from zero
helm_status vcycle(helm_handle* h, int level, helm_handle* H, const helm_solve_opts* o, const double2* r, double2* z,
                   int conj) {
    const cudaStream_t s = h->stream;
    double2 *jt, *t;
    if (level == 0) {
        TRY(ensure_tmp(h, 20));
        jt = h->tmp[18];
        t = h->tmp[19];
    } else {
        TRY(ensure_tmp(H, 4));
        jt = H->tmp[0];
        t = H->tmp[3];
    }
    const bool with_tb = level == 0 && o->correction == HELM_CORR_TB;
    auto smooth = [&](bool zero) -> helm_status {
        if (with_tb) {
            TRY(jacobi_sweeps(H, o->omega, o->n_r, r, z, jt, conj, zero, s));
            TRY(tb_correct(H, r, z, z, conj, false));
            return jacobi_sweeps(H, o->omega, o->n_r, r, z, jt, conj, false, s);
        }
        return jacobi_sweeps(H, o->omega, 2 * o->n_r + 1, r, z, jt, conj, zero, s);
    };
    TRY(smooth(true));
    if (level == (int)h->mg.size()) return HELM_OK;
    helm_handle* Cc = h->mg[level];
    TRY(ensure_tmp(Cc, 4));
    Cc->stream = s;
    launch_apply<double>(H->op64, z, r, t, nullptr, conj, true, s);
    launch_restrict_fw<double>(H->dim, H->n, t, Cc->mask, Cc->tmp[1], s);
    h->launches += 2;
    CKL();
    TRY(vcycle(h, level + 1, Cc, o, Cc->tmp[1], Cc->tmp[2], conj));
    launch_prolong_add<double>(H->dim, H->n, Cc->tmp[2], H->mask, z, s);
    h->launches += 1;
    CKL();
    return smooth(false);
}

helm_status precond(helm_handle* h, const helm_solve_opts* o, const double2* r, double2* z, int conj) {
    NvtxRange nvtx("hybrid cycle");
    if (h->precision == HELM_MIXED && o->relax == HELM_MG)
        return fail(h, HELM_BAD_ARG, "the multigrid cycle runs on FP64 handles");
    if (h->precision == HELM_MIXED) {
        TRY(ensure_tmp32(h, 4));
        launch_cvt_f64_to_f32(r, h->tmp32[0], h->N, h->stream);
        TRY(precond32(h, o, h->tmp32[0], h->tmp32[1], conj));
        launch_cvt_f32_to_f64(h->tmp32[1], z, h->N, h->stream);
        h->launches += 2;
        CKL();
        return HELM_OK;
    }
    const bool no_relax = o->relax == HELM_RELAX_NONE || o->n_r <= 0;
    if (no_relax && o->correction == HELM_CORR_NONE) {
        // neither stage: M is the identity (plain Krylov)
        CK(cudaMemcpyAsync(z, r, sizeof(double2) * h->N, cudaMemcpyDeviceToDevice, h->stream));
        return HELM_OK;
    }
    if (o->relax == HELM_MG) return vcycle(h, 0, h, o, r, z, conj);
    if (o->relax == HELM_RBGS && o->n_r > 0 && o->correction == HELM_CORR_TB && !h->k2) return precond_rbgs_tb_df(h, o, r, z, conj);
    TRY(relax_from_zero(h, o->relax, o->omega, o->n_r, r, z, conj));
    if (o->correction == HELM_CORR_TB) {
        const bool zero = o->relax == HELM_RELAX_NONE || o->n_r <= 0;
        TRY(tb_correct(h, r, zero ? nullptr : z, z, conj, o->relax == HELM_RBGS));
    } else if (o->correction == HELM_CORR_NONLINEAR) {
        // M2 acts on the residual after the sweeps: r - A z
        TRY(ensure_tmp(h, 13));
        double2* rr = h->tmp[12];
        if (no_relax) {
            CK(cudaMemcpyAsync(rr, r, sizeof(double2) * h->N, cudaMemcpyDeviceToDevice, h->stream));
        } else {
            launch_apply<double>(h->op64, z, r, rr, nullptr, conj, true, h->stream);
            h->launches += 1;
        }
        TRY(nl_correct(h, rr, z));
    }
    return HELM_OK;
}

helm_status check_opts(helm_handle* h, const helm_solve_opts* o) {
    if (!o) return fail(h, HELM_BAD_ARG, "opts is NULL");
    if (o->method < 0 || o->method > 2) return fail(h, HELM_BAD_ARG, "unknown method");
    if (o->relax < 0 || o->relax > HELM_MG) return fail(h, HELM_BAD_ARG, "unknown relaxation");
    if ((o->relax == HELM_SOR || o->relax == HELM_SSOR || o->relax == HELM_JACOBI || o->relax == HELM_MG) &&
        !(o->omega > 0.0 && o->omega < 2.0))
        return fail(h, HELM_BAD_ARG, "omega must be in (0, 2)");
    if (o->relax == HELM_MG && !h->mg_levels)
        return fail(h, HELM_NOT_READY, "multigrid hierarchy not set up (helm_mg_setup)");
    if (o->correction < 0 || o->correction > 2) return fail(h, HELM_BAD_ARG, "unknown correction");
    if (o->correction == HELM_CORR_TB && !h->Q) return fail(h, HELM_NOT_READY, "trunk basis not loaded");
    if (o->correction == HELM_CORR_NONLINEAR) {
        if (!h->bw) return fail(h, HELM_NOT_READY, "branch network not loaded");
        if (o->method == HELM_METHOD_BICGSTAB)
            return fail(h, HELM_BAD_ARG, "the nonlinear correction cannot precondition BiCGStab (needs a linear M)");
        if (h->precision == HELM_MIXED || o->conj)
            return fail(h, HELM_BAD_ARG, "the nonlinear correction is FP64-handle, non-conjugate only");
    }
    if (o->method == HELM_METHOD_FGMRES && (o->restart < 1 || o->restart > kMaxRestart))
        return fail(h, HELM_BAD_ARG, "restart must be in 1..64");
    if (!(o->tol >= 0) || o->maxit < 0 || o->n_r < 0) return fail(h, HELM_BAD_ARG, "bad tol/maxit/n_r");
    return HELM_OK;
}

struct Hist {
    double* buf;
    int len, n = 0;
    void push(double v) {
        if (buf && n < len) buf[n] = v;
        ++n;
    }
};

// ------------------------------------------------------------- relaxation
helm_status solve_relax(helm_handle* h, const helm_solve_opts* o, const double2* f, double2* x, helm_stats* st,
                        Hist& hist, double bnorm) {
    TRY(ensure_tmp(h, 2));
    double2* r = h->tmp[1];
    int cycles = 0;
    while (true) {
        TRY(residual_norm(h, f, x, r, o->conj, S_RN2));
        ++st->matvecs;
        TRY(poll(h));
        if (barrier_timed_out(h)) { st->status = HELM_TIMEOUT; break; }
        const double res = std::sqrt(hs(h, S_RN2)) / bnorm;
        hist.push(res);
        st->rel_res = res;
        if (res <= o->tol) { st->status = HELM_OK; break; }
        if (!std::isfinite(res) || res > 1e8) { st->status = HELM_DIVERGED; break; }
        if (cycles >= o->maxit) { st->status = HELM_NOT_CONVERGED; break; }
        if (o->relax == HELM_JACOBI) {
            TRY(ensure_tmp(h, 1));
            double2* a = x;
            double2* b = h->tmp[0];
            for (int q = 0; q < o->n_r; ++q) {
                launch_jacobi<double>(h->op64, o->omega, f, a, b, o->conj, false, h->stream);
                std::swap(a, b);
            }
            h->launches += o->n_r;
            if (a != x) CK(cudaMemcpyAsync(x, a, sizeof(double2) * h->N, cudaMemcpyDeviceToDevice, h->stream));
        } else if (red_black(o->relax)) {
            red_black_sweeps<double>(h, h->op64, o->relax, o->omega, o->n_r, f, x, o->conj, false);
        }
        CKL();
        if (o->correction == HELM_CORR_TB) {
            TRY(tb_correct(h, f, x, x, o->conj, o->relax == HELM_RBGS && o->n_r > 0));
            ++st->precond_applies;
        } else if (o->correction == HELM_CORR_NONLINEAR) {
            launch_apply<double>(h->op64, x, f, r, nullptr, o->conj, true, h->stream);
            h->launches += 1;
            TRY(nl_correct(h, r, x));
            ++st->precond_applies;
        }
        ++cycles;
    }
    st->iters = cycles;
    st->cycles = cycles;
    return HELM_OK;
}

// ---------------------------------------------------------------- FGMRES(m)
helm_status ensure_krylov(helm_handle* h, int m) {
    if (h->m_alloc >= m) return HELM_OK;
    dfree(h->V); dfree(h->Z); dfree(h->Hm); dfree(h->cs); dfree(h->sn); dfree(h->g); dfree(h->y); dfree(h->hpart);
    h->m_alloc = 0;
    TRY(dalloc(h, &h->V, (size_t)(m + 1) * h->N));
    TRY(dalloc(h, &h->Z, (size_t)m * h->N));
    TRY(dalloc(h, &h->Hm, (size_t)(m + 1) * m));
    TRY(dalloc(h, &h->cs, (size_t)m));
    TRY(dalloc(h, &h->sn, (size_t)m));
    TRY(dalloc(h, &h->g, (size_t)(m + 1)));
    TRY(dalloc(h, &h->y, (size_t)2 * (kMaxRestart + 1)));
    TRY(dalloc(h, &h->hpart, (size_t)kRedBlocks * (m + 1)));
    h->m_alloc = m;
    return HELM_OK;
}

helm_status solve_fgmres(helm_handle* h, const helm_solve_opts* o, const double2* f, double2* x, helm_stats* st,
                         Hist& hist, double bnorm) {
    const int m = o->restart;
    const bool mixed = h->precision == HELM_MIXED;
    TRY(ensure_krylov(h, m));
    const long long N = h->N;
    cudaStream_t s = h->stream;
    const int ldh = m + 1;
    if (mixed) {
        TRY(ensure_tmp32(h, 4));
        if (h->m32_alloc < m) {
            dfree(h->Z32);
            h->m32_alloc = 0;
            TRY(dalloc(h, &h->Z32, (size_t)m * N));
            h->m32_alloc = m;
        }
    }
    double2* h2 = h->y + (kMaxRestart + 1);
    int iters = 0, cycles = 0;
    while (true) {
        double2* V0 = h->V;
        TRY(residual_norm(h, f, x, V0, o->conj, S_BETA2));
        ++st->matvecs;
        TRY(poll(h));
        const double beta = std::sqrt(hs(h, S_BETA2));
        st->rel_res = beta / bnorm;
        if (cycles == 0) hist.push(beta / bnorm);
        if (beta <= o->tol * bnorm) { st->status = HELM_OK; break; }
        if (!std::isfinite(beta)) { st->status = HELM_DIVERGED; break; }
        if (iters >= o->maxit) { st->status = HELM_NOT_CONVERGED; break; }
        ++cycles;
        launch_init_g(h->g, m + 1, scal(h, S_BETA2), s);
        launch_scale_vec(V0, V0, scal(h, S_BETA2), N, s);
        h->launches += 2;
        CK(cudaMemsetAsync(h->Hm, 0, sizeof(double2) * (m + 1) * m, s));
        int kdim = 0;
        for (int j = 0; j < m; ++j) {
            double2* Vj = h->V + (long long)j * N;
            double2* Zj = h->Z + (long long)j * N;
            double2* w = h->V + (long long)(j + 1) * N;
            double2* Hcol = h->Hm + (long long)j * ldh;
            if (mixed) {
                // complex64 preconditioner and matvec; the product is widened before CGS2
                float2* Z32j = h->Z32 + (long long)j * N;
                launch_cvt_f64_to_f32(Vj, h->tmp32[0], N, s);
                TRY(precond32(h, o, h->tmp32[0], Z32j, o->conj));
                launch_apply<float>(h->op32, Z32j, nullptr, h->tmp32[2], nullptr, o->conj, false, s);
                launch_cvt_f32_to_f64(h->tmp32[2], w, N, s);
                h->launches += 3;
            } else {
                TRY(precond(h, o, Vj, Zj, o->conj));
                launch_apply<double>(h->op64, Zj, nullptr, w, nullptr, o->conj, false, s);
                h->launches += 1;
            }
            ++st->precond_applies;
            ++st->matvecs;
            // CGS2: h = V^H w, w -= V h, h2 = V^H w, w -= V h2, h += h2
            NvtxRange nvtx_a("Arnoldi CGS2 + Givens");
            launch_mdot(h->V, j + 1, w, N, h->hpart, s);
            launch_mdot_finalize(h->hpart, kRedBlocks, j + 1, Hcol, 0, nullptr, s);
            launch_mupdate(h->V, j + 1, Hcol, -1.0, w, N, nullptr, s);
            launch_mdot(h->V, j + 1, w, N, h->hpart, s);
            launch_mdot_finalize(h->hpart, kRedBlocks, j + 1, Hcol, 1, h2, s);
            launch_mupdate(h->V, j + 1, h2, -1.0, w, N, h->red, s);
            launch_sum_real(h->red, kRedBlocks, scal(h, S_WN2), s);
            launch_givens(h->Hm, ldh, j, h->cs, h->sn, h->g, scal(h, S_WN2), scal(h, S_EST), s);
            launch_scale_vec(w, w, scal(h, S_WN2), N, s);
            h->launches += 10;
            CKL();
            ++iters;
            kdim = j + 1;
            TRY(poll(h));
            if (barrier_timed_out(h)) { st->status = HELM_TIMEOUT; break; }
            const double est = hs(h, S_EST) / bnorm;
            hist.push(est);
            const double wn2 = hs(h, S_WN2);
            if (!std::isfinite(est)) break;
            if (wn2 == 0.0 || est <= o->tol || iters >= o->maxit) break;
        }
        if (st->status == HELM_TIMEOUT) break;
        launch_hsolve(h->Hm, ldh, kdim, h->g, h->y, s);
        if (mixed)
            launch_mupdate32(h->Z32, kdim, h->y, 1.0, x, N, s);
        else
            launch_mupdate(h->Z, kdim, h->y, 1.0, x, N, nullptr, s);
        h->launches += 2;
        CKL();
    }
    st->iters = iters;
    st->cycles = cycles;
    return HELM_OK;
}

// ---------------------------------------------------------------- BiCGStab
helm_status solve_bicgstab(helm_handle* h, const helm_solve_opts* o, const double2* f, double2* x,
                           helm_stats* st, Hist& hist, double bnorm) {
    TRY(ensure_tmp(h, 10));
    const long long N = h->N;
    cudaStream_t s = h->stream;
    double2 *r = h->tmp[1], *rh = h->tmp[2], *p = h->tmp[3], *v = h->tmp[4], *sv = h->tmp[5], *t = h->tmp[6],
            *ph = h->tmp[7], *sh = h->tmp[8];
    const double tol_abs = o->tol * bnorm;
    TRY(residual_norm(h, f, x, r, o->conj, S_RN2));
    ++st->matvecs;
    TRY(poll(h));
    double res = std::sqrt(hs(h, S_RN2)) / bnorm;
    hist.push(res);
    st->rel_res = res;
    int iters = 0, restarts = 0;
    if (res <= o->tol) {
        st->status = HELM_OK;
        st->iters = 0;
        return HELM_OK;
    }
    auto restart = [&]() -> helm_status {
        CK(cudaMemcpyAsync(rh, r, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemsetAsync(p, 0, sizeof(double2) * N, s));
        CK(cudaMemsetAsync(v, 0, sizeof(double2) * N, s));
        launch_bicg_scalar(5, h->red, 0, h->sc, 0.0, s);
        // rho = <rhat, r> and beta for the first iteration of this (re)start
        launch_dot(rh, r, N, reinterpret_cast<double2*>(h->red), s);
        launch_bicg_scalar(0, h->red, kRedBlocks, h->sc, tol_abs, s);
        h->launches += 3;
        CKL();
        return HELM_OK;
    };
    TRY(restart());
    st->status = HELM_NOT_CONVERGED;
    // one iteration: p update, M p, v = A p with alpha, s with ||s||, M s, t = A s with
    // omega, x/r update with ||r|| and the next rho/beta -- each reduction and its scalar
    // recurrence fused into the kernel that produces the vector.  The iteration ends by
    // copying the scalars into one of two pinned snapshots.
    // the double-float cycle with a cooperative launch takes the vector updates that
    // feed the preconditioner into its first phase
    const bool fuse = h->precision != HELM_MIXED && o->relax == HELM_RBGS && o->n_r > 0 &&
                      o->correction == HELM_CORR_TB && !h->k2 && h->Q && cycle_df_blocks(N) > 0;
    float4* phdf = nullptr;
    float4* shdf = nullptr;
    if (fuse) {
        TRY(ensure_tmp(h, 18));
        phdf = reinterpret_cast<float4*>(h->tmp[16]);
        shdf = reinterpret_cast<float4*>(h->tmp[17]);
    }
    auto launch_iter = [&](int slot) -> helm_status {
        if (fuse) {
            // p = r + beta (p - omega v) inside the preconditioner's first phase; the
            // preconditioned vector also as FP32 pairs, the operator's input
            TRY(precond_rbgs_tb_df(h, o, r, ph, o->conj, 1, v, p, 0.0, phdf));
            ev_mark(h, 3, 0);
            launch_apply_bicg_df(h->op64, h->dft, 1, phdf, v, rh, o->conj, h->sc, h->fparts, h->counter, s);
            ev_mark(h, 3, 1);
        } else {
            launch_bicg_update_p(r, v, p, h->sc, N, s);
            TRY(precond(h, o, p, ph, o->conj));
            ev_mark(h, 3, 0);
            launch_apply_bicg(h->op64, 1, ph, v, rh, o->conj, h->sc, h->fparts, h->counter, s);
            ev_mark(h, 3, 1);
        }
        if (fuse) {
            // s = r - alpha v and ||s|| inside the preconditioner's first phase
            TRY(precond_rbgs_tb_df(h, o, r, sh, o->conj, 2, v, sv, tol_abs, shdf));
            ev_mark(h, 3, 0);
            launch_apply_bicg_df(h->op64, h->dft, 2, shdf, t, sv, o->conj, h->sc, h->fparts, h->counter, s);
            ev_mark(h, 3, 1);
        } else {
            launch_bicg_s_fused(r, v, sv, h->sc, N, h->fparts, h->counter, tol_abs, s);
            TRY(precond(h, o, sv, sh, o->conj));
            ev_mark(h, 3, 0);
            launch_apply_bicg(h->op64, 2, sh, t, sv, o->conj, h->sc, h->fparts, h->counter, s);
            ev_mark(h, 3, 1);
        }
        launch_bicg_xr_fused(x, r, ph, sh, sv, t, rh, h->sc, N, h->fparts, h->counter, o->tol, bnorm, s);
        h->launches += fuse ? 3 : 5;
        CK(cudaMemcpyAsync(h->hring + 2 * S_NSLOTS * slot, h->sc, S_NSLOTS * sizeof(double2),
                           cudaMemcpyDeviceToHost, s));
        CK(cudaEventRecord(h->evring[slot], s));
        CKL();
        return HELM_OK;
    };
    // Lagged polling: iteration i + 1 is queued before the host waits for the scalars
    // of iteration i, so the GPU does not idle while the host decides.  When iteration
    // i ends the loop, its x/r kernel has set S_STOP on the device and the queued
    // iteration leaves x and r untouched (its other outputs are scratch), so the state
    // is exactly that of iteration i.
    int inflight = 0, head = 0;   // queued but unread iterations; slot of the oldest
    while (true) {
        if (inflight == 0) {
            if (iters >= o->maxit) break;
            TRY(launch_iter(head));
            inflight = 1;
        }
        if (inflight == 1 && iters + 1 < o->maxit) {
            TRY(launch_iter(head ^ 1));
            inflight = 2;
        }
        CK(cudaEventSynchronize(h->evring[head]));
        const double* snap = h->hring + 2 * S_NSLOTS * head;
        head ^= 1;
        --inflight;
        st->precond_applies += 2;
        st->matvecs += 2;
        ++iters;
        const double brk = snap[2 * S_FLAGS + 1];
        if (brk == 4.0) { st->status = HELM_TIMEOUT; break; }
        if (brk == 1.0) { st->status = HELM_BREAKDOWN; break; }
        res = std::sqrt(snap[2 * S_RN2]) / bnorm;
        hist.push(res);
        if (!std::isfinite(res)) { st->status = HELM_DIVERGED; break; }
        if (res <= o->tol) {
            // any queued iteration is a no-op on x and r; drop it
            inflight = 0;
            head = 0;
            TRY(residual_norm(h, f, x, r, o->conj, S_RN2));
            ++st->matvecs;
            TRY(poll(h));
            const double rt = std::sqrt(hs(h, S_RN2)) / bnorm;
            if (rt <= o->tol) {
                st->status = HELM_OK;
                res = rt;
                break;
            }
            ++restarts;
            TRY(restart());
        } else if (brk == 2.0 || brk == 3.0) {
            st->status = HELM_BREAKDOWN;
            break;
        }
    }
    // final true residual
    TRY(residual_norm(h, f, x, t, o->conj, S_RN2));
    TRY(poll(h));
    st->rel_res = std::sqrt(hs(h, S_RN2)) / bnorm;
    st->iters = iters;
    st->cycles = restarts;
    return HELM_OK;
}

// ------------------------------------------- complex64 BiCGStab (MIXED handles)
// BiCGStab with right preconditioning whose vectors, operator and preconditioner are
// complex64, with reliable updates of an FP64 iterate (bicg32.cu): when the recursive
// residual has dropped below kReliableDelta times its largest value since the last
// update, or met the tolerance, the host folds the increment into x, recomputes the
// true residual in FP64 and replaces the recursive one by it (keeping the search
// direction); a breakdown restarts from the true residual (rhat = r, p = v = 0).
// A recursive residual that grows past rel_runaway times the last true one (a
// runaway of the complex64 recursion) drops the increment and restarts from the
// FP64 iterate.  With rel_guard > 0 a fold is first tried: if the true residual of
// x + xl exceeds rel_guard times the best true one so far the increment is taken back
// out and the iteration restarts from x.  Convergence is decided on the FP64 true
// residual only.

// runaway resets and rejected folds after which the complex64 BiCGStab hands the
// solve to the FP64 BiCGStab (with the same complex64 cycle); the largest factor by
// which the final fold of an unconverged solve may raise the best true residual
constexpr int kMixedTroubles = 4;
constexpr double kFinalGuard = 1e2;

helm_status ensure_b32(helm_handle* h) {
    while (h->b32.size() < 9) {
        float2* p = nullptr;
        TRY(dalloc(h, &p, (size_t)h->N));
        h->b32.push_back(p);
    }
    if (!h->b32parts) TRY(dalloc(h, &h->b32parts, (size_t)3 * bicg32_blocks()));
    if (!h->a32parts) TRY(dalloc(h, &h->a32parts, (size_t)5 * apply_grid_blocks(h->op32.dim, h->n)));
    return HELM_OK;
}

helm_status solve_bicgstab32(helm_handle* h, const helm_solve_opts* o, const double2* f, double2* x,
                             helm_stats* st, Hist& hist, double bnorm, bool* gave_up) {
    *gave_up = false;
    TRY(ensure_tmp(h, 2));
    TRY(ensure_tmp32(h, 4));
    TRY(ensure_b32(h));
    const long long N = h->N;
    cudaStream_t s = h->stream;
    double2* r64 = h->tmp[1];
    float2 *r = h->b32[0], *rh = h->b32[1], *p = h->b32[2], *v = h->b32[3], *sv = h->b32[4], *t = h->b32[5],
           *ph = h->b32[6], *sh = h->b32[7], *xl = h->b32[8];
    double* parts = h->b32parts;
    double2* xtry = h->tmp[0];                   // trial folds (copy of x plus the increment)
    const double tol_abs = o->tol * bnorm;
    TRY(residual_norm(h, f, x, r64, o->conj, S_RN2));
    ++st->matvecs;
    TRY(poll(h));
    double res = std::sqrt(hs(h, S_RN2)) / bnorm;
    hist.push(res);
    st->rel_res = res;
    if (res <= o->tol) {
        st->status = HELM_OK;
        st->iters = 0;
        return HELM_OK;
    }
    CK(cudaMemsetAsync(xl, 0, sizeof(float2) * N, s));
    launch_b32_set_tol(h->sc, tol_abs, s);
    launch_b32_replace(r64, r, rh, p, v, 1, h->sc, N, parts, h->counter, s);
    h->launches += 2;
    CKL();
    // the kernels of one iteration, on h->stream
    auto enqueue_iter = [&]() -> helm_status {
        const cudaStream_t q = h->stream;
        launch_b32_update_p(r, v, p, h->sc, N, q);
        TRY(precond32(h, o, p, ph, o->conj));
        // v = A phat with the partial sums of <rhat, v> in its epilogue where the pair
        // kernels apply (k32_s then forms alpha itself); else the operator, then the
        // reduction kernel.  The two parts buffers keep both sets of partials apart.
        ev_mark(h, 3, 0);
        const int na = launch_apply32_bicg(h->op32, 1, ph, v, rh, o->conj, h->sc, h->a32parts, q);
        if (!na) launch_apply<float>(h->op32, ph, nullptr, v, nullptr, o->conj, false, q);
        ev_mark(h, 3, 1);
        if (na) {
            launch_b32_s_dot(r, v, sv, h->sc, N, parts, h->counter, h->a32parts, na, q);
        } else {
            launch_b32_alpha(rh, v, h->sc, N, parts, h->counter, q);
            launch_b32_s(r, v, sv, h->sc, N, parts, h->counter, q);
        }
        TRY(precond32(h, o, sv, sh, o->conj));
        // t = A shat with the partial sums of <t, s> and <t, t> (omega, formed by k32_xr)
        ev_mark(h, 3, 0);
        const int no = launch_apply32_bicg(h->op32, 2, sh, t, sv, o->conj, h->sc, h->a32parts + 2 * (size_t)na, q);
        if (!no) launch_apply<float>(h->op32, sh, nullptr, t, nullptr, o->conj, false, q);
        ev_mark(h, 3, 1);
        if (no) {
            launch_b32_xr_dot(xl, r, ph, sh, sv, t, rh, h->sc, N, parts, h->counter, h->a32parts + 2 * (size_t)na, no,
                              q);
        } else {
            launch_b32_omega(t, sv, h->sc, N, parts, h->counter, q);
            launch_b32_xr(xl, r, ph, sh, sv, t, rh, h->sc, N, parts, h->counter, q);
        }
        const bool fa = na != 0, fo = no != 0;
        h->launches += 5 + (fa ? 0 : 1) + (fo ? 0 : 1);
        CKL();
        return HELM_OK;
    };
    // without per-launch profiling the iteration is captured once as a CUDA graph (on a
    // private stream: the legacy default stream cannot be captured) and replayed
    const bool use_graph = !h->profile;
    const int key[5] = {o->relax, o->n_r, o->correction, o->conj, 1};
    if (use_graph && (!h->g32 || std::memcmp(key, h->g32_key, sizeof(key)) != 0 || h->g32_omega != o->omega)) {
        drop_graphs(h);
        if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        {
            const cudaStream_t saved = h->stream;
            const long long l0 = h->launches;
            const std::string err0 = h->err;
            h->stream = h->cap_stream;
            CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
            const helm_status cst = enqueue_iter();
            cudaGraph_t graph = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &graph);
            h->stream = saved;
            cudaError_t ie = cudaErrorUnknown;
            if (cst == HELM_OK && ce == cudaSuccess) ie = cudaGraphInstantiate(&h->g32, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            h->g32_launches = h->launches - l0;
            h->launches = l0;
            if (ie != cudaSuccess) {
                h->g32 = nullptr;
                cudaGetLastError();
                h->err = err0;
                return cst != HELM_OK ? cst : fail(h, HELM_CUDA_ERROR, "capture of the BiCGStab iteration failed");
            }
        }
        std::memcpy(h->g32_key, key, sizeof(key));
        h->g32_omega = o->omega;
    }
    auto launch_iter = [&](int slot) -> helm_status {
        if (use_graph) {
            CK(cudaGraphLaunch(h->g32, s));
            h->launches += h->g32_launches;
        } else {
            TRY(enqueue_iter());
        }
        CK(cudaMemcpyAsync(h->hring + 2 * S_NSLOTS * slot, h->sc, S_NSLOTS * sizeof(double2),
                           cudaMemcpyDeviceToHost, s));
        CK(cudaEventRecord(h->evring[slot], s));
        CKL();
        return HELM_OK;
    };
    // x += xl; r64 = f - A x (FP64, its norm in S_BETA2); r = complex64(r64) with rho,
    // beta (restart: also rhat = r, p = v = 0); the host waits for the result
    bool rejected = false;
    auto reliable_update = [&](int restart, int drop, double last) -> helm_status {
        rejected = false;
        if (drop || !(h->rel_guard > 0.0)) {
            launch_b32_fold(x, xl, N, s, drop ? 1 : 0);
            TRY(residual_norm(h, f, x, r64, o->conj, S_BETA2));
            launch_b32_replace(r64, r, rh, p, v, restart, h->sc, N, parts, h->counter, s);
            h->launches += 2;
            ++st->matvecs;
            CKL();
            return poll(h);
        }
        // the trial fold goes into a copy of x (taking a large increment back out of x
        // itself would cancel x's digits); accepted, x += xl gives the same values
        CK(cudaMemcpyAsync(xtry, x, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
        launch_b32_fold(xtry, xl, N, s, 2);
        TRY(residual_norm(h, f, xtry, r64, o->conj, S_BETA2));
        ++st->matvecs;
        TRY(poll(h));
        const double rt = std::sqrt(hs(h, S_BETA2)) / bnorm;
        if (std::isfinite(rt) && rt <= h->rel_guard * last) {
            launch_b32_fold(x, xl, N, s, 0);
            launch_b32_replace(r64, r, rh, p, v, restart, h->sc, N, parts, h->counter, s);
            h->launches += 4;
            CKL();
            return poll(h);
        }
        // the increment made the iterate worse: drop it and start afresh from x
        rejected = true;
        launch_b32_fold(x, xl, N, s, 1);
        TRY(residual_norm(h, f, x, r64, o->conj, S_BETA2));
        launch_b32_replace(r64, r, rh, p, v, 1, h->sc, N, parts, h->counter, s);
        h->launches += 4;
        ++st->matvecs;
        CKL();
        return poll(h);
    };
    st->status = HELM_NOT_CONVERGED;
    double maxrr = res, last_true = res, best_true = res;
    int iters = 0, restarts = 0, inflight = 0, head = 0, since_start = 0, troubles = 0;
    while (true) {
        if (inflight == 0) {
            if (iters >= o->maxit) break;
            TRY(launch_iter(head));
            inflight = 1;
        }
        if (inflight == 1 && iters + 1 < o->maxit) {
            TRY(launch_iter(head ^ 1));
            inflight = 2;
        }
        CK(cudaEventSynchronize(h->evring[head]));
        const double* snap = h->hring + 2 * S_NSLOTS * head;
        head ^= 1;
        --inflight;
        st->precond_applies += 2;
        st->matvecs += 2;
        ++iters;
        ++since_start;
        const double brk = snap[2 * S_FLAGS + 1];
        const bool stop = snap[2 * S_STOP] != 0.0;
        if (brk == 4.0) { st->status = HELM_TIMEOUT; break; }
        const double rn = std::sqrt(snap[2 * S_RN2]) / bnorm;
        hist.push(rn);
        // a runaway of the complex64 recursion (or a non-finite value): drop the
        // increment and restart from the FP64 iterate
        const bool reset = !std::isfinite(rn) || rn > h->rel_runaway * last_true;
        if (!stop && !reset && rn >= h->rel_delta * maxrr) {
            maxrr = std::max(maxrr, rn);
            continue;
        }
        // drain the queued iteration: a no-op if this one stopped, else a real one
        if (inflight) {
            CK(cudaEventSynchronize(h->evring[head]));
            if (!stop) {
                st->precond_applies += 2;
                st->matvecs += 2;
                ++iters;
                ++since_start;
            }
            inflight = 0;
        }
        head = 0;
        TRY(reliable_update(reset ? 1 : 0, reset ? 1 : 0, best_true));
        const double rt = std::sqrt(hs(h, S_BETA2)) / bnorm;
        res = rt;
        if (rt <= o->tol) { st->status = HELM_OK; break; }
        if (!std::isfinite(rt)) { st->status = HELM_DIVERGED; break; }
        best_true = std::min(best_true, rt);
        if (reset || rejected) {
            ++restarts;
            since_start = 0;
            maxrr = last_true = rt;
            // the complex64 recursion keeps running away: hand the rest of the solve to
            // the FP64 BiCGStab (from the FP64 iterate, which the guard kept clean)
            if (++troubles >= kMixedTroubles) {
                *gave_up = true;
                break;
            }
            continue;
        }
        if (stop && brk != 0.0) {
            // breakdown (rho, <rhat, v> or <t, t> zero, or omega zero): restart from
            // the true residual just computed, unless the (re)start itself broke down
            if (since_start <= 1) { st->status = HELM_BREAKDOWN; break; }
            since_start = 0;
            launch_b32_replace(r64, r, rh, p, v, 1, h->sc, N, parts, h->counter, s);
            h->launches += 1;
            CKL();
            ++restarts;
        }
        maxrr = last_true = rt;
    }
    // fold what is left of the increment and take the final true residual; without
    // convergence the fold is tried first and taken back out if it left the iterate
    // more than kFinalGuard times worse than the best true residual (an increment
    // that drifted away from its recursive residual)
    if (st->status != HELM_OK) {
        CK(cudaMemcpyAsync(xtry, x, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
        launch_b32_fold(xtry, xl, N, s, 2);
        TRY(residual_norm(h, f, xtry, r64, o->conj, S_RN2));
        TRY(poll(h));
        const double rt = std::sqrt(hs(h, S_RN2)) / bnorm;
        launch_b32_fold(x, xl, N, s, (std::isfinite(rt) && rt <= kFinalGuard * best_true) ? 0 : 1);
        h->launches += 3;
        ++st->matvecs;
    } else {
        launch_b32_fold(x, xl, N, s);
        h->launches += 1;
    }
    TRY(residual_norm(h, f, x, r64, o->conj, S_RN2));
    TRY(poll(h));
    st->rel_res = std::sqrt(hs(h, S_RN2)) / bnorm;
    if (st->status == HELM_NOT_CONVERGED && st->rel_res <= o->tol) st->status = HELM_OK;
    st->iters = iters;
    st->cycles = restarts;
    return HELM_OK;
}

void fill_tables(helm_handle* h) {
    Op<double>& o = h->op64;
    Op<float>& f = h->op32;
    o.dim = f.dim = h->dim;
    o.n = f.n = h->n;
    o.L = f.L = h->L;
    o.N = f.N = h->N;
    o.hinv2 = 1.0 / (h->h * h->h);
    f.hinv2 = (float)o.hinv2;
    o.dre = h->k0 * h->k0 - 2.0 * h->dim / (h->h * h->h);
    f.dre = (float)o.dre;
    o.mask = f.mask = h->mask;
    o.lidx = f.lidx = h->lidx;
    o.nbm = f.nbm = h->nbm;
    o.face = f.face = h->face;
    for (int m = 0; m <= kMaxLayerCells; ++m) {
        double eta = (h->L > 0 && m <= h->L) ? (double)m / (double)h->L : 0.0;
        double im = h->k0 * h->k0 * ((h->strength * eta) * eta);
        o.im[m] = im;
        f.im[m] = (float)im;
        double2 inv = cdiv(make_double2(1.0, 0.0), make_double2(o.dre, im));
        o.invd_tab[m] = inv;
        f.invd_tab[m] = make_float2((float)inv.x, (float)inv.y);
    }
    o.k2 = h->k2;
    o.invd = h->invd;
    f.k2 = h->k2f;
    f.invd = h->invdf;
    // FP32-pair copies (hi = nearest float, lo = nearest float of the remainder)
    auto split = [](double v) {
        const float hi = (float)v;
        return make_float2(hi, (float)(v - (double)hi));
    };
    DfTab& t = h->dft;
    t.hinv2 = split(o.hinv2);
    t.dre = split(o.dre);
    for (int m = 0; m <= kMaxLayerCells; ++m) {
        t.im[m] = split(o.im[m]);
        const float2 re = split(o.invd_tab[m].x), im = split(o.invd_tab[m].y);
        t.invd[m] = make_float4(re.x, re.y, im.x, im.y);
    }
    // the fused sweep's launch shape queries the occupancy once per row width: here,
    // outside any stream capture
    (void)rbgs_sweep32_ok(f, nullptr, nullptr, nullptr);
}

// A_c = Q^T (A Q) and its inverse from a node-major copy of Q (N x ldq)
helm_status build_coarse(helm_handle* h, const double* Qrm, int ldq, int k) {
    const long long N = h->N;
    cudaStream_t s = h->stream;
    double *Wc = nullptr, *Cc = nullptr, *part = nullptr;
    double2* gj = nullptr;
    auto cleanup = [&]() { dfree(Wc); dfree(Cc); dfree(part); dfree(gj); };
    helm_status st;
    if ((st = dalloc(h, &Wc, (size_t)N * 2 * ldq)) != HELM_OK || (st = dalloc(h, &Cc, (size_t)k * 2 * k)) != HELM_OK ||
        (st = dalloc(h, &part, (size_t)(2 * 152 + 64) * 64 * 64 * 2 + (size_t)k * 2 * k * 2)) != HELM_OK ||
        (st = dalloc(h, &gj, (size_t)k * 2 * k)) != HELM_OK) {
        cleanup();
        return st;
    }
    if (!h->Ainv && (st = dalloc(h, &h->Ainv, (size_t)k * k)) != HELM_OK) {
        cleanup();
        return st;
    }
    launch_apply_columns(h->op64, Qrm, ldq, k, Wc, 2 * ldq, s);
    launch_gram(Qrm, ldq, k, Wc, 2 * ldq, 2 * k, N, part, Cc, s);
    cudaMemsetAsync(h->dflag, 0, sizeof(int) * 8, s);
    launch_gauss_jordan(Cc, 2 * k, k, h->Ainv, gj, h->dflag, s);
    int flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) return fail(h, HELM_CUDA_ERROR, cudaGetErrorString(e));
    if (flag) return fail(h, HELM_SINGULAR_COARSE, "coarse operator A_c is singular");
    return HELM_OK;
}

// after a synchronised solve or preconditioner call: HELM_TIMEOUT (with the barrier
// state reset) if a grid-barrier wait of the cooperative cycle gave up
helm_status clear_barrier_timeout(helm_handle* h) {
    int waited_out = 0;
    CK(cudaMemcpy(&waited_out, h->dflag + 2, sizeof(int), cudaMemcpyDeviceToHost));
    if (!waited_out) return HELM_OK;
    CK(cudaMemset(h->dflag + 2, 0, sizeof(int)));
    CK(cudaMemset(h->counter + 2, 0, 2 * sizeof(unsigned)));
    CK(cudaMemset(h->sc + S_FLAGS, 0, sizeof(double2)));
    CK(cudaMemset(h->sc + S_STOP, 0, sizeof(double2)));
    return fail(h, HELM_TIMEOUT, "a grid-barrier wait of the red-black cycle timed out");
}

}  // namespace

// =============================================================== C ABI
extern "C" {

helm_status helm_create(int dim, int n, double k0, int layer_cells, double layer_strength, const uint8_t* mask,
                        const double* k2, int precision, helm_handle** out) {
    helm_handle* h = nullptr;
    if (!out) return HELM_BAD_ARG;
    *out = nullptr;
    if ((dim != 2 && dim != 3) || n < 3 || layer_cells < 0 || layer_cells > kMaxLayerCells || !mask ||
        (precision != HELM_FP64 && precision != HELM_MIXED) || !std::isfinite(k0) || !std::isfinite(layer_strength))
        return HELM_BAD_ARG;
    long long N = 1;
    for (int a = 0; a < dim; ++a) N *= n;
    if (N >= (1LL << 31) || n > 65535) return HELM_BAD_ARG;
    int dev = 0, ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return HELM_NO_DEVICE;
    }
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return HELM_NO_DEVICE;
    if (prop.major * 10 + prop.minor != 103) return HELM_NO_DEVICE;
    h = new helm_handle();
    h->dim = dim;
    h->n = n;
    h->N = N;
    h->L = layer_cells;
    h->k0 = k0;
    h->strength = layer_strength;
    h->precision = precision;
    h->h = 1.0 / (n - 1);
    h->hinv2 = 1.0 / (h->h * h->h);
    auto bail = [&](helm_status st) {
        helm_destroy(h);
        return st;
    };
    if (dalloc(h, &h->mask, (size_t)N) != HELM_OK) return bail(HELM_OUT_OF_MEMORY);
    if (cudaMemcpy(h->mask, mask, (size_t)N, cudaMemcpyDefault) != cudaSuccess) return bail(HELM_CUDA_ERROR);
    h->red_len = std::max<long long>(apply_grid_blocks(dim, n), 4LL * kRedBlocks) * 2;
    if (dalloc(h, &h->red, (size_t)h->red_len) != HELM_OK) return bail(HELM_OUT_OF_MEMORY);
    if (dalloc(h, &h->sc, (size_t)S_NSLOTS) != HELM_OK) return bail(HELM_OUT_OF_MEMORY);
    if (dalloc(h, &h->dflag, 8) != HELM_OK) return bail(HELM_OUT_OF_MEMORY);
    if (dalloc(h, &h->counter, 4) != HELM_OK) return bail(HELM_OUT_OF_MEMORY);
    if (dalloc(h, &h->fparts,
               (size_t)4 * std::max<long long>(std::max(apply_grid_blocks(dim, n), bicg_grid_blocks(dim, n)),
                                               kRedBlocks)) != HELM_OK)
        return bail(HELM_OUT_OF_MEMORY);
    if (cudaMemset(h->counter, 0, 4 * sizeof(unsigned)) != cudaSuccess) return bail(HELM_CUDA_ERROR);
    if (cudaMallocHost((void**)&h->hpin, sizeof(double2) * S_NSLOTS) != cudaSuccess) return bail(HELM_OUT_OF_MEMORY);
    if (cudaMallocHost((void**)&h->hring, 2 * sizeof(double2) * S_NSLOTS) != cudaSuccess)
        return bail(HELM_OUT_OF_MEMORY);
    for (auto& e : h->evring)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return bail(HELM_CUDA_ERROR);
    if (cudaMemset(h->sc, 0, sizeof(double2) * S_NSLOTS) != cudaSuccess) return bail(HELM_CUDA_ERROR);
    if (k2) {
        if (dalloc(h, &h->k2, (size_t)N) != HELM_OK || dalloc(h, &h->invd, (size_t)N) != HELM_OK ||
            dalloc(h, &h->k2f, (size_t)N) != HELM_OK || dalloc(h, &h->invdf, (size_t)N) != HELM_OK)
            return bail(HELM_OUT_OF_MEMORY);
        if (cudaMemcpy(h->k2, k2, sizeof(double2) * N, cudaMemcpyDefault) != cudaSuccess) return bail(HELM_CUDA_ERROR);
    }
    if (dalloc(h, &h->lidx, (size_t)N) != HELM_OK) return bail(HELM_OUT_OF_MEMORY);
    if (dalloc(h, &h->nbm, (size_t)N) != HELM_OK) return bail(HELM_OUT_OF_MEMORY);
    fill_tables(h);
    launch_layer_index(h->op64, h->lidx, nullptr);
    if (k2) {
        launch_invd_field(h->op64, h->invd, nullptr);
        launch_cvt_f64_to_f32(h->k2, h->k2f, N, nullptr);
        launch_cvt_f64_to_f32(h->invd, h->invdf, N, nullptr);
    }
    cudaMemset(h->dflag, 0, sizeof(int) * 8);
    launch_check_ring(h->op64, h->dflag, nullptr);
    int bad = 0;
    if (cudaMemcpy(&bad, h->dflag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return bail(HELM_CUDA_ERROR);
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(HELM_CUDA_ERROR);
    if (bad) return bail(HELM_BAD_ARG);
    launch_nbr_code(h->op64, h->nbm, nullptr);
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(HELM_CUDA_ERROR);
    cudaEventCreate(&h->ev0);
    cudaEventCreate(&h->ev1);
    *out = h;
    return HELM_OK;
}

helm_status helm_create_bvp(int dim, int n, double k0, const uint8_t* mask, const double* k2, int neumann_top,
                            helm_handle** out) {
    helm_handle* h = nullptr;
    if (!out) return HELM_BAD_ARG;
    *out = nullptr;
    if ((dim != 2 && dim != 3) || n < 4 || !mask || !std::isfinite(k0) || k0 < 0) return HELM_BAD_ARG;
    long long N = 1;
    for (int a = 0; a < dim; ++a) N *= n;
    if (N >= (1LL << 31) || n > 65535) return HELM_BAD_ARG;
    int dev = 0, ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return HELM_NO_DEVICE;
    }
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return HELM_NO_DEVICE;
    if (prop.major * 10 + prop.minor != 103) return HELM_NO_DEVICE;
    h = new helm_handle();
    h->dim = dim;
    h->n = n;
    h->N = N;
    h->L = 0;
    h->k0 = k0;
    h->strength = 0.0;
    h->precision = HELM_FP64;
    h->bvp = 1;
    h->neumann_top = neumann_top ? 1 : 0;
    h->h = 1.0 / (n - 1);
    h->hinv2 = 1.0 / (h->h * h->h);
    auto bail = [&](helm_status st) {
        helm_destroy(h);
        return st;
    };
    if (dalloc(h, &h->mask, (size_t)N) != HELM_OK) return bail(HELM_OUT_OF_MEMORY);
    if (cudaMemcpy(h->mask, mask, (size_t)N, cudaMemcpyDefault) != cudaSuccess) return bail(HELM_CUDA_ERROR);
    h->red_len = std::max<long long>(apply_grid_blocks(dim, n), 4LL * kRedBlocks) * 2;
    if (dalloc(h, &h->red, (size_t)h->red_len) != HELM_OK || dalloc(h, &h->sc, (size_t)S_NSLOTS) != HELM_OK ||
        dalloc(h, &h->dflag, 8) != HELM_OK || dalloc(h, &h->counter, 4) != HELM_OK ||
        dalloc(h, &h->fparts, (size_t)4 * std::max<long long>(std::max(apply_grid_blocks(dim, n),
                                                                        bicg_grid_blocks(dim, n)),
                                                               kRedBlocks)) != HELM_OK)
        return bail(HELM_OUT_OF_MEMORY);
    if (cudaMemset(h->counter, 0, 4 * sizeof(unsigned)) != cudaSuccess) return bail(HELM_CUDA_ERROR);
    if (cudaMemset(h->dflag, 0, 8 * sizeof(int)) != cudaSuccess) return bail(HELM_CUDA_ERROR);
    if (cudaMallocHost((void**)&h->hpin, sizeof(double2) * S_NSLOTS) != cudaSuccess ||
        cudaMallocHost((void**)&h->hring, 2 * sizeof(double2) * S_NSLOTS) != cudaSuccess)
        return bail(HELM_OUT_OF_MEMORY);
    for (auto& e : h->evring)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return bail(HELM_CUDA_ERROR);
    if (cudaMemset(h->sc, 0, sizeof(double2) * S_NSLOTS) != cudaSuccess) return bail(HELM_CUDA_ERROR);
    if (dalloc(h, &h->k2, (size_t)N) != HELM_OK || dalloc(h, &h->invd, (size_t)N) != HELM_OK ||
        dalloc(h, &h->k2f, (size_t)N) != HELM_OK || dalloc(h, &h->invdf, (size_t)N) != HELM_OK ||
        dalloc(h, &h->lidx, (size_t)N) != HELM_OK || dalloc(h, &h->nbm, (size_t)N) != HELM_OK ||
        dalloc(h, &h->face, (size_t)N) != HELM_OK)
        return bail(HELM_OUT_OF_MEMORY);
    fill_tables(h);
    launch_face_code(h->op64, h->face, nullptr);
    launch_layer_index(h->op64, h->lidx, nullptr);
    launch_nbr_code(h->op64, h->nbm, nullptr);
    // the scaled boundary diagonals as an effective k^2 field, then 1/diag
    launch_bvp_k2(h->op64, reinterpret_cast<const double2*>(k2), k0, h->neumann_top, h->k2, nullptr);
    launch_invd_field(h->op64, h->invd, nullptr);
    launch_cvt_f64_to_f32(h->k2, h->k2f, N, nullptr);
    launch_cvt_f64_to_f32(h->invd, h->invdf, N, nullptr);
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(HELM_CUDA_ERROR);
    cudaEventCreate(&h->ev0);
    cudaEventCreate(&h->ev1);
    *out = h;
    return HELM_OK;
}

helm_status helm_destroy(helm_handle* h) {
    if (!h) return HELM_BAD_ARG;
    drop_graphs(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (helm_handle* c : h->mg) helm_destroy(c);
    h->mg.clear();
    dfree(h->mask); dfree(h->lidx); dfree(h->nbm); dfree(h->face); dfree(h->k2); dfree(h->invd); dfree(h->k2f);
    dfree(h->invdf);
    dfree(h->red); dfree(h->sc); dfree(h->dflag); dfree(h->counter); dfree(h->fparts);
    if (h->hpin) cudaFreeHost(h->hpin);
    if (h->hring) cudaFreeHost(h->hring);
    for (auto e : h->evring)
        if (e) cudaEventDestroy(e);
    for (auto p : h->tmp) cudaFree(p);
    for (auto p : h->tmp32) cudaFree(p);
    for (auto p : h->b32) cudaFree(p);
    dfree(h->b32parts);
    dfree(h->a32parts);
    dfree(h->Q); dfree(h->Qr); dfree(h->Ainv); dfree(h->coarse_partials); dfree(h->cbuf); dfree(h->ybuf);
    if (h->Qbf) cudaFree(h->Qbf);
    if (h->Qbr) cudaFree(h->Qbr);
    dfree(h->partials32); dfree(h->y32); dfree(h->Z32);
    dfree(h->Traw); dfree(h->bw); dfree(h->nl_x); dfree(h->nl_h0); dfree(h->nl_h1);
    dfree(h->V); dfree(h->Z); dfree(h->Hm); dfree(h->cs); dfree(h->sn); dfree(h->g); dfree(h->y); dfree(h->hpart);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    for (auto& pool : h->evpool)
        for (auto e : pool) cudaEventDestroy(e);
    delete h;
    return HELM_OK;
}

helm_status helm_set_stream(helm_handle* h, void* stream) {
    if (!h) return HELM_BAD_ARG;
    h->stream = (cudaStream_t)stream;
    return HELM_OK;
}

const char* helm_last_error(const helm_handle* h) { return h ? h->err.c_str() : "null handle"; }

helm_status helm_checked_status(int* checked, unsigned long long* first) {
    if (!checked || !first) return HELM_BAD_ARG;
#ifdef HELM_CHECKED
    *checked = 1;
#else
    *checked = 0;
#endif
    *first = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return HELM_CUDA_ERROR;
    for (auto take : checked_units()) {
        const unsigned long long v = take();
        if (v && !*first) *first = v;
    }
    return HELM_OK;
}

helm_status helm_set_profiling(helm_handle* h, int on) {
    if (!h) return HELM_BAD_ARG;
    h->profile = on ? 1 : 0;
    return HELM_OK;
}

helm_status helm_info(const helm_handle* h, long long* N, double* hstep) {
    if (!h) return HELM_BAD_ARG;
    if (N) *N = h->N;
    if (hstep) *hstep = h->h;
    return HELM_OK;
}

helm_status helm_layer_k2(helm_handle* h, const double* scale, double* k2_out) {
    if (!h || !k2_out) return fail(h, HELM_BAD_ARG, "null argument");
    if (h->bvp) return fail(h, HELM_BAD_ARG, "no absorbing layer on an outer-boundary (helm_create_bvp) handle");
    launch_layer_k2(h->op64, h->k0, h->strength, scale, reinterpret_cast<double2*>(k2_out), h->stream);
    CKL();
    return HELM_OK;
}

helm_status helm_rhs(helm_handle* h, const double* src, const double* g, double* b) {
    if (h && h->bvp && src && g && b) {
        launch_rhs_bvp(h->op64, (const double2*)src, (const double2*)g, h->neumann_top, (double2*)b, h->stream);
        CKL();
        return HELM_OK;
    }
    if (!h || !src || !g || !b) return fail(h, HELM_BAD_ARG, "null argument");
    launch_rhs(h->op64, reinterpret_cast<const double2*>(src), reinterpret_cast<const double2*>(g),
               reinterpret_cast<double2*>(b), h->stream);
    CKL();
    return HELM_OK;
}

helm_status helm_apply(helm_handle* h, const void* x, void* y, int conj, int dtype) {
    if (!h || !x || !y) return fail(h, HELM_BAD_ARG, "null argument");
    if (dtype == HELM_C128)
        launch_apply<double>(h->op64, (const double2*)x, nullptr, (double2*)y, nullptr, conj, false, h->stream);
    else if (dtype == HELM_C64)
        launch_apply<float>(h->op32, (const float2*)x, nullptr, (float2*)y, nullptr, conj, false, h->stream);
    else
        return fail(h, HELM_BAD_ARG, "dtype");
    CKL();
    return HELM_OK;
}

helm_status helm_residual(helm_handle* h, const void* f, const void* x, void* r, double* norm2, int conj,
                          int dtype) {
    if (!h || !f || !x || !r) return fail(h, HELM_BAD_ARG, "null argument");
    double* part = norm2 ? h->red : nullptr;
    int nb = 0;
    if (dtype == HELM_C128)
        nb = launch_apply<double>(h->op64, (const double2*)x, (const double2*)f, (double2*)r, part, conj, true,
                                  h->stream);
    else if (dtype == HELM_C64)
        nb = launch_apply<float>(h->op32, (const float2*)x, (const float2*)f, (float2*)r, part, conj, true,
                                 h->stream);
    else
        return fail(h, HELM_BAD_ARG, "dtype");
    if (norm2) launch_sum_real(h->red, nb, norm2, h->stream);
    CKL();
    return HELM_OK;
}

helm_status helm_relax(helm_handle* h, int kind, double omega, int sweeps, const void* f, void* x, int conj,
                       int dtype) {
    if (!h || !f || !x || sweeps < 0) return fail(h, HELM_BAD_ARG, "bad argument");
    if (kind != HELM_JACOBI && !red_black(kind)) return fail(h, HELM_BAD_ARG, "kind");
    cudaStream_t s = h->stream;
    if (dtype == HELM_C128) {
        if (kind == HELM_JACOBI) {
            TRY(ensure_tmp(h, 1));
            double2* a = (double2*)x;
            double2* b = h->tmp[0];
            for (int q = 0; q < sweeps; ++q) {
                launch_jacobi<double>(h->op64, omega, (const double2*)f, a, b, conj, false, s);
                std::swap(a, b);
            }
            if (a != x) CK(cudaMemcpyAsync(x, a, sizeof(double2) * h->N, cudaMemcpyDeviceToDevice, s));
        } else {
            red_black_sweeps<double>(h, h->op64, kind, omega, sweeps, (const double2*)f, (double2*)x, conj, false);
        }
    } else if (dtype == HELM_C64) {
        if (kind == HELM_JACOBI) {
            TRY(ensure_tmp32(h, 1));
            float2* a = (float2*)x;
            float2* b = h->tmp32[0];
            for (int q = 0; q < sweeps; ++q) {
                launch_jacobi<float>(h->op32, omega, (const float2*)f, a, b, conj, false, s);
                std::swap(a, b);
            }
            if (a != x) CK(cudaMemcpyAsync(x, a, sizeof(float2) * h->N, cudaMemcpyDeviceToDevice, s));
        } else {
            TRY(ensure_tmp32(h, 1));
            if (!fused_sweeps32(h, kind, omega, sweeps, (const float2*)f, (float2*)x, h->tmp32[0], conj, false))
                red_black_sweeps<float>(h, h->op32, kind, omega, sweeps, (const float2*)f, (float2*)x, conj, false);
        }
    } else {
        return fail(h, HELM_BAD_ARG, "dtype");
    }
    CKL();
    return HELM_OK;
}

helm_status don_load(helm_handle* h, const double* weights, const int* widths, int n_layers, int act, int p,
                     double tau) {
    NvtxRange nvtx("don_load: trunk basis setup");
    if (!h || !weights || !widths) return fail(h, HELM_BAD_ARG, "null argument");
    if (act != HELM_ACT_TANH && act != HELM_ACT_LEAKY_RELU) return fail(h, HELM_BAD_ARG, "activation");
    drop_graphs(h);
    if (n_layers < 1 || n_layers > 7) return fail(h, HELM_BAD_ARG, "n_layers must be 1..7");
    if (widths[0] != h->dim) return fail(h, HELM_BAD_ARG, "widths[0] must equal dim");
    for (int i = 1; i <= n_layers; ++i)
        if (widths[i] < 1 || widths[i] > 256) return fail(h, HELM_BAD_ARG, "layer widths must be 1..256");
    if (p < 1 || p > kMaxP || widths[n_layers] < p) return fail(h, HELM_BAD_ARG, "p must be 1..min(256, out width)");
    if (!(tau >= 0.0) || tau >= 1.0) return fail(h, HELM_BAD_ARG, "tau must be in [0, 1)");
    cudaStream_t s = h->stream;
    // weights: transpose each W to (in x out) for coalesced reads
    std::vector<double> hw;
    size_t off = 0;
    for (int l = 0; l < n_layers; ++l) {
        const int win = widths[l], wout = widths[l + 1];
        const double* W = weights + off;
        const double* b = W + (size_t)win * wout;
        for (int i = 0; i < win; ++i)
            for (int o = 0; o < wout; ++o) hw.push_back(W[(size_t)o * win + i]);
        for (int o = 0; o < wout; ++o) hw.push_back(b[o]);
        off += (size_t)win * wout + wout;
    }
    dfree(h->Q); dfree(h->Qr); dfree(h->Ainv); dfree(h->coarse_partials); dfree(h->cbuf); dfree(h->ybuf);
    h->k = 0;
    const long long N = h->N;
    const int ldt = round32(p);
    double *dW = nullptr, *T = nullptr, *G = nullptr, *Wk = nullptr, *R = nullptr, *Rinv = nullptr, *Q1 = nullptr,
           *Wc = nullptr, *Cc = nullptr, *part = nullptr;
    double2* gj = nullptr;
    int* kept = nullptr;
    helm_status st = HELM_OK;
    auto cleanup = [&]() {
        dfree(dW); dfree(T); dfree(G); dfree(Wk); dfree(R); dfree(Rinv); dfree(Q1); dfree(Wc); dfree(Cc);
        dfree(part); dfree(gj); dfree(kept);
    };
#define STEP(expr)                \
    do {                          \
        st = (expr);              \
        if (st != HELM_OK) {      \
            cleanup();            \
            return st;            \
        }                         \
    } while (0)
#define STEPC(call)                                                                                   \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) {                                                                      \
            cleanup();                                                                                \
            return fail(h, HELM_CUDA_ERROR, std::string(#call) + ": " + cudaGetErrorString(e_));      \
        }                                                                                             \
    } while (0)
    STEP(dalloc(h, &dW, hw.size()));
    STEPC(cudaMemcpy(dW, hw.data(), hw.size() * sizeof(double), cudaMemcpyHostToDevice));
    STEP(dalloc(h, &T, (size_t)N * ldt));
    STEP(dalloc(h, &G, (size_t)p * p));
    STEP(dalloc(h, &Wk, (size_t)p * p));
    STEP(dalloc(h, &R, (size_t)p * p));
    STEP(dalloc(h, &Rinv, (size_t)p * p));
    STEP(dalloc(h, &kept, (size_t)p));
    STEP(dalloc(h, &part, (size_t)2 * 152 * 64 * 64 * 4 + (size_t)p * 2 * p * 16));
    launch_trunk_eval(h->op64, dW, widths, n_layers, p, act, T, ldt, s);
    dfree(h->Traw);
    STEP(dalloc(h, &h->Traw, (size_t)N * p));
    launch_rm_to_cm_f32(T, ldt, p, h->Traw, N, s);
    launch_gram(T, ldt, p, T, ldt, p, N, part, G, s);
    STEPC(cudaMemsetAsync(h->dflag, 0, sizeof(int) * 8, s));
    launch_select_chol(G, p, p, tau, Wk, R, kept, h->dflag + 1, h->dflag, s);
    STEPC(cudaGetLastError());
    int hk[2] = {0, 0};
    STEPC(cudaMemcpyAsync(hk, h->dflag, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
    STEPC(cudaStreamSynchronize(s));
    const int k = hk[1];
    if (hk[0] != 0 || k == 0) {
        cleanup();
        return fail(h, HELM_SINGULAR_COARSE, "trunk basis is empty (no column kept)");
    }
    h->kept.assign(k, 0);
    STEPC(cudaMemcpy(h->kept.data(), kept, sizeof(int) * k, cudaMemcpyDeviceToHost));
    const int ldq = round32(k);
    launch_tri_inverse(R, k, p, Rinv, s);
    STEP(dalloc(h, &Q1, (size_t)N * ldq));
    launch_gather_times_upper(T, ldt, kept, k, Rinv, p, Q1, ldq, N, s);
    // CholeskyQR2 second pass: Q = Q1 R2^-1 with Q1^T Q1 = R2^T R2
    launch_gram(Q1, ldq, k, Q1, ldq, k, N, part, G, s);
    STEPC(cudaMemsetAsync(h->dflag, 0, sizeof(int) * 8, s));
    launch_select_chol(G, k, k, 0.0, Wk, R, kept, h->dflag + 1, h->dflag, s);
    STEPC(cudaMemcpyAsync(hk, h->dflag, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
    STEPC(cudaStreamSynchronize(s));
    if (hk[1] != k) {
        cleanup();
        return fail(h, HELM_SINGULAR_COARSE, "second CholeskyQR pass lost rank");
    }
    launch_tri_inverse(R, k, k, Rinv, s);
    dfree(T);
    STEP(dalloc(h, &T, (size_t)N * ldq));            // node-major Q for the setup GEMMs
    launch_gather_times_upper(Q1, ldq, nullptr, k, Rinv, k, T, ldq, N, s);
    dfree(Q1);
    if (h->precision == HELM_MIXED) {
        // the coarse operator is built from the same rounded basis the kernels use
        launch_round_bf16(T, ldq, k, N, s);
        dfree(h->Qbf);
        dfree(h->Qbr);
        const long long ldb = basis_ld(N), ldr = basis_ld((N + 1) / 2);
        STEPC(cudaMalloc(&h->Qbf, (size_t)ldb * k * 2));
        STEPC(cudaMemsetAsync(h->Qbf, 0, (size_t)ldb * k * 2, s));
        launch_rm_to_cm_bf16(T, ldq, k, h->Qbf, ldb, N, s);
        STEPC(cudaMalloc(&h->Qbr, (size_t)ldr * k * 2));
        STEPC(cudaMemsetAsync(h->Qbr, 0, (size_t)ldr * k * 2, s));
        launch_red_rows_bf16(h->Qbf, ldb, k, N, h->n, h->Qbr, ldr, s);
    }
    // column-major FP32-pair Q for the per-iteration kernels; T becomes hi + lo so that
    // A_c is built from exactly the basis the kernels apply
    // column strides padded (basis_ld): zero-filled so that padding rows are finite
    STEP(dalloc(h, &h->Q, (size_t)basis_ld(N) * k));
    STEPC(cudaMemsetAsync(h->Q, 0, sizeof(float2) * basis_ld(N) * k, s));
    launch_split_basis(T, ldq, k, h->Q, basis_ld(N), N, s);
    dfree(h->Qr);
    STEP(dalloc(h, &h->Qr, (size_t)basis_ld((N + 1) / 2) * k));
    STEPC(cudaMemsetAsync(h->Qr, 0, sizeof(float2) * basis_ld((N + 1) / 2) * k, s));
    launch_red_rows(h->Q, basis_ld(N), k, N, h->n, h->Qr, basis_ld((N + 1) / 2), s);
    // A_c = Q^T (A Q)
    st = build_coarse(h, T, ldq, k);
    if (st != HELM_OK) {
        cleanup();
        dfree(h->Q); dfree(h->Qr); dfree(h->Ainv);
        return st;
    }
    STEP(dalloc(h, &h->coarse_partials, (size_t)std::max(restrict_blocks(N), project_blocks(N)) * k));
    if (h->precision == HELM_MIXED) {
        dfree(h->partials32); dfree(h->y32);
        STEP(dalloc(h, &h->partials32,
                    (size_t)std::max({restrict_blocks(N), restrict32_red_blocks(N), restrict32_rr_ranges(N)}) * k));
        STEP(dalloc(h, &h->y32, (size_t)kMaxP));
    }
    STEP(dalloc(h, &h->cbuf, (size_t)kMaxP));
    STEP(dalloc(h, &h->ybuf, (size_t)kMaxP));
    h->p = p;
    h->k = k;
    h->ldq = ldq;
    cleanup();
    STEPC(cudaStreamSynchronize(s));
#undef STEP
#undef STEPC
    return HELM_OK;
}

helm_status don_load_branch(helm_handle* h, const float* weights, const int* widths, int n_layers) {
    if (!h || !weights || !widths || n_layers < 1 || n_layers > 8) return fail(h, HELM_BAD_ARG, "bad argument");
    if (!h->Traw) return fail(h, HELM_NOT_READY, "don_load the trunk first");
    if ((long long)widths[0] != 2 * h->N) return fail(h, HELM_BAD_ARG, "branch input width must be 2N");
    if (widths[n_layers] != 2 * h->p) return fail(h, HELM_BAD_ARG, "branch output width must be 2p");
    size_t total = 0;
    int hmax = 1;
    for (int l = 0; l < n_layers; ++l) {
        if (l > 0 && (widths[l] < 1 || widths[l] > 4096)) return fail(h, HELM_BAD_ARG, "hidden widths must be 1..4096");
        total += (size_t)widths[l] * widths[l + 1] + widths[l + 1];
        hmax = std::max(hmax, widths[l + 1]);
    }
    dfree(h->bw); dfree(h->nl_x); dfree(h->nl_h0); dfree(h->nl_h1);
    h->bwidths.assign(widths, widths + n_layers + 1);
    TRY(dalloc(h, &h->bw, total));
    TRY(dalloc(h, &h->nl_x, (size_t)2 * h->N));
    TRY(dalloc(h, &h->nl_h0, (size_t)hmax));
    TRY(dalloc(h, &h->nl_h1, (size_t)hmax));
    CK(cudaMemcpy(h->bw, weights, total * sizeof(float), cudaMemcpyHostToDevice));
    return HELM_OK;
}

helm_status don_info(const helm_handle* h, int* k, int* kept_idx) {
    if (!h) return HELM_BAD_ARG;
    if (k) *k = h->k;
    if (kept_idx)
        for (int i = 0; i < h->k; ++i) kept_idx[i] = h->kept[i];
    return HELM_OK;
}

helm_status don_get_q(const helm_handle* hc, double* q_out) {
    helm_handle* h = const_cast<helm_handle*>(hc);
    if (!h || !q_out) return fail(h, HELM_BAD_ARG, "null argument");
    if (!h->Q) return fail(h, HELM_NOT_READY, "trunk basis not loaded");
    launch_cm_pair_to_rm(h->Q, basis_ld(h->N), h->k, q_out, h->N, h->stream);
    CKL();
    return HELM_OK;
}

helm_status don_get_ainv(const helm_handle* hc, double* out) {
    helm_handle* h = const_cast<helm_handle*>(hc);
    if (!h || !out) return fail(h, HELM_BAD_ARG, "null argument");
    if (!h->Ainv) return fail(h, HELM_NOT_READY, "trunk basis not loaded");
    CK(cudaMemcpyAsync(out, h->Ainv, sizeof(double2) * h->k * h->k, cudaMemcpyDeviceToDevice, h->stream));
    return HELM_OK;
}

helm_status don_correct(helm_handle* h, int mode, const void* r, void* z, int conj, int dtype) {
    if (!h || !r || !z) return fail(h, HELM_BAD_ARG, "null argument");
    if (dtype != HELM_C128) return fail(h, HELM_BAD_ARG, "dtype");
    if (mode == HELM_CORR_NONLINEAR) {
        if (conj) return fail(h, HELM_BAD_ARG, "the nonlinear correction has no conjugate form");
        return nl_correct(h, (const double2*)r, (double2*)z);
    }
    if (mode != HELM_CORR_TB) return fail(h, HELM_BAD_ARG, "mode");
    return tb_correct(h, (const double2*)r, nullptr, (double2*)z, conj);
}

helm_status helm_precond(helm_handle* h, const helm_solve_opts* opts, const void* r, void* z) {
    if (!h || !r || !z) return fail(h, HELM_BAD_ARG, "null argument");
    TRY(check_opts(h, opts));
    TRY(precond(h, opts, (const double2*)r, (double2*)z, opts->conj));
    CK(cudaStreamSynchronize(h->stream));
    return clear_barrier_timeout(h);
}

helm_status helm_mg_setup(helm_handle* h, int levels) {
    NvtxRange nvtx("helm_mg_setup");
    if (!h) return HELM_BAD_ARG;
    if (levels < 1 || levels > 8) return fail(h, HELM_BAD_ARG, "levels must be 1..8");
    if (h->bvp) return fail(h, HELM_BAD_ARG, "the multigrid hierarchy needs the Dirichlet-ring operator");
    if (h->precision != HELM_FP64) return fail(h, HELM_BAD_ARG, "the multigrid cycle runs on FP64 handles");
    for (helm_handle* c : h->mg) helm_destroy(c);
    h->mg.clear();
    h->mg_levels = 0;
    int n = h->n;
    for (int l = 1; l < levels; ++l) {
        if (n % 2 == 0 || n < 5) return fail(h, HELM_BAD_ARG, "vertex coarsening needs an odd n >= 5 on every level");
        n = (n + 1) / 2;
    }
    helm_handle* parent = h;
    cudaStream_t s = h->stream;
    for (int l = 1; l < levels; ++l) {
        const int nf = parent->n, nc = (nf + 1) / 2;
        const long long Nf = parent->N, Nc = h->dim == 3 ? (long long)nc * nc * nc : (long long)nc * nc;
        uint8_t* mc = nullptr;
        double2 *kf = nullptr, *kc = nullptr;
        auto cleanup = [&]() { dfree(mc); dfree(kf); dfree(kc); };
        helm_status st;
        if ((st = dalloc(h, &mc, (size_t)Nc)) != HELM_OK || (st = dalloc(h, &kc, (size_t)Nc)) != HELM_OK) {
            cleanup();
            return st;
        }
        const double2* kfine = parent->k2;
        if (!kfine) {
            if ((st = dalloc(h, &kf, (size_t)Nf)) != HELM_OK) {
                cleanup();
                return st;
            }
            launch_layer_k2(parent->op64, parent->k0, parent->strength, nullptr, kf, s);
            kfine = kf;
        }
        launch_inject_mask(h->dim, nf, parent->mask, mc, s);
        launch_inject_c128(h->dim, nf, kfine, kc, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            cleanup();
            return fail(h, HELM_CUDA_ERROR, "injection to the coarse level");
        }
        helm_handle* c = nullptr;
        st = helm_create(h->dim, nc, h->k0, 0, 0.0, mc, reinterpret_cast<const double*>(kc), HELM_FP64, &c);
        cleanup();
        if (st != HELM_OK) return fail(h, st, "coarse level handle");
        c->stream = s;
        h->mg.push_back(c);
        parent = c;
    }
    h->mg_levels = levels;
    return HELM_OK;
}

helm_status helm_set_reliable(helm_handle* h, double delta, double runaway, double guard) {
    if (!h || !(delta > 0.0 && delta < 1.0) || !(runaway > 1.0) || !(guard >= 0.0))
        return fail(h, HELM_BAD_ARG, "bad argument");
    h->rel_delta = delta;
    h->rel_runaway = runaway;
    h->rel_guard = guard;
    return HELM_OK;
}

helm_status helm_set_wait_limit(helm_handle* h, unsigned polls, unsigned extra_arrivals) {
    if (!h || polls == 0) return fail(h, HELM_BAD_ARG, "bad argument");
    drop_graphs(h);         // the captured iteration holds the old limits
    h->bar_spin = polls;
    h->bar_extra = extra_arrivals;
    return HELM_OK;
}

helm_status helm_solve(helm_handle* h, const helm_solve_opts* o, const void* fv, void* xv, helm_stats* stats,
                       double* res_hist, int hist_len) {
    NvtxRange nvtx(o && o->method == HELM_METHOD_FGMRES ? "helm_solve: FGMRES"
                   : o && o->method == HELM_METHOD_BICGSTAB ? "helm_solve: BiCGStab"
                                                            : "helm_solve: relaxation");
    if (!h || !fv || !xv) return fail(h, HELM_BAD_ARG, "null argument");
    TRY(check_opts(h, o));
    const double2* f = (const double2*)fv;
    double2* x = (double2*)xv;
    helm_stats st{};
    st.status = HELM_NOT_CONVERGED;
    Hist hist{res_hist, hist_len};
    h->launches = 0;
    for (int& e : h->evn) e = 0;
    CK(cudaEventRecord(h->ev0, h->stream));
    CK(cudaMemsetAsync(h->sc + S_FLAGS, 0, sizeof(double2), h->stream));
    launch_set_masked(x, f, h->mask, h->N, h->stream);
    h->launches += 1;
    TRY(norm2_into(h, f, S_BN2));
    TRY(poll(h));
    double bnorm = std::sqrt(hs(h, S_BN2));
    if (bnorm == 0.0) {
        CK(cudaMemsetAsync(x, 0, sizeof(double2) * h->N, h->stream));
        st.status = HELM_OK;
        st.rel_res = 0;
    } else if (o->method == HELM_METHOD_RELAX) {
        TRY(solve_relax(h, o, f, x, &st, hist, bnorm));
    } else if (o->method == HELM_METHOD_FGMRES) {
        TRY(solve_fgmres(h, o, f, x, &st, hist, bnorm));
    } else if (h->precision == HELM_MIXED) {
        bool gave_up = false;
        TRY(solve_bicgstab32(h, o, f, x, &st, hist, bnorm, &gave_up));
        if (gave_up && st.status != HELM_OK && st.iters < o->maxit) {
            // the rest of the iteration budget in the FP64 BiCGStab from the current
            // iterate (complex64 cycle through conversions); the statistics add up
            helm_solve_opts o2 = *o;
            o2.maxit = o->maxit - st.iters;
            helm_stats s2{};
            s2.status = HELM_NOT_CONVERGED;
            TRY(solve_bicgstab(h, &o2, f, x, &s2, hist, bnorm));
            st.status = s2.status;
            st.rel_res = s2.rel_res;
            st.iters += s2.iters;
            st.cycles += s2.cycles + 1;
            st.precond_applies += s2.precond_applies;
            st.matvecs += s2.matvecs;
        }
    } else {
        TRY(solve_bicgstab(h, o, f, x, &st, hist, bnorm));
    }
    CK(cudaEventRecord(h->ev1, h->stream));
    CK(cudaEventSynchronize(h->ev1));
    // a grid-barrier wait that gave up leaves a flag: the blocks that gave up went on
    // unsynchronised, so the barrier's arrival counter and generation are reset before
    // the next launch and the solve reports HELM_TIMEOUT
    const helm_status bst = clear_barrier_timeout(h);
    if (bst == HELM_TIMEOUT) st.status = HELM_TIMEOUT;
    else if (bst != HELM_OK) return bst;
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    st.ms = ms;
    st.launches = h->launches;
    st.n_restrict = h->evn[0];
    st.n_prolong = h->evn[1];
    st.restrict_ms = h->profile ? ev_sum(h, 0) : 0.0;
    st.prolong_ms = h->profile ? ev_sum(h, 1) : 0.0;
    st.n_sweep = h->evn[2];
    st.sweep_ms = h->profile ? ev_sum(h, 2) : 0.0;
    st.n_apply = h->evn[3];
    st.apply_ms = h->profile ? ev_sum(h, 3) : 0.0;
    if (stats) *stats = st;
    return (helm_status)st.status;
}

helm_status helm_solve_concurrent(int nprob, helm_handle** hs, const helm_solve_opts* o, const double* const* f,
                                  double* const* x, helm_stats* stats, int threads) {
    NvtxRange nvtx("helm_solve_concurrent");
    if (nprob < 0 || (nprob > 0 && (!hs || !o || !f || !x))) return HELM_BAD_ARG;
    std::set<helm_handle*> seen;
    for (int i = 0; i < nprob; ++i) {
        if (!hs[i] || !f[i] || !x[i] || hs[i]->precision != HELM_MIXED || !seen.insert(hs[i]).second)
            return HELM_BAD_ARG;
    }
    if (nprob == 0) return HELM_OK;
    // every problem on a private non-blocking stream, ordered after its handle's stream
    std::vector<cudaStream_t> own(nprob, nullptr), saved(nprob, nullptr);
    std::vector<cudaEvent_t> ready(nprob, nullptr);
    auto release = [&]() {
        for (int i = 0; i < nprob; ++i) {
            if (own[i]) {
                hs[i]->stream = saved[i];
                cudaStreamSynchronize(own[i]);
                cudaStreamDestroy(own[i]);
            }
            if (ready[i]) cudaEventDestroy(ready[i]);
        }
    };
    for (int i = 0; i < nprob; ++i) {
        saved[i] = hs[i]->stream;
        if (cudaStreamCreateWithFlags(&own[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ready[i], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(ready[i], saved[i]) != cudaSuccess || cudaStreamWaitEvent(own[i], ready[i], 0) != cudaSuccess) {
            release();
            return HELM_CUDA_ERROR;
        }
        hs[i]->stream = own[i];
    }
    // a pool of host threads takes the problems in index order; each runs the ordinary
    // solve of its problem, which waits on its own stream only
    std::vector<helm_status> st(nprob, HELM_NOT_CONVERGED);
    std::vector<helm_stats> sv(nprob);
    std::atomic<int> next{0};
    auto work = [&]() {
        for (int i = next++; i < nprob; i = next++) st[i] = helm_solve(hs[i], o, f[i], x[i], &sv[i], nullptr, 0);
    };
    int dev = 0;
    cudaGetDevice(&dev);
    const int T = std::max(1, std::min(nprob, threads > 0 ? threads : nprob));
    std::vector<std::thread> pool;
    try {
        for (int q = 1; q < T; ++q)
            pool.emplace_back([&, dev]() {
                cudaSetDevice(dev);
                work();
            });
    } catch (...) {
        // no more threads: the ones started and this one take the remaining problems
    }
    work();
    for (auto& t : pool) t.join();
    release();
    helm_status first = HELM_OK;
    for (int i = 0; i < nprob; ++i) {
        if (stats) stats[i] = sv[i];
        if (first == HELM_OK && st[i] != HELM_OK) first = st[i];
    }
    return first;
}

helm_status helm_receivers_setup(helm_handle* h, int nrec, const double* xyz, int* idx, double* w) {
    if (!h || nrec < 0 || (nrec > 0 && (!xyz || !idx || !w))) return fail(h, HELM_BAD_ARG, "bad argument");
    if (h->dim != 3) return fail(h, HELM_BAD_ARG, "receivers need a 3D handle");
    if (nrec == 0) return HELM_OK;
    launch_receivers_setup(h->n, nrec, xyz, idx, w, h->stream);
    CKL();
    return HELM_OK;
}

helm_status helm_receivers_sample(helm_handle* h, int nrec, const int* idx, const double* w, const double* u,
                                  double* out) {
    if (!h || nrec < 0 || (nrec > 0 && (!idx || !w || !u || !out))) return fail(h, HELM_BAD_ARG, "bad argument");
    if (nrec == 0) return HELM_OK;
    launch_receivers_sample(nrec, idx, w, (const double2*)u, (double2*)out, h->stream);
    CKL();
    return HELM_OK;
}

helm_status helm_receivers_adjoint(helm_handle* h, int nrec, const int* idx, const double* w, const double* e,
                                   double* b) {
    if (!h || nrec < 0 || !b || (nrec > 0 && (!idx || !w || !e))) return fail(h, HELM_BAD_ARG, "bad argument");
    CK(cudaMemsetAsync(b, 0, sizeof(double2) * h->N, h->stream));
    if (nrec > 0) launch_receivers_adjoint(nrec, idx, w, (const double2*)e, (double2*)b, h->stream);
    CKL();
    return HELM_OK;
}

helm_status helm_k2_gradient(helm_handle* h, const double* lambda, const double* u, double* grad) {
    if (!h || !lambda || !u || !grad) return fail(h, HELM_BAD_ARG, "null argument");
    if (h->bvp) return fail(h, HELM_BAD_ARG, "k^2 gradients need the Dirichlet-ring operator");
    launch_k2_gradient(h->N, h->mask, (const double2*)lambda, (const double2*)u, (double2*)grad, h->stream);
    CKL();
    return HELM_OK;
}

helm_status helm_set_k2(helm_handle* h, const double* k2) {
    if (!h || !k2) return fail(h, HELM_BAD_ARG, "null argument");
    if (h->bvp) return fail(h, HELM_BAD_ARG, "an outer-boundary handle takes its k^2 at creation");
    drop_graphs(h);
    const long long N = h->N;
    if (!h->k2) {
        TRY(dalloc(h, &h->k2, (size_t)N));
        TRY(dalloc(h, &h->invd, (size_t)N));
        TRY(dalloc(h, &h->k2f, (size_t)N));
        TRY(dalloc(h, &h->invdf, (size_t)N));
    }
    CK(cudaMemcpyAsync(h->k2, k2, sizeof(double2) * N, cudaMemcpyDefault, h->stream));
    fill_tables(h);
    launch_invd_field(h->op64, h->invd, h->stream);
    launch_cvt_f64_to_f32(h->k2, h->k2f, N, h->stream);
    launch_cvt_f64_to_f32(h->invd, h->invdf, N, h->stream);
    CKL();
    if (h->Q) {
        // rebuild A_c for the new operator from a node-major copy of the (possibly rounded) basis
        double* Qrm = nullptr;
        TRY(dalloc(h, &Qrm, (size_t)N * h->k));
        launch_cm_pair_to_rm(h->Q, basis_ld(N), h->k, Qrm, N, h->stream);
        helm_status st = build_coarse(h, Qrm, h->k, h->k);
        cudaStreamSynchronize(h->stream);
        dfree(Qrm);
        if (st != HELM_OK) return st;
    }
    CK(cudaStreamSynchronize(h->stream));
    return HELM_OK;
}

helm_status helm_solve_host(helm_handle* h, const helm_solve_opts* o, const double* f, double* x,
                            helm_stats* stats, double* res_hist, int hist_len) {
    if (!h || !f || !x) return fail(h, HELM_BAD_ARG, "null argument");
    TRY(ensure_tmp(h, 12));
    double2* df = h->tmp[10];
    double2* dx = h->tmp[11];
    CK(cudaMemcpyAsync(df, f, sizeof(double2) * h->N, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(dx, x, sizeof(double2) * h->N, cudaMemcpyHostToDevice, h->stream));
    helm_status st = helm_solve(h, o, df, dx, stats, res_hist, hist_len);
    CK(cudaMemcpyAsync(x, dx, sizeof(double2) * h->N, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return st;
}

}  // extern "C"
