// Matrix-free Helmholtz operator, residual and relaxation sweeps (Eq. 1-2).
//
// Blocks of 32 x 8 threads over (x, y).  Per node two byte tables (neighbour code,
// layer index) replace the mask loads and the index arithmetic; k^2 and 1/diag
// come from per-layer tables in Op (or the stored field).  Kernel families:
//   k_apply_z        3D operator/residual marching in z (planes in registers,
//                    x-neighbours by warp shuffles), complex128 and complex64
//   k_march_c64      3D complex64 operator and damped Jacobi, two nodes per thread; the
//                    red rows' residual; the operator with the partial sums of a
//                    BiCGStab scalar (DOT)
//   k_rbgs_c64       3D complex64 red-black half-sweep, two nodes per thread
//   k_sweep_c64      3D complex64 full red-black sweep in one launch (old planes
//                    staged in shared memory by cp.async, halo rows recomputed)
//   k_apply, k_jacobi, k_rbgs   the general forms (2D, no tables, complex128)
//   k_apply_bicg(_df)           the BiCGStab operator with its fused reduction
//   k_cycle_df       the red-black part of the FP64 trunk-basis hybrid cycle in
//                    double-float arithmetic, one cooperative launch
// FP64 is the scarce pipe on GB300 (2 instructions per clock per SM against 128
// for FP32), so the FP64 path moves its sweeps onto FP32 pairs.
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "bicg.cuh"
#include "helm_internal.cuh"

namespace helm {

namespace {

constexpr int BX = 32, BY = 8;

__device__ __forceinline__ int layer_index(int i, int n, int L) {
    int d = min(i, n - 1 - i);
    return max(0, L - d);
}

template <typename R>
__device__ __forceinline__ int node_layer(const Op<R>& op, int i, int j, int k) {
    int m = max(layer_index(i, op.n, op.L), layer_index(j, op.n, op.L));
    if (op.dim == 3) m = max(m, layer_index(k, op.n, op.L));
    return m;
}

template <typename R>
__device__ __forceinline__ typename CT<R>::T diag_of(const Op<R>& op, long long l, int m, int conj) {
    typename CT<R>::T d;
    if (op.k2) {
        d = op.k2[l];
        d.x -= (R)(2 * op.dim) * op.hinv2;
    } else {
        d.x = op.dre;
        d.y = op.im[m];
    }
    if (conj) d.y = -d.y;
    return d;
}

template <typename R>
__device__ __forceinline__ typename CT<R>::T invd_of(const Op<R>& op, long long l, int m, int conj) {
    typename CT<R>::T d = op.k2 ? op.invd[l] : op.invd_tab[m];
    if (conj) d.y = -d.y;
    return d;
}

// sum of the fluid neighbours of a fluid node; `code` is the node's neighbour code
// (bit q set: neighbour q is fluid, q = -x, +x, -y, +y, -z, +z), one byte load
// instead of six mask loads
template <typename R>
__device__ __forceinline__ typename CT<R>::T nbr_sum(const Op<R>& op, const typename CT<R>::T* __restrict__ x,
                                                     long long l, unsigned code) {
    using C = typename CT<R>::T;
    const long long sy = op.n, sz = (long long)op.n * op.n;
    C z;
    z.x = 0; z.y = 0;
    // pairwise (tree) sum: three independent adds, then two -- shorter FP64 dependency chains
    const C a = (code & 1u) ? x[HCHK(l - 1, op.N)] : z;
    const C b = (code & 2u) ? x[HCHK(l + 1, op.N)] : z;
    const C c = (code & 4u) ? x[HCHK(l - sy, op.N)] : z;
    const C d = (code & 8u) ? x[HCHK(l + sy, op.N)] : z;
    if (op.face) {
        // Sommerfeld / Neumann boundary rows: axis a weighs 2^-(b - [on an axis-a face])
        const unsigned fc = op.face[l];
        const int nb = (int)(fc >> 4);
        const R wx = ldexp((R)1, -(nb - (int)(fc & 1u))), wy = ldexp((R)1, -(nb - (int)((fc >> 1) & 1u)));
        C s = cadd(cscale(wx, cadd(a, b)), cscale(wy, cadd(c, d)));
        if (op.dim == 3) {
            const R wz = ldexp((R)1, -(nb - (int)((fc >> 2) & 1u)));
            const C e = (code & 16u) ? x[HCHK(l - sz, op.N)] : z;
            const C f = (code & 32u) ? x[HCHK(l + sz, op.N)] : z;
            s = cadd(s, cscale(wz, cadd(e, f)));
        }
        return s;
    }
    C s = cadd(cadd(a, b), cadd(c, d));
    if (op.dim == 3) {
        const C e = (code & 16u) ? x[HCHK(l - sz, op.N)] : z;
        const C f = (code & 32u) ? x[HCHK(l + sz, op.N)] : z;
        s = cadd(s, cadd(e, f));
    }
    return s;
}

constexpr unsigned kMasked = 0x80u;

// neighbour code and layer index of a node: from the handle's tables, or from the
// mask and the indices when the operator carries no tables (no-allocation path)
template <typename R>
__device__ __forceinline__ unsigned node_code(const Op<R>& op, long long l) {
    if (op.nbm) return op.nbm[l];
    if (op.mask[l]) return kMasked;
    const long long sy = op.n, sz = (long long)op.n * op.n;
    unsigned c = 0;
    if (!op.mask[l - 1]) c |= 1u;
    if (!op.mask[l + 1]) c |= 2u;
    if (!op.mask[l - sy]) c |= 4u;
    if (!op.mask[l + sy]) c |= 8u;
    if (op.dim == 3) {
        if (!op.mask[l - sz]) c |= 16u;
        if (!op.mask[l + sz]) c |= 32u;
    }
    return c;
}

template <typename R>
__device__ __forceinline__ int node_lidx(const Op<R>& op, long long l, int i, int j, int k) {
    return op.lidx ? (int)op.lidx[l] : node_layer(op, i, j, k);
}

template <typename R>
__device__ __forceinline__ void block_reduce_store(double v, double* out) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int tid = threadIdx.x + blockDim.x * threadIdx.y;
    int lane = tid & 31, w = tid >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    int nw = (blockDim.x * blockDim.y) >> 5;
    if (w == 0) {
        v = lane < nw ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) *out = v;
    }
}

// y = A x, or y = f - A x (resid), at one node; returns |y_l|^2
template <typename R, bool RESID>
__device__ __forceinline__ double apply_point(const Op<R>& op, const typename CT<R>::T* __restrict__ x,
                                              const typename CT<R>::T* __restrict__ f, typename CT<R>::T* __restrict__ y,
                                              int conj, int i, int j, int k) {
    using C = typename CT<R>::T;
    const long long l = i + (long long)op.n * (j + (long long)op.n * k);
    const C xc = x[l];
    const unsigned code = node_code(op, l);
    C out;
    if (code & kMasked) {
        out = xc;
    } else {
        const C s = nbr_sum(op, x, l, code);
        const C d = diag_of(op, l, node_lidx(op, l, i, j, k), conj);
        out.x = op.hinv2 * s.x + (d.x * xc.x - d.y * xc.y);
        out.y = op.hinv2 * s.y + (d.x * xc.y + d.y * xc.x);
    }
    if (RESID) out = csub(f[l], out);
    y[l] = out;
    return (double)out.x * out.x + (double)out.y * out.y;
}

// 3D operator marching in z: a block owns a 32 x 8 tile of (x, y) and walks zc
// planes (zc chosen so that the grid still has a few blocks per SM).  The
// z-neighbours come from registers (each plane of x is loaded once, two planes
// ahead of its use), the x-neighbours from warp shuffles (a warp is one row of 32
// consecutive nodes; the two row ends load from memory), the y-neighbours from L1.
constexpr int ZC = 16;      // largest z chunk

template <typename R, bool RESID, bool NORM>
__global__ void __launch_bounds__(BX * BY) k_apply_z(Op<R> op, int zc, const typename CT<R>::T* __restrict__ x,
                                                     const typename CT<R>::T* __restrict__ f,
                                                     typename CT<R>::T* __restrict__ y, double* partials, int conj) {
    using C = typename CT<R>::T;
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k0 = blockIdx.z * zc;
    const int k1 = min(op.n, k0 + zc);
    const bool valid = i < op.n && j < op.n;
    const long long sy = op.n, sz = (long long)op.n * op.n;
    const int lane = threadIdx.x;
    C zero;
    zero.x = 0; zero.y = 0;
    long long l = i + (long long)op.n * (j + (long long)op.n * k0);
    C prev = (valid && k0 > 0) ? x[l - sz] : zero;
    C cur = valid ? x[l] : zero;
    C next = (valid && k0 + 1 < op.n) ? x[l + sz] : zero;
    // the per-node tables are read one plane ahead as well, so that no load of
    // the loop is used in the iteration that issues it
    unsigned code = valid ? (unsigned)op.nbm[l] : kMasked;
    int li = valid ? (int)op.lidx[l] : 0;
    double acc = 0.0;
    for (int k = k0; k < k1; ++k, l += sz) {
        const bool more = valid && k + 1 < k1;
        const C next2 = (more && k + 2 < op.n) ? x[l + 2 * sz] : zero;
        const unsigned code_n = more ? (unsigned)op.nbm[l + sz] : kMasked;
        const int li_n = more ? (int)op.lidx[l + sz] : 0;
        C xm, xp;
        xm.x = __shfl_up_sync(0xffffffffu, cur.x, 1);
        xm.y = __shfl_up_sync(0xffffffffu, cur.y, 1);
        xp.x = __shfl_down_sync(0xffffffffu, cur.x, 1);
        xp.y = __shfl_down_sync(0xffffffffu, cur.y, 1);
        if (lane == 0 && (code & 1u)) xm = x[l - 1];
        if (lane == BX - 1 && (code & 2u)) xp = x[l + 1];
        C out;
        if (code & kMasked) {
            out = cur;
        } else {
            const C a = (code & 1u) ? xm : zero;
            const C b = (code & 2u) ? xp : zero;
            const C c = (code & 4u) ? x[l - sy] : zero;
            const C d = (code & 8u) ? x[l + sy] : zero;
            const C e = (code & 16u) ? prev : zero;
            const C g = (code & 32u) ? next : zero;
            const C s = cadd(cadd(cadd(a, b), cadd(c, d)), cadd(e, g));
            const C dg = diag_of(op, l, li, conj);
            out.x = op.hinv2 * s.x + (dg.x * cur.x - dg.y * cur.y);
            out.y = op.hinv2 * s.y + (dg.x * cur.y + dg.y * cur.x);
        }
        if (valid) {
            if (RESID) out = csub(f[l], out);
            y[l] = out;
            if (NORM) acc += (double)out.x * out.x + (double)out.y * out.y;
        }
        prev = cur;
        cur = next;
        next = next2;
        code = code_n;
        li = li_n;
    }
    if (NORM) {
        block_reduce_store<R>(acc, partials + (blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)));
    }
}

// ---- complex64 in 3D: two consecutive x-nodes per thread, so that every vector
// access is one 16-byte load or store and a warp covers 64 nodes of a row.  Needs
// n even (every row starts on a 16-byte boundary) and 16-byte aligned vectors; the
// per-node tables are read as byte pairs.  Marches in z like k_apply_z, with the
// right-hand side prefetched one plane ahead too.  A pair whose two nodes have
// all six neighbours fluid (the common case) takes no selects.
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 pick(unsigned c, unsigned bit, float2 v) {
    return (c & bit) ? v : make_float2(0.f, 0.f);
}

// neighbour sums of the two nodes of a pair (same summation tree as k_apply_z)
__device__ __forceinline__ void pair_sums(unsigned c0, unsigned c1, float2 left, float2 right, float4 cur,
                                          float4 ym, float4 yp, float4 zm, float4 zp, float2& s0, float2& s1) {
    if ((c0 & c1) == 0x3Fu) {
        s0 = cadd(cadd(cadd(left, hi2(cur)), cadd(lo2(ym), lo2(yp))), cadd(lo2(zm), lo2(zp)));
        s1 = cadd(cadd(cadd(lo2(cur), right), cadd(hi2(ym), hi2(yp))), cadd(hi2(zm), hi2(zp)));
    } else {
        s0 = cadd(cadd(cadd(pick(c0, 1u, left), pick(c0, 2u, hi2(cur))),
                       cadd(pick(c0, 4u, lo2(ym)), pick(c0, 8u, lo2(yp)))),
                  cadd(pick(c0, 16u, lo2(zm)), pick(c0, 32u, lo2(zp))));
        s1 = cadd(cadd(cadd(pick(c1, 1u, lo2(cur)), pick(c1, 2u, right)),
                       cadd(pick(c1, 4u, hi2(ym)), pick(c1, 8u, hi2(yp)))),
                  cadd(pick(c1, 16u, hi2(zm)), pick(c1, 32u, hi2(zp))));
    }
}

// KIND 0: y = A x (FLAG: y = f - A x); KIND 1: damped-Jacobi sweep y = x + omega
// D^-1 (f - A x) (FLAG: from x = 0, x not read); KIND 2: the residual f - A x of the
// red node of each pair (colour 0), written compactly as one float2 per pair
// (zero on masked nodes)
// DOT (KIND 0 only): the BiCGStab reduction of launch_apply32_bicg in the epilogue,
// 1: conj(w) y (for alpha), 2: conj(y) w and |y|^2 (for omega); FP32 sums per
// thread and across the block in a fixed order, one partial per block
struct Dot32 {
    const float4* w;
    double2* sc;
    float* parts;
};

template <int KIND, bool FLAG, bool NORM, int DOT = 0>
__global__ void __launch_bounds__(BX * BY) k_march_c64(Op<float> op, int zc, float omega,
                                                       const float4* __restrict__ x, const float4* __restrict__ f,
                                                       float4* __restrict__ y, double* partials, int conj,
                                                       Dot32 dot = Dot32{}) {
    static_assert(DOT == 0 || (KIND == 0 && !FLAG && !NORM), "the fused reduction follows y = A x only");
    constexpr bool NBR = !(KIND == 1 && FLAG);             // neighbours (and x) are read
    constexpr bool RHS = KIND >= 1 || FLAG;                // f is read
    constexpr unsigned kMM = kMasked | (kMasked << 8);
    const int n = op.n, h = n >> 1;
    const int i2 = blockIdx.x * BX + threadIdx.x;          // pair index within the row
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k0 = blockIdx.z * zc;
    const int k1 = min(n, k0 + zc);
    const bool valid = i2 < h && j < n;
    const int sy = h, sz = h * n;                          // strides in pairs (N < 2^31)
    [[maybe_unused]] const long long NP = op.N >> 1;       // pairs (bounds of the checked build)
    const int lane = threadIdx.x;
    const unsigned short* code2 = reinterpret_cast<const unsigned short*>(op.nbm);
    const unsigned short* lidx2 = reinterpret_cast<const unsigned short*>(op.lidx);
    const float2* x1 = reinterpret_cast<const float2*>(x);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    int l = i2 + h * (j + n * k0);
    float4 prev = z4, cur = z4, next = z4, fv = z4;
    if (NBR) {
        prev = (valid && k0 > 0) ? x[HCHK(l - sz, NP)] : z4;
        cur = valid ? x[HCHK(l, NP)] : z4;
        next = (valid && k0 + 1 < n) ? x[HCHK(l + sz, NP)] : z4;
    }
    if (RHS) fv = valid ? f[HCHK(l, NP)] : z4;
    unsigned cc = valid ? (unsigned)code2[HCHK(l, NP)] : kMM;
    unsigned li = valid ? (unsigned)lidx2[HCHK(l, NP)] : 0u;
    float acc = 0.f;
    float dre = 0.f, dim = 0.f, dtt = 0.f;                 // DOT sums
    float4 wv = z4;                                        // DOT operand, prefetched one plane ahead
    if (DOT) wv = valid ? dot.w[HCHK(l, NP)] : z4;
    for (int k = k0; k < k1; ++k, l += sz) {
        const bool more = valid && k + 1 < k1;
        float4 next2 = z4, f_n = z4, w_n = z4;
        if (DOT) w_n = more ? dot.w[HCHK(l + sz, NP)] : z4;
        if (NBR) next2 = (more && k + 2 < n) ? x[HCHK(l + 2 * sz, NP)] : z4;
        if (RHS) f_n = more ? f[HCHK(l + sz, NP)] : z4;
        const unsigned cc_n = more ? (unsigned)code2[HCHK(l + sz, NP)] : kMM;
        const unsigned li_n = more ? (unsigned)lidx2[HCHK(l + sz, NP)] : 0u;
        const unsigned c0 = cc & 0xffu, c1 = cc >> 8;
        float2 s0 = make_float2(0.f, 0.f), s1 = s0;
        if (NBR) {
            float2 left, right;
            left.x = __shfl_up_sync(0xffffffffu, cur.z, 1);
            left.y = __shfl_up_sync(0xffffffffu, cur.w, 1);
            right.x = __shfl_down_sync(0xffffffffu, cur.x, 1);
            right.y = __shfl_down_sync(0xffffffffu, cur.y, 1);
            // the row-segment ends: node i-1 of lane 0 and node i+2 of the last lane
            // (fluid nodes are interior, so these exist whenever the bit is set)
            if (lane == 0 && (c0 & 1u)) left = x1[HCHK(2 * l - 1, op.N)];
            if (lane == BX - 1 && (c1 & 2u)) right = x1[HCHK(2 * l + 2, op.N)];
            const unsigned any = c0 | c1;                  // a masked code has no neighbour bits
            const float4 ym = (any & 4u) ? x[HCHK(l - sy, NP)] : z4;
            const float4 yp = (any & 8u) ? x[HCHK(l + sy, NP)] : z4;
            pair_sums(c0, c1, left, right, cur, ym, yp, prev, next, s0, s1);
        }
        float2 o0, o1;
        if (KIND != 1) {
            float2 d0, d1;
            if (op.k2) {
                const float4 kk = reinterpret_cast<const float4*>(op.k2)[HCHK(l, NP)];
                d0 = make_float2(kk.x - 6.f * op.hinv2, kk.y);
                d1 = make_float2(kk.z - 6.f * op.hinv2, kk.w);
            } else {
                d0 = make_float2(op.dre, op.im[HCHK(li & 0xffu, kMaxLayerCells + 1)]);
                d1 = make_float2(op.dre, op.im[HCHK(li >> 8, kMaxLayerCells + 1)]);
            }
            if (conj) { d0.y = -d0.y; d1.y = -d1.y; }
            const float2 x0 = lo2(cur), xh = hi2(cur);
            o0 = (c0 & kMasked) ? x0
                                : make_float2(op.hinv2 * s0.x + (d0.x * x0.x - d0.y * x0.y),
                                              op.hinv2 * s0.y + (d0.x * x0.y + d0.y * x0.x));
            o1 = (c1 & kMasked) ? xh
                                : make_float2(op.hinv2 * s1.x + (d1.x * xh.x - d1.y * xh.y),
                                              op.hinv2 * s1.y + (d1.x * xh.y + d1.y * xh.x));
            if (FLAG || KIND == 2) {
                o0 = csub(lo2(fv), o0);
                o1 = csub(hi2(fv), o1);
            }
        } else {
            float2 id0, id1;
            if (op.k2) {
                const float4 iv = reinterpret_cast<const float4*>(op.invd)[HCHK(l, NP)];
                id0 = lo2(iv);
                id1 = hi2(iv);
            } else {
                id0 = op.invd_tab[HCHK(li & 0xffu, kMaxLayerCells + 1)];
                id1 = op.invd_tab[HCHK(li >> 8, kMaxLayerCells + 1)];
            }
            if (conj) { id0.y = -id0.y; id1.y = -id1.y; }
            const float2 f0 = lo2(fv), fh = hi2(fv);
            if (FLAG) {
                o0 = cscale(omega, (c0 & kMasked) ? f0 : cmul(id0, f0));
                o1 = cscale(omega, (c1 & kMasked) ? fh : cmul(id1, fh));
            } else {
                const float w1 = 1.f - omega;
                const float2 x0 = lo2(cur), xh = hi2(cur);
                if (c0 & kMasked) {
                    o0 = cadd(x0, cscale(omega, csub(f0, x0)));
                } else {
                    const float2 t = cmul(id0, make_float2(f0.x - op.hinv2 * s0.x, f0.y - op.hinv2 * s0.y));
                    o0 = make_float2(w1 * x0.x + omega * t.x, w1 * x0.y + omega * t.y);
                }
                if (c1 & kMasked) {
                    o1 = cadd(xh, cscale(omega, csub(fh, xh)));
                } else {
                    const float2 t = cmul(id1, make_float2(fh.x - op.hinv2 * s1.x, fh.y - op.hinv2 * s1.y));
                    o1 = make_float2(w1 * xh.x + omega * t.x, w1 * xh.y + omega * t.y);
                }
            }
        }
        if (valid && KIND == 2) {
            const int a = (j + k) & 1;                     // the red node of the pair
            const unsigned ca = a ? c1 : c0;
            reinterpret_cast<float2*>(y)[HCHK(l, NP)] = (ca & kMasked) ? make_float2(0.f, 0.f) : (a ? o1 : o0);
        } else if (valid) {
            y[HCHK(l, NP)] = make_float4(o0.x, o0.y, o1.x, o1.y);
            if (NORM) acc += (o0.x * o0.x + o0.y * o0.y) + (o1.x * o1.x + o1.y * o1.y);
            if (DOT == 1) {                                // conj(w) y
                const float2 w0 = lo2(wv), w1 = hi2(wv);
                dre = fmaf(w0.x, o0.x, fmaf(w0.y, o0.y, dre));
                dim = fmaf(w0.x, o0.y, fmaf(-w0.y, o0.x, dim));
                dre = fmaf(w1.x, o1.x, fmaf(w1.y, o1.y, dre));
                dim = fmaf(w1.x, o1.y, fmaf(-w1.y, o1.x, dim));
            } else if (DOT == 2) {                         // conj(y) w, |y|^2
                const float2 w0 = lo2(wv), w1 = hi2(wv);
                dre = fmaf(o0.x, w0.x, fmaf(o0.y, w0.y, dre));
                dim = fmaf(o0.x, w0.y, fmaf(-o0.y, w0.x, dim));
                dre = fmaf(o1.x, w1.x, fmaf(o1.y, w1.y, dre));
                dim = fmaf(o1.x, w1.y, fmaf(-o1.y, w1.x, dim));
                dtt = fmaf(o0.x, o0.x, fmaf(o0.y, o0.y, dtt));
                dtt = fmaf(o1.x, o1.x, fmaf(o1.y, o1.y, dtt));
            }
        }
        prev = cur;
        cur = next;
        next = next2;
        fv = f_n;
        wv = w_n;
        cc = cc_n;
        li = li_n;
    }
    if (NORM) {
        block_reduce_store<float>((double)acc, partials + (blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)));
    }
    if (DOT) {
        // S_STOP was set, if at all, by an earlier launch: every block takes the same
        // branch.  The block's partial sums only: the kernel that needs the scalar
        // (k32_s for alpha, k32_xr for omega) sums them itself.
        if (dot.sc[S_STOP].x != 0.0) return;
        // (FP32 butterflies and the warps in order: FP64 adds and shuffles run at a
        // small fraction of the FP32 rate on this GPU)
        constexpr int W = DOT == 1 ? 2 : 3;
        const int tid = threadIdx.x + BX * threadIdx.y;
        const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
        float v[3] = {dre, dim, dtt};
        __shared__ float red[3][BX * BY / 32];
        for (int q = 0; q < W; ++q)
            for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
        if ((tid & 31) == 0)
            for (int q = 0; q < W; ++q) red[q][tid >> 5] = v[q];
        __syncthreads();
        if (tid < W) {
            float t = 0.f;
            for (int w = 0; w < BX * BY / 32; ++w) t += red[tid][w];
            dot.parts[W * bid + tid] = t;
        }
    }
}

// new value of a swept node (Gauss-Seidel, or SOR for omega != 1): a masked node
// takes f, a fluid node D^-1 (f - h^-2 s) from its neighbour sum s (D^-1 f when the
// old iterate is zero); SOR moves the old value xo by omega times the step
__device__ __forceinline__ float2 gs_value(const Op<float>& op, unsigned c, float2 fa, float2 s, float2 id,
                                           float2 xo, float omega, bool xzero) {
    float2 out;
    if (c & kMasked) {
        out = fa;
    } else if (xzero) {
        out = cmul(id, fa);
    } else {
        out = cmul(id, make_float2(fa.x - op.hinv2 * s.x, fa.y - op.hinv2 * s.y));
    }
    if (omega != 1.f) out = xzero ? cscale(omega, out) : cadd(xo, cscale(omega, csub(out, xo)));
    return out;
}

// complex64 red-black half-sweep in 3D with the pair layout of k_march_c64: each
// thread owns the node pair (2 i2, 2 i2 + 1) of a row, one node of each colour
// (n even), and updates the one of the swept colour in place.  The neighbours of
// that node are of the other colour and are not written by this launch, so the
// z-march keeps the planes in registers as in k_march_c64.  XZERO: the first
// half-sweep from x = 0 (no neighbours read).  SOR (omega != 1): the node moves by
// omega times its Gauss-Seidel step.
template <bool XZERO>
__global__ void __launch_bounds__(BX * BY) k_rbgs_c64(Op<float> op, int zc, int colour, const float4* __restrict__ f,
                                                      float4* x, int conj, float omega) {
    constexpr unsigned kMM = kMasked | (kMasked << 8);
    const int n = op.n, h = n >> 1;
    const int i2 = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k0 = blockIdx.z * zc;
    const int k1 = min(n, k0 + zc);
    const bool valid = i2 < h && j < n;
    [[maybe_unused]] const long long NP = op.N >> 1;
    const int sy = h, sz = h * n;
    const int lane = threadIdx.x;
    const unsigned short* code2 = reinterpret_cast<const unsigned short*>(op.nbm);
    const unsigned short* lidx2 = reinterpret_cast<const unsigned short*>(op.lidx);
    const float2* x1 = reinterpret_cast<const float2*>(x);
    float2* xw = reinterpret_cast<float2*>(x);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    int l = i2 + h * (j + n * k0);
    float4 prev = z4, cur = z4, next = z4;
    if (!XZERO) {
        prev = (valid && k0 > 0) ? x[HCHK(l - sz, NP)] : z4;
        cur = valid ? x[HCHK(l, NP)] : z4;
        next = (valid && k0 + 1 < n) ? x[HCHK(l + sz, NP)] : z4;
    }
    float4 fv = valid ? f[HCHK(l, NP)] : z4;
    unsigned cc = valid ? (unsigned)code2[HCHK(l, NP)] : kMM;
    unsigned li = valid ? (unsigned)lidx2[HCHK(l, NP)] : 0u;
    for (int k = k0; k < k1; ++k, l += sz) {
        const bool more = valid && k + 1 < k1;
        float4 next2 = z4;
        if (!XZERO) next2 = (more && k + 2 < n) ? x[HCHK(l + 2 * sz, NP)] : z4;
        const float4 f_n = more ? f[HCHK(l + sz, NP)] : z4;
        const unsigned cc_n = more ? (unsigned)code2[HCHK(l + sz, NP)] : kMM;
        const unsigned li_n = more ? (unsigned)lidx2[HCHK(l + sz, NP)] : 0u;
        const int a = ((j + k) & 1) ^ colour;               // swept node of the pair
        const unsigned ca = a ? (cc >> 8) : (cc & 0xffu);
        float2 s0 = make_float2(0.f, 0.f), s1 = s0;
        if (!XZERO) {
            float2 left, right;
            left.x = __shfl_up_sync(0xffffffffu, cur.z, 1);
            left.y = __shfl_up_sync(0xffffffffu, cur.w, 1);
            right.x = __shfl_down_sync(0xffffffffu, cur.x, 1);
            right.y = __shfl_down_sync(0xffffffffu, cur.y, 1);
            if (lane == 0 && a == 0 && (ca & 1u)) left = x1[HCHK(2 * l - 1, op.N)];
            if (lane == BX - 1 && a == 1 && (ca & 2u)) right = x1[HCHK(2 * l + 2, op.N)];
            const float4 ym = (ca & 4u) ? x[HCHK(l - sy, NP)] : z4;
            const float4 yp = (ca & 8u) ? x[HCHK(l + sy, NP)] : z4;
            pair_sums(a ? 0u : ca, a ? ca : 0u, left, right, cur, ym, yp, prev, next, s0, s1);
        }
        if (valid) {
            float2 id = make_float2(0.f, 0.f);
            if (!(ca & kMasked)) {
                if (op.k2) {
                    const float4 iv = reinterpret_cast<const float4*>(op.invd)[HCHK(l, NP)];
                    id = a ? hi2(iv) : lo2(iv);
                } else {
                    id = op.invd_tab[HCHK(a ? (li >> 8) : (li & 0xffu), kMaxLayerCells + 1)];
                }
                if (conj) id.y = -id.y;
            }
            const float2 out = gs_value(op, ca, a ? hi2(fv) : lo2(fv), a ? s1 : s0, id, a ? hi2(cur) : lo2(cur),
                                        omega, XZERO);
            xw[HCHK(2 * l + a, op.N)] = out;
        }
        prev = cur;
        cur = next;
        next = next2;
        fv = f_n;
        cc = cc_n;
        li = li_n;
    }
}

// ---- one full red-black sweep per launch (complex64, 3D, n even, pair layout)
//
// Colour c0 on every node, then colour 1 - c0, read from xin and written to xout
// (out of place).  A block owns whole x-rows: blockDim.x threads over the n/2
// pairs of a row (a multiple of 32), blockDim.y = BYI + 2 rows, of which the first
// and last are halo rows: they compute the colour-c0 values of the rows just
// outside the block, which the block's own second-colour nodes need, instead of
// waiting for the neighbouring block.  Each thread marches in z over its pair.
//
// Old values are staged in shared memory: a ring of five z-planes of the block's rows
// plus one more row on each side (the y-neighbours of the halo rows), filled by
// asynchronous copies (cp.async, 16 bytes per thread and row) issued two planes
// ahead, so that no neighbour read waits on global memory and the staging holds no
// registers.  At step t a thread updates colour c0 at plane t from the staged planes
// t - 1, t, t + 1 and puts the new value in a ring of three shared planes; after one
// barrier it updates colour 1 - c0 at plane t - 1 from the new colour-c0 values
// (x and y neighbours from the shared plane, z neighbours from its registers) and
// writes the pair.  Blocks split z into chunks and recompute the colour-c0 planes
// just outside their chunk.  1/diag of the layer comes from a shared copy of the
// per-layer table.  Every node value comes from the arithmetic of k_rbgs_c64
// (gs_value) with the neighbour sums in the same order, so one launch equals two
// half-sweeps.
__device__ __forceinline__ float2 pair_node(float4 v, int a) { return a ? hi2(v) : lo2(v); }

// neighbour sum of one node from its six neighbour values (code bits select the
// fluid ones), in the order of pair_sums
__device__ __forceinline__ float2 six_sum(unsigned c, float2 xm, float2 xp, float2 ym, float2 yp, float2 zm,
                                          float2 zp) {
    if ((c & 0x3Fu) == 0x3Fu) return cadd(cadd(cadd(xm, xp), cadd(ym, yp)), cadd(zm, zp));
    return cadd(cadd(cadd(pick(c, 1u, xm), pick(c, 2u, xp)), cadd(pick(c, 4u, ym), pick(c, 8u, yp))),
                cadd(pick(c, 16u, zm), pick(c, 32u, zp)));
}

// 16-byte asynchronous copy global -> shared (L2 only); valid = false fills zeros
// without reading (src must still be a mapped address)
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's copy groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int kSweepMaxThreads = 1024;
constexpr int kSweepXPlanes = 5;     // staged old-value planes: t - 1, t, t + 1, and two in flight

// 1/diag of node a of the pair at pair index l with layer byte m: the stored field's
// per-node value, or the shared copy of the layer table (conjugated already)
__device__ __forceinline__ float2 sweep_invd(const Op<float>& op, const float2* stab, int l, int a, unsigned m,
                                             int conj) {
    if (op.k2) {
        const float4 iv = reinterpret_cast<const float4*>(op.invd)[HCHK(l, op.N >> 1)];
        float2 id = a ? hi2(iv) : lo2(iv);
        if (conj) id.y = -id.y;
        return id;
    }
    return stab[HCHK(m, kMaxLayerCells + 1)];
}

// dynamic shared memory of k_sweep_c64 for a block of txt x tyt threads
__host__ __device__ constexpr size_t sweep_smem_bytes(int txt, int tyt, bool xzero) {
    return (xzero ? 0 : (size_t)kSweepXPlanes * (tyt + 2) * txt * sizeof(float4)) +
           (size_t)3 * tyt * txt * sizeof(float2) + (size_t)(kMaxLayerCells + 1) * sizeof(float2);
}

template <bool XZERO>
__global__ void __launch_bounds__(kSweepMaxThreads, 1)
    k_sweep_c64(Op<float> op, int zc, int c0, const float4* __restrict__ f, const float4* __restrict__ xin,
                float4* __restrict__ xout, int conj, float omega) {
    extern __shared__ float4 sweep_smem[];
    constexpr unsigned kMM = kMasked | (kMasked << 8);
    const int n = op.n, h = n >> 1;
    const int TXT = blockDim.x, TYT = blockDim.y, BYI = TYT - 2;
    const int i2 = threadIdx.x, ty = threadIdx.y;
    const int j0 = blockIdx.y * BYI;                       // first inner row of the block
    const int j = j0 - 1 + ty;                             // this thread's row
    const int k0 = blockIdx.z * zc, k1 = min(n, k0 + zc);
    const bool row_ok = i2 < h && j >= 0 && j < n;
    const bool inner = row_ok && ty >= 1 && ty <= BYI;
    const int sz = h * n;
    [[maybe_unused]] const long long NP = op.N >> 1;
    const int RS = TYT + 2;                                // staged rows j0 - 2 .. j0 + BYI + 1
    const int PX = RS * TXT, PR = TYT * TXT;
    float4* xs = sweep_smem;                               // [5][RS][TXT] old pairs (not with XZERO)
    float2* ring = reinterpret_cast<float2*>(sweep_smem + (XZERO ? 0 : kSweepXPlanes * PX));   // [3][TYT][TXT]
    float2* stab = ring + 3 * PR;                          // 1/diag by layer index
    const int me = ty * TXT + i2;                          // this thread in a ring plane
    const int mx = (ty + 1) * TXT + i2;                    // this thread's row in a staged plane
    const int im1 = i2 > 0 ? -1 : 0, ip1 = i2 + 1 < TXT ? 1 : 0;
    const unsigned short* code2 = reinterpret_cast<const unsigned short*>(op.nbm);
    const unsigned short* lidx2 = reinterpret_cast<const unsigned short*>(op.lidx);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float2 z2 = make_float2(0.f, 0.f);
    const int lrow = i2 + h * j;
    for (int q = ty * TXT + i2; q <= op.L && q <= kMaxLayerCells; q += TXT * TYT) {
        float2 v = op.invd_tab[q];
        if (conj) v.y = -v.y;
        stab[q] = v;
    }
    // staged rows of this thread: its own, and the outer row next to a halo row
    const int jx = ty == 0 ? j0 - 2 : (ty == TYT - 1 ? j0 + BYI + 1 : -1);
    const int mo = (ty == 0 ? 0 : RS - 1) * TXT + i2;
    // stage plane p (zeros outside the grid) into the staged plane at offset so
    const bool out_ok = jx != -1 && i2 < h && jx >= 0 && jx < n;
    const int lout = i2 + h * jx;
    auto stage = [&](int p, int so) {
        const bool pin = p >= 0 && p < n;
        cp_async16(xs + so + mx, xin + HCHK(pin && row_ok ? lrow + sz * p : 0, NP), pin && row_ok);
        if (jx != -1) cp_async16(xs + so + mo, xin + HCHK(pin && out_ok ? lout + sz * p : 0, NP), pin && out_ok);
    };
    int t = k0 - 1;
    auto in_t = [&](int q) { return row_ok && q >= 0 && q < n; };
    // offsets of the staged planes t - 1, t, t + 1, t + 2 (in flight) and of the free
    // slot that plane t + 3 goes to (rotated every step: no index arithmetic per access)
    int o_m1 = 0, o_0 = PX, o_p1 = 2 * PX, o_p2 = 3 * PX, o_p3 = 4 * PX;
    if (!XZERO) {
        stage(t - 1, o_m1);
        stage(t, o_0);
        stage(t + 1, o_p1);
        cp_async_commit();
        stage(t + 2, o_p2);
        cp_async_commit();
        cp_async_wait<1>();
    }
    float4 fc = in_t(t) ? f[HCHK(lrow + sz * t, NP)] : z4;
    unsigned cc = in_t(t) ? (unsigned)code2[HCHK(lrow + sz * t, NP)] : kMM;
    unsigned lc = in_t(t) ? (unsigned)lidx2[HCHK(lrow + sz * t, NP)] : 0u;
    float2 rm2 = z2, rm = z2;                              // new colour-c0 values at planes t-2, t-1
    // the colour-(1 - c0) node of this thread's pair at plane t - 1: f, old value,
    // code and layer bytes (kept from the previous step)
    float2 fb = z2, xob = z2;
    unsigned cb = kMasked, lb = 0u;
    int rs = 0, rs_m = 2;                                  // ring slots of planes t and t - 1
    __syncthreads();
    for (; t <= k1; ++t) {
        const int l = lrow + sz * t;
        float4 fn = z4;
        unsigned cn = kMM, ln = 0u;
        if (in_t(t + 1)) {
            fn = f[HCHK(l + sz, NP)];
            cn = code2[HCHK(l + sz, NP)];
            ln = lidx2[HCHK(l + sz, NP)];
        }
        // colour c0 at plane t (old neighbours from the staged planes)
        const int ar = c0 ^ ((j + t) & 1);                 // the colour-c0 node of the pair
        const unsigned ca = ar ? (cc >> 8) : (cc & 0xffu);
        float2 rc = z2;
        float4 own = z4;                                   // this thread's old pair at plane t
        if (!XZERO) own = xs[o_0 + mx];
        if (in_t(t)) {
            float2 sa = z2;
            if (!XZERO && !(ca & kMasked)) {
                const float4* P = xs + o_0;
                // the y and z neighbours: node ar of the neighbouring pairs, read as one
                // complex64 value each (an offset, not a select)
                const float2* P2 = reinterpret_cast<const float2*>(xs) + ar;
                const float2 xm = ar ? lo2(own) : hi2(P[mx + im1]);
                const float2 xp = ar ? lo2(P[mx + ip1]) : hi2(own);
                const float2 ym = P2[2 * (o_0 + mx - TXT)];
                const float2 yp = P2[2 * (o_0 + mx + TXT)];
                const float2 zm = P2[2 * (o_m1 + mx)];
                const float2 zp = P2[2 * (o_p1 + mx)];
                sa = six_sum(ca, xm, xp, ym, yp, zm, zp);
            }
            const float2 id = (ca & kMasked) ? z2 : sweep_invd(op, stab, l, ar, ar ? (lc >> 8) : (lc & 0xffu), conj);
            rc = gs_value(op, ca, pair_node(fc, ar), sa, id, pair_node(own, ar), omega, XZERO);
        }
        ring[rs * PR + me] = rc;
        if (!XZERO) {
            // plane t + 3 into the slot of plane t - 2 (last read in the previous step);
            // plane t + 2 (issued one step ago) must have landed before the barrier
            stage(t + 3, o_p3);
            cp_async_commit();
            cp_async_wait<1>();
        }
        __syncthreads();
        // colour 1 - c0 at plane t - 1 (new colour-c0 neighbours)
        if (inner && t - 1 >= k0 && t - 1 < k1) {
            const int lmi = l - sz;
            const int a = ar;                              // (c0 ^ 1) ^ ((j + t - 1) & 1)
            float2 b;
            if (cb & kMasked) {
                b = gs_value(op, cb, fb, z2, z2, xob, omega, false);
            } else {
                const float2* R = ring + rs_m * PR;
                const float2 xm = a ? rm : R[me + im1];
                const float2 xp = a ? R[me + ip1] : rm;
                const float2 sb = six_sum(cb, xm, xp, R[me - TXT], R[me + TXT], rm2, rc);
                const float2 id = sweep_invd(op, stab, lmi, a, lb, conj);
                b = gs_value(op, cb, fb, sb, id, xob, omega, false);
            }
            xout[HCHK(lmi, NP)] = a ? make_float4(rm.x, rm.y, b.x, b.y) : make_float4(b.x, b.y, rm.x, rm.y);
        }
        rm2 = rm;
        rm = rc;
        // the other node of the pair at plane t (element 1 - ar) is swept next step
        fb = ar ? lo2(fc) : hi2(fc);
        xob = ar ? lo2(own) : hi2(own);
        cb = ar ? (cc & 0xffu) : (cc >> 8);
        lb = ar ? (lc & 0xffu) : (lc >> 8);
        fc = fn;
        cc = cn;
        lc = ln;
        rs_m = rs;
        rs = rs == 2 ? 0 : rs + 1;
        const int o_free = o_m1;
        o_m1 = o_0;
        o_0 = o_p1;
        o_p1 = o_p2;
        o_p2 = o_p3;
        o_p3 = o_free;
    }
    if (!XZERO) cp_async_wait<0>();
}

// y = A x, or y = f - A x (resid); two z-planes per thread; optional per-block ||y||^2 partials.
template <typename R, bool RESID, bool NORM>
__global__ void __launch_bounds__(BX * BY) k_apply(Op<R> op, int zc, const typename CT<R>::T* __restrict__ x,
                                                   const typename CT<R>::T* __restrict__ f,
                                                   typename CT<R>::T* __restrict__ y, double* partials,
                                                   int conj) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    // 3D: zc planes per block (the grid of k_apply_z, so partial counts agree)
    const int k0 = op.dim == 3 ? zc * blockIdx.z : 0;
    const int k1 = op.dim == 3 ? min(op.n, k0 + zc) : 1;
    double acc = 0.0;
    if (i < op.n && j < op.n)
        for (int kk = k0; kk < k1; ++kk) acc += apply_point<R, RESID>(op, x, f, y, conj, i, j, kk);
    if (NORM) {
        block_reduce_store<R>(acc, partials + (blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)));
    }
}

// y = A x with a BiCGStab reduction in the epilogue and its scalar update in the
// last block.  mode 1: <w, y> -> alpha = rho / <rhat, v> (w = rhat);
// mode 2: <y, w>, <y, y> -> omega (w = s).
template <int MODE>
__global__ void __launch_bounds__(BX * BY) k_apply_bicg(Op<double> op, const double2* __restrict__ x,
                                                        double2* __restrict__ y, const double2* __restrict__ w,
                                                        int conj, double2* sc, double* parts, unsigned* counter) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k0 = op.dim == 3 ? 2 * blockIdx.z : 0;
    double a = 0, b = 0, c = 0;
    if (i < op.n && j < op.n) {
        for (int kk = k0; kk < (op.dim == 3 ? min(k0 + 2, op.n) : 1); ++kk) {
            apply_point<double, false>(op, x, nullptr, y, conj, i, j, kk);
            const long long l = i + (long long)op.n * (j + (long long)op.n * kk);
            const double2 yv = y[l], wv = w[l];
            if (MODE == 1) {          // conj(w) y
                a += wv.x * yv.x + wv.y * yv.y;
                b += wv.x * yv.y - wv.y * yv.x;
            } else {                  // conj(y) w and |y|^2
                a += yv.x * wv.x + yv.y * wv.y;
                b += yv.x * wv.y - yv.y * wv.x;
                c += yv.x * yv.x + yv.y * yv.y;
            }
        }
    }
    const int tid = threadIdx.x + BX * threadIdx.y;
    const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
    const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    __shared__ double red[3][BX * BY / 32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((tid & 31) == 0) { red[0][tid >> 5] = a; red[1][tid >> 5] = b; red[2][tid >> 5] = c; }
    __syncthreads();
    if (tid == 0) {
        double sa = 0, sb = 0, scc = 0;
        for (int q = 0; q < BX * BY / 32; ++q) { sa += red[0][q]; sb += red[1][q]; scc += red[2][q]; }
        parts[3 * bid + 0] = sa;
        parts[3 * bid + 1] = sb;
        parts[3 * bid + 2] = scc;
    }
    if (last_block_done(counter, nblk)) {
        double tot[3];
        sum_parts<3>(parts, nblk, tid, tot);
        if (tid == 0) {
            if (MODE == 1) bicg_alpha(sc, make_double2(tot[0], tot[1]));
            else bicg_omega(sc, make_double2(tot[0], tot[1]), tot[2]);
            *counter = 0;
        }
    }
}

// one damped-Jacobi sweep: xout = xin + omega D^-1 (f - A xin), evaluated on a
// fluid node as (1 - omega) x + omega D^-1 (f - h^-2 sum of fluid neighbours)
// (the diagonal term cancels: fewer FP64 operations, same value up to rounding)
template <typename R, bool XZERO>
__device__ __forceinline__ void jacobi_point(const Op<R>& op, R omega, const typename CT<R>::T* __restrict__ f,
                                             const typename CT<R>::T* __restrict__ xin,
                                             typename CT<R>::T* __restrict__ xout, int conj, int i, int j, int k) {
    using C = typename CT<R>::T;
    const long long l = i + (long long)op.n * (j + (long long)op.n * k);
    const C fl = f[l];
    const unsigned code = node_code(op, l);
    C out;
    if (code & kMasked) {
        if (XZERO) {
            out = cscale(omega, fl);
        } else {
            const C xc = xin[l];
            out = cadd(xc, cscale(omega, csub(fl, xc)));
        }
    } else {
        C id = invd_of(op, l, node_lidx(op, l, i, j, k), conj);
        if (XZERO) {
            out = cscale(omega, cmul(id, fl));
        } else {
            const C xc = xin[l];
            const C s = nbr_sum(op, xin, l, code);
            C g;
            g.x = fl.x - op.hinv2 * s.x;
            g.y = fl.y - op.hinv2 * s.y;
            const C t = cmul(id, g);
            const R w1 = (R)1 - omega;
            out.x = w1 * xc.x + omega * t.x;
            out.y = w1 * xc.y + omega * t.y;
        }
    }
    xout[l] = out;
}

// Two z-planes per thread (independent points: more FP64 work in flight per warp).
template <typename R, bool XZERO>
__global__ void __launch_bounds__(BX * BY) k_jacobi(Op<R> op, R omega, const typename CT<R>::T* __restrict__ f,
                                                    const typename CT<R>::T* __restrict__ xin,
                                                    typename CT<R>::T* __restrict__ xout, int conj) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k0 = op.dim == 3 ? 2 * blockIdx.z : 0;
    if (i >= op.n || j >= op.n) return;
    jacobi_point<R, XZERO>(op, omega, f, xin, xout, conj, i, j, k0);
    if (op.dim == 3 && k0 + 1 < op.n) jacobi_point<R, XZERO>(op, omega, f, xin, xout, conj, i, j, k0 + 1);
}

// red-black Gauss-Seidel update of one node of the swept colour, in place:
// x_l = D_l^-1 (f_l - h^-2 sum of fluid neighbours) on fluid nodes (the Gauss-Seidel
// value x + D^-1 (f - A x) with the diagonal term cancelled), f_l on masked nodes;
// SOR (omega != 1): x_l + omega (that value - x_l)
template <typename R, bool XZERO>
__device__ __forceinline__ void rbgs_point(const Op<R>& op, const typename CT<R>::T* __restrict__ f,
                                           typename CT<R>::T* x, int conj, int i, int j, int k, R omega) {
    using C = typename CT<R>::T;
    const long long l = i + (long long)op.n * (j + (long long)op.n * k);
    const C fl = f[l];
    const unsigned code = node_code(op, l);
    C out;
    if (code & kMasked) {
        out = fl;
    } else {
        const C id = invd_of(op, l, node_lidx(op, l, i, j, k), conj);
        if (XZERO) {
            out = cmul(id, fl);
        } else {
            const C s = nbr_sum(op, x, l, code);
            C g;
            g.x = fl.x - op.hinv2 * s.x;
            g.y = fl.y - op.hinv2 * s.y;
            out = cmul(id, g);
        }
    }
    if (omega != (R)1) {
        if (XZERO) {
            out = cscale(omega, out);
        } else {
            const C xo = x[l];
            out = cadd(xo, cscale(omega, csub(out, xo)));
        }
    }
    x[l] = out;
}

template <typename R, bool XZERO>
__global__ void __launch_bounds__(BX * BY) k_rbgs(Op<R> op, int colour, const typename CT<R>::T* __restrict__ f,
                                                  typename CT<R>::T* x, int conj, R omega) {
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = op.dim == 3 ? blockIdx.z : 0;
    if (j >= op.n) return;
    const int i = 2 * (blockIdx.x * BX + threadIdx.x) + ((j + k + colour) & 1);
    if (i < op.n) rbgs_point<R, XZERO>(op, f, x, conj, i, j, k, omega);
}

// r_red[l / 2] = (v - A z)_l at the red nodes l (one per node pair (2m, 2m + 1))
__global__ void __launch_bounds__(BX * BY) k_residual_red(Op<double> op, const double2* __restrict__ z,
                                                          const double2* __restrict__ v,
                                                          double2* __restrict__ r_red, int conj) {
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = op.dim == 3 ? blockIdx.z : 0;
    if (j >= op.n) return;
    const int i = 2 * (blockIdx.x * BX + threadIdx.x) + ((j + k) & 1);
    if (i >= op.n) return;
    const long long l = i + (long long)op.n * (j + (long long)op.n * k);
    const double2 xc = z[l];
    const unsigned code = node_code(op, l);
    double2 out;
    if (code & kMasked) {
        out = xc;
    } else {
        const double2 s = nbr_sum(op, z, l, code);
        const double2 d = diag_of(op, l, node_lidx(op, l, i, j, k), conj);
        out.x = op.hinv2 * s.x + (d.x * xc.x - d.y * xc.y);
        out.y = op.hinv2 * s.y + (d.x * xc.y + d.y * xc.x);
    }
    r_red[l >> 1] = csub(v[l], out);
}

// ---- double-float red-black Gauss-Seidel for FP64 handles.  The sweeps of the
// hybrid cycle keep f and x as FP32 pairs (value = hi + lo, a 48-bit significand)
// and run on the FP32 pipes, which this GPU has ~64x more of than FP64 pipes:
// f is split once (the first red half-sweep), the residual leaves as pairs for the
// projection, and the prolongation converts back to FP64 once.  Additions are
// two-sums with one renormalisation, products an FMA-exact product plus the cross
// terms (the lo*lo term, ~2^-48 relative, is dropped).
__device__ __forceinline__ float2 df_norm(float s, float e) {
    const float h = s + e;
    return make_float2(h, e - (h - s));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    const float s = a.x + b.x;
    const float bb = s - a.x;
    float e = (a.x - (s - bb)) + (b.x - bb);
    e += a.y + b.y;
    return df_norm(s, e);
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    return df_norm(p, e);
}
__device__ __forceinline__ float2 df_split(double v) {
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
}

struct Cdf {          // complex double-float
    float2 re, im;
};
__device__ __forceinline__ Cdf cdf_load(const float4* p, long long l) {
    const float4 v = p[l];
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ float4 cdf_pack(Cdf a) { return make_float4(a.re.x, a.re.y, a.im.x, a.im.y); }
__device__ __forceinline__ Cdf cdf_add(Cdf a, Cdf b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ Cdf cdf_sub(Cdf a, Cdf b) { return {df_add(a.re, df_neg(b.re)), df_add(a.im, df_neg(b.im))}; }
__device__ __forceinline__ Cdf cdf_scale(float2 s, Cdf a) { return {df_mul(s, a.re), df_mul(s, a.im)}; }
__device__ __forceinline__ Cdf cdf_mul(Cdf a, Cdf b) {
    return {df_add(df_mul(a.re, b.re), df_neg(df_mul(a.im, b.im))), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ Cdf cdf_zero() { return {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
__device__ __forceinline__ Cdf invd_df(const DfTab& t, int m, int conj) {
    const float4 v = t.invd[m];
    Cdf d = {make_float2(v.x, v.y), make_float2(v.z, v.w)};
    if (conj) d.im = df_neg(d.im);
    return d;
}

// sum of the fluid neighbours (same tree as nbr_sum)
__device__ __forceinline__ Cdf nbr_sum_df(const Op<double>& op, const float4* __restrict__ x, long long l,
                                          unsigned code) {
    const long long sy = op.n, sz = (long long)op.n * op.n;
    const Cdf a = (code & 1u) ? cdf_load(x, HCHK(l - 1, op.N)) : cdf_zero();
    const Cdf b = (code & 2u) ? cdf_load(x, HCHK(l + 1, op.N)) : cdf_zero();
    const Cdf c = (code & 4u) ? cdf_load(x, HCHK(l - sy, op.N)) : cdf_zero();
    const Cdf d = (code & 8u) ? cdf_load(x, HCHK(l + sy, op.N)) : cdf_zero();
    Cdf s = cdf_add(cdf_add(a, b), cdf_add(c, d));
    if (op.dim == 3) {
        const Cdf e = (code & 16u) ? cdf_load(x, HCHK(l - sz, op.N)) : cdf_zero();
        const Cdf f = (code & 32u) ? cdf_load(x, HCHK(l + sz, op.N)) : cdf_zero();
        s = cdf_add(s, cdf_add(e, f));
    }
    return s;
}

// fs = f as pairs on every node; x = D^-1 f on red fluid nodes, f on red masked
// nodes, 0 on black nodes (the first red half-sweep from x = 0)
__global__ void k_rbgs_df_first(Op<double> op, DfTab t, const double2* __restrict__ f, float4* __restrict__ fs,
                                float4* __restrict__ xs, int conj) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = op.dim == 3 ? blockIdx.z : 0;
    if (i >= op.n || j >= op.n) return;
    const long long l = i + (long long)op.n * (j + (long long)op.n * k);
    const double2 fv = f[l];
    const Cdf F = {df_split(fv.x), df_split(fv.y)};
    fs[l] = cdf_pack(F);
    Cdf x = cdf_zero();
    if (((i + j + k) & 1) == 0) {
        const unsigned code = node_code(op, l);
        x = (code & kMasked) ? F : cdf_mul(invd_df(t, node_lidx(op, l, i, j, k), conj), F);
    }
    xs[l] = cdf_pack(x);
}

// one half-sweep of colour `colour`: x = D^-1 (f - h^-2 s) on fluid nodes, f on masked
__global__ void __launch_bounds__(BX * BY) k_rbgs_df(Op<double> op, DfTab t, int colour,
                                                     const float4* __restrict__ fs, float4* xs, int conj) {
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = op.dim == 3 ? blockIdx.z : 0;
    if (j >= op.n) return;
    const int i = 2 * (blockIdx.x * BX + threadIdx.x) + ((j + k + colour) & 1);
    if (i >= op.n) return;
    const long long l = i + (long long)op.n * (j + (long long)op.n * k);
    const unsigned code = node_code(op, l);
    const Cdf F = cdf_load(fs, l);
    Cdf x;
    if (code & kMasked) {
        x = F;
    } else {
        const Cdf sum = nbr_sum_df(op, xs, l, code);
        x = cdf_mul(invd_df(t, node_lidx(op, l, i, j, k), conj), cdf_sub(F, cdf_scale(t.hinv2, sum)));
    }
    xs[l] = cdf_pack(x);
}

// r_red[l / 2] = (f - A x)_l on the red nodes, as pairs
__global__ void __launch_bounds__(BX * BY) k_residual_red_df(Op<double> op, DfTab t, const float4* __restrict__ fs,
                                                             const float4* __restrict__ xs,
                                                             float4* __restrict__ r_red, int conj) {
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = op.dim == 3 ? blockIdx.z : 0;
    if (j >= op.n) return;
    const int i = 2 * (blockIdx.x * BX + threadIdx.x) + ((j + k) & 1);
    if (i >= op.n) return;
    const long long l = i + (long long)op.n * (j + (long long)op.n * k);
    const unsigned code = node_code(op, l);
    const Cdf x = cdf_load(xs, l);
    Cdf out;
    if (code & kMasked) {
        out = x;
    } else {
        const Cdf sum = nbr_sum_df(op, xs, l, code);
        const int m = node_lidx(op, l, i, j, k);
        const Cdf d = {t.dre, conj ? df_neg(t.im[m]) : t.im[m]};
        out = cdf_add(cdf_scale(t.hinv2, sum), cdf_mul(d, x));
    }
    r_red[l >> 1] = cdf_pack(cdf_sub(cdf_load(fs, l), out));
}

// y = A x with the BiCGStab reduction of k_apply_bicg, for an x given as FP32 pairs
// (the output of the double-float hybrid cycle): the operator in double-float on
// the FP32 pipes, y converted to FP64 once, the dots in FP64
// (or, IN32, for a complex64 x: exact pairs with lo = 0)
__device__ __forceinline__ Cdf cdf_load(const float2* p, long long l) {
    const float2 v = p[l];
    return {make_float2(v.x, 0.f), make_float2(v.y, 0.f)};
}

template <typename XT>
__device__ __forceinline__ Cdf nbr_sum_any(const Op<double>& op, const XT* __restrict__ x, long long l,
                                           unsigned code) {
    const long long sy = op.n, sz = (long long)op.n * op.n;
    const Cdf a = (code & 1u) ? cdf_load(x, HCHK(l - 1, op.N)) : cdf_zero();
    const Cdf b = (code & 2u) ? cdf_load(x, HCHK(l + 1, op.N)) : cdf_zero();
    const Cdf c = (code & 4u) ? cdf_load(x, HCHK(l - sy, op.N)) : cdf_zero();
    const Cdf d = (code & 8u) ? cdf_load(x, HCHK(l + sy, op.N)) : cdf_zero();
    Cdf s = cdf_add(cdf_add(a, b), cdf_add(c, d));
    if (op.dim == 3) {
        const Cdf e = (code & 16u) ? cdf_load(x, HCHK(l - sz, op.N)) : cdf_zero();
        const Cdf f = (code & 32u) ? cdf_load(x, HCHK(l + sz, op.N)) : cdf_zero();
        s = cdf_add(s, cdf_add(e, f));
    }
    return s;
}

template <int MODE, typename XT>
__global__ void __launch_bounds__(BX * BY) k_apply_bicg_df(Op<double> op, DfTab t, const XT* __restrict__ x,
                                                           double2* __restrict__ y, const double2* __restrict__ w,
                                                           int conj, double2* sc, double* parts, unsigned* counter) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k0 = op.dim == 3 ? 2 * blockIdx.z : 0;
    double a = 0, b = 0, c = 0;
    if (i < op.n && j < op.n) {
        for (int kk = k0; kk < (op.dim == 3 ? min(k0 + 2, op.n) : 1); ++kk) {
            const long long l = i + (long long)op.n * (j + (long long)op.n * kk);
            const unsigned code = node_code(op, l);
            const Cdf X = cdf_load(x, l);
            Cdf out;
            if (code & kMasked) {
                out = X;
            } else {
                const Cdf sum = nbr_sum_any(op, x, l, code);
                const int m = node_lidx(op, l, i, j, kk);
                const Cdf d = {t.dre, conj ? df_neg(t.im[m]) : t.im[m]};
                out = cdf_add(cdf_scale(t.hinv2, sum), cdf_mul(d, X));
            }
            const double2 yv = make_double2((double)out.re.x + (double)out.re.y, (double)out.im.x + (double)out.im.y);
            y[l] = yv;
            const double2 wv = w[l];
            if (MODE == 1) {          // conj(w) y
                a += wv.x * yv.x + wv.y * yv.y;
                b += wv.x * yv.y - wv.y * yv.x;
            } else {                  // conj(y) w and |y|^2
                a += yv.x * wv.x + yv.y * wv.y;
                b += yv.x * wv.y - yv.y * wv.x;
                c += yv.x * yv.x + yv.y * yv.y;
            }
        }
    }
    const int tid = threadIdx.x + BX * threadIdx.y;
    const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
    const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    __shared__ double red[3][BX * BY / 32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((tid & 31) == 0) { red[0][tid >> 5] = a; red[1][tid >> 5] = b; red[2][tid >> 5] = c; }
    __syncthreads();
    if (tid == 0) {
        double sa = 0, sb = 0, scc = 0;
        for (int q = 0; q < BX * BY / 32; ++q) { sa += red[0][q]; sb += red[1][q]; scc += red[2][q]; }
        parts[3 * bid + 0] = sa;
        parts[3 * bid + 1] = sb;
        parts[3 * bid + 2] = scc;
    }
    if (last_block_done(counter, nblk)) {
        double tot[3];
        sum_parts<3>(parts, nblk, tid, tot);
        if (tid == 0) {
            if (MODE == 1) bicg_alpha(sc, make_double2(tot[0], tot[1]));
            else bicg_omega(sc, make_double2(tot[0], tot[1]), tot[2]);
            *counter = 0;
        }
    }
}

// ---- the red-black part of the trunk-basis hybrid cycle in one cooperative
// launch: f as pairs with the first red half-sweep from x = 0, the remaining
// half-sweeps, and the red-row residual, each phase over the whole grid and the
// phases separated by a grid barrier (one block per SM, all blocks resident).
// Values written in an earlier phase by other blocks are read past L1 (ld.cg).
// The barrier's wait is bounded: on a timeout it records *err and lets the block
// go on (the host reports the solve as failed).
struct GridBar {
    unsigned* count;        // arrivals in the current barrier
    unsigned* gen;          // barrier generation
    int* err;               // set to 1 when a wait gives up
    double2* sc;            // Krylov scalars or null: a timeout also stops the BiCGStab loop
    unsigned spin_limit;    // polls of the generation word before a wait gives up
    unsigned target;        // arrivals that complete a barrier (gridDim.x; more only to inject a timeout)
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// arrival is an acquire-release add on the counter (each block's writes, ordered
// before it by the block barrier, are released; the last arrival acquires them all),
// the last block resets the counter and releases the next generation, and the
// others acquire it.  Thread 0 waits for all; the block barrier passes it on.
__device__ __forceinline__ void grid_barrier(const GridBar& b) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g = ld_acquire_gpu(b.gen);
        unsigned old;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(b.count) : "memory");
        if (old == b.target - 1) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(b.count) : "memory");
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(b.gen) : "memory");
        } else {
            for (unsigned it = 0; ld_acquire_gpu(b.gen) == g; ++it)
                if (it >= b.spin_limit) {
                    // give up: record it and mark the BiCGStab iteration as stopped
                    // (flag 4 = timeout); the block goes on with its phases, reading
                    // and writing only in-range entries
                    atomicExch(b.err, 1);
                    if (b.sc) {
                        b.sc[S_FLAGS].y = 4.0;
                        b.sc[S_STOP].x = 1.0;
                    }
                    break;
                }
        }
    }
    __syncthreads();
}

__device__ __forceinline__ int colour_of(long long l, int n) {
    const unsigned ul = (unsigned)l, un = (unsigned)n;
    const unsigned r = ul / un;          // row index j + n k
    const unsigned kk = r / un;
    return (int)(((ul - r * un) + (r - kk * un) + kk) & 1u);
}

__device__ __forceinline__ Cdf cdf_load_cg(const float4* p, long long l) {
    const float4 v = __ldcg(p + l);
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}

__device__ __forceinline__ Cdf nbr_sum_df_cg(const Op<double>& op, const float4* x, long long l, unsigned code) {
    const long long sy = op.n, sz = (long long)op.n * op.n;
    const Cdf a = (code & 1u) ? cdf_load_cg(x, HCHK(l - 1, op.N)) : cdf_zero();
    const Cdf b = (code & 2u) ? cdf_load_cg(x, HCHK(l + 1, op.N)) : cdf_zero();
    const Cdf c = (code & 4u) ? cdf_load_cg(x, HCHK(l - sy, op.N)) : cdf_zero();
    const Cdf d = (code & 8u) ? cdf_load_cg(x, HCHK(l + sy, op.N)) : cdf_zero();
    Cdf s = cdf_add(cdf_add(a, b), cdf_add(c, d));
    if (op.dim == 3) {
        const Cdf e = (code & 16u) ? cdf_load_cg(x, HCHK(l - sz, op.N)) : cdf_zero();
        const Cdf f = (code & 32u) ? cdf_load_cg(x, HCHK(l + sz, op.N)) : cdf_zero();
        s = cdf_add(s, cdf_add(e, f));
    }
    return s;
}

constexpr int kCycleThreads = 1024;

// PRE selects where the cycle's right-hand side comes from: 0, f as given; 1, the
// BiCGStab direction update p = r + beta (p - omega v) (p written back); 2, the
// BiCGStab half step s = r - alpha v (written to w) with ||s||^2 summed per block
// and, after the first barrier, in block 0 in a fixed order (scalar recurrence of
// the BiCGStab driver, slot S_SN2 and the tolerance flag)
template <int PRE>
__global__ void __launch_bounds__(kCycleThreads, 1) k_cycle_df(Op<double> op, DfTab t, const double2* __restrict__ f,
                                                               const double2* __restrict__ v, double2* w, double2* sc,
                                                               double* parts, double tol_abs, float4* fs, float4* xs,
                                                               float4* r_red, int n_r, int conj, GridBar bar) {
    const long long N = op.N, M = (N + 1) / 2;
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    double2 c1 = make_double2(0, 0), c2 = c1;
    if (PRE == 1) { c1 = sc[S_BETA]; c2 = sc[S_OMEGA]; }
    if (PRE == 2) c1 = sc[S_ALPHA];
    double acc = 0.0;
    // fs = f as pairs; x = D^-1 f on red fluid nodes, f on red masked nodes, 0 on black
    for (long long l = tid; l < N; l += nth) {
        double2 fv;
        if (PRE == 0) {
            fv = f[l];
        } else if (PRE == 1) {
            const double2 tt = csub(w[l], cmul(c2, v[l]));
            fv = cadd(f[l], cmul(c1, tt));
            w[l] = fv;
        } else {
            fv = csub(f[l], cmul(c1, v[l]));
            w[l] = fv;
            acc += fv.x * fv.x + fv.y * fv.y;
        }
        const Cdf F = {df_split(fv.x), df_split(fv.y)};
        __stcg(fs + l, cdf_pack(F));
        Cdf x = cdf_zero();
        if (colour_of(l, op.n) == 0) {
            const unsigned code = op.nbm[l];
            x = (code & kMasked) ? F : cdf_mul(invd_df(t, op.lidx[l], conj), F);
        }
        __stcg(xs + l, cdf_pack(x));
    }
    if (PRE == 2) {
        __shared__ double red[kCycleThreads / 32];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = 0.0;
            for (int q = 0; q < kCycleThreads / 32; ++q) b += red[q];
            parts[blockIdx.x] = b;
        }
    }
    grid_barrier(bar);
    if (PRE == 2 && blockIdx.x == 0 && threadIdx.x == 0) {
        double sn = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) sn += __ldcg(parts + b);
        bicg_snorm(sc, sn, tol_abs);
    }
    for (int q = 0; q < n_r; ++q) {
        for (int colour = (q == 0 ? 1 : 0); colour < 2; ++colour) {
            for (long long m = tid; m < M; m += nth) {
                const long long l = 2 * m + (colour_of(2 * m, op.n) != colour);
                if (l >= N) continue;
                const unsigned code = op.nbm[l];
                const Cdf F = cdf_load_cg(fs, l);
                Cdf x;
                if (code & kMasked) {
                    x = F;
                } else {
                    const Cdf sum = nbr_sum_df_cg(op, xs, l, code);
                    x = cdf_mul(invd_df(t, op.lidx[l], conj), cdf_sub(F, cdf_scale(t.hinv2, sum)));
                }
                __stcg(xs + l, cdf_pack(x));
            }
            grid_barrier(bar);
        }
    }
    // r_red[m] = (f - A x) at the red node of pair m
    for (long long m = tid; m < M; m += nth) {
        const long long l = 2 * m + (colour_of(2 * m, op.n) != 0);
        const unsigned code = op.nbm[l];
        const Cdf x = cdf_load_cg(xs, l);
        Cdf out;
        if (code & kMasked) {
            out = x;
        } else {
            const Cdf sum = nbr_sum_df_cg(op, xs, l, code);
            const int mm = op.lidx[l];
            const Cdf d = {t.dre, conj ? df_neg(t.im[mm]) : t.im[mm]};
            out = cdf_add(cdf_scale(t.hinv2, sum), cdf_mul(d, x));
        }
        r_red[m] = cdf_pack(cdf_sub(cdf_load_cg(fs, l), out));
    }
}

__global__ void k_rhs(Op<double> op, const double2* __restrict__ src, const double2* __restrict__ g,
                      double2* __restrict__ b) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= op.n || j >= op.n) return;
    const long long l = i + (long long)op.n * (j + (long long)op.n * k);
    if (op.mask[l]) {
        b[l] = g[l];
        return;
    }
    const long long sy = op.n, sz = (long long)op.n * op.n;
    double2 v = src[l];
    long long nb[6] = {l - 1, l + 1, l - sy, l + sy, l - sz, l + sz};
    const int nn = 2 * op.dim;
    for (int q = 0; q < nn; ++q) {
        if (op.mask[nb[q]]) {
            double2 gm = g[nb[q]];
            v.x -= gm.x * op.hinv2;
            v.y -= gm.y * op.hinv2;
        }
    }
    b[l] = v;
}

__global__ void k_layer_k2(Op<double> op, double k0sq, double strength, const double* __restrict__ scale,
                           double2* __restrict__ k2) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= op.n || j >= op.n) return;
    const long long l = i + (long long)op.n * (j + (long long)op.n * k);
    const int m = node_layer(op, i, j, k);
    const double eta = op.L > 0 ? (double)m / (double)op.L : 0.0;
    const double base = scale ? k0sq * scale[l] : k0sq;
    k2[l] = make_double2(base, base * (strength * eta * eta));
}

__global__ void k_invd_field(Op<double> op, double2* __restrict__ invd) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= op.n || j >= op.n) return;
    const long long l = i + (long long)op.n * (j + (long long)op.n * k);
    double2 d = op.k2[l];
    d.x -= 2.0 * op.dim * op.hinv2;
    invd[l] = op.mask[l] ? make_double2(1.0, 0.0) : cdiv(make_double2(1.0, 0.0), d);
}

__global__ void k_layer_index(Op<double> op, uint8_t* __restrict__ lidx) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= op.n || j >= op.n) return;
    const long long l = i + (long long)op.n * (j + (long long)op.n * k);
    lidx[l] = (uint8_t)node_layer(op, i, j, k);
}

__global__ void k_nbr_code(Op<double> op, uint8_t* __restrict__ code) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= op.n || j >= op.n) return;
    const long long l = i + (long long)op.n * (j + (long long)op.n * k);
    const long long sy = op.n, sz = (long long)op.n * op.n;
    unsigned c = 0;
    if (op.mask[l]) {
        c = kMasked;
    } else if (op.face) {
        // outer-boundary problem: a neighbour counts if it is in the grid and unmasked
        const int n = op.n;
        if (i > 0 && !op.mask[l - 1]) c |= 1u;
        if (i < n - 1 && !op.mask[l + 1]) c |= 2u;
        if (j > 0 && !op.mask[l - sy]) c |= 4u;
        if (j < n - 1 && !op.mask[l + sy]) c |= 8u;
        if (op.dim == 3) {
            if (k > 0 && !op.mask[l - sz]) c |= 16u;
            if (k < n - 1 && !op.mask[l + sz]) c |= 32u;
        }
    } else {
        // fluid nodes are interior (the outer ring is masked), so all neighbours exist
        if (!op.mask[l - 1]) c |= 1u;
        if (!op.mask[l + 1]) c |= 2u;
        if (!op.mask[l - sy]) c |= 4u;
        if (!op.mask[l + sy]) c |= 8u;
        if (op.dim == 3) {
            if (!op.mask[l - sz]) c |= 16u;
            if (!op.mask[l + sz]) c |= 32u;
        }
    }
    code[l] = (uint8_t)c;
}

// face byte of a node: (number of boundary faces << 4) | axis bits
__global__ void k_face_code(Op<double> op, uint8_t* __restrict__ face) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= op.n || j >= op.n) return;
    const long long l = i + (long long)op.n * (j + (long long)op.n * k);
    const int n = op.n;
    const unsigned ax = (i == 0 || i == n - 1) ? 1u : 0u, ay = (j == 0 || j == n - 1) ? 1u : 0u;
    const unsigned az = (op.dim == 3 && (k == 0 || k == n - 1)) ? 1u : 0u;
    face[l] = (uint8_t)(((ax + ay + az) << 4) | ax | (ay << 1) | (az << 2));
}

// effective k^2 of the outer-boundary problem: with it diag_of returns the scaled
// boundary diagonal 2^-b (k^2 - 2d h^-2 + 2 i k0 a / h), a = number of Sommerfeld
// faces of the node (all its faces but the Neumann top face y = 1 in 2D, z = 1 in 3D)
__global__ void k_bvp_k2(Op<double> op, const double2* __restrict__ k2phys, double k0, int neumann_top,
                         double2* __restrict__ k2eff) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= op.n || j >= op.n) return;
    const long long l = i + (long long)op.n * (j + (long long)op.n * k);
    const int n = op.n;
    const int top = op.dim == 3 ? (k == n - 1) : (j == n - 1);
    const int nb = (i == 0) + (i == n - 1) + (j == 0) + (j == n - 1) + (op.dim == 3 ? (k == 0) + (k == n - 1) : 0);
    const int a = nb - (neumann_top && top ? 1 : 0);
    const double sigma = ldexp(1.0, -nb), h = sqrt(1.0 / op.hinv2), two_d = 2.0 * op.dim * op.hinv2;
    const double2 kp = k2phys ? k2phys[l] : make_double2(k0 * k0, 0.0);
    // K - 2d h^-2 = sigma (k^2 - 2d h^-2) + i sigma 2 k0 a / h
    k2eff[l] = make_double2(sigma * (kp.x - two_d) + two_d, sigma * (kp.y + 2.0 * k0 * a / h));
}

// right-hand side of the outer-boundary problem: masked nodes carry the Dirichlet
// value g; a fluid node gets 2^-b (src - (2 / h) g [on the Neumann top face]) minus the
// weighted Dirichlet values of its masked neighbours
__global__ void k_rhs_bvp(Op<double> op, const double2* __restrict__ src, const double2* __restrict__ g,
                          int neumann_top, double2* __restrict__ b) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= op.n || j >= op.n) return;
    const long long l = i + (long long)op.n * (j + (long long)op.n * k);
    if (op.mask[l]) {
        b[l] = g[l];
        return;
    }
    const int n = op.n;
    const unsigned fc = op.face[l];
    const int nb = (int)(fc >> 4);
    const double sigma = ldexp(1.0, -nb), h = sqrt(1.0 / op.hinv2);
    const int top = op.dim == 3 ? (k == n - 1) : (j == n - 1);
    double2 v = src[l];
    if (neumann_top && top) {
        v.x -= 2.0 / h * g[l].x;
        v.y -= 2.0 / h * g[l].y;
    }
    v = cscale(sigma, v);
    const long long sy = n, sz = (long long)n * n;
    const double wx = ldexp(1.0, -(nb - (int)(fc & 1u))), wy = ldexp(1.0, -(nb - (int)((fc >> 1) & 1u)));
    const double wz = ldexp(1.0, -(nb - (int)((fc >> 2) & 1u)));
    auto lift = [&](bool exists, long long m, double w) {
        if (exists && op.mask[m]) {
            v.x -= op.hinv2 * w * g[m].x;
            v.y -= op.hinv2 * w * g[m].y;
        }
    };
    lift(i > 0, l - 1, wx);
    lift(i < n - 1, l + 1, wx);
    lift(j > 0, l - sy, wy);
    lift(j < n - 1, l + sy, wy);
    if (op.dim == 3) {
        lift(k > 0, l - sz, wz);
        lift(k < n - 1, l + sz, wz);
    }
    b[l] = v;
}

__global__ void k_check_ring(Op<double> op, int* bad) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= op.n || j >= op.n) return;
    bool ring = i == 0 || j == 0 || i == op.n - 1 || j == op.n - 1;
    if (op.dim == 3) ring = ring || k == 0 || k == op.n - 1;
    const long long l = i + (long long)op.n * (j + (long long)op.n * k);
    if (ring && !op.mask[l]) atomicOr(bad, 1);
}

dim3 grid_for(int dim, int n, int xdiv = 1, int zdiv = 1) {
    int nx = (n + xdiv - 1) / xdiv;
    return dim3((nx + BX - 1) / BX, (n + BY - 1) / BY, dim == 3 ? (n + zdiv - 1) / zdiv : 1);
}

}  // namespace

int bicg_grid_blocks(int dim, int n) {
    dim3 g = grid_for(dim, n, 1, 2);
    return g.x * g.y * g.z;
}

// z chunk of a 3D marching grid with xy blocks per plane: the largest of 16, 8,
// 4, 2, 1 that leaves at least four blocks per SM
int march_zc(long long xy, int n) {
    int zc = ZC;
    while (zc > 1 && xy * ((n + zc - 1) / zc) < 4 * 152) zc /= 2;
    return zc;
}

int apply_zc(int dim, int n) {
    if (dim != 3) return 1;
    return march_zc((long long)((n + BX - 1) / BX) * ((n + BY - 1) / BY), n);
}

// grid of the two-nodes-per-thread complex64 kernels
dim3 pair_grid(int n, int* zc) {
    const int h = n / 2;
    const int gx = (h + BX - 1) / BX, gy = (n + BY - 1) / BY;
    *zc = march_zc((long long)gx * gy, n);
    return dim3(gx, gy, (n + *zc - 1) / *zc);
}

bool aligned16(const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// the complex64 pair kernels apply: 3D, tables present, n even, 16-byte aligned vectors
bool pair_ok(const Op<float>& op, const void* a, const void* b, const void* c) {
    return op.dim == 3 && op.nbm && op.lidx && !op.face && (op.n % 2) == 0 && aligned16(a) && aligned16(b) && aligned16(c) &&
           aligned16(op.k2) && aligned16(op.invd);
}

// an upper bound on the partial sums any operator launch writes (buffer sizing)
int apply_grid_blocks(int dim, int n) {
    dim3 g = grid_for(dim, n, 1, apply_zc(dim, n));
    long long b = (long long)g.x * g.y * g.z;
    if (dim == 3 && n % 2 == 0) {
        int zc;
        dim3 p = pair_grid(n, &zc);
        b = std::max(b, (long long)p.x * p.y * p.z);
    }
    return (int)b;
}

template <typename R>
int launch_apply(const Op<R>& op, const typename CT<R>::T* x, const typename CT<R>::T* f, typename CT<R>::T* y,
                 double* partials, int conj, bool resid, cudaStream_t s) {
    if constexpr (std::is_same<R, float>::value) {
        if (pair_ok(op, x, resid ? f : nullptr, y)) {
            int zc;
            const dim3 g = pair_grid(op.n, &zc), b(BX, BY);
            const float4* x4 = reinterpret_cast<const float4*>(x);
            const float4* f4 = reinterpret_cast<const float4*>(f);
            float4* y4 = reinterpret_cast<float4*>(y);
            if (resid) {
                if (partials) k_march_c64<0, true, true><<<g, b, 0, s>>>(op, zc, 0.f, x4, f4, y4, partials, conj);
                else k_march_c64<0, true, false><<<g, b, 0, s>>>(op, zc, 0.f, x4, f4, y4, partials, conj);
            } else {
                if (partials) k_march_c64<0, false, true><<<g, b, 0, s>>>(op, zc, 0.f, x4, f4, y4, partials, conj);
                else k_march_c64<0, false, false><<<g, b, 0, s>>>(op, zc, 0.f, x4, f4, y4, partials, conj);
            }
            return (int)(g.x * g.y * g.z);
        }
    }
    const int zc = apply_zc(op.dim, op.n);
    dim3 g = grid_for(op.dim, op.n, 1, zc), b(BX, BY);
    if (op.dim == 3 && op.nbm && op.lidx && !op.face) {
        if (resid) {
            if (partials) k_apply_z<R, true, true><<<g, b, 0, s>>>(op, zc, x, f, y, partials, conj);
            else k_apply_z<R, true, false><<<g, b, 0, s>>>(op, zc, x, f, y, partials, conj);
        } else {
            if (partials) k_apply_z<R, false, true><<<g, b, 0, s>>>(op, zc, x, f, y, partials, conj);
            else k_apply_z<R, false, false><<<g, b, 0, s>>>(op, zc, x, f, y, partials, conj);
        }
        return (int)(g.x * g.y * g.z);
    }
    // 2D, or an operator without the per-node tables (the allocation-free path)
    if (resid) {
        if (partials) k_apply<R, true, true><<<g, b, 0, s>>>(op, zc, x, f, y, partials, conj);
        else k_apply<R, true, false><<<g, b, 0, s>>>(op, zc, x, f, y, partials, conj);
    } else {
        if (partials) k_apply<R, false, true><<<g, b, 0, s>>>(op, zc, x, f, y, partials, conj);
        else k_apply<R, false, false><<<g, b, 0, s>>>(op, zc, x, f, y, partials, conj);
    }
    return (int)(g.x * g.y * g.z);
}

template <typename R>
void launch_jacobi(const Op<R>& op, double omega, const typename CT<R>::T* f, const typename CT<R>::T* xin,
                   typename CT<R>::T* xout, int conj, bool xzero, cudaStream_t s) {
    if constexpr (std::is_same<R, float>::value) {
        if (pair_ok(op, f, xzero ? nullptr : xin, xout)) {
            int zc;
            const dim3 g = pair_grid(op.n, &zc), b(BX, BY);
            const float4* x4 = reinterpret_cast<const float4*>(xin);
            const float4* f4 = reinterpret_cast<const float4*>(f);
            float4* y4 = reinterpret_cast<float4*>(xout);
            if (xzero) k_march_c64<1, true, false><<<g, b, 0, s>>>(op, zc, (float)omega, x4, f4, y4, nullptr, conj);
            else k_march_c64<1, false, false><<<g, b, 0, s>>>(op, zc, (float)omega, x4, f4, y4, nullptr, conj);
            return;
        }
    }
    dim3 g = grid_for(op.dim, op.n, 1, 2), b(BX, BY);
    if (xzero) k_jacobi<R, true><<<g, b, 0, s>>>(op, (R)omega, f, xin, xout, conj);
    else k_jacobi<R, false><<<g, b, 0, s>>>(op, (R)omega, f, xin, xout, conj);
}

template <typename R>
void launch_rbgs_half(const Op<R>& op, int colour, const typename CT<R>::T* f, typename CT<R>::T* x, int conj,
                      bool xzero, cudaStream_t s, double omega) {
    if constexpr (std::is_same<R, float>::value) {
        if (pair_ok(op, f, x, nullptr)) {
            int zc;
            const dim3 g = pair_grid(op.n, &zc), b(BX, BY);
            const float4* f4 = reinterpret_cast<const float4*>(f);
            float4* x4 = reinterpret_cast<float4*>(x);
            if (xzero) k_rbgs_c64<true><<<g, b, 0, s>>>(op, zc, colour, f4, x4, conj, (float)omega);
            else k_rbgs_c64<false><<<g, b, 0, s>>>(op, zc, colour, f4, x4, conj, (float)omega);
            return;
        }
    }
    dim3 g = grid_for(op.dim, op.n, 2, 1), b(BX, BY);
    if (xzero) k_rbgs<R, true><<<g, b, 0, s>>>(op, colour, f, x, conj, (R)omega);
    else k_rbgs<R, false><<<g, b, 0, s>>>(op, colour, f, x, conj, (R)omega);
}

bool launch_red_residual32(const Op<float>& op, const float2* f, const float2* x, float2* r_red, int conj,
                           cudaStream_t s) {
    if (!pair_ok(op, f, x, r_red)) return false;
    int zc;
    const dim3 g = pair_grid(op.n, &zc), b(BX, BY);
    k_march_c64<2, false, false><<<g, b, 0, s>>>(op, zc, 0.f, reinterpret_cast<const float4*>(x),
                                                 reinterpret_cast<const float4*>(f), reinterpret_cast<float4*>(r_red),
                                                 nullptr, conj);
    return true;
}

int launch_apply32_bicg(const Op<float>& op, int mode, const float2* x, float2* y, const float2* w, int conj,
                        const double2* sc, float* parts, cudaStream_t s) {
    if (!pair_ok(op, x, y, w) || (mode != 1 && mode != 2)) return 0;
    int zc;
    const dim3 g = pair_grid(op.n, &zc), b(BX, BY);
    const Dot32 d{reinterpret_cast<const float4*>(w), const_cast<double2*>(sc), parts};
    const float4* x4 = reinterpret_cast<const float4*>(x);
    float4* y4 = reinterpret_cast<float4*>(y);
    if (mode == 1) k_march_c64<0, false, false, 1><<<g, b, 0, s>>>(op, zc, 0.f, x4, nullptr, y4, nullptr, conj, d);
    else k_march_c64<0, false, false, 2><<<g, b, 0, s>>>(op, zc, 0.f, x4, nullptr, y4, nullptr, conj, d);
    return (int)(g.x * g.y * g.z);
}

namespace {

// launch shape of k_sweep_c64 on an n^3 grid: whole rows per block (n/2 pairs, at
// most 128), as many rows as fill 1024 threads (8 to 32) including the two halo rows;
// z chunks of 4..16 planes, as many as fill the resident block slots once
struct SweepShape {
    dim3 g, b;
    int zc;
    size_t smem, smem0;         // dynamic shared memory: from xin, from zero
};

bool sweep_shape(int n, SweepShape& sh) {
    const int h = n / 2;
    if (n % 2 != 0 || h < 1 || h > 128) return false;
    const int txt = (h + 31) / 32 * 32;
    const int tyt = std::max(8, std::min(32, kSweepMaxThreads / txt));
    const int byi = tyt - 2;
    sh.b = dim3(txt, tyt);
    sh.smem = sweep_smem_bytes(txt, tyt, false);
    sh.smem0 = sweep_smem_bytes(txt, tyt, true);
    static int sms = 0;
    static int occ[5] = {0, 0, 0, 0, 0};
    const int w = txt / 32;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // the largest block shape (128 x 8 threads) needs about 127 KB
        cudaFuncSetAttribute(k_sweep_c64<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 136 * 1024);
        cudaFuncSetAttribute(k_sweep_c64<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 136 * 1024);
    }
    if (occ[w] == 0) {
        int o0 = 0, o1 = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o0, k_sweep_c64<false>, txt * tyt, sh.smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_sweep_c64<true>, txt * tyt, sh.smem0);
        occ[w] = std::max(1, std::min(o0, o1));
    }
    const int gy = (n + byi - 1) / byi;
    const long long slots = (long long)std::max(sms, 1) * occ[w];
    const int chunks = (int)std::max<long long>(1, slots / gy);
    sh.zc = std::max(4, std::min(16, (n + chunks - 1) / chunks));
    sh.g = dim3(1, gy, (n + sh.zc - 1) / sh.zc);
    return true;
}

}  // namespace

bool rbgs_sweep32_ok(const Op<float>& op, const void* f, const void* x, const void* tmp) {
    SweepShape sh;
    const bool shape = op.dim == 3 && sweep_shape(op.n, sh);      // (also fills the occupancy cache)
    return shape && pair_ok(op, f, x, tmp) && x != tmp;
}

bool launch_rbgs_sweep32(const Op<float>& op, int c0, const float2* f, const float2* xin, float2* xout, int conj,
                         double omega, cudaStream_t s) {
    SweepShape sh;
    if (!pair_ok(op, f, xin, xout) || !sweep_shape(op.n, sh) || xin == xout) return false;
    const float4* f4 = reinterpret_cast<const float4*>(f);
    const float4* x4 = reinterpret_cast<const float4*>(xin);
    float4* y4 = reinterpret_cast<float4*>(xout);
    if (xin) k_sweep_c64<false><<<sh.g, sh.b, sh.smem, s>>>(op, sh.zc, c0, f4, x4, y4, conj, (float)omega);
    else k_sweep_c64<true><<<sh.g, sh.b, sh.smem0, s>>>(op, sh.zc, c0, f4, x4, y4, conj, (float)omega);
    return true;
}

void launch_apply_bicg_df(const Op<double>& op, const DfTab& t, int mode, const float4* x, double2* y,
                          const double2* w, int conj, double2* sc, double* parts, unsigned* counter, cudaStream_t s) {
    dim3 g = grid_for(op.dim, op.n, 1, 2), b(BX, BY);
    if (mode == 1) k_apply_bicg_df<1, float4><<<g, b, 0, s>>>(op, t, x, y, w, conj, sc, parts, counter);
    else k_apply_bicg_df<2, float4><<<g, b, 0, s>>>(op, t, x, y, w, conj, sc, parts, counter);
}

void launch_apply_bicg(const Op<double>& op, int mode, const double2* x, double2* y, const double2* w, int conj,
                       double2* sc, double* parts, unsigned* counter, cudaStream_t s) {
    dim3 g = grid_for(op.dim, op.n, 1, 2), b(BX, BY);
    if (mode == 1) k_apply_bicg<1><<<g, b, 0, s>>>(op, x, y, w, conj, sc, parts, counter);
    else k_apply_bicg<2><<<g, b, 0, s>>>(op, x, y, w, conj, sc, parts, counter);
}

template int launch_apply<double>(const Op<double>&, const double2*, const double2*, double2*, double*, int,
                                  bool, cudaStream_t);
template int launch_apply<float>(const Op<float>&, const float2*, const float2*, float2*, double*, int, bool,
                                 cudaStream_t);
template void launch_jacobi<double>(const Op<double>&, double, const double2*, const double2*, double2*, int,
                                    bool, cudaStream_t);
template void launch_jacobi<float>(const Op<float>&, double, const float2*, const float2*, float2*, int, bool,
                                   cudaStream_t);
template void launch_rbgs_half<double>(const Op<double>&, int, const double2*, double2*, int, bool,
                                       cudaStream_t, double);
template void launch_rbgs_half<float>(const Op<float>&, int, const float2*, float2*, int, bool, cudaStream_t,
                                      double);

void launch_residual_red(const Op<double>& op, const double2* z, const double2* v, double2* r_red, int conj,
                         cudaStream_t s) {
    k_residual_red<<<grid_for(op.dim, op.n, 2, 1), dim3(BX, BY), 0, s>>>(op, z, v, r_red, conj);
}

void launch_rbgs_df_first(const Op<double>& op, const DfTab& t, const double2* f, float4* fs, float4* xs, int conj,
                          cudaStream_t s) {
    k_rbgs_df_first<<<grid_for(op.dim, op.n), dim3(BX, BY), 0, s>>>(op, t, f, fs, xs, conj);
}

void launch_rbgs_df(const Op<double>& op, const DfTab& t, int colour, const float4* fs, float4* xs, int conj,
                    cudaStream_t s) {
    k_rbgs_df<<<grid_for(op.dim, op.n, 2, 1), dim3(BX, BY), 0, s>>>(op, t, colour, fs, xs, conj);
}

void launch_residual_red_df(const Op<double>& op, const DfTab& t, const float4* fs, const float4* xs, float4* r_red,
                            int conj, cudaStream_t s) {
    k_residual_red_df<<<grid_for(op.dim, op.n, 2, 1), dim3(BX, BY), 0, s>>>(op, t, fs, xs, r_red, conj);
}

// blocks of the cooperative cycle: one per SM (at most), 0 if the device cannot
// launch it cooperatively
int cycle_df_blocks(long long N) {
    static int sms = -1;
    if (sms < 0) {
        int dev = 0, coop = 0, occ = 0, count = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev);
        if (coop) {
            int o0 = 0, o1 = 0, o2 = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o0, k_cycle_df<0>, kCycleThreads, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_cycle_df<1>, kCycleThreads, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k_cycle_df<2>, kCycleThreads, 0);
            occ = std::min(o0, std::min(o1, o2));
        }
        sms = (coop && occ >= 1) ? count : 0;
    }
    if (sms < 1) return 0;
    const long long need = (N + kCycleThreads - 1) / kCycleThreads;
    return (int)(need < sms ? (need < 1 ? 1 : need) : sms);
}

cudaError_t launch_cycle_df(const Op<double>& op, const DfTab& t, int pre, const double2* f, const double2* v,
                            double2* w, double2* sc, double* parts, double tol_abs, float4* fs, float4* xs,
                            float4* r_red, int n_r, int conj, unsigned* bar2, int* err, unsigned spin_limit,
                            unsigned extra_arrivals, cudaStream_t s) {
    const int nb = cycle_df_blocks(op.N);
    if (nb < 1) return cudaErrorNotSupported;
    GridBar b{bar2, bar2 + 1, err, sc, spin_limit, (unsigned)nb + extra_arrivals};
    Op<double> opv = op;
    DfTab tv = t;
    const double2* fv = f;
    const double2* vv = v;
    void* args[] = {&opv, &tv, (void*)&fv, (void*)&vv, &w, &sc, &parts, &tol_abs, &fs, &xs, &r_red, &n_r, &conj, &b};
    const void* fn = pre == 0 ? (const void*)k_cycle_df<0> : pre == 1 ? (const void*)k_cycle_df<1>
                                                                      : (const void*)k_cycle_df<2>;
    return cudaLaunchCooperativeKernel(fn, dim3(nb), dim3(kCycleThreads), args, 0, s);
}

void launch_rhs(const Op<double>& op, const double2* src, const double2* g, double2* b, cudaStream_t s) {
    k_rhs<<<grid_for(op.dim, op.n), dim3(BX, BY), 0, s>>>(op, src, g, b);
}

void launch_layer_k2(const Op<double>& op, double k0, double strength, const double* scale, double2* k2,
                     cudaStream_t s) {
    k_layer_k2<<<grid_for(op.dim, op.n), dim3(BX, BY), 0, s>>>(op, k0 * k0, strength, scale, k2);
}

void launch_invd_field(const Op<double>& op, double2* invd, cudaStream_t s) {
    k_invd_field<<<grid_for(op.dim, op.n), dim3(BX, BY), 0, s>>>(op, invd);
}

void launch_layer_index(const Op<double>& op, uint8_t* lidx, cudaStream_t s) {
    k_layer_index<<<grid_for(op.dim, op.n), dim3(BX, BY), 0, s>>>(op, lidx);
}

void launch_nbr_code(const Op<double>& op, uint8_t* code, cudaStream_t s) {
    k_nbr_code<<<grid_for(op.dim, op.n), dim3(BX, BY), 0, s>>>(op, code);
}

void launch_face_code(const Op<double>& op, uint8_t* face, cudaStream_t s) {
    k_face_code<<<grid_for(op.dim, op.n), dim3(BX, BY), 0, s>>>(op, face);
}
void launch_bvp_k2(const Op<double>& op, const double2* k2phys, double k0, int neumann_top, double2* k2eff,
                   cudaStream_t s) {
    k_bvp_k2<<<grid_for(op.dim, op.n), dim3(BX, BY), 0, s>>>(op, k2phys, k0, neumann_top, k2eff);
}
void launch_rhs_bvp(const Op<double>& op, const double2* src, const double2* g, int neumann_top, double2* b,
                    cudaStream_t s) {
    k_rhs_bvp<<<grid_for(op.dim, op.n), dim3(BX, BY), 0, s>>>(op, src, g, neumann_top, b);
}

void launch_check_ring(const Op<double>& op, int* bad, cudaStream_t s) {
    k_check_ring<<<grid_for(op.dim, op.n), dim3(BX, BY), 0, s>>>(op, bad);
}

}  // namespace helm
