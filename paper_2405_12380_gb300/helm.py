"""Thin Python layer over libhelm's C ABI: torch tensors in, torch tensors out.

Device memory and streams come from PyTorch; every arithmetic step runs in the
CUDA kernels behind include/helm.h.  Complex vectors are torch.complex128 (or
complex64) CUDA tensors of N = n^dim entries, flat index i + n (j + n k).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L
from ._lib import SolveOpts, Stats


class HelmError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"libhelm: {L.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def opts(method="fgmres", relax="jacobi", n_r=1, omega=0.6, correction="tb", tol=1e-8,
         restart=30, maxit=1000, conj=False) -> SolveOpts:
    m = {"relax": L.HELM_METHOD_RELAX, "fgmres": L.HELM_METHOD_FGMRES,
         "bicgstab": L.HELM_METHOD_BICGSTAB}[method]
    r = {"none": L.HELM_RELAX_NONE, "jacobi": L.HELM_JACOBI, "rbgs": L.HELM_RBGS, "sor": L.HELM_SOR,
         "ssor": L.HELM_SSOR, "mg": L.HELM_MG}[relax]
    c = {"none": L.HELM_CORR_NONE, "tb": L.HELM_CORR_TB, "nonlinear": L.HELM_CORR_NONLINEAR}[correction]
    return SolveOpts(m, r, int(n_r), float(omega), c, float(tol), int(restart), int(maxit), int(bool(conj)))


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _dtype_code(t):
    if t.dtype == torch.complex128:
        return L.HELM_C128
    if t.dtype == torch.complex64:
        return L.HELM_C64
    raise TypeError(f"unsupported dtype {t.dtype}")


class Problem:
    """One discretised Helmholtz problem (helm_create) on the current CUDA device."""

    def __init__(self, dim, n, k0, mask, layer_cells=8, layer_strength=0.5, k2=None, precision="fp64",
                 boundary="dirichlet", neumann_top=True):
        """boundary "dirichlet": the outer ring is masked and an absorbing layer of
        layer_cells cells damps the waves (helm_create); "sommerfeld": the paper's
        first-order absorbing condition on the outer faces, with the Neumann
        incoming-wave face on top when neumann_top (helm_create_bvp)."""
        self.lib = L.lib()
        self.dim, self.n = int(dim), int(n)
        self.N = self.n ** self.dim
        dev = torch.device("cuda")
        self.mask = torch.as_tensor(mask, dtype=torch.uint8).reshape(-1).to(dev).contiguous()
        k2t = None
        if k2 is not None:
            k2t = torch.as_tensor(k2).to(dev, torch.complex128).reshape(-1).contiguous()
        prec = {"fp64": L.HELM_FP64, "mixed": L.HELM_MIXED}[precision]
        h = C.c_void_p()
        if boundary == "sommerfeld":
            st = self.lib.helm_create_bvp(self.dim, self.n, float(k0), _ptr(self.mask), _ptr(k2t),
                                          int(bool(neumann_top)), C.byref(h))
        else:
            st = self.lib.helm_create(self.dim, self.n, float(k0), int(layer_cells), float(layer_strength),
                                      _ptr(self.mask), _ptr(k2t), prec, C.byref(h))
        if st != 0:
            raise HelmError(st, "helm_create")
        self.h = h
        self.set_stream(torch.cuda.current_stream())

    # ------------------------------------------------------------ plumbing
    def _check(self, st, what=""):
        if st != 0:
            msg = self.lib.helm_last_error(self.h)
            raise HelmError(st, f"{what}: {msg.decode() if msg else ''}")

    def set_stream(self, stream):
        self._check(self.lib.helm_set_stream(self.h, C.c_void_p(stream.cuda_stream)), "set_stream")

    def set_profiling(self, on=True):
        self._check(self.lib.helm_set_profiling(self.h, int(bool(on))), "set_profiling")

    def mg_setup(self, levels):
        """Multigrid hierarchy of `levels` grids for the HELM_MG cycle (n odd down
        to the coarsest level)."""
        self._check(self.lib.helm_mg_setup(self.h, int(levels)), "mg_setup")

    def set_wait_limit(self, polls=1 << 20, extra_arrivals=0):
        """Bounded grid-barrier waits of the cooperative red-black cycle: polls
        before a wait gives up, and arrivals added to every barrier's target
        (> 0 injects a timeout for tests)."""
        self._check(self.lib.helm_set_wait_limit(self.h, int(polls), int(extra_arrivals)), "set_wait_limit")

    def set_reliable(self, delta=0.1, runaway=1e3, guard=0.0):
        """Reliable-update parameters of the complex64 BiCGStab (helm_set_reliable)."""
        self._check(self.lib.helm_set_reliable(self.h, float(delta), float(runaway), float(guard)), "set_reliable")

    def close(self):
        if getattr(self, "h", None):
            self.lib.helm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vec(self, dtype=torch.complex128):
        return torch.zeros(self.N, dtype=dtype, device="cuda")

    # ---------------------------------------------------------- operations
    def layer_k2(self, scale=None):
        out = self.vec()
        sc = None if scale is None else torch.as_tensor(scale, dtype=torch.float64).reshape(-1).cuda().contiguous()
        self._check(self.lib.helm_layer_k2(self.h, _ptr(sc), _ptr(out)), "layer_k2")
        return out

    def rhs(self, src, g):
        b = self.vec()
        self._check(self.lib.helm_rhs(self.h, _ptr(src.contiguous()), _ptr(g.contiguous()), _ptr(b)), "rhs")
        return b

    def apply(self, x, conj=False, out=None):
        y = torch.empty_like(x) if out is None else out
        self._check(self.lib.helm_apply(self.h, _ptr(x), _ptr(y), int(conj), _dtype_code(x)), "apply")
        return y

    def residual(self, f, x, conj=False, want_norm=True):
        r = torch.empty_like(x)
        nrm = torch.zeros(1, dtype=torch.float64, device="cuda") if want_norm else None
        self._check(self.lib.helm_residual(self.h, _ptr(f), _ptr(x), _ptr(r), _ptr(nrm), int(conj),
                                           _dtype_code(x)), "residual")
        return (r, nrm) if want_norm else r

    def relax(self, kind, f, x, sweeps=1, omega=0.6, conj=False):
        k = {"jacobi": L.HELM_JACOBI, "rbgs": L.HELM_RBGS, "sor": L.HELM_SOR, "ssor": L.HELM_SSOR}[kind]
        self._check(self.lib.helm_relax(self.h, k, float(omega), int(sweeps), _ptr(f), _ptr(x), int(conj),
                                        _dtype_code(x)), "relax")
        return x

    def don_load(self, layers, p, tau=0.0, act="tanh"):
        """layers: [(W[out, in], b[out])] float64; act on hidden layers: "tanh" or
        "leaky_relu" (App. B's trunk)."""
        widths = [layers[0][0].shape[1]] + [W.shape[0] for W, _ in layers]
        flat = np.ascontiguousarray(np.concatenate(
            [np.concatenate([np.asarray(W, np.float64).reshape(-1), np.asarray(b, np.float64)])
             for W, b in layers]))
        wd = (C.c_int * len(widths))(*widths)
        self._check(self.lib.don_load(self.h, flat.ctypes.data_as(C.c_void_p), wd, len(layers),
                                      {"tanh": L.HELM_ACT_TANH, "leaky_relu": L.HELM_ACT_LEAKY_RELU}[act],
                                      int(p), float(tau)), "don_load")
        k = C.c_int()
        idx = (C.c_int * int(p))()
        self.lib.don_info(self.h, C.byref(k), idx)
        self.k = k.value
        self.kept = list(idx)[: self.k]
        return self.k

    def don_load_branch(self, layers):
        """layers: [(W[out, in], b[out])] (FP32 values), ReLU on hidden layers;
        input width 2N, output width 2p."""
        widths = [layers[0][0].shape[1]] + [W.shape[0] for W, _ in layers]
        flat = np.ascontiguousarray(np.concatenate(
            [np.concatenate([np.asarray(W, np.float32).reshape(-1), np.asarray(b, np.float32)]) for W, b in layers]))
        wd = (C.c_int * len(widths))(*widths)
        self._check(self.lib.don_load_branch(self.h, flat.ctypes.data_as(C.c_void_p), wd, len(layers)),
                    "don_load_branch")

    def don_correct_nonlinear(self, r, z=None):
        z = torch.zeros_like(r) if z is None else z
        self._check(self.lib.don_correct(self.h, L.HELM_CORR_NONLINEAR, _ptr(r), _ptr(z), 0, _dtype_code(r)),
                    "don_correct")
        return z

    def basis(self):
        Q = torch.empty(self.N, self.k, dtype=torch.float64, device="cuda")
        self._check(self.lib.don_get_q(self.h, _ptr(Q)), "don_get_q")
        return Q

    def coarse_inverse(self):
        A = torch.empty(self.k, self.k, dtype=torch.complex128, device="cuda")
        self._check(self.lib.don_get_ainv(self.h, _ptr(A)), "don_get_ainv")
        return A

    def don_correct(self, r, z=None, conj=False):
        z = torch.zeros_like(r) if z is None else z
        self._check(self.lib.don_correct(self.h, L.HELM_CORR_TB, _ptr(r), _ptr(z), int(conj), _dtype_code(r)),
                    "don_correct")
        return z

    def precond(self, r, o: SolveOpts):
        z = torch.empty_like(r)
        self._check(self.lib.helm_precond(self.h, C.byref(o), _ptr(r), _ptr(z)), "precond")
        return z

    def solve(self, f, x0=None, o: SolveOpts | None = None, hist_len=4096, raise_on_fail=False):
        o = o or opts()
        x = torch.zeros_like(f) if x0 is None else x0.clone()
        st = Stats()
        hist = np.zeros(hist_len)
        rc = self.lib.helm_solve(self.h, C.byref(o), _ptr(f), _ptr(x), C.byref(st),
                                 hist.ctypes.data_as(C.c_void_p), hist_len)
        if rc in (L.HELM_BAD_ARG, L.HELM_CUDA_ERROR, L.HELM_NOT_READY, L.HELM_OUT_OF_MEMORY) or (
                raise_on_fail and rc != 0):
            self._check(rc, "solve")
        d = st.as_dict()
        d["status_name"] = L.STATUS_NAMES.get(d["status"], d["status"])
        n_hist = min(hist_len, self._hist_count(d, o))
        d["hist"] = hist[:n_hist]
        return x, d

    @staticmethod
    def _hist_count(d, o):
        if o.method == L.HELM_METHOD_RELAX:
            return d["iters"] + 1
        return d["iters"] + 1

    # ------------------------------------------------------------ adjoint
    def set_k2(self, k2):
        k2t = torch.as_tensor(k2).to("cuda", torch.complex128).reshape(-1).contiguous()
        self._check(self.lib.helm_set_k2(self.h, _ptr(k2t)), "set_k2")

    def receivers(self, xyz):
        """(idx, w) device tensors of the trilinear sampling of receivers xyz (R x 3)."""
        x = torch.as_tensor(xyz, dtype=torch.float64).reshape(-1, 3).cuda().contiguous()
        R = x.shape[0]
        idx = torch.empty(8 * R, dtype=torch.int32, device="cuda")
        w = torch.empty(8 * R, dtype=torch.float64, device="cuda")
        self._check(self.lib.helm_receivers_setup(self.h, R, _ptr(x), _ptr(idx), _ptr(w)), "receivers_setup")
        return idx, w

    def sample(self, idx, w, u):
        R = idx.numel() // 8
        out = torch.empty(R, dtype=torch.complex128, device="cuda")
        self._check(self.lib.helm_receivers_sample(self.h, R, _ptr(idx), _ptr(w), _ptr(u.contiguous()), _ptr(out)),
                    "receivers_sample")
        return out

    def sample_adjoint(self, idx, w, e):
        R = idx.numel() // 8
        b = self.vec()
        self._check(self.lib.helm_receivers_adjoint(self.h, R, _ptr(idx), _ptr(w), _ptr(e.contiguous()), _ptr(b)),
                    "receivers_adjoint")
        return b

    def k2_gradient(self, lam, u):
        g = self.vec()
        self._check(self.lib.helm_k2_gradient(self.h, _ptr(lam.contiguous()), _ptr(u.contiguous()), _ptr(g)),
                    "k2_gradient")
        return g

    def solve_host(self, f: np.ndarray, x: np.ndarray, o: SolveOpts | None = None):
        """Host buffers in and out (complex128 numpy arrays, x updated in place)."""
        o = o or opts()
        st = Stats()
        rc = self.lib.helm_solve_host(self.h, C.byref(o), f.ctypes.data_as(C.c_void_p),
                                      x.ctypes.data_as(C.c_void_p), C.byref(st), None, 0)
        if rc in (L.HELM_BAD_ARG, L.HELM_CUDA_ERROR, L.HELM_NOT_READY, L.HELM_OUT_OF_MEMORY):
            self._check(rc, "solve_host")
        return st.as_dict()


def _driver_version():
    """CUDA driver version (e.g. 13000), the tile cache key's driver part."""
    v = C.c_int(0)
    try:
        C.CDLL("libcuda.so.1").cuDriverGetVersion(C.byref(v))
    except OSError:
        return "unknown"
    return v.value


def solve_concurrent(problems, fs, xs=None, o: "SolveOpts | None" = None, threads: int = 0):
    """helm_solve_concurrent: every problem (distinct HELM_MIXED Problems) solved by its
    own solve on its own stream, overlapped on the GPU, each stopping at its own
    convergence.  Returns (solutions, per-problem statistics)."""
    lib = L.lib()
    o = o or opts("bicgstab", "rbgs", 3, tol=1e-6, maxit=20000)
    n = len(problems)
    xs = [torch.zeros_like(f) for f in fs] if xs is None else [x.clone() for x in xs]
    hs = (C.c_void_p * n)(*[P.h for P in problems])
    fp = (C.c_void_p * n)(*[f.data_ptr() for f in fs])
    xp = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
    stats = (Stats * n)()
    rc = lib.helm_solve_concurrent(n, hs, C.byref(o), fp, xp, stats, int(threads))
    if rc in (L.HELM_BAD_ARG, L.HELM_CUDA_ERROR, L.HELM_NOT_READY, L.HELM_OUT_OF_MEMORY):
        raise HelmError(rc, "helm_solve_concurrent")
    out = []
    for s_ in stats:
        d = s_.as_dict()
        d["status_name"] = L.STATUS_NAMES.get(d["status"], d["status"])
        out.append(d)
    return xs, out


class Batch:
    """Many independent problems (HELM_MIXED Problems with a loaded trunk basis)
    solved together by batched FGMRES: one launch per phase over all problems."""

    def __init__(self, problems):
        self.lib = L.lib()
        self.problems = list(problems)
        hs = (C.c_void_p * len(self.problems))(*[P.h for P in self.problems])
        b = C.c_void_p()
        st = self.lib.helm_batch_create(len(self.problems), hs, C.byref(b))
        if st != 0:
            raise HelmError(st, "helm_batch_create")
        self.b = b
        self.tile = (1024, 4 * 152)

    def set_tile(self, tile_rows, grid=4 * 152):
        st = self.lib.helm_batch_set_tile(self.b, int(tile_rows), int(grid))
        if st != 0:
            raise HelmError(st, "helm_batch_set_tile")
        self.tile = (int(tile_rows), int(grid))

    def solve(self, fs, xs=None, o: SolveOpts | None = None):
        o = o or opts("fgmres", "jacobi", 1, tol=1e-6, restart=30, maxit=5000)
        n = len(self.problems)
        xs = [torch.zeros_like(f) for f in fs] if xs is None else [x.clone() for x in xs]
        fp = (C.c_void_p * n)(*[f.data_ptr() for f in fs])
        xp = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
        stats = (Stats * n)()
        rc = self.lib.helm_batch_solve(self.b, C.byref(o), fp, xp, stats)
        if rc in (L.HELM_BAD_ARG, L.HELM_CUDA_ERROR, L.HELM_NOT_READY, L.HELM_OUT_OF_MEMORY):
            raise HelmError(rc, "helm_batch_solve")
        out = []
        for s in stats:
            d = s.as_dict()
            d["status_name"] = L.STATUS_NAMES.get(d["status"], d["status"])
            out.append(d)
        return xs, out

    def autotune(self, fs, o: SolveOpts | None = None, candidates=(256, 512, 1024, 2048, 4096), trial_iters=6,
                 cache=None):
        """Pick the tile length by timing a few iterations of the given method for each
        candidate; results are cached per GPU, driver version, method, problem count
        and total size."""
        import json
        import os
        import time
        key = None
        if cache:
            prop = torch.cuda.get_device_properties(0)
            key = (f"{prop.name}|driver {_driver_version()}|{o.method if o is not None else 1}|"
                   f"{len(self.problems)}|{sum(P.N for P in self.problems)}")
            try:
                table = json.load(open(cache))
                if key in table:
                    self.set_tile(table[key])
                    return table[key], {}
            except Exception:
                table = {}
        o = o or opts("fgmres", "jacobi", 1, tol=1e-12, restart=30, maxit=trial_iters)
        trial = SolveOpts(o.method, o.relax, o.n_r, o.omega, o.correction, 1e-30, o.restart, trial_iters, o.conj)
        times = {}
        for t in candidates:
            self.set_tile(t)
            self.solve(fs, None, trial)                   # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            self.solve(fs, None, trial)
            torch.cuda.synchronize()
            times[t] = time.perf_counter() - t0
        best = min(times, key=times.get)
        self.set_tile(best)
        if cache and key:
            try:
                table = json.load(open(cache)) if os.path.exists(cache) else {}
            except Exception:
                table = {}
            table[key] = best
            os.makedirs(os.path.dirname(cache) or ".", exist_ok=True)
            json.dump(table, open(cache, "w"), indent=1)
        return best, times

    def close(self):
        if getattr(self, "b", None):
            self.lib.helm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
