"""Command-line runner: set up a named workload and solve it on cuda:0.

    python -m paper_2405_12380_gb300.cli --workload cube3d-64 [--maxit M] [--solves S] [--precision P]
    python -m paper_2405_12380_gb300.cli --stencil N          # operator bandwidth on N^3
    python -m paper_2405_12380_gb300.cli --experiment mixed   # 128^3 submarine, mixed vs FP64
    python -m paper_2405_12380_gb300.cli --experiment batch [--count C]
    python -m paper_2405_12380_gb300.cli --experiment adjoint [--fd V]

Prints one JSON line per solve (or per experiment result) with the library's
statistics.  Used to drive profiler captures of a bounded number of iterations
and the measurements of the mixed-precision, batched and adjoint forms.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    import torch

    import scenes
    import paper_2405_12380_gb300 as hm

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cube3d-64")
    ap.add_argument("--maxit", type=int, default=None)
    ap.add_argument("--solves", type=int, default=1)
    ap.add_argument("--stencil", type=int, default=0, help="time y = A x on an n^3 grid instead of solving")
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--experiment", choices=["mixed", "batch", "adjoint"], default=None)
    ap.add_argument("--count", type=int, default=64, help="batch: number of problems")
    ap.add_argument("--fd", type=int, default=32, help="adjoint: voxels checked by central differences")
    ap.add_argument("--relax", default=None, help="experiments: jacobi | rbgs (default: the workload's)")
    ap.add_argument("--n-r", type=int, default=None, help="experiments: sweeps per preconditioner application")
    ap.add_argument("--method", default=None, help="experiments: fgmres | bicgstab")
    ap.add_argument("--precision", default=None, help="fp64 | mixed (default: the workload's)")
    ap.add_argument("--form", default="both", choices=["lockstep", "concurrent", "both"],
                    help="batch: lockstep batched solve (helm_batch_solve), concurrent solves "
                         "(helm_solve_concurrent), or both")
    a = ap.parse_args(argv)
    if a.stencil:
        return stencil(a.stencil, a.reps)
    over = {k: v for k, v in (("relax", a.relax), ("n_r", a.n_r), ("method", a.method)) if v is not None}
    if a.experiment == "mixed":
        return exp_mixed(a.maxit, over)
    if a.experiment == "batch":
        return exp_batch(a.count, a.maxit, over, a.form)
    if a.experiment == "adjoint":
        return exp_adjoint(a.fd, a.maxit, over)
    w = dict(scenes.BENCH_WORKLOADS[a.workload])
    if a.maxit is not None:
        w["maxit"] = a.maxit
    sc = scenes.make_scene(w["scene"], seed=w["seed"], n=w["n"])
    torch.cuda.set_device(0)
    prec = a.precision or w.get("precision", "fp64")
    P = hm.Problem(sc.dim, sc.n, sc.k0, sc.mask, layer_cells=sc.layer_cells, layer_strength=sc.layer_strength,
                   precision=prec)
    f = P.rhs(torch.from_numpy(sc.src).cuda(), torch.from_numpy(sc.g).cuda())
    k = P.don_load(sc.trunk, sc.p, tau=w["tau"]) if w["correction"] == "tb" else 0
    o = hm.opts(w["method"], w["relax"], w["n_r"], correction=w["correction"], tol=w["tol"],
                restart=w["restart"], maxit=w["maxit"])
    for _ in range(a.solves):
        x, st = P.solve(f, None, o)
        st.pop("hist", None)
        st["kept"] = k
        st["precision"] = prec
        print(json.dumps(st), flush=True)


def stencil(n, reps):
    """Operator throughput: y = A x on n^3 (complex64 and complex128), one JSON line each."""
    import torch

    import scenes
    import paper_2405_12380_gb300 as hm
    torch.cuda.set_device(0)
    mask = (scenes.ring_mask(3, n) | scenes.box_mask(3, n, *scenes.centred_box_nodes(n, n // 4)))
    P = hm.Problem(3, n, 16.0, mask.reshape(-1).astype("uint8"), layer_cells=8, layer_strength=0.5)
    for dt, nbytes in ((torch.complex64, 17), (torch.complex128, 33)):
        xs = [torch.randn(P.N, dtype=dt, device="cuda") for _ in range(3)]
        y = torch.empty_like(xs[0])
        for q in range(3):
            P.apply(xs[q], out=y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for q in range(reps):
            P.apply(xs[q % 3], out=y)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        print(json.dumps({"dtype": str(dt), "n": n, "us": ms * 1e3, "GBps": nbytes * P.N / (ms * 1e-3) / 1e9}))
    # complex64 sweeps: per full sweep read x and f, write x, two table bytes (26 B per node)
    f = torch.randn(P.N, dtype=torch.complex64, device="cuda")
    x = torch.randn(P.N, dtype=torch.complex64, device="cuda")
    for kind, sweeps in (("jacobi", 2), ("rbgs", 1)):
        P.relax(kind, f, x, sweeps=sweeps)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for q in range(reps):
            P.relax(kind, f, x, sweeps=sweeps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps / sweeps
        print(json.dumps({"sweep": kind, "dtype": "complex64", "n": n, "us_per_sweep": ms * 1e3,
                          "GBps": 26 * P.N / (ms * 1e-3) / 1e9}))


def _emit(d):
    print(json.dumps(d), flush=True)


def exp_mixed(maxit=None, over=None):
    """The 128^3 submarine scattering problem solved by DeepONet-FGMRES(50) (one Jacobi
    sweep + trunk-basis correction per preconditioner application) to 1e-6, once with
    the mixed-precision handle (complex64 preconditioner, BF16 basis, FP64 Arnoldi and
    residuals) and once with the FP64 handle; same input, same options."""
    import torch

    import scenes
    import paper_2405_12380_gb300 as hm
    w = dict(scenes.BENCH_WORKLOADS["submarine3d-128"])
    w.update(over or {})
    sc = scenes.make_scene(w["scene"], seed=w["seed"], n=w["n"])
    torch.cuda.set_device(0)
    o = hm.opts(w["method"], w["relax"], w["n_r"], correction=w["correction"], tol=w["tol"],
                restart=w["restart"], maxit=maxit or w["maxit"])
    xs = {}
    for prec in ("mixed", "fp64"):
        P = hm.Problem(sc.dim, sc.n, sc.k0, sc.mask, layer_cells=sc.layer_cells,
                       layer_strength=sc.layer_strength, precision=prec)
        f = P.rhs(torch.from_numpy(sc.src).cuda(), torch.from_numpy(sc.g).cuda())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k = P.don_load(sc.trunk, sc.p, tau=w["tau"])
        torch.cuda.synchronize()
        setup = time.perf_counter() - t0
        x, st = P.solve(f, None, o)
        st.pop("hist", None)
        xs[prec] = x
        _emit({"experiment": "mixed", "precision": prec, "workload": "submarine3d-128", "kept": k,
               "method": w["method"], "relax": w["relax"], "n_r": w["n_r"],
               "setup_s": setup, "solve_s": st["ms"] / 1e3, "iters": st["iters"], "cycles": st["cycles"],
               "rel_res_fp64": st["rel_res"], "status": st["status_name"]})
        P.close()
        del P, f
        torch.cuda.empty_cache()
    d = torch.linalg.vector_norm(xs["mixed"] - xs["fp64"]) / torch.linalg.vector_norm(xs["fp64"])
    _emit({"experiment": "mixed", "rel_diff_mixed_vs_fp64_solution": float(d)})


def exp_batch(count=64, maxit=None, over=None, form="both"):
    """`count` problems on uneven grids 48^3-128^3 (seeded k, scatterers, sources) on
    mixed-precision handles, to 1e-6: the lockstep batched solve (default
    DeepONet-FGMRES(30) with Jacobi + trunk basis; --method bicgstab --relax rbgs
    --n-r 3 for the batched complex64 BiCGStab) and/or the concurrent solves (each
    problem's own solve on its own stream, helm_solve_concurrent), against the same
    problems solved one after another with the FP64 handle; every mixed solution's
    FP64 residual is recomputed by the library."""
    import torch

    import scenes
    import paper_2405_12380_gb300 as hm
    torch.cuda.set_device(0)
    scs = scenes.batch_scenes(0, count=count)
    ov = over or {}
    o = hm.opts(ov.get("method", "fgmres"), ov.get("relax", "jacobi"), ov.get("n_r", 1), tol=1e-6, restart=30,
                maxit=maxit or 20000)
    probs, fs = [], []
    for sc in scs:
        P = hm.Problem(3, sc.n, sc.k0, sc.mask, layer_cells=sc.layer_cells, precision="mixed")
        P.don_load(sc.trunk, sc.p, tau=1e-6)
        probs.append(P)
        fs.append(P.rhs(torch.from_numpy(sc.src).cuda(), torch.from_numpy(sc.g).cuda()))
    results = {}
    forms = ["lockstep", "concurrent"] if form == "both" else [form]
    for fm in forms:
        tile = None
        if fm == "lockstep":
            B = hm.Batch(probs)
            tile, _ = B.autotune(fs, o)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if fm == "lockstep":
            xb, stb = B.solve(fs, None, o)
        else:
            xb, stb = hm.solve_concurrent(probs, fs, None, o)
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
        ok = sum(1 for s_ in stb if s_["status"] == 0)
        res_check = []
        for P, f, x in zip(probs, fs, xb):
            _, nrm = P.residual(f, x)
            res_check.append(float(nrm.sqrt().item() / torch.linalg.vector_norm(f).item()))
        _emit({"experiment": "batch", "form": ("batched mixed, lockstep" if fm == "lockstep"
                                               else "mixed, concurrent solves"),
               "problems": count, "relax": o.relax, "n_r": o.n_r, "nodes": int(sum(P.N for P in probs)),
               "tile": tile, "wall_s": tb, "converged": ok, "iters_max": max(s_["iters"] for s_ in stb),
               "rel_res_max": max(s_["rel_res"] for s_ in stb), "fp64_residual_recomputed_max": max(res_check),
               "converged_by_fp64_residual": sum(1 for r_ in res_check if r_ <= 1.0001e-6),
               "method": o.method, "iters_each": [s_["iters"] for s_ in stb]})
        results[fm] = (tb, xb)
        if fm == "lockstep":
            B.close()
            del B
    for P in probs:
        P.close()
    del probs
    torch.cuda.empty_cache()
    # the same problems, one FP64 handle at a time
    t_seq, ok64, it64 = 0.0, 0, []
    diffs = {fm: [] for fm in results}
    for i, sc in enumerate(scs):
        P = hm.Problem(3, sc.n, sc.k0, sc.mask, layer_cells=sc.layer_cells)
        f = P.rhs(torch.from_numpy(sc.src).cuda(), torch.from_numpy(sc.g).cuda())
        P.don_load(sc.trunk, sc.p, tau=1e-6)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x64, st = P.solve(f, None, o)
        torch.cuda.synchronize()
        t_seq += time.perf_counter() - t0
        ok64 += st["status"] == 0
        it64.append(st["iters"])
        for fm, (_, xb) in results.items():
            diffs[fm].append(float(torch.linalg.vector_norm(xb[i] - x64) / torch.linalg.vector_norm(x64)))
        P.close()
    _emit({"experiment": "batch", "form": "sequential FP64", "problems": count, "wall_s": t_seq,
           "converged": ok64, "iters_max": max(it64), "iters_each": it64,
           **{f"rel_diff_{fm}_vs_fp64_max": max(v) for fm, v in diffs.items()},
           **{f"speedup_{fm}": t_seq / results[fm][0] for fm in results}})


def exp_adjoint(n_fd=32, maxit=None, over=None):
    """The 96^3 adjoint workload: receiver misfit of the bump-perturbed k^2 against
    data from the unperturbed field (here from a GPU solve; the tests use the
    oracle's), gradient by the adjoint DeepONet-FGMRES solve, timed, and checked
    against central differences of the loss on `n_fd` seeded fluid voxels."""
    import numpy as np
    import torch

    import scenes
    import paper_2405_12380_gb300 as hm
    from paper_2405_12380_gb300.autograd import misfit_loss
    torch.cuda.set_device(0)
    sc = scenes.bump_cube3d(0, n=96)
    P0 = hm.Problem(3, sc.n, sc.k0, sc.mask, layer_cells=sc.layer_cells, layer_strength=sc.layer_strength)
    k2 = P0.layer_k2(sc.k2_scale)
    k20 = P0.layer_k2(None)
    P = hm.Problem(3, sc.n, sc.k0, sc.mask, layer_cells=sc.layer_cells, layer_strength=sc.layer_strength, k2=k2)
    f = P.rhs(torch.from_numpy(sc.src).cuda(), torch.from_numpy(sc.g).cuda())
    k = P.don_load(sc.trunk, sc.p, tau=1e-6)
    ov = over or {}
    o = hm.opts(ov.get("method", "fgmres"), ov.get("relax", "rbgs"), ov.get("n_r", 3), tol=1e-10, restart=30,
                maxit=maxit or 20000)
    idx, w = P.receivers(sc.extra["receivers"])
    P.set_k2(k20)
    u0, st0 = P.solve(f, None, o)
    d = P.sample(idx, w, u0)
    P.set_k2(k2)
    times = []
    for rep in range(3):
        k2t = k2.clone().requires_grad_(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L, u = misfit_loss(k2t, f, P, o, idx, w, d)
        L.backward()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    g = k2t.grad.clone()
    _emit({"experiment": "adjoint", "workload": "bump_cube3d-96", "kept": k, "loss": float(L), "method": o.method,
           "relax": o.relax, "n_r": o.n_r,
           "forward_backward_s": min(times), "forward_iters": st0["iters"]})
    # central differences on seeded fluid voxels (real and imaginary directions)
    rng = np.random.default_rng(7)
    fluid = np.flatnonzero(sc.mask.reshape(-1) == 0)
    worst = 0.0
    gmax = float(g.abs().max())
    rows = []
    for l in rng.choice(fluid, n_fd, replace=False):
        for unit, part in ((1.0, "re"), (1j, "im")):
            eps = 1e-3 * float(abs(k2[l]))
            vals = []
            for sgn in (1, -1):
                kk = k2.clone()
                kk[l] += sgn * eps * unit
                P.set_k2(kk)
                uu, st = P.solve(f, None, o)
                e = P.sample(idx, w, uu) - d
                vals.append(float((e.real ** 2 + e.imag ** 2).sum()))
            fd = (vals[0] - vals[1]) / (2 * eps)
            an = float(g[l].real if part == "re" else g[l].imag)
            err = abs(fd - an) / max(abs(fd), 1e-2 * gmax)
            worst = max(worst, err)
            rows.append((int(l), part, fd, an))
    P.set_k2(k2)
    _emit({"experiment": "adjoint", "fd_voxels": n_fd, "fd_directions": 2 * n_fd,
           "max_rel_err_vs_central_differences": worst, "grad_max_abs": gmax, "samples": rows[:4]})


if __name__ == "__main__":
    main()
