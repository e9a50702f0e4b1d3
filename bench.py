"""Benchmark of the space-time BEM hot path on GB300 (prints one JSON line).

Workload (square256): unit-square boundary with N_x = 256 uniform segments,
N_t = 256 uniform steps on T = 1, alpha = 1, Dirichlet datum
g = U*(x - y*, t) with y* = (1.5, 1.5), u_0 = 0 (synthetic, seeded geometry).

One step = the whole hot path on one GPU, inputs (the mesh) resident:
  assembly of V_h, K_h, D_h (FP64, 3 x 256 x 256 x 256 Toeplitz entries),
  right-hand side f = 1/2 M_h g + K_h g, lumped mass,
  right-preconditioned GMRES to a relative residual of 1e-8 (FP64) with the
  direct block-Toeplitz products (the paper's method).  The same step with
  the products through time FFTs of the lag blocks (an optional extra, not
  the paper's method; --solve fft makes it the timed step) is timed beside
  it.
value = distinct Toeplitz entries assembled per second of whole-step time.
Component figures (assembly entries/s, Toeplitz-apply GB/s and GFLOP/s, GMRES
time) are reported beside it.  Between timed steps a 256 MB buffer is written
to flush L2 (outside the step's CUDA events).

--impl reference times the FP64 CPU oracle on this machine's host cores on a
bounded random sample of the same entries (the oracle has no GPU code).
Multi-GPU (torchrun, N > 1): the one problem is sharded by lag (chunks of 16
lags dealt to ranks in snake order); every rank assembles its lag blocks, and
each K, V and D product is its partial sum followed by an NCCL all-reduce of
the n_t x n_x result (strong scaling: value = the problem's entries per second
of the slowest rank's step).
"""
import argparse
import ctypes
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "assembly entries/s; Toeplitz matvec GB/s; GMRES time to 1e-8 res, mixed vs FP64"
UNIT = "entries/s"
WORKLOAD = "square256"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# FP64 pipe: 1.25 TFLOP/s nominal dense FP64 for GB300 (recipe table); the
# roofline divides by the FP64 FMA rate measured in the same run
# (stbem_pipe_peaks) and reports the nominal fraction beside it.
FP64_NOMINAL_TFLOPS = 1.25
# DRAM bytes (read + write) of the lags >= 2 launch of the FP64 D tile kernel
# at square256 (one launch over lags 2..255) from the ncu capture of the
# current kernel (profiles/k_tile_D_f64_lag2.md gives the command); set to None
# whenever that kernel changes until it is captured again
TRAFFIC_D2_BYTES = 2673664 + 80304384


def _oracle_sample(n_entries, seed, rng_lags=None):
    """Time the oracle on a bounded random sample of (op, lag, i, j) entries."""
    import workloads as W
    from oracle import assembly as OA
    from oracle.geometry import BoundaryMesh
    p = W.config(WORKLOAD)
    om = BoundaryMesh(p.vertices, p.T, p.n_t, p.alpha)
    rng = np.random.default_rng(seed)
    per_op = n_entries // 3
    t0 = time.perf_counter()
    done = 0
    for op, fn in (("V", OA.V_entries), ("K", OA.K_entries), ("D", OA.D_entries)):
        lags = rng.integers(0, p.n_t, size=per_op)
        I = rng.integers(0, p.n_x, size=per_op)
        J = rng.integers(0, p.n_x, size=per_op)
        for d in np.unique(lags):
            sel = lags == d
            fn(om, int(d), I[sel], J[sel])
            done += int(sel.sum())
    return done, time.perf_counter() - t0


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def W_config():
    import workloads as W
    return W.config(WORKLOAD)


def _config(p, l2, solve="direct"):
    return {"workload": WORKLOAD, "n_x": p.n_x, "n_t": p.n_t, "alpha": p.alpha, "T": p.T,
            "y_star": list(p.y_star), "precision": "fp64 assembly + fp64 GMRES", "l2": l2,
            "gmres_products": "time FFTs of the lag blocks (fp64)" if solve == "fft" else "direct block sums"}


def _oracle_worker(args):
    n, seed = args
    return _oracle_sample(n, seed)


class OraclePool:
    """The oracle on every host core: one single-threaded worker process per
    core (BLAS and OpenMP pinned to one thread each), started with 'spawn' so
    that it is safe after CUDA has been initialised in the parent."""

    def __init__(self, cores=None):
        import multiprocessing as mp
        self.cores = cores or _cores()
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        self.blas_threads = 1
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.pool.map(_oracle_worker, [(3, 1 + w) for w in range(self.cores)])    # imports, warm-up

    def step(self, per_worker, seed):
        """Every worker evaluates per_worker random entries; returns (entries,
        wall seconds of the parallel region)."""
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, [(per_worker, seed * 1000 + w) for w in range(self.cores)])
        return sum(c for c, _ in res), time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


ORACLE_PER_WORKER = 1024     # entries per worker per step (about 1 s of one core)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    pool = OraclePool()
    for k in range(args.warmup):
        pool.step(64, 100 + k)
    times, counts = [], []
    for k in range(args.steps):
        c, t = pool.step(ORACLE_PER_WORKER, 2000 + k)
        counts.append(c)
        times.append(t)
    pool.close()
    value = sum(counts) / sum(times)
    sample = ("%d random (op, lag, i, j) entries of %s per step (%d per worker), uniform over the 3 "
              "operators, lags and index pairs; %d single-threaded numpy worker processes"
              % (ORACLE_PER_WORKER * pool.cores, WORKLOAD, ORACLE_PER_WORKER, pool.cores))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(W_config(), "n/a (CPU oracle)"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "blas_threads": pool.blas_threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw nvidia-smi samples; STBEM_BENCH_OUT chooses the directory
        out_dir = os.environ.get("STBEM_BENCH_OUT") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, "clocks_bench_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_batched(ctx, dev, stream, n_src=256, fp64_residual=False):
    """square512 with 256 right-hand sides g_k = U*(x - y_k, t), y_k seeded on
    the annulus 1.2 < |y - (0.5, 0.5)| < 3: batched tensor-core solve to
    FP64-solve accuracy, timed with CUDA events, beside one FP64
    single-right-hand-side solve.  F and the final refinement residuals use
    the exact-slice tensor-core product (7 slices); with fp64_residual the
    same solve on FP64 CUDA-core residuals is timed as well."""
    import torch
    import workloads as W
    import paper_1811_05224_gb300 as P
    p = W.config("square512")
    nt, nx = p.n_t, p.n_x
    mesh = P.Mesh(ctx, p.vertices, p.T, p.n_t, p.alpha)
    ev = lambda: torch.cuda.Event(enable_timing=True)       # noqa: E731
    e = [ev() for _ in range(8)]
    e[0].record(stream)
    V = P.assemble(ctx, mesh, "V")
    e[1].record(stream)
    K = P.assemble(ctx, mesh, "K")
    e[2].record(stream)
    D32 = P.assemble(ctx, mesh, "D", "f32")
    e[3].record(stream)
    V3 = P.bf16_split3(ctx, V)
    Db = P.to_bf16(ctx, D32)
    L = P.lumped_mass(ctx, mesh)
    Vx = P.exact_slices(ctx, V, 7)
    Kx = P.exact_slices(ctx, K, 7)
    ys = W.annulus_sources(n_src, seed=4)
    e[4].record(stream)
    # F = 1/2 M G + K G with the exact-slice K product of all 256 right-hand sides
    G, F = P.rhs_batched(ctx, mesh, Kx, ys)
    e[5].record(stream)
    # BF16 tensor-core inner solves; refinement on the three-slice residual,
    # then on the exact-slice residual to 1e-8 (FP64-solve accuracy)
    Wb, infos = P.solve_batched(ctx, V3, F, Db, L, tol=1e-8, inner_tol=1e-2, restart=40, max_iter=600, V64=Vx)
    e[6].record(stream)
    torch.cuda.synchronize(dev)
    s0, s1 = ev(), ev()
    # products alone on all right-hand sides: BF16, compensated BF16, exact-slice
    xb = P.to_bf16(ctx, Wb)
    for _ in range(2):
        P.apply_tc(ctx, V3[0], xb)

    def timed(fn):
        s0.record(stream)
        r = fn()
        s1.record(stream)
        torch.cuda.synchronize(dev)
        return r, s0.elapsed_time(s1)

    _, tc_ms = timed(lambda: P.apply_tc(ctx, V3[0], xb))
    # the compensated accumulation (partials of 4 K steps) of the hi x hi slice
    # product of the three-slice residual
    _, tc4_ms = timed(lambda: P.apply_tc(ctx, V3[0], xb, chunk=4))
    xwork = torch.empty(int(_exact_work_bytes(ctx, nt, nx, n_src, 7)), dtype=torch.uint8, device=dev)
    yx = torch.empty_like(Wb)
    P.apply_exact(ctx, Vx, Wb, out=yx, work=xwork)
    _, ex_ms = timed(lambda: P.apply_exact(ctx, Vx, Wb, out=yx, work=xwork))
    _, sl_ms = timed(lambda: P.exact_slices(ctx, Wb, 7))
    tc_flops = 2.0 * nx * nx * nt * (nt + 1) / 2 * n_src
    # FP64 CUDA-core product of 8 right-hand sides: accuracy of the exact-slice
    # product and of F, and the FP64 rate
    y64, y64_ms = timed(lambda: P.apply(ctx, V, Wb[:8]))
    # error against the row-scale bound n_x sum_d max|V[d][i]| max|W[b][m - d]|
    # (the exact-slice error is relative to row maxima, not to |V| |W|
    # elementwise: early steps of W span hundreds of decades along a row)
    ra = V.abs().amax(dim=2)
    rx = Wb[:8].abs().amax(dim=2)
    Mb = torch.zeros_like(y64)
    for d in range(nt):
        Mb[:, d:, :] += rx[:, :nt - d, None] * ra[d][None, None, :]
    Mb *= nx
    ex_err = float(((yx[:8] - y64).abs() / Mb.clamp_min(1e-300)).max())
    ex_norm = float(max((yx[b] - y64[b]).norm() / y64[b].norm() for b in range(8)))
    del ra, rx, Mb
    _, F8 = P.rhs_batched(ctx, mesh, K, ys[:8])
    f_rel = float(max((F[b] - F8[b]).norm() / F8[b].norm() for b in range(8)))
    fp64_solve = None
    if fp64_residual:
        s0.record(stream)
        _, F64 = P.rhs_batched(ctx, mesh, K, ys)
        s1.record(stream)
        torch.cuda.synchronize(dev)
        rhs64_ms = s0.elapsed_time(s1)
        (W64, inf64), solve64_ms = timed(lambda: P.solve_batched(ctx, V3, F64, Db, L, tol=1e-8, inner_tol=1e-2,
                                                                 restart=40, max_iter=600, V64=V))
        fp64_solve = {"rhs_ms": rhs64_ms, "solve_ms": solve64_ms,
                      "inner_iterations": max(i["iterations"] for i in inf64),
                      "note": "the same solve with F and the final residuals from the FP64 CUDA-core product"}
        del F64, W64
    # the same solve with F and the final residuals through time FFTs (the
    # frequency blocks of K and V), and the FFT product of all right-hand sides
    s0.record(stream)
    Kh, Vh = P.fft_operator(ctx, K), P.fft_operator(ctx, V)
    s1.record(stream)
    torch.cuda.synchronize(dev)
    fft_transforms_ms = s0.elapsed_time(s1)
    (_, Ff), rhsf_ms = timed(lambda: P.rhs_batched(ctx, mesh, Kh, ys))
    nbw = ctypes.c_size_t()
    ctx.check(ctx.lib.stbem_solve_batched_fft_workspace_bytes(nt, nx, n_src, 40, ctypes.byref(nbw)))
    fwork = torch.empty(nbw.value, dtype=torch.uint8, device=dev)
    (Wf, inff), solvef_ms = timed(lambda: P.solve_batched(ctx, V3, Ff, Db, L, tol=1e-8, inner_tol=1e-2,
                                                          restart=40, max_iter=600, V64=Vh, work=fwork))
    del fwork
    yf = torch.empty_like(Wb)
    awf = P.api.apply_fft_workspace(ctx, nt, nx, n_src)
    P.apply_fft(ctx, Vh, Wb, work=awf, out=yf)
    _, fft_apply_ms = timed(lambda: P.apply_fft(ctx, Vh, Wb, work=awf, out=yf))
    fft_apply_rel = float(max((yf[b] - y64[b]).norm() / y64[b].norm() for b in range(8)))
    del awf, Kh, Vh
    # one FP64 single-right-hand-side solve of the same system for comparison
    D64 = P.assemble(ctx, mesh, "D")
    g1, f1 = P.rhs(ctx, mesh, K, ys[0])
    (w1, info1), one_ms = timed(lambda: P.solve(ctx, V, f1, D64, L, tol=1e-8))
    # accuracy reference: the FP64 solve of right-hand side 0 to 1e-11
    w_acc, _ = P.solve(ctx, V, f1, D64, L, tol=1e-11)
    rel = float((Wb[0] - w_acc).norm() / w_acc.norm())
    rel_fft = float((Wf[0] - w_acc).norm() / w_acc.norm())
    r0f = f1 - P.apply(ctx, V, Wf[0])
    rel_fp64_path = float((w1 - w_acc).norm() / w_acc.norm())
    r0 = f1 - P.apply(ctx, V, Wb[0])
    peaks = _peaks()
    bf16_peak = float(peaks.get("bf16_tflops", 1867.6))
    ex_exec = tc_flops * 28                                   # 7 slices: 28 slice-pair products
    out = {
        "workload": "square512 x 256 sources (annulus 1.2..3, seed 4)",
        "assembly_ms": {"V_f64": e[0].elapsed_time(e[1]), "K_f64": e[1].elapsed_time(e[2]),
                        "D_f32": e[2].elapsed_time(e[3])},
        "slices_ms": e[3].elapsed_time(e[4]),
        "slices_note": "three BF16 slices of V, BF16 D, exact slices (7 x 6 bits) of V and K",
        "rhs_ms": e[4].elapsed_time(e[5]),
        "rhs_note": "F = 1/2 M G + K G, exact-slice tensor-core K product of all right-hand sides",
        "F_rel_diff_vs_fp64_product_8rhs": f_rel,
        "solve_ms": e[5].elapsed_time(e[6]),
        "solve_note": "BF16 tensor-core lockstep GMRES, refinement on three-slice then exact-slice residuals, tol 1e-8",
        "inner_iterations": max(i["iterations"] for i in infos),
        "max_rel_residual": max(i["rel_residual"] for i in infos),
        "fp64_rel_residual_rhs0": float(r0.norm() / f1.norm()),
        "w_rel_diff_vs_fp64_solve_1e-11_rhs0": rel,
        "fp64_path_1e-8_w_rel_diff_vs_fp64_solve_1e-11_rhs0": rel_fp64_path,
        "fp64_single_solve_ms": one_ms, "fp64_single_solve_iterations": info1["iterations"],
        "fp64_256_sequential_solves_ms_projected": one_ms * n_src,
        "fp64_residual_solve": fp64_solve,
        "fft_residual_solve": {
            "transforms_ms": fft_transforms_ms, "rhs_ms": rhsf_ms, "solve_ms": solvef_ms,
            "inner_iterations": max(i["iterations"] for i in inff),
            "max_rel_residual": max(i["rel_residual"] for i in inff),
            "fp64_rel_residual_rhs0": float(r0f.norm() / f1.norm()),
            "w_rel_diff_vs_fp64_solve_1e-11_rhs0": rel_fft,
            "apply_ms_all_rhs": fft_apply_ms, "apply_rel_diff_vs_fp64_8rhs": fft_apply_rel,
            "note": "the same solve with F and the final refinement residuals from the FP64 products through "
                    "time FFTs (frequency blocks of K and V, transformed once: transforms_ms)"},
        "tc_apply": {"ms": tc_ms, "tflops": tc_flops / (tc_ms * 1e-3) / 1e12,
                     "frac_of_bf16_peak": tc_flops / (tc_ms * 1e-3) / 1e12 / bf16_peak,
                     "peak_tflops": bf16_peak, "peak": "measured bf16 burst (MEASURED_PEAKS.json)"},
        "tc_apply_compensated_chunk4": {"ms": tc4_ms, "tflops": tc_flops / (tc4_ms * 1e-3) / 1e12,
                                        "frac_of_bf16_peak": tc_flops / (tc4_ms * 1e-3) / 1e12 / bf16_peak},
        "exact_apply": {"ms": ex_ms, "slice_x_ms": sl_ms,
                        "fp64_equivalent_tflops": tc_flops / (ex_ms * 1e-3) / 1e12,
                        "bf16_tflops_executed": ex_exec / (ex_ms * 1e-3) / 1e12,
                        "frac_of_bf16_peak": ex_exec / (ex_ms * 1e-3) / 1e12 / bf16_peak,
                        "max_err_over_rowmax_bound_8rhs": ex_err,
                        "max_normwise_rel_err_8rhs": ex_norm,
                        "fp64_cuda_core_8rhs_ms": y64_ms,
                        "fp64_cuda_core_tflops": tc_flops * 8 / n_src / (y64_ms * 1e-3) / 1e12,
                        "note": "7 slices x 6 bits, 28 slice-pair BF16 products, exact FP32 group sums, "
                                "double-float combination; includes slicing W"},
    }
    del V, K, D32, D64, V3, Db, G, F, Wb, Vx, Kx, xwork, yx, Ff, Wf, yf
    torch.cuda.empty_cache()
    return out


def _exact_work_bytes(ctx, nt, nx, B, S):
    import ctypes
    nb = ctypes.c_size_t()
    ctx.check(ctx.lib.stbem_apply_exact_workspace_bytes(nt, nx, B, S, ctypes.byref(nb)))
    return nb.value


def run_grad(ctx, dev, stream):
    """The differentiation workload: 16-corner star (seeded radii), N_x = 256,
    N_t = 256, alpha = 1, y* = (1.5, 1.5); loss ||w_h - w_target||^2 with
    w_target from seeded perturbed corners.  Times the forward solve, the
    adjoint solve and the assembly-derivative kernels (CUDA events), and checks
    the gradient in one random direction of (corners, alpha) against an FP64
    central difference (h = 1e-6)."""
    import torch
    import workloads as W
    import paper_1811_05224_gb300 as P
    C0 = W.star_corners(16, seed=5)
    S = W.subdivision_matrix(16, 16)
    T, nt, ys, al = 1.0, 256, (1.5, 1.5), 1.0
    rng = np.random.default_rng(23)
    ev = lambda: torch.cuda.Event(enable_timing=True)       # noqa: E731

    def forward(C, a):
        mesh = P.Mesh(ctx, S @ C, T, nt, a)
        V = P.assemble(ctx, mesh, "V")
        K = P.assemble(ctx, mesh, "K")
        D = P.assemble(ctx, mesh, "D")
        L = P.lumped_mass(ctx, mesh)
        g, f = P.rhs(ctx, mesh, K, ys)
        w, info = P.solve(ctx, V, f, D, L, tol=1e-12, restart=100, max_iter=2000)
        return mesh, V, K, D, L, g, w, info

    wt = forward(C0 + 0.01 * rng.standard_normal(C0.shape), al)[6]
    e = [ev() for _ in range(6)]
    e[0].record(stream)
    mesh, V, K, D, L, g, w, info = forward(C0, al)
    e[1].record(stream)
    # workspaces and the adjoint right-hand side outside the timed intervals
    awork = P.api.solve_workspace(ctx, nt, mesh.n_x, 100)
    gwork = P.api.grad_workspace(ctx, nt, mesh.n_x)
    rhs_adj = 2.0 * (w - wt)
    torch.cuda.synchronize(dev)
    e[2].record(stream)
    lam, ainfo = P.solve_adjoint(ctx, V, rhs_adj, D, L, tol=1e-12, restart=100, max_iter=2000, work=awork)
    e[3].record(stream)
    e[4].record(stream)
    dxy, dal = P.grad(ctx, mesh, K, ys, g, w, lam, work=gwork)
    e[5].record(stream)
    torch.cuda.synchronize(dev)
    # the forward solve alone with the same options and workspace, for the
    # per-iteration comparison with the adjoint solve
    _, f_fwd = P.rhs(ctx, mesh, K, ys)
    torch.cuda.synchronize(dev)
    s0, s1 = ev(), ev()
    s0.record(stream)
    _, finfo = P.solve(ctx, V, f_fwd, D, L, tol=1e-12, restart=100, max_iter=2000, work=awork)
    s1.record(stream)
    torch.cuda.synchronize(dev)
    # the derivative kernels alone, once more
    k0, k1 = ev(), ev()
    k0.record(stream)
    P.grad(ctx, mesh, K, ys, g, w, lam, work=gwork)
    k1.record(stream)
    torch.cuda.synchronize(dev)
    # the forward and adjoint solves with the products through time FFTs
    fwork = P.api.solve_fft_workspace(ctx, nt, mesh.n_x, 100)
    q = [ev() for _ in range(5)]
    q[0].record(stream)
    Vh, Dh = P.fft_operator(ctx, V), P.fft_operator(ctx, D)
    q[1].record(stream)
    w_f, finfo_f = P.solve_fft(ctx, Vh, f_fwd, Dh, L, tol=1e-12, restart=100, max_iter=2000, work=fwork)
    q[2].record(stream)
    q[3].record(stream)
    lam_f, ainfo_f = P.solve_fft(ctx, Vh, rhs_adj, Dh, L, tol=1e-12, restart=100, max_iter=2000, transpose=True,
                                 work=fwork)
    q[4].record(stream)
    torch.cuda.synchronize(dev)
    fft_out = {"transforms_ms": q[0].elapsed_time(q[1]),
               "forward_solve_ms": q[1].elapsed_time(q[2]), "forward_iterations": finfo_f["iterations"],
               "adjoint_solve_ms": q[3].elapsed_time(q[4]), "adjoint_iterations": ainfo_f["iterations"],
               "w_rel_diff": float((w_f - w).norm() / w.norm()),
               "lambda_rel_diff": float((lam_f - lam).norm() / lam.norm())}
    del Vh, Dh, w_f, lam_f, fwork
    gC = S.T @ dxy.cpu().numpy()
    ga = float(dal)
    v, va, h = rng.standard_normal(C0.shape), float(rng.standard_normal()), 1e-6
    Lp = float(((forward(C0 + h * v, al + h * va)[6] - wt) ** 2).sum())
    Lm = float(((forward(C0 - h * v, al - h * va)[6] - wt) ** 2).sum())
    fd = (Lp - Lm) / (2 * h)
    an = float((gC * v).sum() + ga * va)
    out = {
        "workload": "star256: 16 corners (radii seed 5), N_x = 256, N_t = 256, alpha = 1, 33 parameters",
        "forward_ms": e[0].elapsed_time(e[1]), "forward_gmres_iterations": info["iterations"],
        "adjoint_solve_ms": e[2].elapsed_time(e[3]), "adjoint_iterations": ainfo["iterations"],
        "forward_solve_ms": s0.elapsed_time(s1), "forward_solve_iterations": finfo["iterations"],
        "adjoint_vs_forward_ms_per_iteration": (e[2].elapsed_time(e[3]) / max(1, ainfo["iterations"])) /
                                               (s0.elapsed_time(s1) / max(1, finfo["iterations"])),
        "grad_kernels_ms": k0.elapsed_time(k1),
        "backward_ms": e[2].elapsed_time(e[3]) + e[4].elapsed_time(e[5]),
        "fd_check": {"directional_derivative": an, "central_difference": fd,
                     "rel_diff": abs(fd - an) / abs(an), "h": h},
        "fft_products": fft_out,
    }
    del V, K, D, g, w, lam, gwork, awork
    torch.cuda.empty_cache()
    return out


def m0_evaluations(n_x, nodes, tris, n_t, alpha, T=1.0):
    """Algorithmic count of kernel evaluations G(r, t_k) of the M_h^0 rule on a
    triangulation: per (segment, triangle) pair and order range [b, e) of the
    rule, order^3 points times the distinct times t_b .. t_e (t_0 = 0 costs
    nothing), plus 2*8*3*12*12 polar points per touching pair at m = 0.  The
    pair classes and orders follow the rule (touching by shared vertex,
    rho^2 = 4 m ht / (alpha s^2) steps); the near class only changes the
    order at m = 0 and is counted as regular there (a lower bound)."""
    ht = T / n_t
    X = np.asarray(nodes, dtype=np.float64)
    tr = np.asarray(tris)
    e = [np.sqrt(((X[tr[:, a]] - X[tr[:, (a + 1) % 3]]) ** 2).sum(1)) for a in range(3)]
    diam = np.maximum.reduce(e)
    # unit square boundary: segment length 1 / (n_x / 4); s = max(h, diam)
    h = 4.0 / n_x
    s = np.maximum(h, diam)
    steps = ((1e4, 3), (144.0, 4), (5.0, 6), (1.44, 8), (0.0, 12))
    tot = 0.0
    for sk in np.unique(s):
        cnt = n_x * float((s == sk).sum())
        orders = []
        for m in range(1, n_t):
            r2 = (4.0 * m * ht) / (alpha * sk * sk)
            orders.append(next(o for thr, o in steps if r2 >= thr))
        # runs of equal order: points x (steps + 1)
        m = 0
        while m < len(orders):
            o, k = orders[m], m
            while k < len(orders) and orders[k] == o:
                k += 1
            tot += cnt * o ** 3 * (k - m + 1)
            m = k
        tot += cnt * 8 ** 3            # m = 0, regular order
    return tot


def run_initial(ctx, dev, stream, L=6):
    """The paper's Section 4 example at level L (Q = (0,1)^3, alpha = 10,
    u = exp(-t/alpha) sin(x1 cos(pi/8) + x2 sin(pi/8)), 2^L segments per side,
    N_t = 2^L, structured triangulation of Omega): times the matrix-free
    M_h^0 u_0 product and the assembled M_h^0, the whole right-hand side and
    both GMRES solves; reports the iteration counts next to Table 1's and the
    error of w_h against the exact Neumann datum."""
    import torch
    import workloads as W
    import paper_1811_05224_gb300 as P
    n = 2 ** L
    al = 10.0
    X = W.unit_square(n)
    nodes, tris = W.square_triangulation(n)
    ev = lambda: torch.cuda.Event(enable_timing=True)       # noqa: E731
    e = [ev() for _ in range(6)]
    e[0].record(stream)
    mesh = P.Mesh(ctx, X, 1.0, n, al)
    dom = P.Domain(ctx, mesh, nodes, tris)
    V = P.assemble(ctx, mesh, "V")
    K = P.assemble(ctx, mesh, "K")
    D = P.assemble(ctx, mesh, "D")
    Lm = P.lumped_mass(ctx, mesh)
    e[1].record(stream)
    g, u0 = P.planewave_data(ctx, dom)
    work = P.api.m0_workspace(ctx, dom)
    f = P.rhs_initial(ctx, dom, K, g, u0, work=work)
    e[2].record(stream)
    w, info = P.solve(ctx, V, f, D, Lm, tol=1e-8)
    e[3].record(stream)
    w0, info0 = P.solve(ctx, V, f, tol=1e-8, max_iter=1000)
    e[4].record(stream)
    torch.cuda.synchronize(dev)
    # the M_h^0 product alone (matrix-free), and the stored operator
    y = torch.zeros((n, 4 * n), dtype=torch.float64, device=dev)
    k0, k1 = ev(), ev()
    k0.record(stream)
    P.m0_apply(ctx, dom, u0, out=y, work=work)
    k1.record(stream)
    torch.cuda.synchronize(dev)
    asm_ms = None
    if n * 4 * n * dom.n_nodes * 8 <= 4e9:
        M0 = torch.empty((n, 4 * n, dom.n_nodes), dtype=torch.float64, device=dev)
        a0, a1 = ev(), ev()
        a0.record(stream)
        P.m0_assemble(ctx, dom, M0)
        a1.record(stream)
        torch.cuda.synchronize(dev)
        asm_ms = a0.elapsed_time(a1)
        del M0
    # exact Neumann datum w = d_n u averaged over the elements (closed form)
    th = np.pi / 8
    dd = np.array([np.cos(th), np.sin(th)])
    Xb = np.roll(X, -1, axis=0)
    hseg = np.sqrt(((Xb - X) ** 2).sum(1))
    tt = (Xb - X) / hseg[:, None]
    nn = np.stack([tt[:, 1], -tt[:, 0]], axis=1)
    t = np.arange(n + 1) / n
    tavg = al * n * (np.exp(-t[:-1] / al) - np.exp(-t[1:] / al))
    savg = np.cos(0.5 * (X + Xb) @ dd) * np.sinc(0.5 * hseg * (tt @ dd) / np.pi)
    wex = tavg[:, None] * (savg * (nn @ dd))[None, :]
    wn = w.cpu().numpy()
    wts = hseg[None, :] / n
    err = float(np.sqrt((wts * (wn - wex) ** 2).sum() / (wts * wex ** 2).sum()))
    # u in Q at a 32 x 32 grid of interior points at t = T (representation formula)
    gx = (np.arange(32) + 0.5) / 32
    P2 = np.stack(np.meshgrid(gx, gx), -1).reshape(-1, 2)
    T2 = np.ones(P2.shape[0])
    pts_d = torch.as_tensor(P2).to(dev)
    ts_d = torch.as_tensor(T2).to(dev)
    P.evaluate(ctx, mesh, pts_d, ts_d, w, g, dom, u0)
    v0, v1 = ev(), ev()
    v0.record(stream)
    uq = P.evaluate(ctx, mesh, pts_d, ts_d, w, g, dom, u0)
    v1.record(stream)
    torch.cuda.synchronize(dev)
    uex = np.exp(-T2 / al) * np.sin(P2 @ dd)
    u_err = float(np.abs(uq.cpu().numpy() - uex).max() / np.abs(uex).max())
    table1 = {2: (14, 17), 3: (19, 18), 4: (24, 20), 5: (35, 20), 6: (50, 20), 7: (67, 20), 8: (91, 19),
              9: (122, 19)}
    m0_ms = k0.elapsed_time(k1)
    evals = m0_evaluations(4 * n, nodes, tris, n, al)
    out = {
        "workload": "Section 4 example, level %d: unit square, N_x = %d, N_t = %d, N = %d, alpha = 10, "
                    "%d nodes / %d triangles" % (L, 4 * n, n, 4 * n * n, dom.n_nodes, dom.n_tris),
        "m0_apply_ms": m0_ms, "m0_assemble_ms": asm_ms,
        "m0_kernel_evaluations": evals, "m0_evaluations_per_s": evals / (m0_ms * 1e-3),
        "setup_assembly_ms": e[0].elapsed_time(e[1]), "rhs_ms": e[1].elapsed_time(e[2]),
        "gmres_prec_ms": e[2].elapsed_time(e[3]), "gmres_prec_iterations": info["iterations"],
        "gmres_plain_ms": e[3].elapsed_time(e[4]), "gmres_plain_iterations": info0["iterations"],
        "table1_iterations": {"plain": table1[L][0], "preconditioned": table1[L][1]},
        "w_l2_rel_error_vs_exact": err,
        "evaluate_u": {"points": int(P2.shape[0]), "t": 1.0, "ms": v0.elapsed_time(v1),
                       "max_rel_error_vs_exact": u_err},
    }
    del V, K, D, w, w0, f, g, u0, y, work
    torch.cuda.empty_cache()
    return out


def run_ragged(ctx, dev, stream):
    """Ragged batch: 64 unit squares with N_x = 4k (k seeded in [16, 128]) and
    N_t seeded in [64, 512] (seed 41), alpha = 1, T = 1, sources seeded on the
    annulus 1.2..3 (seed 4).  FP32 operators (FP64 singular pairs), one
    persistent launch per operator for all 64 problems; the product's lag
    chunk autotuned; lockstep GMRES (FP64 vectors, graph-captured Arnoldi
    steps) inside FP64 refinement (FP64 V residuals) to 1e-8 on all problems,
    beside the same 64 solves one at a time."""
    import torch
    import workloads as W
    import paper_1811_05224_gb300 as P
    pr = W.ragged_squares()
    probs = [(W.unit_square(nx // 4), 1.0, nt, 1.0) for nx, nt in pr]
    R = P.Ragged(ctx, probs)
    ev = lambda: torch.cuda.Event(enable_timing=True)       # noqa: E731
    e = [ev() for _ in range(4)]
    e[0].record(stream)
    V = R.assemble("V", "f32")
    e[1].record(stream)
    K = R.assemble("K", "f32")
    e[2].record(stream)
    D = R.assemble("D", "f32")
    e[3].record(stream)
    torch.cuda.synchronize(dev)
    asm_ms = {k: e[i].elapsed_time(e[i + 1]) for i, k in enumerate("VKD")}
    L = R.lumped_mass()
    ys = W.annulus_sources(len(probs), seed=4)
    g, f = R.rhs(K, ys)
    y = torch.empty_like(f)
    best, report = R.tune(V, f, y)
    a0, a1 = ev(), ev()
    a0.record(stream)
    R.apply(V, f, out=y)
    a1.record(stream)
    torch.cuda.synchronize(dev)
    apply_ms = a0.elapsed_time(a1)
    flops = sum(2.0 * nx * nx * nt * (nt + 1) / 2 for nx, nt in pr)
    # FP64 V for the refinement residuals (FP64 accuracy of every solution)
    v0, v1 = ev(), ev()
    v0.record(stream)
    V64 = R.assemble("V", "f64")
    v1.record(stream)
    torch.cuda.synchronize(dev)
    work = R.solve_mixed_workspace(40)
    R.solve_mixed(V64, V, f, D, L, tol=1e-8, inner_tol=1e-4, restart=40, max_iter=600, work=work)   # graphs
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    w, infos = R.solve_mixed(V64, V, f, D, L, tol=1e-8, inner_tol=1e-4, restart=40, max_iter=600, work=work)
    torch.cuda.synchronize(dev)
    solve_ms = 1e3 * (time.perf_counter() - t0)
    # the same systems one at a time (single-problem mixed solve, same operators)
    nt_max, nx_max = max(nt for _, nt in pr), max(nx for nx, _ in pr)
    nb = ctypes.c_size_t()
    ctx.check(ctx.lib.stbem_solve_mixed_workspace_bytes(nt_max, nx_max, 40, ctypes.byref(nb)))
    sw = torch.empty(nb.value, dtype=torch.uint8, device=dev)
    t0 = time.perf_counter()
    worst, worst_res = 0.0, 0.0
    for p in range(len(probs)):
        fp = R.view_vec(f, p)
        wp, _ = P.solve_mixed(ctx, R.view_op(V64, p), R.view_op(V, p), fp, R.view_op(D, p), R.view_mass(L, p),
                              tol=1e-8, inner_tol=1e-4, restart=40, max_iter=600, work=sw)
        worst = max(worst, float((wp - R.view_vec(w, p)).norm() / wp.norm()))
    torch.cuda.synchronize(dev)
    seq_ms = 1e3 * (time.perf_counter() - t0)
    for p in range(len(probs)):
        fp = R.view_vec(f, p)
        rp = fp - P.apply(ctx, R.view_op(V64, p), R.view_vec(w, p))
        worst_res = max(worst_res, float(rp.norm() / fp.norm()))
    entries = 3 * R.op_elems
    out = {
        "workload": "64 unit squares, N_x = 4k (k in [16,128]), N_t in [64,512] (seed 41), alpha = 1",
        "precision": "FP32 operators (FP64 singular pairs), FP64 vectors",
        "entries": entries,
        "assembly_ms": asm_ms,
        "assembly_entries_per_s": entries / (sum(asm_ms.values()) * 1e-3),
        "apply_ms": apply_ms, "apply_gflops": flops / (apply_ms * 1e-3) / 1e9,
        "tuned": best, "tuner_ms": report,
        "assembly_V_f64_ms": v0.elapsed_time(v1),
        "solve_ms": solve_ms, "lockstep_inner_iterations": max(i["iterations"] for i in infos),
        "solve_note": "FP32 lockstep GMRES inside FP64 refinement (FP64 V residuals), tol 1e-8",
        "max_fp64_rel_residual": worst_res,
        "sequential_solves_ms": seq_ms,
        "sequential_note": "the 64 single-problem mixed solves (stbem_solve_mixed), same operators and tolerance",
        "max_w_rel_diff_vs_sequential": worst,
    }
    del V, K, D, V64, f, g, y, w, work, sw
    R.close()
    torch.cuda.empty_cache()
    return out


def run_nonuniform(ctx, dev, stream, n=128, q=1.5):
    """Non-uniform time grid (Section 1 allows any decomposition of (0, T)):
    unit square with N_x = n, graded nodes t_j = (j / n)^q on T = 1, alpha = 1,
    g = U*(x - y*, t), y* = (1.5, 1.5).  All n (n + 1) / 2 blocks of V, K, D
    assembled and stored packed (no Toeplitz structure), the block product
    (every block read once) timed against max(bytes / HBM, flops / FP64) and
    the preconditioned GMRES (lumped mass per step) to 1e-8."""
    import torch
    import workloads as W
    import paper_1811_05224_gb300 as P
    t = (np.arange(n + 1) / n) ** q
    mesh = P.GradedMesh(ctx, W.unit_square(n // 4), t, 1.0)
    ev = lambda: torch.cuda.Event(enable_timing=True)       # noqa: E731
    blocks = n * (n + 1) // 2
    ops, asm_ms = {}, {}
    for op in "VKD":
        a0, a1 = ev(), ev()
        a0.record(stream)
        ops[op] = P.nu_assemble(ctx, mesh, op)
        a1.record(stream)
        torch.cuda.synchronize(dev)
        asm_ms[op] = a0.elapsed_time(a1)
    g, f = P.nu_rhs(ctx, mesh, ops["K"], (1.5, 1.5))
    L = P.nu_lumped_mass(ctx, mesh)
    x = torch.randn(n, n, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    for _ in range(3):
        P.nu_apply(ctx, ops["V"], n, x, out=y)
    reps = 10
    p0, p1 = ev(), ev()
    p0.record(stream)
    for _ in range(reps):
        P.nu_apply(ctx, ops["V"], n, x, out=y)
    p1.record(stream)
    torch.cuda.synchronize(dev)
    apply_ms = p0.elapsed_time(p1) / reps
    nbytes = blocks * n * n * 8 + 2 * n * n * 8
    flops = 2.0 * blocks * n * n
    s0, s1 = ev(), ev()
    s0.record(stream)
    w, info = P.nu_solve(ctx, ops["V"], f, ops["D"], L, tol=1e-8)
    s1.record(stream)
    torch.cuda.synchronize(dev)
    w0, info0 = P.nu_solve(ctx, ops["V"], f, tol=1e-8, max_iter=1000)
    # the same problem on a uniform grid of n steps: iteration counts
    mu = P.Mesh(ctx, W.unit_square(n // 4), 1.0, n, 1.0)
    Vu, Ku, Du = (P.assemble(ctx, mu, o) for o in "VKD")
    _, fu = P.rhs(ctx, mu, Ku, (1.5, 1.5))
    _, infou = P.solve(ctx, Vu, fu, Du, P.lumped_mass(ctx, mu), tol=1e-8)
    hbm = float(_peaks().get("hbm_gbs", 6784.2))
    fp64 = P.pipe_peaks(ctx)["fp64_tflops"]
    out = {
        "workload": "unit square N_x = %d, graded t_j = (j / %d)^%g (step ratio up to %.2f), alpha = 1, "
                    "%d packed blocks per operator (%.2f GB)" % (n, n, q, float(np.max(np.diff(t)[1:] /
                                                                                      np.diff(t)[:-1])),
                                                                  blocks, blocks * n * n * 8 / 1e9),
        "assembly_ms": asm_ms,
        "assembly_entries_per_s": 3 * blocks * n * n / (sum(asm_ms.values()) * 1e-3),
        "block_apply_ms": apply_ms, "block_apply_gbs": nbytes / (apply_ms * 1e-3) / 1e9,
        "block_apply_gflops": flops / (apply_ms * 1e-3) / 1e9,
        "block_apply_roofline_ms": 1e3 * max(nbytes / (hbm * 1e9), flops / (fp64 * 1e12)),
        "block_apply_roofline_frac": 1e3 * max(nbytes / (hbm * 1e9), flops / (fp64 * 1e12)) / apply_ms,
        "block_apply_note": "roofline max(bytes / HBM, flops / FP64): 2 flops per 8 bytes need 1.7 TFLOP/s at "
                            "the HBM rate, above GB300's FP64 rate, so the product is FP64-bound",
        "gmres_prec_ms": s0.elapsed_time(s1), "gmres_prec_iterations": info["iterations"],
        "gmres_prec_rel_residual": info["rel_residual"],
        "gmres_plain_iterations": info0["iterations"],
        "uniform_grid_prec_iterations": infou["iterations"],
    }
    del ops, g, f, L, x, y, w, w0, Vu, Ku, Du, fu
    torch.cuda.empty_cache()
    return out


def max_over_ranks(ms, device):
    """The slowest rank's time: all ranks run their own problem and the job
    ends with the last one (a no-op without an initialised process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def strong_value(units_total, ms_max):
    """Whole-job throughput under strong scaling: all ranks together process
    units_total (one sharded problem) in the slowest rank's time."""
    return units_total / (ms_max * 1e-3)


def weak_value(units_per_rank, world, ms_max):
    """Whole-job throughput under weak scaling: every rank processes
    units_per_rank in the slowest rank's time."""
    return world * units_per_rank / (ms_max * 1e-3)


def run_ours(args):
    import torch
    import torch.distributed as dist

    import workloads as W
    import paper_1811_05224_gb300 as P
    from paper_1811_05224_gb300 import capi

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ctx = P.Context(local, stream)
    lib = capi.load()
    p = W.config(WORKLOAD)
    mesh = P.Mesh(ctx, p.vertices, p.T, p.n_t, p.alpha)
    nt, nx = p.n_t, p.n_x
    V = ctx.empty((nt, nx, nx))
    K = ctx.empty((nt, nx, nx))
    D = ctx.empty((nt, nx, nx))
    awork = P.api.apply_workspace(ctx, nt, nx, 1)
    swork = P.api.solve_workspace(ctx, nt, nx, 200)
    w = ctx.empty((nt, nx))
    # frequency blocks of V and D for the products through time FFTs
    nf, nfb = ctypes.c_int(), ctypes.c_size_t()
    ctx.check(lib.stbem_fft_operator_bytes(nt, nx, ctypes.byref(nf), ctypes.byref(nfb)))
    Vh, Kh, Dh = (P.FFTOperator(torch.empty((nf.value, nx, nx), dtype=torch.complex128, device=dev), nt, nx)
                  for _ in range(3))
    fswork = P.api.solve_fft_workspace(ctx, nt, nx, 200)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)       # noqa: E731
    infos = []

    # N > 1: one problem sharded by lag (chunks of 16 lags dealt in snake
    # order); each rank assembles its lag blocks, and the K, V and D products
    # are its partial sums followed by an NCCL all-reduce (strong scaling)
    sharded = world > 1
    if sharded:
        ranges = P.shard.lag_ranges(nt, world, rank, 16)
        Vs, Ks, Ds = (P.shard.ShardedOperator(ctx, mesh, o, ranges) for o in "VKD")

    def step(m, events=None, solve_mode=args.solve, infos_out=infos):
        e = [ev() for _ in range(5)] if events is None else events
        e[0].record(stream)
        if sharded:
            for S in (Vs, Ks, Ds):
                S.assemble(m)
            e[1].record(stream)
            g, f = P.shard.rhs_sharded(ctx, m, Ks, p.y_star)
            L = P.lumped_mass(ctx, m)
            e[2].record(stream)
            _, info = P.shard.solve_sharded(ctx, Vs, f, Ds, L, tol=1e-8, max_iter=500, restart=200, out=w)
        else:
            P.assemble_ops(ctx, m, "f64", out={"V": V, "K": K, "D": D})
            e[1].record(stream)
            if solve_mode == "fft":
                # K g through the frequency blocks of K as well
                P.fft_operator(ctx, K, out=Kh.data)
                g, f = P.rhs_batched(ctx, m, Kh, [p.y_star])
                g, f = g[0], f[0]
            else:
                g, f = P.rhs(ctx, m, K, p.y_star, work=awork)
            L = P.lumped_mass(ctx, m)
            e[2].record(stream)
            if solve_mode == "fft":
                P.fft_operator(ctx, V, out=Vh.data)
                P.fft_operator(ctx, D, out=Dh.data)
                _, info = P.solve_fft(ctx, Vh, f, Dh, L, tol=1e-8, max_iter=500, restart=200, work=fswork, out=w)
            else:
                _, info = P.solve(ctx, V, f, D, L, tol=1e-8, max_iter=500, restart=200, work=swork, out=w)
        e[3].record(stream)
        infos_out.append(info)
        return e

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()

    for _ in range(max(args.warmup, 0)):
        step(mesh)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    n0 = lib.stbem_launch_count()
    step_events = []
    barrier()
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        step_events.append(step(mesh))
    barrier()
    t_wall = time.perf_counter() - t_wall
    launches = lib.stbem_launch_count() - n0
    ck = clocks.stop()
    ms = [e[0].elapsed_time(e[3]) for e in step_events]
    ms_asm = [e[0].elapsed_time(e[1]) for e in step_events]
    ms_solve = [e[2].elapsed_time(e[3]) for e in step_events]
    ms_step = max_over_ranks(sum(ms) / len(ms), dev)
    entries = 3 * nt * nx * nx
    # sharded: all ranks together assemble and solve one problem (strong);
    # replicas: every rank its own (weak)
    value = strong_value(entries, ms_step) if sharded else weak_value(entries, world, ms_step)
    asm_rate = entries / (statistics.mean(ms_asm) * 1e-3)
    # the same step with the other product (direct block sums or time FFTs),
    # timed the same way, and the distance between the two solutions
    step_alt = None
    if not sharded:
        alt_mode = "direct" if args.solve == "fft" else "fft"
        w_main = w.clone()
        alt_infos = []
        for _ in range(max(args.warmup, 1)):
            step(mesh, solve_mode=alt_mode, infos_out=alt_infos)
        torch.cuda.synchronize(dev)
        alt_events = []
        for _ in range(args.steps):
            flush.zero_()
            alt_events.append(step(mesh, solve_mode=alt_mode, infos_out=alt_infos))
        torch.cuda.synchronize(dev)
        step_alt = {"solve": alt_mode,
                    "ms_per_step": statistics.mean(e[0].elapsed_time(e[3]) for e in alt_events),
                    "gmres_ms": statistics.mean(e[2].elapsed_time(e[3]) for e in alt_events),
                    "gmres_iterations": alt_infos[-1]["iterations"],
                    "gmres_rel_residual": alt_infos[-1]["rel_residual"],
                    "w_rel_diff": float((w - w_main).norm() / w_main.norm())}
        w.copy_(w_main)
    if sharded:
        # the per-kernel components below use full operators on every rank
        for op, buf in (("V", V), ("K", K), ("D", D)):
            P.assemble(ctx, mesh, op, out=buf)
        torch.cuda.synchronize(dev)

    # Toeplitz apply (V, FP64): kernel time with CUDA events on the launch stream
    x = torch.randn(nt, nx, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    for _ in range(3):
        P.apply(ctx, V, x, work=awork, out=y)
    reps = 10
    a0, a1 = ev(), ev()
    flush.zero_()
    a0.record(stream)
    for _ in range(reps):
        P.apply(ctx, V, x, work=awork, out=y)
    a1.record(stream)
    torch.cuda.synchronize(dev)
    ms_apply = a0.elapsed_time(a1) / reps
    apply_flops = 2.0 * nx * nx * nt * (nt + 1) / 2
    apply_bytes = nt * nx * nx * 8 + 2 * nt * nx * 8
    # the same product through the frequency blocks (three launches: the
    # transform of x, one complex matrix-vector product per frequency, the
    # inverse transform); algorithmic bytes: the frequency blocks once, x and
    # y, and the two transforms written and read once each
    P.fft_operator(ctx, V, out=Vh.data)
    fawork = P.api.apply_fft_workspace(ctx, nt, nx, 1)
    yf = torch.empty_like(x)
    for _ in range(3):
        P.apply_fft(ctx, Vh, x, work=fawork, out=yf)
    f0, f1 = ev(), ev()
    flush.zero_()
    f0.record(stream)
    for _ in range(reps):
        P.apply_fft(ctx, Vh, x, work=fawork, out=yf)
    f1.record(stream)
    o0, o1 = ev(), ev()
    flush.zero_()
    o0.record(stream)
    for _ in range(reps):
        P.fft_operator(ctx, V, out=Vh.data)
    o1.record(stream)
    torch.cuda.synchronize(dev)
    ms_apply_fft = f0.elapsed_time(f1) / reps
    ms_fft_op = o0.elapsed_time(o1) / reps
    fft_apply_bytes = nf.value * nx * nx * 16 + 2 * nt * nx * 8 + 4 * nf.value * nx * 16
    fft_op_bytes = nt * nx * nx * 8 + nf.value * nx * nx * 16
    # flops: 8 per complex multiply-add of the frequency products, and
    # 5 L log2 L per complex transform of length L (two real columns each)
    Lf = 2 * (nf.value - 1)
    fft_len_flops = 5.0 * Lf * np.log2(Lf)
    fft_apply_flops = 8.0 * nf.value * nx * nx + 2 * (nx / 2) * fft_len_flops
    fft_op_flops = (nx * nx / 2) * fft_len_flops
    apply_fft_rel = float((yf - y).norm() / y.norm())
    # dominant kernel: the FP64 D tile kernel at lags >= 2 (four lags per CTA,
    # chunks within one space order each, one launch), timed alone with CUDA
    # events on the launching stream; launches counted
    l2 = []
    for _ in range(2):
        c0, c1 = ev(), ev()
        flush.zero_()
        n_before = lib.stbem_launch_count()
        c0.record(stream)
        P.assemble_lags(ctx, mesh, "D", 2, nt, out=D)
        c1.record(stream)
        torch.cuda.synchronize(dev)
        n_lag2_launches = max(1, lib.stbem_launch_count() - n_before)
        l2.append(c0.elapsed_time(c1))
    d2_ms_launch = min(l2) / n_lag2_launches
    d2_flops_launch = d_lag2_flops(nx, nt) / n_lag2_launches
    # per-operator assembly time (separate events, same kernels)
    op_ms = {}
    for op, buf in (("V", V), ("K", K), ("D", D)):
        b0, b1 = ev(), ev()
        b0.record(stream)
        P.assemble(ctx, mesh, op, out=buf)
        b1.record(stream)
        torch.cuda.synchronize(dev)
        op_ms[op] = b0.elapsed_time(b1)

    # mixed precision pipeline on the same workload: FP64 V and K, FP32 D from
    # the mixed assembly, FP32 V rounded from FP64, FP64 refinement around FP32
    # inner GMRES; compared with the plain FP64 solution w
    w_plain = w.clone()
    D32 = torch.empty((nt, nx, nx), dtype=torch.float32, device=dev)
    mwork = None
    mixed_ms, mixed_solve_ms, mixed_info, w_mixed = [], [], None, None
    for k in range(max(args.warmup, 1) + max(1, min(args.steps, 3))):
        flush.zero_()
        e0, e1, e2 = ev(), ev(), ev()
        e0.record(stream)
        P.assemble_ops(ctx, mesh, {"V": "f64", "K": "f64", "D": "f32"}, out={"V": V, "K": K, "D": D32})
        V32 = P.round_f32(ctx, V)
        g, f = P.rhs(ctx, mesh, K, p.y_star, work=awork)
        L = P.lumped_mass(ctx, mesh)
        e1.record(stream)
        w_mixed, mixed_info = P.solve_mixed(ctx, V, V32, f, D32, L, tol=1e-8, inner_tol=1e-4, work=mwork)
        e2.record(stream)
        torch.cuda.synchronize(dev)
        if k >= max(args.warmup, 1):
            mixed_ms.append(e0.elapsed_time(e2))
            mixed_solve_ms.append(e1.elapsed_time(e2))
    mixed_rel = float((w_mixed - w_plain).norm() / w_plain.norm())
    # the same step with FP64 GMRES on the products through time FFTs: the
    # FP32 D enters only the preconditioner (its frequency blocks)
    mf_ms, mf_solve_ms, mf_info, w_mf = [], [], None, None
    for k in range(max(args.warmup, 1) + max(1, min(args.steps, 3))):
        flush.zero_()
        e0, e1, e2 = ev(), ev(), ev()
        e0.record(stream)
        P.assemble_ops(ctx, mesh, {"V": "f64", "K": "f64", "D": "f32"}, out={"V": V, "K": K, "D": D32})
        g, f = P.rhs(ctx, mesh, K, p.y_star, work=awork)
        L = P.lumped_mass(ctx, mesh)
        e1.record(stream)
        P.fft_operator(ctx, V, out=Vh.data)
        P.fft_operator(ctx, D32, out=Dh.data)
        w_mf, mf_info = P.solve_fft(ctx, Vh, f, Dh, L, tol=1e-8, max_iter=500, restart=200, work=fswork)
        e2.record(stream)
        torch.cuda.synchronize(dev)
        if k >= max(args.warmup, 1):
            mf_ms.append(e0.elapsed_time(e2))
            mf_solve_ms.append(e1.elapsed_time(e2))
    mf_rel = float((w_mf - w_plain).norm() / w_plain.norm())
    d32_ms = None
    b0, b1 = ev(), ev()
    b0.record(stream)
    P.assemble(ctx, mesh, "D", "f32", out=D32)
    b1.record(stream)
    torch.cuda.synchronize(dev)
    d32_ms = b0.elapsed_time(b1)

    batched = None
    if not args.no_batched and world == 1:
        batched = run_batched(ctx, dev, stream, fp64_residual=args.batched_fp64_residual)
    grad = None
    if not args.no_grad and world == 1:
        grad = run_grad(ctx, dev, stream)
    initial = None
    if not args.no_initial and world == 1:
        initial = run_initial(ctx, dev, stream)
    ragged = None
    if not args.no_ragged and world == 1:
        ragged = run_ragged(ctx, dev, stream)
    precision = None
    if not args.no_precision and world == 1:
        precision = run_precision(ctx, dev, stream)
    nonuniform = None
    if not args.no_nonuniform and world == 1:
        nonuniform = run_nonuniform(ctx, dev, stream)
    # measured pipe peaks of this GPU (FP64 FMA is the assembly's and the
    # single-right-hand-side product's roofline)
    peaks = P.pipe_peaks(ctx)
    fp64_peak = peaks["fp64_tflops"]
    hbm_gbs = float(_peaks().get("hbm_gbs", 6784.2))
    # GMRES roofline: per iteration k (from 0) one V and one D apply at their
    # roofline times plus the two Gram-Schmidt passes over k + 1 basis vectors
    # (read twice, updated once: 4 (k + 1) N doubles through HBM), and one
    # more V apply for the final true residual
    it_last = infos[-1]["iterations"]
    t_apply = max(apply_bytes / (hbm_gbs * 1e9), apply_flops / (fp64_peak * 1e12))
    t_gs = sum(4.0 * (k + 1) * nt * nx * 8 / (hbm_gbs * 1e9) for k in range(it_last))
    if args.solve == "fft" and not sharded:
        # products through the frequency blocks, plus the two operator
        # transforms inside the timed solve interval, each at
        # max(bytes / HBM, flops / measured FP64)
        t_apply = max(fft_apply_bytes / (hbm_gbs * 1e9), fft_apply_flops / (fp64_peak * 1e12))
        t_gs += 2 * max(fft_op_bytes / (hbm_gbs * 1e9), fft_op_flops / (fp64_peak * 1e12))
    gmres_roof_ms = 1e3 * ((2 * it_last + 1) * t_apply + t_gs)

    # end to end through the public API with host buffers: vertices in, w out
    verts = np.ascontiguousarray(p.vertices)
    w_host = torch.empty((nt, nx), dtype=torch.float64).pin_memory()
    e2e_ms = []
    for k in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        m2 = P.Mesh(ctx, verts, p.T, p.n_t, p.alpha)
        step(m2)
        w_host.copy_(w, non_blocking=True)
        torch.cuda.synchronize(dev)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        m2.close()
    e2e_ms_max = max_over_ranks(statistics.mean(e2e_ms), dev)
    e2e_val = strong_value(entries, e2e_ms_max) if sharded else weak_value(entries, world, e2e_ms_max)

    if rank != 0:
        if world > 1:
            dist.barrier()
        return 0
    # oracle CPU baseline on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        pool = OraclePool()
        c, t = pool.step(ORACLE_PER_WORKER, 12345)
        pool.close()
        cpu = {"value": c / t, "unit": UNIT, "cores": pool.cores, "blas_threads": pool.blas_threads,
               "kind": "oracle",
               "sample": "%d random (op, lag, i, j) entries of %s (%d per worker), uniform over the 3 operators, "
                         "lags and index pairs; %d single-threaded numpy worker processes (spawn)"
                         % (c, WORKLOAD, ORACLE_PER_WORKER, pool.cores)}
    asm_tflops = d2_flops_launch / (d2_ms_launch * 1e-3) / 1e12
    last = infos[-1]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(_config(p, "256 MB buffer written between steps", args.solve),
                       parallelism=("lag-sharded over %d GPUs (chunks of 16 lags, snake order), NCCL all-reduce "
                                    "per product" % world) if sharded else
                       ("%d independent replicas" % world if world > 1 else "1 GPU")),
        "components": {
            "assembly_entries_per_s": asm_rate,
            "assembly_ms": {k: round(v, 3) for k, v in op_ms.items()},
            "assembly_step_ms": statistics.mean(ms_asm),
            "assembly_note": "assembly_ms: each operator alone; assembly_step_ms: V, K and D of the step, "
                             "assembled concurrently (stbem_assemble_ops)",
            "dense_equivalent_entries_per_s": asm_rate * (nt + 1) / 2,
            "apply_f64_ms": ms_apply, "apply_f64_gbs": apply_bytes / (ms_apply * 1e-3) / 1e9,
            "apply_f64_gflops": apply_flops / (ms_apply * 1e-3) / 1e9,
            "gmres_ms": statistics.mean(ms_solve), "gmres_iterations": last["iterations"],
            "gmres_rel_residual": last["rel_residual"],
            "gmres_roofline_ms": gmres_roof_ms,
            "gmres_roofline_frac": gmres_roof_ms / statistics.mean(ms_solve),
            "gmres_roofline_note": "iterations x (V apply + D apply at their roofline: direct products at "
                                   "max(bytes / HBM, flops / measured FP64), products through the frequency "
                                   "blocks at bytes / HBM plus the two operator transforms) + Gram-Schmidt "
                                   "traffic + final residual apply, over the GMRES time (right-hand side "
                                   "excluded)",
            "solve": args.solve,
            "step_other_product": step_alt,
            "apply_fft": {
                "ms": ms_apply_fft, "gbs": fft_apply_bytes / (ms_apply_fft * 1e-3) / 1e9,
                "tflops": fft_apply_flops / (ms_apply_fft * 1e-3) / 1e12,
                "bound": "alu", "frac_of_fp64": fft_apply_flops / (ms_apply_fft * 1e-3) / 1e12 / fp64_peak,
                "frac_of_hbm": fft_apply_bytes / (ms_apply_fft * 1e-3) / 1e9 / hbm_gbs,
                "bytes": fft_apply_bytes, "flops": fft_apply_flops, "rel_diff_vs_direct": apply_fft_rel,
                "note": "three launches (transform of x, frequency products, inverse transform); 8 flops "
                        "per complex multiply-add and 16 bytes per frequency-block entry: 0.5 flop/byte, "
                        "above the FP64/HBM balance, so FP64-bound"},
            "fft_operator": {
                "ms": ms_fft_op, "gbs": fft_op_bytes / (ms_fft_op * 1e-3) / 1e9,
                "tflops": fft_op_flops / (ms_fft_op * 1e-3) / 1e12,
                "bound": "alu", "frac_of_fp64": fft_op_flops / (ms_fft_op * 1e-3) / 1e12 / fp64_peak,
                "bytes": fft_op_bytes, "flops": fft_op_flops},
            "peaks": dict(peaks, hbm_gbs=hbm_gbs, note="fp64/fp32/ex2 measured in this run by stbem_pipe_peaks; "
                                                       "hbm from MEASURED_PEAKS.json"),
            "precision": precision,
            "nonuniform": nonuniform,
            "mixed": {"step_ms": statistics.mean(mixed_ms), "solve_ms": statistics.mean(mixed_solve_ms),
                      "inner_iterations": mixed_info["iterations"],
                      "rel_residual_fp64": mixed_info["rel_residual"],
                      "w_rel_diff_vs_fp64": mixed_rel, "assembly_D_f32_ms": d32_ms,
                      "note": "FP64 V,K; FP32 D (FP64 singular pairs); FP64 refinement around FP32 GMRES"},
            "mixed_fft": {"step_ms": statistics.mean(mf_ms), "solve_ms": statistics.mean(mf_solve_ms),
                          "iterations": mf_info["iterations"], "rel_residual": mf_info["rel_residual"],
                          "w_rel_diff_vs_fp64": mf_rel,
                          "note": "FP64 V,K; FP32 D (FP64 singular pairs) as the preconditioner only; FP64 "
                                  "GMRES with every product through the frequency blocks (time FFTs) of V "
                                  "and of the FP32 D, transformed inside the step"},
            "batched": batched,
            "grad": grad,
            "ragged": ragged,
            "initial": initial,
        },
        "roofline": {"kernel": "k_tile_ml<D, f64, 4 lags> lags >= 2", "bound": "alu",
                     "achieved": asm_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": asm_tflops / fp64_peak, "traffic": TRAFFIC_D2_BYTES,
                     "launch_ms": d2_ms_launch, "flops_per_launch": d2_flops_launch,
                     "nominal_peak": FP64_NOMINAL_TFLOPS, "frac_of_nominal": asm_tflops / FP64_NOMINAL_TFLOPS,
                     "note": "peak: FP64 FMA rate measured in this run (stbem_pipe_peaks), nominal 1.25 "
                             "TFLOP/s beside it; FP64-ALU bound (DRAM traffic is only "
                             "the written lag blocks); algorithmic flops: unique half-segment pairs, each "
                             "group of 4 lags evaluating its 5 Peano intervals once"},
        "apply_roofline": {"bound": "alu", "achieved": apply_flops / (ms_apply * 1e-3) / 1e12,
                           "peak": fp64_peak, "unit": "TFLOP/s",
                           "frac": apply_flops / (ms_apply * 1e-3) / 1e12 / fp64_peak,
                           "frac_of_nominal": apply_flops / (ms_apply * 1e-3) / 1e12 / FP64_NOMINAL_TFLOPS},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(verts.nbytes),
                "d2h_bytes_per_step": int(nt * nx * 8)},
        "gpu_launches": int(launches),
        "clocks": ck,
        "wall_s_timed": t_wall,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
    return 0


def _space_order(d):      # Gauss points per piece at lag d >= 2 (discretisation rule)
    return 4 if d >= 32 else (6 if d >= 8 else 8)


def _peano_order(k):      # Gauss nodes on time interval k
    return 6 if k >= 32 else (8 if k >= 2 else 16)


# FP64 flops of one Peano node of the D kernel: e^{-c sigma} (c sigma, x 256/ln2,
# two reduction FMAs, four polynomial FMAs, the table product: 15; the power
# of two is an integer exponent add) and the kernel accumulations, 6 flops per
# role (one FMA for F_V, two for the w3 c - w2 factor of F_1); in a group of 4
# lags the 5 intervals serve 8 roles, 1.6 per node: 15 + 9.6 ~ 24.
D_NODE_FLOPS = 24
# per quadrature point: x - y (4 FMAs), c (4), weight (1), switch (1), five
# moments with their bilinear weights (~23)
D_POINT_FLOPS = 33


def d_lag2_flops(n_x, n_t, lags_per_group=4):
    """Algorithmic FP64 flops of the D_h assembly at lags 2..n_t-1: every
    unordered half-segment pair integrated once per lag (H (H + 1) / 2 with
    H = 2 n_x), n(d)^2 points per pair; each group of consecutive lags (as the
    kernel assembles them: runs of lags_per_group within the space-order
    segments [2, 8), [8, 32), [32, n_t), split every 64 lags) evaluates the
    Peano nodes of its L + 1 time intervals once per point, plus the per-lag
    point work.  (The kernel cuts each segment into chunks of lags_per_group
    from the segment's first lag; 64 is a multiple of 4, so the 64-lag runs
    here give the same chunks.)"""
    H = 2 * n_x
    pairs = H * (H + 1) // 2
    tot = 0.0
    for lo, hi in ((2, 8), (8, 32), (32, n_t)):
        hi = min(hi, n_t)
        for d0 in range(lo, hi, 64):
            d1 = min(d0 + 64, hi)
            for g0 in range(d0, d1, lags_per_group):
                L = min(lags_per_group, d1 - g0)
                nodes = sum(_peano_order(g0 - 1 + i) for i in range(L + 1))
                tot += pairs * _space_order(g0) ** 2 * (D_NODE_FLOPS * nodes + D_POINT_FLOPS * L)
    return tot


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--solve", choices=["direct", "fft"], default="direct",
                    help="products inside the step's right-hand side and GMRES: the direct block sums (default, "
                         "the paper's method) or through time FFTs of the lag blocks; the other is timed beside it")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-right-hand-side square512 component")
    ap.add_argument("--batched-fp64-residual", action="store_true",
                    help="also time the batched solve on FP64 CUDA-core residuals (about a minute)")
    ap.add_argument("--no-grad", action="store_true", help="skip the star256 differentiation component")
    ap.add_argument("--no-ragged", action="store_true", help="skip the 64-problem ragged component")
    ap.add_argument("--no-initial", action="store_true", help="skip the Section 4 example (M_h^0) component")
    ap.add_argument("--no-nonuniform", action="store_true",
                    help="skip the graded-time-grid (packed blocks) component")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the L-shape N_x = N_t = 1024 mixed-versus-FP64 component")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="named workload (default square256; smaller ones are for profiling)")
    ap.add_argument("--component", choices=["tc", "grad", "precision", "initial", "f32apply", "fftapply"],
                    default=None,
                    help="run one kernel family alone on a small case (for ncu captures) and print its timing")
    ap.add_argument("--size", type=int, default=256, help="N_x = N_t of --component's case")
    ap.add_argument("--rhs", type=int, default=64, help="right-hand sides of --component tc")
    args = ap.parse_args()
    globals()["WORKLOAD"] = args.workload
    if args.component:
        return run_component(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


def run_precision(ctx, dev, stream):
    """The precision workload at full size: L-shape (seeded lengths),
    N_x = N_t = 1024, alpha = 0.5.  FP64 path: V, K, D in FP64 (8.6 GB each),
    GMRES to 1e-8 preconditioned with M_h^{-1} D_h M_h^{-T} (the consistent
    mixed mass: on this non-uniform mesh the lumped mass needs ~30x more
    iterations).  Mixed path: V and K in FP64 (the right-hand side and the
    refinement residual), D in FP32 with FP64 singular pairs, V rounded to
    FP32; FP32 inner GMRES, FP64 refinement to 1e-8.  Both timed with CUDA
    events; w compared."""
    import torch
    import workloads as W
    import paper_1811_05224_gb300 as P
    p = W.config("lshape1024")
    m = P.Mesh(ctx, p.vertices, p.T, p.n_t, p.alpha)
    ev = lambda: torch.cuda.Event(enable_timing=True)       # noqa: E731
    e = [ev() for _ in range(8)]
    e[0].record(stream)
    V = P.assemble(ctx, m, "V")
    e[1].record(stream)
    K = P.assemble(ctx, m, "K")
    e[2].record(stream)
    g, f = P.rhs(ctx, m, K, p.y_star)
    L = P.lumped_mass(ctx, m)
    del K
    torch.cuda.empty_cache()
    e[3].record(stream)
    D32 = P.assemble(ctx, m, "D", "f32")
    V32 = P.round_f32(ctx, V)
    Minv = P.mixed_mass_inverse(ctx, m)
    e[4].record(stream)
    wm, im = P.solve_mixed(ctx, V, V32, f, D32, Minv, tol=1e-8, inner_tol=1e-4, max_iter=400, restart=60)
    e[5].record(stream)
    # the same mixed solve with exact-slice outer residuals (no FP64 product)
    x = [ev() for _ in range(3)]
    x[0].record(stream)
    Vx = P.exact_slices(ctx, V, 7)
    x[1].record(stream)
    wx, ix = P.solve_mixed(ctx, Vx, V32, f, D32, Minv, tol=1e-8, inner_tol=1e-4, max_iter=400, restart=60)
    x[2].record(stream)
    del V32
    # and with the inner GMRES on the tensor cores: three BF16 slices of V and
    # of the FP32 D (the preconditioner), exact-slice residuals
    t = [ev() for _ in range(3)]
    t[0].record(stream)
    V3 = P.bf16_split3(ctx, V)
    D3 = P.bf16_split3(ctx, D32.double())
    t[1].record(stream)
    wt, it3 = P.solve_mixed(ctx, Vx, V3, f, D3, Minv, tol=1e-8, inner_tol=1e-4, max_iter=400, restart=60)
    t[2].record(stream)
    del Vx, V3, D3
    torch.cuda.empty_cache()
    # FP64 GMRES with the products through time FFTs: frequency blocks of the
    # FP64 V and of the FP32 D (the preconditioner), no FP32 product anywhere
    q = [ev() for _ in range(3)]
    q[0].record(stream)
    Vh = P.fft_operator(ctx, V)
    Dh = P.fft_operator(ctx, D32)
    q[1].record(stream)
    wf, i_f = P.solve_fft(ctx, Vh, f, Dh, Minv, tol=1e-8, max_iter=400, restart=60)
    q[2].record(stream)
    f0 = ev()
    f0.record(stream)         # the FP64 path starts here
    D = P.assemble(ctx, m, "D")
    e[6].record(stream)
    w, i64 = P.solve(ctx, V, f, D, Minv, tol=1e-8, max_iter=400, restart=60)
    e[7].record(stream)
    # the FP64 path's GMRES with the products through time FFTs
    h = [ev() for _ in range(3)]
    h[0].record(stream)
    P.fft_operator(ctx, D, out=Dh.data)
    h[1].record(stream)
    wf64, i_f64 = P.solve_fft(ctx, Vh, f, Dh, Minv, tol=1e-8, max_iter=400, restart=60)
    h[2].record(stream)
    torch.cuda.synchronize(dev)
    del Vh, Dh
    torch.cuda.empty_cache()
    r = f - P.apply(ctx, V, wm)
    out = {
        "workload": "lshape1024: N_x = N_t = 1024, alpha = 0.5, seeded lengths (seed 3)",
        "assembly_ms": {"V_f64": e[0].elapsed_time(e[1]), "K_f64": e[1].elapsed_time(e[2]),
                        "D_f32_and_V_round": e[3].elapsed_time(e[4]), "D_f64": f0.elapsed_time(e[6])},
        "mixed_solve_ms": e[4].elapsed_time(e[5]), "mixed_inner_iterations": im["iterations"],
        "fp64_solve_ms": e[6].elapsed_time(e[7]), "fp64_iterations": i64["iterations"],
        "mixed_fp64_rel_residual": float(r.norm() / f.norm()),
        "w_rel_diff_mixed_vs_fp64": float((wm - w).norm() / w.norm()),
        "mixed_path_ms": e[3].elapsed_time(e[5]), "fp64_path_ms": f0.elapsed_time(e[7]),
    }
    r2 = f - P.apply(ctx, V, w)
    out["fp64_rel_residual"] = float(r2.norm() / f.norm())
    r3 = f - P.apply(ctx, V, wx)
    out["mixed_exact"] = {
        "exact_slices_ms": x[0].elapsed_time(x[1]), "solve_ms": x[1].elapsed_time(x[2]),
        "inner_iterations": ix["iterations"],
        "path_ms": e[3].elapsed_time(e[4]) + x[0].elapsed_time(x[2]),
        "fp64_rel_residual": float(r3.norm() / f.norm()),
        "w_rel_diff_vs_fp64": float((wx - w).norm() / w.norm()),
        "note": "FP32 D and V inner GMRES; outer residuals from the exact-slice V product (7 slices) "
                "on the tensor cores instead of the FP64 CUDA-core product; path = D32 + V32 + mass + "
                "slicing V + solve"}
    r5 = f - P.apply(ctx, V, wf)
    out["mixed_fft"] = {
        "transforms_ms": q[0].elapsed_time(q[1]), "solve_ms": q[1].elapsed_time(q[2]),
        "iterations": i_f["iterations"],
        "path_ms": e[3].elapsed_time(e[4]) + q[0].elapsed_time(q[2]),
        "fp64_rel_residual": float(r5.norm() / f.norm()),
        "w_rel_diff_vs_fp64": float((wf - w).norm() / w.norm()),
        "note": "FP64 GMRES, every product through the frequency blocks (time FFTs) of the FP64 V and of "
                "the FP32 D; path = D32 + V32 + mass + both transforms + solve"}
    r6 = f - P.apply(ctx, V, wf64)
    out["fp64_fft"] = {
        "transform_D_ms": h[0].elapsed_time(h[1]), "transform_V_ms": q[0].elapsed_time(q[1]) - h[0].elapsed_time(h[1]),
        "solve_ms": h[1].elapsed_time(h[2]), "iterations": i_f64["iterations"],
        "path_ms": f0.elapsed_time(e[6]) + q[0].elapsed_time(q[1]) + h[1].elapsed_time(h[2]),
        "fp64_rel_residual": float(r6.norm() / f.norm()),
        "w_rel_diff_vs_fp64": float((wf64 - w).norm() / w.norm()),
        "note": "the FP64 path with its GMRES products through the frequency blocks of V and D (FP64); "
                "path = D FP64 assembly + both transforms + solve (transform_V_ms: the two transforms of "
                "the mixed_fft entry less that of D)"}
    r4 = f - P.apply(ctx, V, wt)
    out["mixed_tc"] = {
        "slices_ms": t[0].elapsed_time(t[1]), "solve_ms": t[1].elapsed_time(t[2]),
        "inner_iterations": it3["iterations"],
        "path_ms": e[3].elapsed_time(e[4]) + x[0].elapsed_time(x[1]) + t[0].elapsed_time(t[2]),
        "fp64_rel_residual": float(r4.norm() / f.norm()),
        "w_rel_diff_vs_fp64": float((wt - w).norm() / w.norm()),
        "note": "inner GMRES on the BF16 tensor cores (three-slice V and D, compensated products, "
                "lag chunks for one right-hand side), exact-slice outer residuals; path = D32 + mass + "
                "exact slices of V + BF16 slices of V and D + solve"}
    del V, D, D32, wm, w, wx, wt, wf, wf64, f, g, L, Minv, r, r2, r3, r4, r5, r6
    torch.cuda.empty_cache()
    return out


def run_component(args):
    """One kernel family on a small case, for profiling: 'tc' = the BF16
    tensor-core products (plain, compensated and exact-slice) of a
    unit-square V with --rhs right-hand sides; 'grad' = the gradient kernels on a 16-corner star
    with N_x = N_t = --size.  Warm-up, then timed calls with CUDA events."""
    import torch
    import workloads as W
    import paper_1811_05224_gb300 as P
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = P.Context(0, stream)
    n = args.size
    out = {"component": args.component, "size": n}
    ev = lambda: torch.cuda.Event(enable_timing=True)       # noqa: E731
    if args.component == "precision":
        print(json.dumps(run_precision(ctx, dev, stream)), flush=True)
        return 0
    if args.component == "initial":
        # --size is the level L of the Section 4 example (2^L segments per side)
        res = run_initial(ctx, dev, stream, L=n if n <= 9 else 6)
        print(json.dumps(res), flush=True)
        return 0
    if args.component == "f32apply":
        # the FP32 CUDA-core product (register-tiled kernel) of a unit-square V
        # with n_t = N_x = --size, one right-hand side
        mesh = P.Mesh(ctx, W.unit_square(n // 4), 1.0, n, 1.0)
        V32 = P.assemble(ctx, mesh, "V", "f32")
        g = torch.Generator(device="cpu").manual_seed(3)
        x = torch.randn((n, n), generator=g, dtype=torch.float64).to(dev)
        work = P.api.apply_workspace(ctx, n, n, 1, "f32")
        y = torch.empty_like(x)
        for _ in range(2):
            P.apply(ctx, V32, x, work=work, out=y)
        e0, e1 = ev(), ev()
        e0.record(stream)
        P.apply(ctx, V32, x, work=work, out=y)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        flops = 2.0 * n * n * n * (n + 1) / 2
        out.update({"ms": ms, "tflops": flops / (ms * 1e-3) / 1e12,
                    "frac_of_fp32_peak": flops / (ms * 1e-3) / 1e12 / P.pipe_peaks(ctx)["fp32_tflops"]})
        print(json.dumps(out))
        return 0
    if args.component == "fftapply":
        # the product through the frequency blocks of a unit-square V with
        # n_t = N_x = --size, one right-hand side: the operator transform
        # (first launch of k_rfft_cols), then forward and transposed products
        mesh = P.Mesh(ctx, W.unit_square(n // 4), 1.0, n, 1.0)
        V = P.assemble(ctx, mesh, "V")
        Vh = P.fft_operator(ctx, V)
        g = torch.Generator(device="cpu").manual_seed(3)
        x = torch.randn((n, n), generator=g, dtype=torch.float64).to(dev)
        work = P.api.apply_fft_workspace(ctx, n, n, 1)
        y = torch.empty_like(x)
        nf = Vh.data.shape[0]
        res = {}
        for name, call, reps in (("apply_fft", lambda: P.apply_fft(ctx, Vh, x, work=work, out=y), 20),
                                 ("apply_fft_t", lambda: P.apply_fft(ctx, Vh, x, True, work=work, out=y), 20),
                                 ("fft_operator", lambda: P.fft_operator(ctx, V, out=Vh.data), 5)):
            for _ in range(3):
                call()
            e0, e1 = ev(), ev()
            e0.record(stream)
            for _ in range(reps):
                call()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            res[name] = e0.elapsed_time(e1) / reps
        prod_bytes = nf * n * n * 16 + 2 * n * n * 8 + 4 * nf * n * 16
        op_bytes = n * n * n * 8 + nf * n * n * 16
        Lf = 2 * (nf - 1)
        tflops = 5.0 * Lf * np.log2(Lf)
        prod_flops = 8.0 * nf * n * n + n * tflops
        op_flops = (n * n / 2) * tflops
        fp64 = P.pipe_peaks(ctx)["fp64_tflops"]
        out.update({"ms": res, "apply_fft_gbs": prod_bytes / (res["apply_fft"] * 1e-3) / 1e9,
                    "apply_fft_frac_of_fp64": prod_flops / (res["apply_fft"] * 1e-3) / 1e12 / fp64,
                    "fft_operator_frac_of_fp64": op_flops / (res["fft_operator"] * 1e-3) / 1e12 / fp64,
                    "fp64_tflops_measured": fp64,
                    "bytes": {"apply_fft": prod_bytes, "fft_operator": op_bytes},
                    "flops": {"apply_fft": prod_flops, "fft_operator": op_flops}})
        print(json.dumps(out))
        return 0
    if args.component == "tc":
        mesh = P.Mesh(ctx, W.unit_square(n // 4), 1.0, n, 1.0)
        V = P.assemble(ctx, mesh, "V")
        Vb = P.to_bf16(ctx, V)
        Vx = P.exact_slices(ctx, V, 7)
        del V
        g = torch.Generator(device="cpu").manual_seed(3)
        x64 = torch.randn((args.rhs, n, n), generator=g, dtype=torch.float64).to(dev)
        xb = x64.to(torch.bfloat16)
        y = torch.empty((args.rhs, n, n), dtype=torch.float64, device=dev)
        xwork = torch.empty(int(_exact_work_bytes(ctx, n, n, args.rhs, 7)), dtype=torch.uint8, device=dev)
        flops = 2.0 * n * n * n * (n + 1) / 2 * args.rhs
        runs = {"plain": lambda: P.apply_tc(ctx, Vb, xb, out=y),
                "compensated4": lambda: P.apply_tc(ctx, Vb, xb, out=y, chunk=4),
                "exact7": lambda: P.apply_exact(ctx, Vx, x64, out=y, work=xwork)}
        for name, fn in runs.items():
            for _ in range(2):
                fn()
            e0, e1 = ev(), ev()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
            out[name] = {"ms": ms, "tflops": flops / (ms * 1e-3) / 1e12}
        out["exact7"]["bf16_tflops_executed"] = out["exact7"]["tflops"] * 28
        out["rhs"] = args.rhs
    else:
        S = W.subdivision_matrix(16, n // 16)
        mesh = P.Mesh(ctx, S @ W.star_corners(16, seed=5), 1.0, n, 1.0)
        K = P.assemble(ctx, mesh, "K")
        g, _ = P.rhs(ctx, mesh, K, (1.5, 1.5))
        gen = torch.Generator(device="cpu").manual_seed(5)
        lam = torch.randn((n, n), generator=gen, dtype=torch.float64).to(dev)
        w = torch.randn((n, n), generator=gen, dtype=torch.float64).to(dev)
        work = P.api.grad_workspace(ctx, n, n)
        for _ in range(2):
            P.grad(ctx, mesh, K, (1.5, 1.5), g, w, lam, work=work)
        e0, e1 = ev(), ev()
        e0.record(stream)
        P.grad(ctx, mesh, K, (1.5, 1.5), g, w, lam, work=work)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        out["grad_ms"] = e0.elapsed_time(e1)
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
