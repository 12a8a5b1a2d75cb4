"""Benchmark of the solve phase: V-cycle preconditioned CG on the CDG Poisson
operator of a 512 x 512 jittered square (524,288 triangles, p = 3, 5.24M
dofs, 7 agglomeration levels, V(2,2), FP64, relative residual 1e-10).

One step = one complete solve from f sampled at the quadrature points (device
resident) to the DG coefficients u (device), i.e. right-hand-side assembly +
PCG iterations to 1e-10.  value = solved DOF/s over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload tri512_p3|tri256_p3|tri32_p2|tet48_p2]

Under torchrun (N > 1) every rank solves its own copy (replicas, weak scaling);
the timed region is bracketed by barriers and the max over ranks is taken.
"""
from __future__ import annotations

import os

# the CPU-baseline legs time the single-threaded oracle: keep numpy's BLAS on one core
for _v in ("OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import math
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (generator, n, p, levels, nu, precision)
    "tri512_p3": ("square", 512, 3, 7, 2, "fp64"),
    "tri256_p3": ("square", 256, 3, 6, 2, "fp64"),
    "tri32_p2": ("square", 32, 2, 4, 1, "fp64"),
    "tet48_p2": ("cube", 48, 2, 6, 2, "fp32"),
    "tet48_p2_primal": ("cube", 48, 2, 6, 2, "fp32"),
}
# hierarchy options per workload (default: flux coarsening, no p-multigrid front end).  The
# tetrahedral workload runs the paper's flux coarsening (Section 4.1) behind the p-multigrid
# front end (Section 4.4): flux-coarsened p = 2 tetrahedral levels alone stall the FP32
# V-cycle.  Primal coarsening (Section 3.5) is kept as a labelled ablation.
WORKLOAD_HIERARCHY = {"tet48_p2": dict(coarsen="flux", pmg=True),
                      "tet48_p2_primal": dict(coarsen="primal", pmg=False)}
METRIC = "solved DOF/s (PCG+V-cycle to 1e-10)"
HBM_FALLBACK_GBS = 6800.0           # profiling-recipe fallback when no measured peak file exists
# GB300 FP64 rate derived from the unit counts and the clock: 152 SMs x 2 FP64 FMA per clock
# x 2 flops x 2.07 GHz; the roofline divides by the rate the FMA probe measures in the same run
FP64_DERIVED_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM bytes (read + write) of one level-0 apply as ncu captured them on the 256 x 256 p = 3
# square (523,264 blocks): FP64 443,725,568 (profiles/bsr_kernel_tri256_p3_fp64.md), FP32
# 223,440,896 (profiles/bsr_kernel_tri256_p3_fp32.md).  Other squares at p = 3 report them scaled by
# their level-0 block count (the traffic is 1.003-1.005x the algorithmic bytes, which grow with
# the blocks); other workloads report null.  Set to None whenever bsr_kernel changes, until it is
# captured again.
CAPTURED_APPLY = {"blocks": 523_264, "fp64": 443_725_568, "fp32": 223_440_896}


def apply_traffic(kind, p, nnzb0, dtype):
    """Per-launch DRAM traffic of the level-0 apply, from the capture scaled by the block count."""
    if CAPTURED_APPLY.get(dtype) is None or kind != "square" or p != 3:
        return None
    return round(CAPTURED_APPLY[dtype] * nnzb0 / CAPTURED_APPLY["blocks"])


def make_mesh(kind, n):
    from synthetic import jittered_square, kuhn_cube
    return jittered_square(n) if kind == "square" else kuhn_cube(n)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        for k in ("hbm_gbs", "hbm_GBs", "hbm"):
            if k in d:
                return float(d[k]), "measured"
    return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:6]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest x over all ranks (the slowest replica's time); x itself without a
    process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world_size: int, ms: float) -> float:
    """Replicas (weak scaling): every rank solves its own copy, so the whole job
    processes world_size x the units in the slowest rank's time."""
    return units_per_rank * world_size / (ms * 1e-3)


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def fp64_fma_peak(pkg, dev, stream):
    """FP64 FMA rate of this GPU (TFLOP/s), measured with the library's FMA probe
    (16 independent register-operand chains per thread, 8 CTAs of 256 threads per
    SM), best of 5 timed launches."""
    import torch
    sink = torch.zeros(1, dtype=torch.float64, device=dev)
    blocks, iters = 152 * 8, 4096
    fmas = blocks * 256 * 16 * ((iters + 1) // 2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    L = pkg.lib()
    best = 0.0
    for _ in range(6):
        e0.record(stream)
        rc = L.cdg_fp64_fma_probe(blocks, iters, sink.data_ptr(), stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if rc:
            return None
        best = max(best, 2.0 * fmas / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    return best


def cpu_baseline(kind, p, nu, seconds_target=10.0, coarsen="flux", pmg=False):
    """Oracle (plain FP64 numpy/scipy, Python, one core) on a bounded sample of
    the workload: the same generator and discretisation on a 64 x 64 square
    (8,192 triangles) or a 12^3 cube, oracle set-up untimed, its PCG + V-cycle
    solve timed."""
    from oracle.cdg import Level0
    from oracle.hierarchy import MGHierarchy
    from oracle.solver import VCycle, pcg
    from synthetic import sin_source
    n = 64 if kind == "square" else 12
    mesh = make_mesh(kind, n)
    L0 = Level0(mesh, p)
    H = MGHierarchy(L0, max_levels=5, coarsen=coarsen, pmg=pmg)
    V = VCycle(H.A, H.L, H.nps, nu, nu)
    b = L0.rhs(sin_source(L0.all_volume_points()))
    times, its = [], []
    t_end = time.perf_counter() + seconds_target
    while True:
        t0 = time.perf_counter()
        x, hist, it = pcg(H.A[0], b, V.apply, tol=1e-10)
        times.append(time.perf_counter() - t0)
        its.append(it)
        if time.perf_counter() > t_end or len(times) >= 50:
            break
    ndof = H.A[0].shape[0]
    return {"value": ndof / statistics.median(times), "unit": "DOF/s", "cores": 1, "kind": "oracle",
            "sample": f"Python oracle, 1 core, {'square' if kind == 'square' else 'cube'} n={n} sample "
                      f"({mesh.n_elements} elements, {ndof} dofs), p={p}, {H.n_levels} levels, V({nu},{nu}), "
                      f"tol 1e-10, {its[0]} iterations, median of {len(times)} solves, set-up untimed"}


def _time(fn, stream, reps):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def run_extras(pkg, dev, stream, barrier, only=None):
    """The other workloads of the solve phase, each timed after one warm-up:
    64 meshes of 500-20000 triangles in one batched handle (p = 2) against the
    same meshes solved one after another; one 158 x 158 x 2 triangle mesh
    (p = 3) with 256 right-hand sides (sine combinations; FP32 and BF16 V-cycle blocks)
    against 256 single solves estimated from 8; the differentiable 24^3 x 6
    tetrahedra workload (p = 2, smoothed log-normal kappa): forward + adjoint.
    only: one of "latency", "batched", "multi_rhs", "adjoint", "tet48" (None = all)."""
    out = {}
    if only in (None, "latency"):
        out.update(extra_latency_tri32(pkg, dev, stream))
    if only in (None, "batched"):
        out.update(extra_batched(pkg, dev, stream))
    if only in (None, "multi_rhs"):
        out.update(extra_multi_rhs(pkg, dev, stream))
    if only == "tc_small":
        out.update(extra_tc_small(pkg, dev, stream))
    if only == "mr_small":
        out.update(extra_mr_small(pkg, dev, stream))
    if only in ("multi_rhs_bf16", "multi_rhs_bf16_cuda_cores", "multi_rhs_fp32_tc_fp64_apply"):
        out.update(extra_multi_rhs(pkg, dev, stream, variants=(only[10:],), singles=False))   # one variant
    if only in (None, "adjoint"):
        out.update(extra_adjoint(pkg, dev, stream))
    if only in (None, "tet48"):
        out.update(extra_tet48(pkg, dev, stream))
    return out


def extra_tet48(pkg, dev, stream, steps=3):
    """48^3 x 6 Kuhn cube (663,552 tetrahedra, p = 2, 6.6M dofs): the paper's flux
    coarsening behind the p-multigrid front end, FP32 V-cycle inside FP64 CG to
    1e-10, and its distance to the FP64 V-cycle solve of the same hierarchy
    (one host set-up, bound twice)."""
    import torch
    from synthetic import kuhn_cube, sin_source
    kind, n, p, lv, nu, _ = WORKLOADS["tet48_p2"]
    t0 = time.perf_counter()
    S = pkg.Solver(kuhn_cube(n), p=p, max_levels=lv, nu_pre=nu, nu_post=nu, precision="fp32", tol=1e-10,
                   maxit=500, **WORKLOAD_HIERARCHY["tet48_p2"])
    setup_s = time.perf_counter() - t0
    S.bind(dev)
    fq = torch.tensor(sin_source(S.quadrature_points()[0]), device=dev)
    ms32, (u32, h32, it32, rc32) = _time(lambda: S.solve(fq), stream, steps)
    u32 = u32.clone()
    S.set_precision("fp64").bind(dev)
    ms64, (u64, h64, it64, rc64) = _time(lambda: S.solve(fq), stream, 1)
    ndof = S.info["n_dofs"]
    line = {"value": ndof / (ms32 * 1e-3), "unit": "DOF/s", "ms_per_solve": ms32, "iterations": it32, "rc": rc32,
            "dofs": ndof, "levels": S.n_levels, "np_l": S.info["np_l"], "coarsening": "flux",
            "front_end": "p-multigrid", "vcycle": "fp32", "final_rel_residual": float(h32[-1]),
            "fp64_vcycle_ms_per_solve": ms64, "fp64_vcycle_iterations": it64, "fp64_vcycle_rc": rc64,
            "rel_l2_diff_vs_fp64_vcycle_solve": float((u32 - u64).norm() / u64.norm()),
            "setup_s": round(setup_s, 2)}
    del S
    return {"tet48_p2_flux_pmg_fp32": line}


def extra_latency_tri32(pkg, dev, stream):
    """32 x 32 jittered square (2,048 triangles, p = 2, 12,288 dofs, 4 levels, V(1,1),
    FP64): solve latency; the operator is L2-resident, so this is a latency number."""
    import torch
    from synthetic import sin_source
    kind, n, p, lv, nu, prec = WORKLOADS["tri32_p2"]
    S = pkg.Solver(make_mesh(kind, n), p=p, max_levels=lv, nu_pre=nu, nu_post=nu, precision=prec, tol=1e-10,
                   maxit=500).bind(dev)
    fq = torch.tensor(sin_source(S.quadrature_points()[0]), device=dev)
    for _ in range(3):
        S.solve(fq)
    ms, (u, h, it, rc) = _time(lambda: S.solve(fq), stream, 20)
    return {"tri32_p2_latency": {"ms_per_solve": ms, "iterations": it, "rc": rc, "dofs": S.info["n_dofs"],
                                 "us_per_iteration": ms * 1e3 / max(it, 1)}}


def extra_tc_small(pkg, dev, stream):
    """A small case of the tensor-core kernels (the size ncu captures in full):
    100 x 100 square (20,000 triangles, p = 3, 200,000 dofs), 128 right-hand
    sides (x: 205 MB FP64, above L2): three split FP64 applies (tc_fp64_apply),
    then one BF16-block multi-RHS solve of two iterations (tcgen05 sweeps)."""
    import torch
    from synthetic import jittered_square, sine_combination_sources
    mesh = jittered_square(100)
    R = 128
    S = pkg.Solver(mesh, p=3, max_levels=4, precision="fp32", nrhs=R, tc_fp64_apply=True).bind(dev)
    x = torch.tensor(np.random.default_rng(1).standard_normal((S.info["n_dofs"], R)), device=dev)
    y = torch.empty_like(x)
    ms, _ = _time(lambda: S.apply_multi(x, y), stream, 2)
    del S, x, y
    S = pkg.Solver(mesh, p=3, max_levels=4, nu_pre=2, nu_post=2, precision="bf16", nrhs=R, maxit=2,
                   tensor_cores=True).bind(dev)
    fq = torch.tensor(sine_combination_sources(S.quadrature_points()[0], R, mmax=8, seed0=0), device=dev)
    S.solve_multi(fq)
    torch.cuda.synchronize(dev)
    return {"tc_small": {"split_fp64_apply_ms": ms, "dofs": int(mesh.n_elements * 10), "nrhs": R}}


def extra_mr_small(pkg, dev, stream):
    """A small case of the many-right-hand-side V-cycle sweeps (the size ncu
    captures in full): 100 x 100 square (20,000 triangles, p = 3, 200,000
    dofs), 256 right-hand sides (one FP32 V-cycle vector: 205 MB, above L2),
    two CG iterations with FP32 blocks (CUDA-core sweeps, autotuned), then two
    with BF16 blocks and tcgen05 sweeps.  Each solve runs inside an NVTX range
    ("mr_fp32", "mr_bf16_tc") so that a profiler can pick its kernels out."""
    import torch
    from synthetic import jittered_square, sine_combination_sources
    mesh = jittered_square(100)
    R = 256
    out = {}
    for prec, tc, tag in (("fp32", False, "mr_fp32"), ("bf16", True, "mr_bf16_tc")):
        S = pkg.Solver(mesh, p=3, max_levels=4, nu_pre=2, nu_post=2, precision=prec, nrhs=R, maxit=2,
                       tensor_cores=tc).bind(dev)
        fq = torch.tensor(sine_combination_sources(S.quadrature_points()[0], R, mmax=8, seed0=0), device=dev)
        S.solve_multi(fq)   # the autotuner's timings run here, outside the range
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_push(tag)
        ms, _ = _time(lambda: S.solve_multi(fq), stream, 1)
        torch.cuda.nvtx.range_pop()
        out[tag + "_two_iterations_ms"] = ms
        del S
    return {"mr_small": out}


def extra_batched(pkg, dev, stream):
    import torch
    from synthetic import batched_squares, sin_source
    out = {}
    # ---- batched meshes
    meshes = batched_squares(64, 500, 20000, seed=1)
    # the V-cycle as one persistent cooperative kernel per cycle, then as one kernel per phase
    B = pkg.BatchSolver(meshes, p=2, max_levels=4, persistent_vcycle=True).bind(dev)
    xq = B.quadrature_points()[0]
    fq = torch.tensor(sin_source(xq), device=dev)
    l0 = pkg.kernel_launches()
    ms_p, (u, hists, its_p, rc_p) = _time(lambda: B.solve(fq), stream, 5)
    nl_p = (pkg.kernel_launches() - l0) / 6
    del B
    B = pkg.BatchSolver(meshes, p=2, max_levels=4).bind(dev)
    l0 = pkg.kernel_launches()
    ms, (u, hists, its, rc) = _time(lambda: B.solve(fq), stream, 5)
    nl = (pkg.kernel_launches() - l0) / 6
    seq = 0.0
    for m in meshes:
        S = pkg.Solver(m, p=2, max_levels=4).bind(dev)
        f1 = torch.tensor(sin_source(S.quadrature_points()[0]), device=dev)
        t, _ = _time(lambda: S.solve(f1), stream, 1)
        seq += t
        del S
    out["batched_64_meshes"] = {"value": B.info["n_dofs"] / (ms * 1e-3), "unit": "DOF/s", "ms_per_solve": ms,
                                "dofs": B.info["n_dofs"], "iterations_min_max": [int(its.min()), int(its.max())],
                                "rc": rc, "launches_per_solve": nl, "sequential_ms": seq,
                                "speedup_vs_sequential": seq / ms,
                                "persistent_vcycle": {"value": B.info["n_dofs"] / (ms_p * 1e-3), "ms_per_solve": ms_p,
                                                      "iterations_min_max": [int(its_p.min()), int(its_p.max())],
                                                      "rc": rc_p, "launches_per_solve": nl_p}}
    del B
    return out


def extra_multi_rhs(pkg, dev, stream, variants=("fp32", "fp32_tc_fp64_apply", "bf16", "bf16_tc_fp64_apply",
                                                 "bf16_cuda_cores"), singles=True):
    import torch
    from synthetic import jittered_square, sine_combination_sources
    out = {}
    # ---- many right-hand sides on one mesh
    mesh = jittered_square(158)
    R = 256
    S1 = pkg.Solver(mesh, p=3, max_levels=5, nu_pre=2, nu_post=2, precision="fp32").bind(dev)
    xq = S1.quadrature_points()[0]
    fq = torch.tensor(sine_combination_sources(xq, R, mmax=8, seed0=0), device=dev)
    single = []
    for r in range(8 if singles else 0):
        t, _ = _time(lambda: S1.solve(fq[r].contiguous()), stream, 1)
        single.append(t)
    del S1
    # BF16 blocks: smoother sweeps on tcgen05 tensor cores (default) and on CUDA cores
    for prec, tc, tca, name in (("fp32", False, False, "fp32"), ("fp32", False, True, "fp32_tc_fp64_apply"),
                                ("bf16", True, False, "bf16"), ("bf16", True, True, "bf16_tc_fp64_apply"),
                                ("bf16", False, False, "bf16_cuda_cores")):
        if name not in variants:
            continue
        S = pkg.Solver(mesh, p=3, max_levels=5, nu_pre=2, nu_post=2, precision=prec, nrhs=R,
                       tensor_cores=tc, tc_fp64_apply=tca).bind(dev)
        ms, (u, hists, its, rc) = _time(lambda: S.solve_multi(fq), stream, 2 if singles else 1)
        out["multi_rhs_256_" + name] = {
            "value": R * S.info["n_dofs"] / (ms * 1e-3), "unit": "DOF/s", "ms_per_solve": ms,
            "dofs_per_rhs": S.info["n_dofs"], "nrhs": R, "vcycle_blocks": prec,
            "smoother_sweeps": "tcgen05" if tc else "cuda cores",
            "outer_fp64_apply": "tcgen05 exact split" if tca else "cuda cores",
            "iterations_min_max": [int(its.min()), int(its.max())], "rc": rc,
            "single_rhs_fp32_vcycle_ms": float(np.mean(single)) if single else None,
            "speedup_vs_single_solves": R * float(np.mean(single)) / ms if single else None}
        del S
    return out


def extra_adjoint(pkg, dev, stream):
    import torch
    from synthetic import face_neighbors, kuhn_cube, sin_source, smoothed_lognormal_kappa
    out = {}
    # ---- differentiable solve
    from paper_2012_08024_gb300.autograd import CDGSolve, SolverCache
    mesh = kuhn_cube(24)
    nb = face_neighbors(mesh)
    kappa = smoothed_lognormal_kappa(nb, seed=2)
    kstar = smoothed_lognormal_kappa(nb, seed=3)
    # primal coarsening: with this kappa contrast (~1e3) the flux-coarsened 3D operators are indefinite
    cache = SolverCache(mesh, p=2, max_levels=5, coarsen="primal")
    xq = cache.get(torch.tensor(kstar), dev).quadrature_points()[0]
    fq = torch.tensor(sin_source(xq), device=dev)
    with torch.no_grad():
        ut = CDGSolve.apply(fq, torch.tensor(kstar, device=dev), cache)
    k = torch.tensor(kappa, device=dev, requires_grad=True)
    f = fq.clone().requires_grad_(True)
    t0 = time.perf_counter()
    loss = ((CDGSolve.apply(f, k, cache) - ut) ** 2).sum()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    S = cache.solver
    fw, _ = _time(lambda: S.solve(fq), stream, 2)
    u = S.solve(fq)[0]
    lam = S.solve_adjoint(2 * (u - ut))[0]
    bw, _ = _time(lambda: (S.solve_adjoint(2 * (u - ut)), S.rhs_adjoint(lam), S.kappa_gradient(lam, u)), stream, 2)
    kg, _ = _time(lambda: S.kappa_gradient(lam, u), stream, 10)
    out["adjoint_24cube"] = {"elements": mesh.n_elements, "dofs": S.info["n_dofs"],
                             "forward_ms": fw, "backward_ms": bw, "kappa_gradient_kernel_ms": kg,
                             "first_forward_with_setup_s": t1 - t0, "first_backward_s": t2 - t1,
                             "loss": float(loss.detach())}
    return out


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    kind, n, p, lv, nu, prec = WORKLOADS[args.workload]
    from oracle.cdg import Level0
    from oracle.hierarchy import MGHierarchy
    from oracle.solver import VCycle, pcg
    from synthetic import sin_source
    ns = 64 if kind == "square" else 12
    mesh = make_mesh(kind, ns)
    L0 = Level0(mesh, p)
    hier = WORKLOAD_HIERARCHY.get(args.workload, {})
    H = MGHierarchy(L0, max_levels=5, coarsen=hier.get("coarsen", "flux"), pmg=hier.get("pmg", False))
    V = VCycle(H.A, H.L, H.nps, nu, nu)
    fq = sin_source(L0.all_volume_points())
    for _ in range(args.warmup):
        pcg(H.A[0], L0.rhs(fq), V.apply, tol=1e-10)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        b = L0.rhs(fq)
        x, hist, it = pcg(H.A[0], b, V.apply, tol=1e-10)
    dt = (time.perf_counter() - t0) / args.steps
    ndof = H.A[0].shape[0]
    val = ndof / dt
    sample = (f"Python oracle, 1 core, on a {ns}^{2 if kind == 'square' else 3} "
              f"{'square' if kind == 'square' else 'cube'} sample "
              f"({mesh.n_elements} elements, {ndof} dofs), p={p}, V({nu},{nu}), each step = rhs + PCG to 1e-10")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "DOF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload},
        "cpu_baseline": {"value": val, "unit": "DOF/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tri512_p3", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the batched / multi-RHS / adjoint workloads")
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32"],
                    help="override the workload's V-cycle precision")
    ap.add_argument("--fuse-transfers", type=int, default=0, choices=[0, 1, 2, 3],
                    help="V-cycle transfer fusion: bit 0 residual + restriction + first coarse smoothing step, "
                         "bit 1 prolongation in the coarse level's last sweep (default 0: separate kernels)")
    ap.add_argument("--per-iteration-graphs", action="store_true",
                    help="run the CG loop as graphs per iteration half with a host read each (the same "
                         "kernels; the form a kernel profiler lists launch by launch)")
    ap.add_argument("--only-extra", default=None,
                    choices=["latency", "batched", "multi_rhs", "adjoint", "tet48", "multi_rhs_bf16",
                             "multi_rhs_bf16_cuda_cores", "multi_rhs_fp32_tc_fp64_apply", "tc_small", "mr_small"],
                    help="run one extra workload alone and print its numbers (for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.only_extra:
        import torch
        import paper_2012_08024_gb300 as pkg
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        print(json.dumps(run_extras(pkg, dev, torch.cuda.current_stream(dev), None, only=args.only_extra)))
        return
    import torch
    ws, rank, local = dist_info()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    import paper_2012_08024_gb300 as pkg
    from synthetic import sin_source
    kind, n, p, lv, nu, prec = WORKLOADS[args.workload]
    hier = WORKLOAD_HIERARCHY.get(args.workload, {})
    coarsen, pmg = hier.get("coarsen", "flux"), hier.get("pmg", False)
    if args.precision:
        prec = args.precision
    mesh = make_mesh(kind, n)
    t0 = time.perf_counter()
    S = pkg.Solver(mesh, p=p, max_levels=lv, nu_pre=nu, nu_post=nu, precision=prec, tol=1e-10, maxit=500,
                   coarsen=coarsen, pmg=pmg, single_graph=not args.per_iteration_graphs,
                   fuse_transfers=args.fuse_transfers)
    setup_s = time.perf_counter() - t0
    S.bind(dev)
    xq, _, _ = S.quadrature_points()
    fq_host = sin_source(xq)
    fq = torch.tensor(fq_host, device=dev)
    ndof = S.info["n_dofs"]
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # ---- device-resident solves (the clock sampler starts before the warm-up: nvidia-smi's
    # own start-up must not fall inside a short timed region)
    cs = ClockSampler(dev.index)
    with cs:
        time.sleep(1.0)
        for _ in range(max(args.warmup, 3)):
            u, hist, it, rc = S.solve(fq)
        barrier()
        l0 = pkg.kernel_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        iters = []
        e0.record(stream)
        for _ in range(args.steps):
            u, hist, it, rc = S.solve(fq)
            iters.append(it)
        e1.record(stream)
        barrier()
    launches = pkg.kernel_launches() - l0
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
    value = whole_job_rate(ndof, ws, ms)
    # ---- end to end through the C ABI with pinned host buffers
    fq_pin = torch.tensor(fq_host).pin_memory()
    u_pin = torch.empty((S.ne, S.np_), dtype=torch.float64).pin_memory()
    import ctypes as C
    hist_h = np.zeros(S.maxit + 1)
    itc = C.c_int32(0)

    def solve_host():
        return pkg.lib().cdg_solve(S._h, fq_pin.data_ptr(), None, None, u_pin.data_ptr(), 0,
                                   hist_h.ctypes.data, C.byref(itc), 1, stream.cuda_stream)
    for _ in range(2):
        solve_host()
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        solve_host()
    e1.record(stream)
    barrier()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
    # ---- dominant kernel: level-0 FP64 block-sparse apply, timed on the launching stream
    x0 = torch.randn(ndof, dtype=torch.float64, device=dev)
    y0 = torch.empty_like(x0)
    for _ in range(3):
        S.apply(0, x0, y0)
    reps = 20
    e0.record(stream)
    for _ in range(reps):
        S.apply(0, x0, y0)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    k_us = e0.elapsed_time(e1) / reps * 1e3
    nnzb0 = S.info["nnzb_l"][0]
    npb = S.np_
    alg_bytes = nnzb0 * npb * npb * 8 + nnzb0 * 4 + (S.ne + 1) * 4 + 2 * ndof * 8
    achieved = alg_bytes / (k_us * 1e-6) / 1e9
    peak, peak_src = peaks()
    flops = 2.0 * nnzb0 * npb * npb
    # ---- same workload with the FP32 V-cycle inside the FP64 CG (precision mode 1)
    mixed = None
    fma_peak = fp64_fma_peak(pkg, dev, stream)
    if prec == "fp64":
        u64 = u.clone()
        S32 = S.set_precision("fp32").bind(dev)   # same host set-up, FP32 V-cycle
        for _ in range(3):
            u32, h32, it32, rc32 = S32.solve(fq)
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            u32, h32, it32, rc32 = S32.solve(fq)
        e1.record(stream)
        barrier()
        ms32 = e0.elapsed_time(e1) / args.steps
        # the FP32 V-cycle's block-sparse kernel (HBM-bound): level-0 FP32 apply
        x32 = torch.randn(ndof, dtype=torch.float32, device=dev)
        y32 = torch.empty_like(x32)
        for _ in range(3):
            S32.apply_f32(0, x32, y32)
        e0.record(stream)
        for _ in range(reps):
            S32.apply_f32(0, x32, y32)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        k32_us = e0.elapsed_time(e1) / reps * 1e3
        alg32 = nnzb0 * npb * npb * 4 + nnzb0 * 4 + (S.ne + 1) * 4 + 2 * ndof * 4
        roof32 = {"bound": "hbm", "achieved": alg32 / (k32_us * 1e-6) / 1e9, "peak": peak, "unit": "GB/s",
                  "frac": alg32 / (k32_us * 1e-6) / 1e9 / peak, "traffic": apply_traffic(kind, p, nnzb0, "fp32"),
                  "peak_source": peak_src,
                  "kernel": "level-0 FP32 block-sparse apply (bsr_kernel<float,%d,0,true>)" % npb,
                  "alg_bytes_per_launch": alg32, "launch_us": k32_us}
        mixed = {"value": ndof * ws / (ms32 * 1e-3), "ms_per_step": ms32, "iterations": it32,
                 "roofline_fp32_kernel": roof32,
                 "final_rel_residual": float(h32[-1]),
                 "rel_l2_diff_vs_fp64_solve": float((u32 - u64).norm() / u64.norm()),
                 "speedup_vs_fp64": ms / ms32}
        del S32
    # ---- the paper's own solver settings on the same mesh (Section 5): GMRES(50) right-
    # preconditioned by V(0,3), tol 1e-8, hierarchy to one element
    paper_solver = None
    if args.extras and prec == "fp64":
        paper_solver = {}
        try:
            Sg = pkg.Solver(mesh, p=p, max_levels=16, nu_pre=0, nu_post=3, precision="fp64", tol=1e-8,
                            maxit=500, krylov="gmres", restart=50)
            for pr in ("fp64", "fp32"):
                Sg.set_precision(pr).bind(dev)
                for _ in range(2):
                    ug, hg, itg, rcg = Sg.solve(fq)
                barrier()
                e0.record(stream)
                for _ in range(args.steps):
                    ug, hg, itg, rcg = Sg.solve(fq)
                e1.record(stream)
                barrier()
                msg = e0.elapsed_time(e1) / args.steps
                paper_solver["vcycle_" + pr] = {
                    "value": ndof * ws / (msg * 1e-3), "unit": "DOF/s", "ms_per_step": msg, "iterations": itg,
                    "levels": Sg.n_levels, "rc": rcg, "final_rel_residual": float(hg[-1]),
                    "ms_per_arnoldi_step": msg / max(itg, 1)}
            del Sg
        except Exception as e:
            paper_solver["error"] = repr(e)[:300]
    # ---- the same solve with the p-multigrid front end (Section 4.4): degrees p..2 on the
    # fine mesh before the agglomeration levels (built at p = 1)
    pmg_line = None
    if args.extras and prec == "fp64" and p > 1:
        pmg_line = {}
        try:
            Sp = pkg.Solver(mesh, p=p, max_levels=lv, nu_pre=nu, nu_post=nu, precision="fp64", tol=1e-10,
                            maxit=500, pmg=True)
            for pr in ("fp64", "fp32"):
                Sp.set_precision(pr).bind(dev)
                for _ in range(2):
                    up, hp, itp, rcp = Sp.solve(fq)
                barrier()
                e0.record(stream)
                for _ in range(args.steps):
                    up, hp, itp, rcp = Sp.solve(fq)
                e1.record(stream)
                barrier()
                msp = e0.elapsed_time(e1) / args.steps
                pmg_line["vcycle_" + pr] = {
                    "value": ndof * ws / (msp * 1e-3), "unit": "DOF/s", "ms_per_step": msp, "iterations": itp,
                    "levels": Sp.n_levels, "np_l": Sp.info["np_l"], "rc": rcp, "final_rel_residual": float(hp[-1]),
                    "speedup_vs_fp64_headline": ms / msp}
            del Sp
        except Exception as e:
            pmg_line["error"] = repr(e)[:300]
    extras = {}
    if args.extras and prec == "fp64":
        try:
            extras = run_extras(pkg, dev, stream, barrier)
        except Exception as e:   # the headline line is printed regardless
            extras = {"extras_error": repr(e)[:300]}
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline(kind, p, nu, coarsen=coarsen, pmg=pmg)
    clocks = cs.summary()
    achieved_tf = flops / (k_us * 1e-6) / 1e12
    fp64_peak = fma_peak if fma_peak else FP64_DERIVED_TFLOPS
    roofline = {"bound": "alu", "achieved": achieved_tf, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved_tf / fp64_peak, "traffic": apply_traffic(kind, p, nnzb0, "fp64"),
                "peak_source": ("measured in this run: FP64 FMA probe (cdg_fp64_fma_probe)" if fma_peak else
                                "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz"),
                "peak_derived_tflops": FP64_DERIVED_TFLOPS, "frac_of_derived": achieved_tf / FP64_DERIVED_TFLOPS,
                "kernel": "level-0 FP64 block-sparse apply (bsr_kernel<double,%d,0,true>)" % npb,
                "alg_bytes_per_launch": alg_bytes, "alg_flops_per_launch": flops, "launch_us": k_us,
                "hbm_gbs": achieved, "hbm_peak_gbs": peak, "hbm_peak_source": peak_src,
                "hbm_frac": achieved / peak}
    if mixed:   # the FP32 V-cycle's block-sparse kernel, HBM-bound
        r32 = mixed["roofline_fp32_kernel"]
        roofline.update({"fp32_apply_gbs": r32["achieved"], "fp32_apply_hbm_frac": r32["frac"],
                         "fp32_apply_launch_us": r32["launch_us"], "fp32_apply_alg_bytes": r32["alg_bytes_per_launch"],
                         "fp32_apply_traffic": r32["traffic"]})
    config = {"workload": args.workload, "mesh": f"{kind} {n}", "elements": S.ne, "p": p, "dofs": ndof,
              "levels": S.n_levels, "n_l": S.info["n_l"], "nnzb_l": S.info["nnzb_l"],
              "smoother": f"V({nu},{nu}) block Jacobi omega=2/3", "coarsening": coarsen,
              "p_multigrid_front_end": pmg, "tol": 1e-10, "precision": prec,
              "iterations": iters[-1], "setup_s": round(setup_s, 3), "parallelism": f"replicas x{ws}",
              "l2": "inputs larger than L2 (operator %.2f GB)" % (S.info["device_bytes"] / 1e9)}
    # the other BASELINE workloads' headline numbers, as scalars beside the workload's own
    lat = extras.get("tri32_p2_latency")
    if lat:
        config.update({"tri32_p2_ms_per_solve": lat["ms_per_solve"], "tri32_p2_iterations": lat["iterations"]})
    t48 = extras.get("tet48_p2_flux_pmg_fp32")
    if t48:
        config.update({"tet48_p2_flux_pmg_fp32_ms_per_solve": t48["ms_per_solve"],
                       "tet48_p2_flux_pmg_fp32_dofs_per_s": t48["value"],
                       "tet48_p2_flux_pmg_fp32_iterations": t48["iterations"],
                       "tet48_p2_flux_pmg_fp32_rel_l2_vs_fp64": t48["rel_l2_diff_vs_fp64_vcycle_solve"]})
    if mixed:
        config.update({"mixed_fp32_vcycle_ms_per_solve": mixed["ms_per_step"],
                       "mixed_fp32_vcycle_iterations": mixed["iterations"]})
    line = {
        "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f64+f32", "data": "synthetic",
        "config": config,
        "roofline": roofline,
        "e2e": {"value": whole_job_rate(ndof, ws, ms_e2e), "unit": "DOF/s",
                "h2d_bytes_per_step": int(fq_pin.numel() * 8), "d2h_bytes_per_step": int(u_pin.numel() * 8)},
        "mixed_fp32_vcycle": mixed,
        "paper_solver_gmres50_v03_tol1e-8": paper_solver,
        "pmg_front_end": pmg_line,
        **{k: v for k, v in extras.items() if k != "tet48_p2_flux_pmg_fp32"},
        "tet48_p2_flux_pmg_fp32": t48,
        "gpu_launches": launches,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
