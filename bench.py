#!/usr/bin/env python
"""Benchmark: deflated overlap propagator solve on one GB300.

Workload (the paper's method at the size of its deflated-overlap runs, on
synthetic inputs): 16^3 x 32 lattice, random SU(3) links U = exp(i 0.2 H)
(seed 0) standing in for the paper's smeared 2+1-flavour ensemble, Wilson
mass m0 = -1.5, sign(H_w) ~ Q P(Q^2) with the degree-527 Chebyshev
approximation of x^{-1/2} on [4e-4, 1] (sqrt(eps) = 0.02, delta ~ 1e-10 by
eq. 2), the 50 lowest |lambda| eigenvectors of Q treated exactly, quark mass
0.02, one spin-colour point source solved to ||b - D x|| / ||b|| <= 1e-10.

A step is one solve (every row of the hot path: Wilson kernels, Clenshaw
polynomial, small-space projection, sign, D(m), chiral-sector CG in FP32
with FP64 true-residual correction; by default the inner cycles run at the
adaptive order's lower degrees, every true residual at the full degree).
``value`` counts D_ov applications at the full degree per second sustained
inside the timed solves: Wilson applications of the solves (any precision)
divided by 2n + 1.  Also reported: the FP64-only solve
(time-to-solution against the mixed one), isolated FP32/FP64 D(m)
applications, the Wilson-kernel bandwidth of the Clenshaw loops (roofline),
and the CPU oracle's rate on a bounded sample.

``--impl reference`` times the CPU oracle (the plain FP64 restatement of the
method) on the same workload instead.  Multi-GPU runs (torchrun) are
independent replicas: the method's solves do not shard here.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DIMS = (16, 16, 16, 32)
LINK_EPS = 0.2
M0 = -1.5
SQRT_EPS = 0.02
DEGREE = 527
N_EV = 50
N_DEFL = 32  # D_ov low modes per chiral sector deflating the inner CG
MASS = 0.02
TOL = 1e-10
BC = (0, 0, 0, 1)  # periodic x, y, z; antiperiodic t
METRIC = "D_ov applies/s, dslash HBM GB/s, time-to-1e-10 solve (mixed vs FP64)"
UNIT = "D_ov applies/s"
WORKLOAD = f"16^3x32 deflated overlap point-source solve, n={DEGREE}, N_ev={N_EV}, m={MASS}, tol={TOL}"
# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum) over algorithmic bytes of the Wilson
# kernel, measured on the kernel source whose hash is KERNEL_SHA: at 16^3x32 inside the timed solve
# (one pass, caches as the solve leaves them: the loop's links and vectors stay in L2), at 24^3x48 in
# the kernel case (cold caches).  When the kernel source changes the ratios are stale and `traffic`
# is reported as null until they are measured again.
KERNEL_SHA = "f7f9e39adeb0aa18"
DRAM_OVER_ALGORITHMIC = {"f32_16x16x16x32_solve": 0.09, "f32_24x24x24x48": 0.87, "f16_24x24x24x48": 0.83,
                         "bf16_24x24x24x48": 0.83}
HBM_DIMS = (24, 24, 24, 48)  # the HBM-bound case: links and vectors far beyond the 129 MB L2


def kernel_sha():
    import hashlib

    h = hashlib.sha256()
    for f in ("dslash.cu", "half_store.h"):
        with open(os.path.join(ROOT, "paper_1111_6288_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def dram_ratio(key):
    """The measured DRAM/algorithmic ratio, or None once the kernel source has changed since."""
    return DRAM_OVER_ALGORITHMIC.get(key) if kernel_sha() == KERNEL_SHA else None


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate(local_ms, local_units, world):
    """Max of the step time and sum of the work over ranks (identity for one rank)."""
    if world == 1:
        return local_ms, local_units
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
    u = torch.tensor([local_units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline leg)
# ---------------------------------------------------------------------------

_ORACLE_INPUTS = {}


def _oracle_inputs():
    if not _ORACLE_INPUTS:
        import numpy as np

        import synth
        from oracle import overlap as ov

        U = synth.random_su3_field(DIMS, LINK_EPS, 0)
        x = synth.gaussian_spinor(DIMS, 1, 1)[0]
        rng = np.random.default_rng(3)
        V = (rng.standard_normal((N_EV,) + x.shape) + 0j).astype(np.complex128)
        _ORACLE_INPUTS.update(U=U, x=x, small=ov.SmallSpace(V, np.ones(N_EV)))
    return _ORACLE_INPUTS


def oracle_sample(n_wilson=4):
    """Time the oracle's Wilson application at the workload size; return seconds per
    D_ov application (2n + 1 Wilson applications plus the small-space projection)."""
    from oracle import dirac
    from oracle import overlap as ov

    d = _oracle_inputs()
    bcf = (1.0, 1.0, 1.0, -1.0)
    t0 = time.perf_counter()
    y = d["x"]
    for _ in range(n_wilson):
        y = dirac.hermitian_wilson(d["U"], y, M0, bcf)
    t_w = (time.perf_counter() - t0) / n_wilson
    t0 = time.perf_counter()
    ov.project(d["small"], d["x"])
    t_p = time.perf_counter() - t0
    return (2 * DEGREE + 1) * t_w + t_p, t_w


_CORE_INPUTS = {}


def _oracle_core_init():
    """Per-process inputs of the all-cores oracle sample (built once per worker)."""
    import synth

    _CORE_INPUTS["U"] = synth.random_su3_field(DIMS, LINK_EPS, 0)
    _CORE_INPUTS["y"] = synth.gaussian_spinor(DIMS, 1, 1)[0]


def _oracle_core_worker(task):
    """One process's share of the all-cores oracle sample: waits for the common start time, applies the
    oracle's H_w n times; returns (n, start, end)."""
    n, start_at = task
    from oracle import dirac

    U, y = _CORE_INPUTS["U"], _CORE_INPUTS["y"]
    while time.time() < start_at:
        time.sleep(0.005)
    t0 = time.time()
    for _ in range(n):
        y = dirac.hermitian_wilson(U, y, M0, (1.0, 1.0, 1.0, -1.0))
    return n, t0, time.time()


class OracleCores:
    """The oracle's H_w on every host core at once: one process per core, started by spawn (so that no
    CUDA state is inherited), each holding the workload's inputs."""

    def __init__(self, cores=None):
        import multiprocessing as mp

        self.cores = cores or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_core_init)
        self.rate(1)  # every process has built its inputs

    def rate(self, n_per_core):
        """Wilson applications per second of the whole host, n_per_core applications on each core."""
        start_at = time.time() + 0.5
        res = self.pool.map(_oracle_core_worker, [(n_per_core, start_at)] * self.cores, chunksize=1)
        total = sum(r[0] for r in res)
        return total / (max(r[2] for r in res) - min(r[1] for r in res))

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_full_solve():
    """A whole solve by the oracle at a size it finishes in seconds: 2^4, links exp(i 0.3 H), the 8
    lowest |lambda| modes of Q exact (dense), Chebyshev degree 200 on [0.01, 1], m = 0.1, CGNE from
    x0 = 0 to a true residual of 1e-10 (the first configuration's solve, on the 2^4 lattice)."""
    import synth
    from oracle import dense
    from oracle import overlap as ov
    from oracle import solver

    dims, bcf = (2, 2, 2, 2), (1.0, 1.0, 1.0, -1.0)
    U = synth.random_su3_field(dims, 0.3, 0)
    t0 = time.perf_counter()
    H = dense.hw_matrix(U, M0, bcf)
    lam, W, _, _ = dense.low_modes(H, 6.5, 8)
    small = ov.SmallSpace.from_eigenpairs(dense.vectors_to_fields(W, synth.site_shape(dims)), lam)
    p = ov.OverlapParams(m0=M0, hw_norm=6.5, eps=0.01, degree=200, bc=bcf)
    b = synth.gaussian_spinor(dims, 1, 1)[0]
    _, iters, res = solver.cgne(lambda v: ov.overlap(U, v, 0.1, p, small),
                                lambda v: ov.overlap_dag(U, v, 0.1, p, small), b, tol=1e-10, check_every=10)
    return {"lattice": list(dims), "degree": 200, "n_ev": 8, "mass": 0.1, "seconds": time.perf_counter() - t0,
            "cgne_iterations": iters, "true_residual": res, "cores": 1}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    # every step: one bounded sample on every host core (2 oracle Wilson applications per core, one Y
    # of the polynomial), plus the projection once; scaled to D_ov applications
    _, t_w1 = oracle_sample(1)  # warm (imports, inputs) and the single-core projection time below
    from oracle import overlap as ov

    d = _oracle_inputs()
    tp0 = time.perf_counter()
    ov.project(d["small"], d["x"])
    t_p = time.perf_counter() - tp0
    oc = OracleCores()
    cores = oc.cores
    for _ in range(args.warmup):
        oc.rate(1)
    t0 = time.perf_counter()
    rates = [oc.rate(1) for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    oc.close()
    wilson_rate = sum(rates) / len(rates)
    value = 1.0 / ((2 * DEGREE + 1) / wilson_rate + t_p / cores)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": list(DIMS), "precision": "FP64 CPU oracle (numpy)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"per step: 1 oracle H_w application at 16^3x32 on each of {cores} cores at once "
                                   "(one process each) plus one 50-vector projection, scaled to "
                                   f"{2 * DEGREE + 1} Wilson applications per D_ov application",
                         "paper_context": PAPER_CORE_EQUIVALENCE},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def hbm_roofline(P, U_dims, peak, peak_kind, degree=100, reps=3):
    """Wilson kernel of the Clenshaw loop on a lattice whose working set is far beyond L2 (one
    right-hand side): CUDA events around each polynomial loop on its stream, algorithmic bytes per
    launch as in the library's profile (links once + every spinor stream).  FP32, FP16 and BF16."""
    import torch

    import synth

    U = torch.from_numpy(synth.random_su3_field(U_dims, LINK_EPS, 0)).cuda()
    x0 = torch.from_numpy(synth.gaussian_spinor(U_dims, 1, 1)).to(torch.complex64).cuda()
    out = {}
    for name, prec in (("f32", P.OV_PREC_F32), ("f16", P.OV_PREC_F16), ("bf16", P.OV_PREC_BF16)):
        ctx = P.Context(P.Params(dims=U_dims, bc=BC, m0=M0, eps=SQRT_EPS ** 2, poly_degree=degree, poly_kind=1,
                                 precision=prec, inner_precision=P.OV_PREC_F32, max_nrhs=1))
        ctx.set_gauge(U)
        y = torch.empty_like(x0)
        P.apply_sign_Hw(ctx, x0, y)  # launch shape timed, loop graph captured
        torch.cuda.synchronize()
        ctx.read_profile(prec)
        ctx.set_profiling(True)
        for _ in range(reps):
            P.apply_sign_Hw(ctx, x0, y)
        torch.cuda.synchronize()
        ctx.set_profiling(False)
        pr = ctx.read_profile(prec)
        achieved = pr["clenshaw_bytes"] / (pr["clenshaw_ms"] / 1e3) / 1e9
        per_launch = pr["clenshaw_bytes"] / pr["clenshaw_launches"]
        ratio = dram_ratio(f"{name}_24x24x24x48") if tuple(U_dims) == HBM_DIMS else None
        out[name] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": ratio * per_launch if ratio else None, "traffic_unit": "B/launch",
                     "peak_source": peak_kind, "avg_launch_us": 1e3 * pr["clenshaw_ms"] / pr["clenshaw_launches"],
                     "bytes_per_launch": per_launch, "launches": pr["clenshaw_launches"],
                     "launch_shape": ctx.tune_info}
        ctx.close()
    del U
    return out


def kernel_case(dims, precision="f32", shape=0):
    """A few Wilson-kernel launches (plain and Clenshaw-epilogue) on one lattice.

    The first D(m) application times the launch shapes and captures the loop's graph; the
    second, inside the NVTX range "kernel_case", runs the Clenshaw steps (plain, epilogue,
    ...) with the shape the library picked."""
    import torch

    import paper_1111_6288_gb300 as P
    import synth

    prec = {"f32": P.OV_PREC_F32, "f64": P.OV_PREC_F64, "f16": P.OV_PREC_F16, "bf16": P.OV_PREC_BF16}[precision]
    U = torch.from_numpy(synth.random_su3_field(dims, LINK_EPS, 0)).cuda()
    ctx = P.Context(P.Params(dims=dims, bc=BC, m0=M0, eps=SQRT_EPS ** 2, poly_degree=4, precision=prec,
                             inner_precision=P.OV_PREC_F64 if prec == P.OV_PREC_F64 else P.OV_PREC_F32,
                             max_nrhs=1, launch_shape=shape))
    ctx.set_gauge(U)
    del U
    x = torch.from_numpy(synth.gaussian_spinor(dims, 1, 1)).to(ctx.spinor_dtype()).cuda()
    y = torch.empty_like(x)
    P.apply_overlap(ctx, x, y, mass=MASS)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("kernel_case")
    P.apply_overlap(ctx, x, y, mass=MASS)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print("launch shapes timed:", ctx.tune_info)
    ctx.close()


# The paper's GPU-to-CPU-core equivalence, for context only (other hardware, other codes).
PAPER_CORE_EQUIVALENCE = ("about 30 Cray XT-5 cores per GPU for the paper's all-GPU code on its 2011 cluster "
                          "(6 GB per GPU, 16 GPUs, QDR InfiniBand; CPU runs on 256 cores): 34 for the H_w "
                          "eigensystem and 37 for the D_ov eigensystem (Sec. 3.1, abstract, conclusions)")

MULTI_MASSES = (0.02, 0.03, 0.045, 0.06, 0.08, 0.1, 0.15)  # a ladder of seven masses (Sec. 4 uses seven)


def multimass_case(n_defl):
    """Seven masses from one point source on the solve's workload (16^3x32, 50 H_w modes,
    n_defl D_ov low modes per sector, adaptive order, minimax polynomial): the multi-mass solve
    against single-mass solves of the same masses, all to 1e-10 true residual.  Prints one JSON
    object (a case study, not the bench line)."""
    import torch

    import paper_1111_6288_gb300 as P
    import synth

    torch.cuda.set_device(0)
    U = torch.from_numpy(synth.random_su3_field(DIMS, LINK_EPS, 0)).cuda()
    ctx = P.Context(P.Params(dims=DIMS, bc=BC, m0=M0, eps=SQRT_EPS ** 2, poly_degree=DEGREE, max_nrhs=2, poly_kind=1,
                             precision=P.OV_PREC_F32, inner_precision=P.OV_PREC_F32, adaptive_order=1))
    ctx.set_gauge(U)
    del U
    t0 = time.perf_counter()
    P.eigensolve_Q(ctx, N_EV, tol=1e-10, max_iter=200, register=True)
    for chi in (1, -1) if n_defl > 0 else ():
        P.eigensolve_overlap(ctx, n_defl, chirality=chi)
    setup_s = time.perf_counter() - t0
    print(f"multimass_case: setup {setup_s:.1f} s", flush=True)
    b = torch.from_numpy(synth.point_sources(DIMS, [(0, 0)])).cuda()
    x = torch.zeros_like(b)
    P.solve_overlap(ctx, b, x, MULTI_MASSES[0], tol=TOL)  # graphs, launch shapes
    torch.cuda.synchronize()
    X = torch.empty((len(MULTI_MASSES),) + tuple(b.shape), dtype=b.dtype, device=b.device)
    t0 = time.perf_counter()
    sts = P.solve_overlap_multimass(ctx, b, X, MULTI_MASSES, tol=TOL)
    torch.cuda.synchronize()
    t_multi = time.perf_counter() - t0
    info = ctx.last_info
    print(f"multimass_case: multi-mass {t_multi:.2f} s: {info}", flush=True)
    t_single, single, diff = 0.0, [], 0.0
    for i, m in enumerate(MULTI_MASSES):
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = P.solve_overlap(ctx, b, x, m, tol=TOL)
        torch.cuda.synchronize()
        t_single += time.perf_counter() - t0
        single.append(st)
        diff = max(diff, float((X[i] - x).norm() / x.norm()))
    out = {"multimass_case": {
        "workload": WORKLOAD, "masses": list(MULTI_MASSES), "n_defl_per_sector": n_defl, "setup_s": setup_s,
        "multi_s": t_multi, "single_s": t_single, "speedup": t_single / t_multi,
        "multi_sign_applies": sum(s.sign_applies for s in sts),
        "single_sign_applies": sum(s.sign_applies for s in single),
        "multi_wilson_applies": sum(s.dslash_calls for s in sts),
        "single_wilson_applies": sum(s.dslash_calls for s in single),
        "worst_true_residual": max(s.true_residual for s in sts + single),
        "max_rel_diff_multi_vs_single": diff, "multi_info": info,
        "single_inner_iters": [s.inner_iters for s in single]}}
    print(json.dumps(out), flush=True)
    ctx.close()


BATCH_DIMS = (24, 24, 24, 48)
BATCH_BC = (2, 0, 0, 2)  # Dirichlet x and t (the field direction and time, Sec. 4)
BATCH_CHARGES = (2.0 / 3.0, -1.0 / 3.0)


def batched_case(args):
    """The batched configuration (defaults: 24^3x48, links exp(i 0.2 H), minimax n = 527 on
    [4e-4, 1], m = 0.02; --batch-dims, --batch-link-eps, --batch-degree, --batch-sqrt-eps and
    --batch-mass change them), Dirichlet x and t, --batch-sources spin-colour point sources (12) at
    each of the field values E in --batch-fields (phases q E for q = 2/3, then -1/3, in that order;
    the first --batch-phases of them), the --batch-nev lowest |lambda| eigenvectors of Q per phase
    (eigensolver to 2e-6, an FP32-level bank; each phase after the first warm-started from the
    nearest bank), every right-hand side solved to 1e-10 in one solve_overlap call, in each inner
    precision of --batch-inner.  Against it: single-source solves of one source for each of the
    first --batch-single phases.  Prints one JSON object (a case study, not the bench line)."""
    import numpy as np
    import torch

    import paper_1111_6288_gb300 as P
    import synth

    torch.cuda.set_device(0)
    dims = tuple(int(v) for v in args.batch_dims.split(","))
    degree, sqrt_eps, mass, nsrc = args.batch_degree, args.batch_sqrt_eps, args.batch_mass, args.batch_sources
    fields = [float(v) for v in args.batch_fields.split(",")]
    phases = []
    for E in fields:
        for q in BATCH_CHARGES:
            ph = q * E
            if ph not in phases:
                phases.append(ph)
    phases = phases[:args.batch_phases]
    U = torch.from_numpy(synth.random_su3_field(dims, args.batch_link_eps, 0)).cuda()
    out = {"workload": f"{dims[0]}^3x{dims[3]} Dirichlet x,t, links exp(i {args.batch_link_eps} H), {nsrc} point sources x "
                       f"{len(phases)} field phases, N_ev {args.batch_nev}, n {degree} minimax on [{sqrt_eps ** 2:g}, 1], "
                       f"m {mass}, tol {TOL}", "phases": phases, "runs": {}}
    sc = [(s, c) for s in range(4) for c in range(3)][:nsrc]
    b1 = synth.point_sources(dims, sc)
    for inner in args.batch_inner.split(","):
        prec = {"f32": P.OV_PREC_F32, "f16": P.OV_PREC_F16, "bf16": P.OV_PREC_BF16}[inner]
        nrhs = nsrc * len(phases)
        ctx = P.Context(P.Params(dims=dims, bc=BATCH_BC, m0=M0, eps=sqrt_eps ** 2, poly_degree=degree,
                                 poly_kind=1, precision=prec, inner_precision=prec, max_nrhs=nrhs, adaptive_order=1))
        ctx.set_gauge(U)
        t0 = time.perf_counter()
        eig = []
        for ph in phases:
            t1 = time.perf_counter()
            lam, _ = P.eigensolve_Q(ctx, args.batch_nev, phase=ph, tol=2e-6, max_iter=300, register=True)
            eig.append({"phase": ph, "seconds": time.perf_counter() - t1, "lambda_min": float(abs(lam).min()),
                        "lambda_max": float(abs(lam).max()), "info": ctx.last_info})
            print(f"batched_case {inner}: eigensolver phase {ph:.3e}: {eig[-1]['seconds']:.1f} s", flush=True)
        setup_s = time.perf_counter() - t0
        free, total = torch.cuda.mem_get_info()
        used_after_eig = (total - free) / 1e9
        b = torch.from_numpy(np.concatenate([b1] * len(phases))).cuda()
        ph_rhs = [ph for ph in phases for _ in range(nsrc)]
        # single-source reference solves (one per phase; the first also times the launch shapes)
        single = []
        for ph in phases[:args.batch_single]:
            bs = b[:1].clone()
            xs = torch.zeros_like(bs)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            st = P.solve_overlap(ctx, bs, xs, mass, tol=TOL, phase=[ph])
            torch.cuda.synchronize()
            single.append({"phase": ph, "seconds": time.perf_counter() - t1, "outer": st.outer_iters,
                           "inner": st.inner_iters, "wilson": st.dslash_calls, "residual": st.true_residual})
            print(f"batched_case {inner}: single source phase {ph:.3e}: {single[-1]['seconds']:.1f} s", flush=True)
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = P.solve_overlap(ctx, b, x, mass, tol=TOL, phase=ph_rhs)
        e1.record()
        torch.cuda.synchronize()
        secs = e0.elapsed_time(e1) / 1e3
        free, total = torch.cuda.mem_get_info()
        applies = st.dslash_calls / (2 * degree + 1)
        single_per_source = sum(r["seconds"] for r in single) / len(single) if single else float("nan")
        out["runs"][inner] = {
            "setup_s": setup_s, "eigensolver": eig, "batch_seconds": secs, "nrhs": nrhs,
            "seconds_per_source": secs / nrhs, "single_source_seconds": single_per_source,
            "batch_speedup_per_source": single_per_source / (secs / nrhs),
            "dov_applies_per_s": applies / secs, "dov_applies_per_s_per_rhs": applies / secs / nrhs,
            "outer": st.outer_iters, "inner": st.inner_iters, "sign_applies": st.sign_applies,
            "worst_true_residual": st.true_residual, "cycles": ctx.last_info, "tuning": ctx.tune_info,
            "single": single, "device_gb_in_use": {"after_eigensolver": used_after_eig,
                                                   "after_solve": (total - free) / 1e9}}
        print(f"batched_case {inner}: {nrhs} rhs in {secs:.1f} s ({secs / nrhs:.2f} s per source, single "
              f"{single_per_source:.2f} s), residual {st.true_residual:.2e}", flush=True)
        ctx.close()
    print(json.dumps({"batched_case": out}), flush=True)


def projection_case(args):
    """The small-space projection alone (ov_project_small): a bank of --proj-nev FP32 vectors on the
    lattice --proj-dims and batches of --proj-k vectors (seeded Gaussian, drawn on the device), on the
    tensor cores (three calls first, the ones a profiler capture skips into) and on the CUDA cores,
    CUDA-event timed.  Prints one JSON object (a case study, not the bench line)."""
    import numpy as np
    import torch

    import paper_1111_6288_gb300 as P

    torch.cuda.set_device(0)
    dims = tuple(int(v) for v in args.proj_dims.split(","))
    ks = [int(v) for v in args.proj_k.split(",")]
    site = tuple(reversed(dims)) + (4, 3)
    ctx = P.Context(P.Params(dims=dims, eps=SQRT_EPS ** 2, poly_degree=4, precision=P.OV_PREC_F32,
                             inner_precision=P.OV_PREC_F32, max_nrhs=max(ks)))
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    V = torch.randn((args.proj_nev,) + site, dtype=torch.complex64, device="cuda", generator=g)
    P.deflate(ctx, V, np.linspace(-1.0, 1.0, args.proj_nev))
    del V
    out = {"lattice": list(dims), "n_ev": args.proj_nev, "bank_bytes": args.proj_nev * 12 * int(np.prod(dims)) * 8,
           "runs": {}}
    for k in ks:
        x = torch.randn((k,) + site, dtype=torch.complex64, device="cuda", generator=g)
        ys, xp = torch.empty_like(x), torch.empty_like(x)
        ms = {}
        for method, name in ((2, "tensor_cores"), (1, "cuda_cores")):
            ctx.set_projection(method)
            for _ in range(3):
                P.project_small(ctx, x, ys, xp)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                P.project_small(ctx, x, ys, xp)
            e1.record()
            torch.cuda.synchronize()
            ms[name] = e0.elapsed_time(e1) / 3
        P.sync(ctx)
        out["runs"][str(k)] = ms
        print(f"projection_case N {args.proj_nev} k {k}: tensor cores {ms['tensor_cores']:.2f} ms, "
              f"CUDA cores {ms['cuda_cores']:.2f} ms", flush=True)
        del x, ys, xp
    ctx.close()
    print(json.dumps({"projection_case": out}), flush=True)


def precision_case(args):
    """The bench's solve (16^3x32, 50 H_w modes, 32 D_ov low modes per chiral sector, adaptive order,
    minimax n = 527, m = 0.02, one point source, 1e-10) with each inner precision: FP32, FP16- and
    BF16-stored polynomial loops (FP32 arithmetic), and FP64 with the same algorithm.  Each 16-bit
    run uses a context of that storage (its 16-bit links) with the same bank and its own D_ov
    low modes.  Prints one JSON object (a case study, not the bench line)."""
    import torch

    import paper_1111_6288_gb300 as P
    import synth

    torch.cuda.set_device(0)
    U = torch.from_numpy(synth.random_su3_field(DIMS, LINK_EPS, 0)).cuda()
    common = dict(dims=DIMS, bc=BC, m0=M0, eps=SQRT_EPS ** 2, poly_degree=DEGREE, max_nrhs=2, poly_kind=1,
                  adaptive_order=1)
    c64 = P.Context(P.Params(precision=P.OV_PREC_F64, inner_precision=P.OV_PREC_F64, **common))
    c64.set_gauge(U)
    lam, V = P.eigensolve_Q(c64, N_EV, tol=1e-10, max_iter=200, register=False, want_vectors=True)
    c64.close()
    b = torch.from_numpy(synth.point_sources(DIMS, [(0, 0)])).cuda()
    out = {"workload": WORKLOAD, "runs": {}}
    for name, prec in (("f32", P.OV_PREC_F32), ("f16", P.OV_PREC_F16), ("bf16", P.OV_PREC_BF16)):
        ctx = P.Context(P.Params(precision=prec, inner_precision=prec, **common))
        ctx.set_gauge(U)
        P.deflate(ctx, V, lam)
        for chi in (1, -1):
            P.eigensolve_overlap(ctx, args.n_defl, chirality=chi)
        arms = [(name, prec)] + ([("f64_same_algorithm", P.OV_PREC_F64)] if name == "f32" else [])
        for arm, inner in arms:
            ctx.set_inner_precision(inner)
            x = torch.zeros_like(b)
            P.solve_overlap(ctx, b, x, MASS, tol=TOL)  # launch shapes, graphs
            times = []
            for _ in range(2):
                x.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st = P.solve_overlap(ctx, b, x, MASS, tol=TOL, raise_on_error=False)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
            out["runs"][arm] = {"seconds": min(times), "status": st.status, "outer": st.outer_iters,
                                "inner": st.inner_iters, "sign_applies": st.sign_applies,
                                "true_residual": st.true_residual, "cycles": ctx.last_info}
            print(f"precision_case {arm}: {min(times):.2f} s, {st.outer_iters} outer, {st.inner_iters} inner, "
                  f"residual {st.true_residual:.2e}", flush=True)
        ctx.close()
    print(json.dumps({"precision_case": out}), flush=True)


def derivative_case(args):
    """The field derivative at the configuration of the background-field runs: 16^3x32, Dirichlet x and
    t, links exp(i 0.2 H), 50 eigenvectors of Q per phase (recomputed at every phase), minimax n = 527 on
    [4e-4, 1], m = 0.02, the 12 spin-colour point sources at (8, 0, 0, 8), charge 2/3, E = 1e-4.
    dC(t)/dE by the tangent solve (ov_dcorr_dE) against central differences of C at E +- h for
    h = 1e-5 and 5e-6 (solves to 1e-13, the eigen-split recomputed at each E), with the Richardson
    estimate and the difference of the two steps as the finite difference's noise floor; then the
    derivative from solves to 1e-6 with FP32 and with BF16-stored inner CGs, with their error against
    the 1e-13 one.  Prints one JSON object (a case study, not the bench line)."""
    import numpy as np
    import torch

    import paper_1111_6288_gb300 as P
    import synth

    torch.cuda.set_device(0)
    dims, bc, charge, E, h = DIMS, (2, 0, 0, 2), 2.0 / 3.0, 1e-4, 1e-5
    U = torch.from_numpy(synth.random_su3_field(dims, LINK_EPS, 0)).cuda()
    src = torch.from_numpy(synth.point_sources(dims, site=(8, 0, 0, 8))).cuda()
    Es = [E, E + h, E - h, E + h / 2, E - h / 2]
    out = {"workload": f"16^3x32 Dirichlet x,t, 12 point sources, N_ev {args.deriv_nev}, n {DEGREE}, m {MASS}, "
                       f"q {charge:.4f}, E {E}", "steps": [h, h / 2]}
    t0 = time.perf_counter()

    def context(prec, inner):
        ctx = P.Context(P.Params(dims=dims, bc=bc, m0=M0, eps=SQRT_EPS ** 2, poly_degree=DEGREE, poly_kind=1,
                                 precision=prec, inner_precision=inner, max_nrhs=12, adaptive_order=1))
        ctx.set_gauge(U)
        return ctx

    ctx = context(P.OV_PREC_F64, P.OV_PREC_F32)
    banks = {}
    for e in Es:
        lam, V = P.eigensolve_Q(ctx, args.deriv_nev, phase=charge * e, tol=1e-11, max_iter=300, register=True,
                                want_vectors=True)
        banks[e] = (lam, V)
    out["setup_s"] = time.perf_counter() - t0
    print(f"derivative_case: banks for {len(Es)} phases in {out['setup_s']:.1f} s", flush=True)
    t1 = time.perf_counter()
    C0, dC = P.correlator_jacobian(ctx, src, E, charge, MASS, tol=1e-13)
    out["tangent_s"] = time.perf_counter() - t1
    Cs = {}
    for e in Es[1:]:
        x = torch.zeros_like(src)
        P.solve_overlap(ctx, src, x, MASS, tol=1e-13, phase=[charge * e] * 12)
        Cs[e] = P.correlator(ctx, x)
    fd1 = (Cs[E + h] - Cs[E - h]) / (2 * h)
    fd2 = (Cs[E + h / 2] - Cs[E - h / 2]) / h
    rich = (4 * fd2 - fd1) / 3
    scale = float(np.abs(fd1).max())
    out.update({"C": C0.tolist(), "dC_dE": dC.tolist(), "fd_h": fd1.tolist(), "fd_h2": fd2.tolist(),
                "rel_err_vs_fd_h": float(np.abs(dC - fd1).max()) / scale,
                "rel_err_vs_fd_h2": float(np.abs(dC - fd2).max()) / scale,
                "rel_err_vs_richardson": float(np.abs(dC - rich).max()) / scale,
                "fd_noise_floor": float(np.abs(fd1 - fd2).max()) / scale,
                "max_abs_dC": float(np.abs(dC).max()), "max_abs_C": float(np.abs(C0).max())})
    print(f"derivative_case: dC/dE vs FD: {out['rel_err_vs_fd_h']:.2e} (h), {out['rel_err_vs_fd_h2']:.2e} (h/2), "
          f"{out['rel_err_vs_richardson']:.2e} (Richardson); FD noise floor {out['fd_noise_floor']:.2e}", flush=True)
    ctx.close()
    # lower-precision variants: solves to 1e-6 with FP32 / BF16-stored inner CGs, same banks
    variants = {}
    for name, prec in (("f32", P.OV_PREC_F32), ("bf16", P.OV_PREC_BF16)):
        cv = context(prec, prec)
        lam, V = banks[E]
        P.deflate(cv, V, lam, phase=charge * E)
        t1 = time.perf_counter()
        Cv, dCv = P.correlator_jacobian(cv, src, E, charge, MASS, tol=1e-6)
        variants[name] = {"seconds": time.perf_counter() - t1,
                          "rel_err_dC_vs_f64": float(np.abs(dCv - dC).max()) / float(np.abs(dC).max()),
                          "rel_err_C_vs_f64": float(np.abs(Cv - C0).max()) / float(np.abs(C0).max()),
                          "rel_err_dC_vs_fd_h": float(np.abs(dCv - fd1).max()) / scale}
        print(f"derivative_case {name}: {variants[name]}", flush=True)
        cv.close()
    out["variants"] = variants
    print(json.dumps({"derivative_case": out}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64-solve", action="store_true", help="skip the FP64-only comparison solve")
    ap.add_argument("--fixed-order", action="store_true",
                    help="inner solves at the full polynomial degree (default: adaptive order per outer cycle)")
    ap.add_argument("--n-defl", type=int, default=N_DEFL,
                    help="D_ov low modes per chiral sector for the CG deflation (0: none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel-case", action="store_true",
                    help="profiling case: a few FP32 Wilson-kernel launches (default 24^3x48), "
                         "then exit without a JSON line")
    ap.add_argument("--kernel-dims", default="24,24,24,48", help="lattice of the profiling case: Lx,Ly,Lz,Lt")
    ap.add_argument("--kernel-precision", default="f32", choices=["f32", "f64", "f16", "bf16"],
                    help="precision of the profiling case")
    ap.add_argument("--kernel-shape", type=int, default=0,
                    help="launch shape of the profiling case (ov_params.launch_shape; 0 = timed by the library)")
    ap.add_argument("--batched-case", action="store_true",
                    help="case study: the batched 24^3x48 configuration (point sources x field phases in one "
                         "solve), then exit without a bench line")
    ap.add_argument("--batch-fields", default="0,1e-4", help="field values E of the batched case")
    ap.add_argument("--batch-phases", type=int, default=2, help="distinct phases q E used (first ones)")
    ap.add_argument("--batch-nev", type=int, default=100, help="eigenvectors of Q per phase")
    ap.add_argument("--batch-inner", default="f32", help="inner precisions of the batched case (f32,f16,bf16)")
    ap.add_argument("--batch-dims", default="24,24,24,48", help="lattice of the batched case")
    ap.add_argument("--batch-link-eps", type=float, default=LINK_EPS, help="link spread of the batched case")
    ap.add_argument("--batch-degree", type=int, default=DEGREE, help="polynomial degree of the batched case")
    ap.add_argument("--batch-sqrt-eps", type=float, default=SQRT_EPS, help="sqrt(eps) of the batched case")
    ap.add_argument("--batch-mass", type=float, default=MASS, help="quark mass of the batched case")
    ap.add_argument("--batch-sources", type=int, default=12, help="spin-colour point sources per field phase")
    ap.add_argument("--batch-single", type=int, default=2, help="phases with a single-source reference solve")
    ap.add_argument("--projection-case", action="store_true",
                    help="case study: the small-space projection on the tensor cores and on the CUDA cores, then "
                         "exit without a bench line")
    ap.add_argument("--proj-dims", default="24,24,24,48", help="lattice of the projection case")
    ap.add_argument("--proj-nev", type=int, default=100, help="bank size of the projection case")
    ap.add_argument("--proj-k", default="8,12,24,32", help="batch sizes of the projection case")
    ap.add_argument("--precision-case", action="store_true",
                    help="case study: the bench's solve with FP32, FP16-, BF16-stored and FP64 inner CGs, then "
                         "exit without a bench line")
    ap.add_argument("--derivative-case", action="store_true",
                    help="case study: dC/dE at 16^3x32 against central finite differences in E, then exit "
                         "without a bench line")
    ap.add_argument("--deriv-nev", type=int, default=50, help="eigenvectors of Q per phase in the derivative case")
    ap.add_argument("--multimass-case", action="store_true",
                    help="case study: seven masses by the multi-mass solve against single-mass solves, "
                         "then exit without a bench line")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.multimass_case:
        multimass_case(args.n_defl)
        return
    if args.batched_case:
        batched_case(args)
        return
    if args.derivative_case:
        derivative_case(args)
        return
    if args.precision_case:
        precision_case(args)
        return
    if args.projection_case:
        projection_case(args)
        return
    if args.kernel_case:
        kernel_case(tuple(int(v) for v in args.kernel_dims.split(",")), args.kernel_precision, args.kernel_shape)
        return

    import numpy as np
    import torch

    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import paper_1111_6288_gb300 as P

    if not os.path.exists(P.library_path()):
        from paper_1111_6288_gb300 import build as _b

        _b.build()
    import synth

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    U = torch.from_numpy(synth.random_su3_field(DIMS, LINK_EPS, 0)).to(dev)
    # the minimax polynomial: delta(527) = 1.17e-10, the configuration's 1e-10 at order ~530 (eq. 2)
    common = dict(dims=DIMS, bc=BC, m0=M0, eps=SQRT_EPS ** 2, poly_degree=DEGREE, max_nrhs=2, poly_kind=1)
    ctx_mix = P.Context(P.Params(precision=P.OV_PREC_F32, inner_precision=P.OV_PREC_F32,
                                 adaptive_order=0 if args.fixed_order else 1, **common))
    ctx_64 = P.Context(P.Params(precision=P.OV_PREC_F64, inner_precision=P.OV_PREC_F64, **common))
    ctx_mix.set_gauge(U)
    ctx_64.set_gauge(U)
    t0 = time.perf_counter()
    lam, V = P.eigensolve_Q(ctx_64, N_EV, tol=1e-10, max_iter=200, register=True, want_vectors=True)
    t_eig = time.perf_counter() - t0
    eig_info = ctx_64.last_info
    P.deflate(ctx_mix, V, lam)
    defl_info = None
    if args.n_defl > 0:
        t1 = time.perf_counter()
        modes, lanczos = {}, []
        for chi in (1, -1):
            modes[chi] = P.eigensolve_overlap(ctx_mix, args.n_defl, chirality=chi)
            lanczos.append(ctx_mix.last_info)
        defl_info = {"seconds": time.perf_counter() - t1, "n_per_sector": args.n_defl, "lanczos": lanczos,
                     "ritz_range": [float(min(m[0][0] for m in modes.values())),
                                    float(max(m[0][-1] for m in modes.values()))],
                     "worst_residual": float(max(m[1].max() for m in modes.values()))}
    # 16-bit storage of links and recurrence vectors (FP32 arithmetic): isolated D(m) rate and error
    ctx_half = {}
    for name, prec in (("f16", P.OV_PREC_F16), ("bf16", P.OV_PREC_BF16)):
        ctx_half[name] = P.Context(P.Params(precision=prec, inner_precision=P.OV_PREC_F32, **common))
        ctx_half[name].set_gauge(U)
        P.deflate(ctx_half[name], V, lam)
    del V
    # replicas solve different spin-colour point sources
    sc = (rank % 4, (rank // 4) % 3)
    b = torch.from_numpy(synth.point_sources(DIMS, [sc])).to(dev)
    x = torch.zeros_like(b)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def step(ctx):
        flush.zero_()
        x.zero_()
        return P.solve_overlap(ctx, b, x, MASS, tol=TOL)

    for _ in range(args.warmup):
        step(ctx_mix)
    torch.cuda.synchronize()

    # ---- timed region: K mixed-precision solves ----
    ctx_mix.read_profile(P.OV_PREC_F32)
    ctx_mix.read_profile(P.OV_PREC_F64)
    ctx_mix.set_profiling(True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    launches0 = P.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    ev0.record(stream)
    stats = [step(ctx_mix) for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    launches = P.launch_count() - launches0
    mixed_cycles = ctx_mix.last_info  # before later calls on this context replace it
    barrier(world)
    clk = clocks.stop()
    ctx_mix.set_profiling(False)
    prof32 = ctx_mix.read_profile(P.OV_PREC_F32)
    prof64 = ctx_mix.read_profile(P.OV_PREC_F64)
    local_ms = ev0.elapsed_time(ev1)
    # D_ov applications at the full degree n: Wilson applications / (2n + 1), so that the lower
    # degrees of the adaptive order's inner cycles count for the work they do
    per_apply = 2 * DEGREE + 1
    applies = float(sum(s.dslash_calls for s in stats)) / per_apply
    max_ms, total_applies = aggregate(local_ms, applies, world)
    value = total_applies / (max_ms / 1e3)
    worst_res = max(s.true_residual for s in stats)

    # ---- end to end: host (pinned) b in, host x out, through the public API ----
    b_host = b.cpu().pin_memory()
    x_host = torch.empty_like(b_host).pin_memory()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_applies = 0.0
    for _ in range(args.steps):
        flush.zero_()
        b.copy_(b_host, non_blocking=True)
        x.zero_()
        st = P.solve_overlap(ctx_mix, b, x, MASS, tol=TOL)
        x_host.copy_(x, non_blocking=True)
        e2e_applies += st.dslash_calls / per_apply
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms, e2e_total = aggregate(e0.elapsed_time(e1), e2e_applies, world)
    nbytes = b.numel() * b.element_size()

    # ---- isolated operator applications ----
    def dov_rate(ctx, reps):
        xi = b.to(ctx.spinor_dtype())
        yi = torch.empty_like(xi)
        P.apply_overlap(ctx, xi, yi, mass=MASS)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(reps):
            P.apply_overlap(ctx, xi, yi, mass=MASS)
        a1.record(stream)
        torch.cuda.synchronize()
        return reps / (a0.elapsed_time(a1) / 1e3)

    rate32 = dov_rate(ctx_mix, 5)
    rate64 = dov_rate(ctx_64, 2)
    rates_half = {name: dov_rate(c, 5) for name, c in ctx_half.items()}

    # error of one D(m) application on a Gaussian vector against the FP64 path (max |diff| / max |FP64|)
    xg = torch.from_numpy(synth.gaussian_spinor(DIMS, 1, 7)).to(dev)
    y64 = torch.empty_like(xg)
    P.apply_overlap(ctx_64, xg, y64, mass=MASS)
    errors = {}
    for name, c in [("f32", ctx_mix)] + list(ctx_half.items()):
        x32 = xg.to(torch.complex64)
        y = torch.empty_like(x32)
        P.apply_overlap(c, x32, y, mass=MASS)
        errors[name] = float((y.to(torch.complex128) - y64).abs().max() / y64.abs().max())
    for c in ctx_half.values():
        c.close()

    # ---- FP64-only solve (time-to-solution comparison) ----
    fp64 = None
    if not args.no_fp64_solve:
        flush.zero_()
        x.zero_()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        st64 = P.solve_overlap(ctx_64, b, x, MASS, tol=TOL)
        f1.record(stream)
        torch.cuda.synchronize()
        fp64 = {"seconds": f0.elapsed_time(f1) / 1e3, "outer_iters": st64.outer_iters,
                "inner_iters": st64.inner_iters, "sign_applies": st64.sign_applies,
                "true_residual": st64.true_residual}

    # ---- FP64 inner CG with the mixed solve's algorithm (the same D_ov deflation spaces, in their FP64
    # vectors, and the adaptive order): separates what precision buys from what the algorithm buys ----
    fp64_same = None
    if not args.no_fp64_solve:
        ctx_mix.set_inner_precision(P.OV_PREC_F64)
        flush.zero_()
        x.zero_()
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        stf = P.solve_overlap(ctx_mix, b, x, MASS, tol=TOL)
        g1.record(stream)
        torch.cuda.synchronize()
        fp64_same = {"seconds": g0.elapsed_time(g1) / 1e3, "outer_iters": stf.outer_iters,
                     "inner_iters": stf.inner_iters, "sign_applies": stf.sign_applies,
                     "true_residual": stf.true_residual, "cycles": ctx_mix.last_info}
        ctx_mix.set_inner_precision(P.OV_PREC_F32)

    # ---- roofline of the dominant kernel: the FP32 Wilson kernel of the Clenshaw loops ----
    peak, peak_kind = measured_peaks()
    roof_hbm = hbm_roofline(P, HBM_DIMS, peak, peak_kind)
    achieved = prof32["clenshaw_bytes"] / (prof32["clenshaw_ms"] / 1e3) / 1e9 if prof32["clenshaw_ms"] > 0 else 0.0
    bytes_per_launch = prof32["clenshaw_bytes"] / max(prof32["clenshaw_launches"], 1)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                # DRAM bytes per launch: ncu's DRAM bytes of this kernel on this lattice over its algorithmic
                # bytes, scaled to this launch mix (None once the kernel has changed since the capture)
                "traffic": (dram_ratio("f32_16x16x16x32_solve") * bytes_per_launch
                            if dram_ratio("f32_16x16x16x32_solve") else None),
                "traffic_unit": "B/launch",
                "peak_source": peak_kind,
                "kernel": "dslash_kernel<float> (Clenshaw step launches, 16^3x32, 1-2 systems per launch)",
                "note": ("L2-resident effective bandwidth: at 16^3x32 the loop's links (25 MB) and vectors (12.6 MB "
                         "each) stay in the 129 MB L2, so this is algorithmic bytes over time against the HBM "
                         "peak; roofline_hbm holds the HBM-bound measurement"),
                "avg_launch_us": 1e3 * prof32["clenshaw_ms"] / max(prof32["clenshaw_launches"], 1),
                "bytes_per_launch": bytes_per_launch,
                "clenshaw_share_of_step": prof32["clenshaw_ms"] / local_ms}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_apply, t_w = oracle_sample(2)
        oc = OracleCores()
        wilson_rate, cores = oc.rate(2), oc.cores
        oc.close()
        from oracle import overlap as ov

        d = _oracle_inputs()
        tp0 = time.perf_counter()
        ov.project(d["small"], d["x"])
        t_p = time.perf_counter() - tp0
        all_value = 1.0 / ((2 * DEGREE + 1) / wilson_rate + t_p / cores)
        cpu = {"value": all_value, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"2 oracle H_w applications at 16^3x32 on each of {cores} host cores at once (one process "
                         f"each) plus one 50-vector projection, scaled to {2 * DEGREE + 1} Wilson applications per "
                         "D_ov application",
               "one_core": {"value": 1.0 / t_apply, "unit": UNIT,
                            "sample": f"2 oracle H_w applications ({t_w:.2f} s each) plus the projection"},
               "full_solve": oracle_full_solve(),
               "gpu_over_oracle_all_cores": value / all_value, "gpu_over_oracle_core": value * t_apply,
               "paper_context": PAPER_CORE_EQUIVALENCE}

    if rank == 0:
        mean_mixed_s = max_ms / 1e3 / args.steps
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": list(DIMS), "links": f"exp(i {LINK_EPS} H), seed 0",
                       "m0": M0, "poly_degree": DEGREE, "poly": "minimax (Remez), delta = %.2e" % ctx_mix.delta,
                       "sqrt_eps": SQRT_EPS, "n_ev": N_EV, "mass": MASS,
                       "tol": TOL, "precision": "FP32 inner CG and Clenshaw, FP64 true residual and update",
                       "polynomial": (f"n = {DEGREE} everywhere" if args.fixed_order else
                                      f"n = {DEGREE} in every true residual; each inner cycle at the lowest degree "
                                      "with delta <= 0.5 m g (adaptive order)"),
                       "value_unit": f"D_ov applications at n = {DEGREE}: Wilson applications / {2 * DEGREE + 1}",
                       "deflation": (f"{args.n_defl} low modes of D_ov per chiral sector (setup) deflate the inner CG"
                                     if args.n_defl > 0 else "none"),
                       "parallelism": f"replicas x{world}", "l2": "256 MB flush before every step"},
            "time_to_solution": {"mixed_s": mean_mixed_s, "fp64_s": fp64["seconds"] if fp64 else None,
                                 "speedup": (fp64["seconds"] / mean_mixed_s) if fp64 else None,
                                 "fp64_same_algorithm_s": fp64_same["seconds"] if fp64_same else None,
                                 "speedup_precision_only": (fp64_same["seconds"] / mean_mixed_s) if fp64_same else None,
                                 "fp64_same_algorithm": fp64_same,
                                 "mixed_outer_iters": stats[0].outer_iters, "mixed_inner_iters": stats[0].inner_iters,
                                 "mixed_sign_applies": stats[0].sign_applies,
                                 "mixed_wilson_applies": stats[0].dslash_calls,
                                 "mixed_cycles": mixed_cycles,
                                 "mixed_true_residual": worst_res, "fp64": fp64},
            "dov_apply_per_s": {"f32": rate32, "f64": rate64, **rates_half},
            "dov_error_vs_f64": errors,
            "dslash_gbs": achieved,
            "roofline": roofline,
            "roofline_hbm": {"lattice": list(HBM_DIMS), "kernel": "dslash_kernel (Clenshaw loop, n = 100, one rhs)",
                             **roof_hbm["f32"], "f16": roof_hbm["f16"], "bf16": roof_hbm["bf16"]},
            "clocks": clk,
            "e2e": {"value": e2e_total / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes},
            "gpu_launches": launches,
            "cpu_baseline": cpu,
            "setup": {"eigensolver_s": t_eig, "eigensolver": eig_info, "dov_low_modes": defl_info, "hw_norm": ctx_mix.hw_norm, "lambda_min": float(abs(lam).min()),
                      "lambda_max_in_bank": float(abs(lam).max())},
        }
        print(json.dumps(line))
    ctx_mix.close()
    ctx_64.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
