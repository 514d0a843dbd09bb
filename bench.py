#!/usr/bin/env python
"""Benchmark: MG-GCR solve time to 1e-10 vs plain FP64 EO-GCR on GB300, and the
fine dslash as a fraction of HBM peak.

Workload (one step = one MG-GCR solve of one right-hand side to a true
relative residual of 1e-10, setup excluded and timed separately): the
16^3x32 Wilson-clover lattice with links exp(i eps H), eps = 0.25, H
Gaussian traceless Hermitian, 5 APE steps (alpha = 0.5), csw = 1.0, at the
lightest mass of the sweep, m0 = -0.35; 2-level multigrid with 4^4 blocks
and Nv = 24 null vectors; FP32 preconditioner, FP64 outer GCR.

Prints one JSON line (rank 0).  Under torchrun every rank solves its own
replica of the workload on its own GPU (no data-path collective); timings
are the max over ranks.  ``--impl reference`` times the FP64 CPU oracle on
the host cores instead (a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MG-GCR solve time to 1e-10 vs plain EO-GCR on GB300; dslash % HBM peak"
DIMS = (16, 16, 16, 32)
EPS, APE, ALPHA, CSW = 0.25, 5, 0.5, 1.0
MASSES = (-0.2, -0.3, -0.35)
GAUGE_SEED, SOURCE_SEED, NULLVEC_SEED = 2001, 2002, 2003
# the paper's coarse tolerance 0.1 (a sweep of 0.05 ... 0.3 on GB300 with the
# streamed coarsest solver is flat within 2% between 0.1 and 0.3); 0.3 is timed
# beside it as extra.coarse_tolerance
MG = dict(levels=2, blocks=[(4, 4, 4, 4)], nv=[24], tol_coarse=0.1, restart_coarse=64)
ALT_COARSE_TOL = 0.3
TOL = 1e-10
HBM_DIMS = (32, 32, 32, 64)          # 1.1 GB per FP32 fused-dslash launch: far beyond the 129 MB L2
L2_FLUSH_BYTES = 512 << 20
# The CPU oracle sample: the oracle's complete MG-GCR on an 8^4 lattice of the
# same construction and parameters (4^4 blocks, Nv = 24), its setup cut to 4
# inverse-iteration passes per vector to bound the sample; one process per host
# core (independent sources), so that all cores work.  The per-outer-iteration
# cost (fine and coarse work) is projected to the 16^3x32 workload by volume.
CPU_DIMS = (8, 8, 8, 8)
CPU_SETUP_ITERS = 4
CPU_STEP_ITERS = 2                   # outer iterations per step of the reference arm
CPU_MAX_PROCS = 16
BATCH_RHS = 12                       # right-hand sides of the batched solve
MRHS = (4, 12)                       # right-hand sides of the multi-RHS D_r measurements
PROFILE_MRHS = 4                     # --profile dslash_mrhs: right-hand sides per launch
PROFILE_MRHS_DIMS = (32, 32, 32, 32) # ... on a lattice that keeps an ncu capture to a few GB
# outer iterations of the GPU arm's MG-GCR solve of the 16^3x32 workload at
# m0 = -0.35 on GB300 (coarse tolerance 0.1): projects the reference arm's
# per-iteration sample to one solve
REFERENCE_OUTER_PER_SOLVE = 42
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the FP32 fused
# dslash on 32^3x64, from the ncu capture in profiles/dslash_fp32_32x32x32x64.md
# (set to None whenever that kernel changes)
DSLASH_TRAFFIC_BYTES = 1.125e9
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the streamed
# coarsest-level solve on this workload (None whenever that kernel changes)
COARSE_TRAFFIC_BYTES = 79.13e6        # profiles/coarse_gcr_stream_4x4x4x8.md: 76.46 MB read + 2.67 MB written
                                      # per launch of COARSE_PROFILE_ITERS iterations (the links' first touch
                                      # after the fine-level work; L2 hits afterwards)
DSLASH_FLOPS_PER_SITE = 1824        # fused hop + clover inverse, per output site
COARSE_PROFILE_ITERS = 34            # --profile coarse: GCR iterations per launch (the step's average)


SECTIONS = {}                        # wall seconds of the bench's sections (reported in the JSON line)


def workload_name(m0):
    return (f"wilson-clover {DIMS[0]}^3x{DIMS[3]}, eps={EPS}+{APE} APE(alpha={ALPHA}), csw={CSW}, m0={m0}, "
            f"2-level MG 4^4 blocks Nv=24, tol 1e-10")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------- distributed plumbing
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as td
            td.init_process_group(backend="gloo")  # barrier and timing reductions only
            self.pg = td

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ----------------------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle sample
def oracle_worker(job):
    """One host process: the oracle's multigrid on CPU_DIMS (setup with
    CPU_SETUP_ITERS passes), then either one complete solve ("solve") or
    `steps` samples of CPU_STEP_ITERS outer iterations ("steps").  Runs in a
    spawned process with one thread."""
    mode, seed, steps, dims = job
    from oracle.dirac import WilsonClover
    from oracle.multigrid import MGParams, Multigrid
    from paper_1011_2775_gb300 import inputs as I
    U = I.make_gauge(dims, EPS, APE, ALPHA, GAUGE_SEED)
    W = WilsonClover(U, CSW, MASSES[-1])
    if mode == "dr":   # `steps` applications of the oracle's D_r on even-site vectors
        y = I.gaussian_source(dims, SOURCE_SEED + seed).reshape(W.shape + (12,)) * W.even
        W.Dr(y)
        times = []
        for _ in range(steps):
            t0 = time.perf_counter()
            W.Dr(y)
            times.append(time.perf_counter() - t0)
        return {"dr_s": statistics.median(times)}
    prm = MGParams(blocks=[(4, 4, 4, 4)], nv=[24], tol_coarse=MG["tol_coarse"], restart_coarse=MG["restart_coarse"],
                   setup_iters=CPU_SETUP_ITERS, seed=NULLVEC_SEED)
    t0 = time.perf_counter()
    mg = Multigrid(W, prm)
    setup_s = time.perf_counter() - t0
    eta = I.gaussian_source(dims, SOURCE_SEED + seed).reshape(W.shape + (12,))
    if mode == "solve":
        t0 = time.perf_counter()
        _, info = mg.solve(eta, TOL)
        dt = time.perf_counter() - t0
        return {"setup_s": setup_s, "solve_s": dt, "outer_iterations": info.outer_iterations,
                "true_residual": info.true_residual}
    mg.params.maxit_fine = CPU_STEP_ITERS
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        mg.solve(eta, TOL, max_attempts=1)
        times.append(time.perf_counter() - t0)
    return {"setup_s": setup_s, "step_s": times}


def oracle_pool(jobs):
    """Runs the jobs in spawned single-thread processes, one per host core (at most CPU_MAX_PROCS)."""
    import multiprocessing as mp
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        return pool.map(oracle_worker, jobs)


def links_worker(job):
    """exp(i eps H) on one block of time slices (site-local), in a spawned process."""
    from paper_1011_2775_gb300 import inputs as I
    h, eps = job
    return I.links_from_normals(h, eps)


def ape_worker(job):
    """One APE step on a block of time slices carrying one halo slice on each
    side; returns the block's own slices."""
    from paper_1011_2775_gb300 import inputs as I
    u, alpha = job
    return I.ape_step(u, alpha)[1:-1]


def parallel_gauge(pool, nproc: int, spec) -> "np.ndarray":
    """make_gauge(*spec) with the site-local link construction and every APE
    step split into blocks of time slices over the pool's processes: the same
    operations on the same numbers, so the same field."""
    import numpy as np
    from paper_1011_2775_gb300 import inputs as I
    dims, eps, ape_steps, alpha, seed = spec
    lt = dims[3]
    cuts = np.linspace(0, lt, min(nproc, lt) + 1).astype(int)
    blocks = [(a, b) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
    h = I.gauge_normals(dims, seed)
    u = np.concatenate(pool.map(links_worker, [(h[a:b], eps) for a, b in blocks]), axis=0)
    del h
    for _ in range(int(ape_steps)):
        jobs = [(np.take(u, np.arange(a - 1, b + 1), axis=0, mode="wrap"), alpha) for a, b in blocks]
        u = np.concatenate(pool.map(ape_worker, jobs), axis=0)
    return np.ascontiguousarray(u)


def big_fields(specs, nproc: int = 0) -> dict:
    """The large synthetic gauge fields of the extra configurations, each built
    by parallel_gauge over spawned processes (the fields make_gauge gives),
    keyed by their spec."""
    import multiprocessing as mp
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    n = nproc or host_cores()
    out = {}
    with mp.get_context("spawn").Pool(n) as pool:
        for sp in dict.fromkeys(specs):
            out[sp] = parallel_gauge(pool, n, sp)
    return out


def extra_field_specs() -> list:
    """Specs (dims, eps, ape_steps, alpha, seed) of the fields run_multi and run_config3 use."""
    return ([(dims, EPS, APE, ALPHA, 4001 + 10 * k) for k, (dims, _, _) in enumerate(MULTI)] +
            [(CONFIG3_DIMS, eps, APE, ALPHA, 3001) for eps in (EPS, ROUGH_EPS)])


def host_cores(limit: int = 0) -> int:
    n = max(1, min(CPU_MAX_PROCS, os.cpu_count() or 1))
    return min(n, limit) if limit > 0 else n


def cpu_baseline(gpu_outer: int, gpu_small_ms: float) -> dict:
    """The oracle's complete MG-GCR solve of CPU_DIMS in every host process at
    once; the per-outer-iteration wall time (fine and coarse work), divided by
    the processes working concurrently, projected to one solve of the
    16^3x32 workload by volume and the GPU's outer-iteration count."""
    n = host_cores()
    res = oracle_pool([("solve", q, 0, CPU_DIMS) for q in range(n)])
    per_it = statistics.median(r["solve_s"] / r["outer_iterations"] for r in res)
    vol = (DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3]) / (CPU_DIMS[0] * CPU_DIMS[1] * CPU_DIMS[2] * CPU_DIMS[3])
    value = 1e3 * per_it * vol * gpu_outer / n
    # the oracle's fine D_r on the 16^3x32 workload: one process alone, then one per core at once
    one = oracle_pool([("dr", 0, 2, DIMS)])[0]["dr_s"]
    alln = oracle_pool([("dr", q, 2, DIMS) for q in range(n)])
    per_all = statistics.median(r["dr_s"] for r in alln)
    return {"value": value, "unit": "ms", "cores": n, "kind": "oracle",
            "dr_16x16x16x32": {"single_core_ms": 1e3 * one, "all_cores_ms_per_apply": 1e3 * per_all / n,
                               "processes": n},
            "sample": (f"{n} concurrent single-thread processes, each the oracle's complete MG-GCR solve (setup "
                       f"{CPU_SETUP_ITERS} passes per vector, then to 1e-10) of an 8^4 lattice of the same "
                       f"construction and parameters (4^4 blocks, Nv=24); projection: median wall time per outer "
                       f"iteration x {vol:.0f} (volume) x {gpu_outer} (outer iterations of the GPU solve) / {n} "
                       f"(processes)"),
            "measured_8x8x8x8": {"solve_ms_median": 1e3 * statistics.median(r["solve_s"] for r in res),
                                 "setup_ms_median": 1e3 * statistics.median(r["setup_s"] for r in res),
                                 "outer_iterations": [r["outer_iterations"] for r in res],
                                 "true_residual_max": max(r["true_residual"] for r in res),
                                 "gpu_solve_ms_same_config": gpu_small_ms}}


def profile_main(args):
    import numpy as np
    import torch
    from paper_1011_2775_gb300 import binding as B
    from paper_1011_2775_gb300 import build as build_mod
    from paper_1011_2775_gb300 import inputs as I
    from paper_1011_2775_gb300.solver import Solver

    build_mod.build()
    U = I.make_gauge(DIMS, EPS, APE, ALPHA, GAUGE_SEED)
    if args.profile == "solve":
        eta = torch.from_numpy(I.gaussian_source(DIMS, SOURCE_SEED)).cuda()
        psi = torch.zeros_like(eta)
        S = Solver(DIMS)
        S.load_gauge(U)
        S.set_clover(CSW, args.mass)
        S.set_params(seed=NULLVEC_SEED, maxit_fine=2000, **MG)
        S.setup()
        for _ in range(args.warmup):
            S.solve(eta, TOL, B.MG_MODE_MG, out=psi)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        for _ in range(args.steps):
            _, info = S.solve(eta, TOL, B.MG_MODE_MG, out=psi)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile": "solve", "steps": args.steps, "kernel_launches": info.kernel_launches,
                          "outer_iterations": info.outer_iterations, "true_residual": info.true_residual}))
        S.close()
    elif args.profile == "coarse":
        # the persistent coarsest-level solve of the workload, `steps` launches of
        # COARSE_PROFILE_ITERS GCR iterations each
        S = Solver(DIMS)
        S.load_gauge(U)
        S.set_clover(CSW, args.mass)
        S.set_params(seed=NULLVEC_SEED, maxit_fine=2000, **MG)
        S.setup()
        S.set_params(tol_coarse=1e-12, maxit_coarse=COARSE_PROFILE_ITERS)
        B.mg_benchmark_coarse_solve(S.ctx, max(1, args.warmup), 1)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        ms, by, its = B.mg_benchmark_coarse_solve(S.ctx, 0, args.steps)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile": "coarse", "launches": args.steps, "gcr_iterations": its, "ms_per_solve": ms,
                          "link_bytes_per_solve": by}))
        S.close()
    elif args.profile == "transfer":
        # the level-0 restriction and prolongation on the even sites of the
        # workload, one launch each for 1 and BATCH_RHS right-hand sides
        S = Solver(DIMS)
        S.load_gauge(U)
        S.set_clover(CSW, args.mass)
        S.set_params(seed=NULLVEC_SEED, maxit_fine=2000, **MG)
        S.setup()
        codes = [(B.MG_KERNEL_RESTRICT, 1), (B.MG_KERNEL_PROLONG, 1), (B.MG_KERNEL_RESTRICT, BATCH_RHS),
                 (B.MG_KERNEL_PROLONG, BATCH_RHS)]
        for code, nrhs in codes:
            B.mg_benchmark_kernel_nrhs(S.ctx, code, B.MG_FP32, nrhs, warmup=max(1, args.warmup), iters=1)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        res = []
        for code, nrhs in codes:
            ms, by = B.mg_benchmark_kernel_nrhs(S.ctx, code, B.MG_FP32, nrhs, warmup=0, iters=args.steps)
            res.append({"kernel": "restrict" if code == B.MG_KERNEL_RESTRICT else "prolong", "nrhs": nrhs,
                        "ms_per_launch": ms, "bytes_per_launch": by})
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile": "transfer", "launches": args.steps, "results": res}))
        S.close()
    elif args.profile == "block_tc":
        # the block solve of BATCH_RHS sources with FP16 links: its coarsest-level
        # solves run on tensor cores (k_coarse_gcr_tc)
        etas = torch.from_numpy(I.gaussian_source(DIMS, SOURCE_SEED + 10, nrhs=BATCH_RHS)).cuda()
        psis = torch.zeros_like(etas)
        S = Solver(DIMS)
        S.load_gauge(U)
        S.set_clover(CSW, args.mass)
        S.set_params(seed=NULLVEC_SEED, maxit_fine=2000, rhs_block=BATCH_RHS, storage=B.MG_STORE_FP16, coarse_impl=4,
                     **MG)
        S.setup()
        for _ in range(args.warmup):
            S.solve(etas, TOL, B.MG_MODE_MG, out=psis)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        for _ in range(args.steps):
            _, info = S.solve(etas, TOL, B.MG_MODE_MG, out=psis)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile": "block_tc", "nrhs": BATCH_RHS, "steps": args.steps,
                          "kernel_launches": info.kernel_launches, "outer_iterations": info.outer_iterations,
                          "true_residual": info.true_residual}))
        S.close()
    elif args.profile == "block":
        etas = torch.from_numpy(I.gaussian_source(DIMS, SOURCE_SEED + 10, nrhs=BATCH_RHS)).cuda()
        psis = torch.zeros_like(etas)
        S = Solver(DIMS)
        S.load_gauge(U)
        S.set_clover(CSW, args.mass)
        S.set_params(seed=NULLVEC_SEED, maxit_fine=2000, rhs_block=BATCH_RHS, **MG)
        S.setup()
        for _ in range(args.warmup):
            S.solve(etas, TOL, B.MG_MODE_MG, out=psis)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        for _ in range(args.steps):
            _, info = S.solve(etas, TOL, B.MG_MODE_MG, out=psis)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile": "block", "nrhs": BATCH_RHS, "steps": args.steps,
                          "kernel_launches": info.kernel_launches, "outer_iterations": info.outer_iterations,
                          "true_residual": info.true_residual}))
        S.close()
    else:
        nrhs = 1 if args.profile == "dslash" else args.profile_nrhs
        dims = HBM_DIMS if args.profile == "dslash" else PROFILE_MRHS_DIMS
        reps = [h // d for h, d in zip(dims, DIMS)]
        H = Solver(dims)
        H.load_gauge(np.tile(U, (reps[3], reps[2], reps[1], reps[0], 1, 1, 1)))
        H.set_clover(CSW, args.mass)
        B.mg_benchmark_kernel_nrhs(H.ctx, B.MG_KERNEL_DSLASH_CLOVER, B.MG_FP32, nrhs, warmup=args.warmup, iters=1)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        ms, by = B.mg_benchmark_kernel_nrhs(H.ctx, B.MG_KERNEL_DSLASH_CLOVER, B.MG_FP32, nrhs, warmup=0,
                                            iters=args.steps)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile": args.profile, "nrhs": nrhs, "launches": args.steps, "bytes_per_launch": by,
                          "ms_per_launch": ms}))
        H.close()


# ----------------------------------------------------------------------------- GPU arm
def run_gpu(args, dist: Dist) -> dict:
    import numpy as np
    import torch
    from paper_1011_2775_gb300 import binding as B
    from paper_1011_2775_gb300 import build as build_mod
    from paper_1011_2775_gb300 import inputs as I
    from paper_1011_2775_gb300.solver import Solver

    build_mod.build()
    dev = dist.local
    torch.cuda.set_device(dev)
    m0 = args.mass
    U = I.make_gauge(DIMS, EPS, APE, ALPHA, GAUGE_SEED)
    eta = I.gaussian_source(DIMS, SOURCE_SEED)
    stream = torch.cuda.current_stream(dev)
    S = Solver(DIMS, device=dev, stream=stream.cuda_stream)
    S.load_gauge(U)
    S.set_clover(CSW, m0)
    S.set_params(seed=NULLVEC_SEED, maxit_fine=2000, **MG)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sinfo = S.setup()
    setup_ms = 1e3 * (time.perf_counter() - t0)

    eta_d = torch.from_numpy(eta).to(f"cuda:{dev}")
    psi_d = torch.zeros_like(eta_d)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{dev}")
    for _ in range(args.warmup):
        S.solve(eta_d, TOL, B.MG_MODE_MG, out=psi_d)
    torch.cuda.synchronize()

    # timed region: K solves, inputs resident in HBM, L2 flushed before each
    clocks = Clocks(dev)
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    times, infos, launches = [], [], 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, info = S.solve(eta_d, TOL, B.MG_MODE_MG, out=psi_d)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        infos.append(info)
        launches += info.kernel_launches
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    ms = dist.max(sum(times) / len(times))
    last = infos[-1]
    assert last.true_residual <= TOL, f"true residual {last.true_residual}"

    # end to end through the C ABI with host buffers (H2D of eta, D2H of psi inside)
    psi_h = np.zeros_like(eta)
    e2e_times = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, einfo = S.solve(eta, TOL, B.MG_MODE_MG, out=psi_h)
        e2e_times.append(1e3 * (time.perf_counter() - t0))
    e2e_ms = dist.max(statistics.median(e2e_times))
    nbytes = eta.nbytes

    # the step's dominant kernel, the persistent coarsest-level solve, timed alone
    # with CUDA events on the solve's stream at the step's average number of GCR
    # iterations per coarse solve (one coarse solve per outer iteration)
    per_solve = last.coarse_iterations[1] / max(1, last.outer_iterations)
    keep = (S.params.tol_coarse, S.params.maxit_coarse)
    S.set_params(tol_coarse=1e-12, maxit_coarse=max(1, round(per_solve)))
    c_ms, c_bytes, c_its = B.mg_benchmark_coarse_solve(S.ctx, 3, 20)
    S.set_params(tol_coarse=keep[0], maxit_coarse=keep[1])
    coarse = {"ms": c_ms, "bytes": c_bytes, "gcr_iterations": c_its, "avg_iterations_in_step": per_solve,
              "share_of_step": c_ms * last.outer_iterations / ms}
    # its floors on the same grid: one grid barrier, and one iteration's link
    # stream L2 -> shared memory without arithmetic (three barriers + one stream
    # per GCR iteration)
    f_bar, f_stream, f_bytes, f_grid = B.mg_benchmark_coarse_floor(S.ctx)
    coarse["floor"] = {"grid": f_grid, "barrier_us": f_bar, "link_stream_us": f_stream, "link_bytes": f_bytes,
                       "link_stream_gbs": f_bytes / f_stream / 1e3, "iteration_floor_us": 3 * f_bar + f_stream,
                       "iteration_us": 1e3 * c_ms / max(1.0, c_its)}
    # the level-0 restriction and prolongation on the even sites (back-to-back
    # launches; P of the even sites, 151 MB in FP32, exceeds the L2)
    transfer = {}
    for name, code in [("restrict", B.MG_KERNEL_RESTRICT), ("prolong", B.MG_KERNEL_PROLONG)]:
        for nrhs in (1, BATCH_RHS):
            ms_t, by = B.mg_benchmark_kernel_nrhs(S.ctx, code, B.MG_FP32, nrhs, warmup=3, iters=20)
            transfer[f"{name}_nrhs{nrhs}"] = {"ms": ms_t, "bytes": by, "gbs": by / ms_t / 1e6}

    extra = {}
    if not args.no_extra:
        t_x = time.perf_counter()
        extra = run_extras(args, S, U, eta, flush, stream, dev)
        SECTIONS["extras"] = time.perf_counter() - t_x

    # plain FP64 even-odd GCR on the same system (bounded)
    eo = None
    if not args.no_eo:
        S.set_params(seed=NULLVEC_SEED, maxit_fine=args.eo_maxit, **MG)
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, ei = B.mg_solve(S.ctx, psi_d, eta_d, 1, TOL, B.MG_MODE_EO_GCR, allow_not_converged=True)
        e1.record(stream)
        torch.cuda.synchronize()
        eo = {"ms": e0.elapsed_time(e1), "iterations": ei.outer_iterations, "true_residual": ei.true_residual,
              "converged": st == B.MG_OK, "restart": 16, "iteration_cap": args.eo_maxit}
    S.close()

    # the fine dslash on a lattice far beyond L2 (HBM-resident)
    reps = [h // d for h, d in zip(HBM_DIMS, DIMS)]
    U_big = np.tile(U, (reps[3], reps[2], reps[1], reps[0], 1, 1, 1))  # periodic copy: valid SU(3) field
    H = Solver(HBM_DIMS, device=dev, stream=stream.cuda_stream)
    H.load_gauge(U_big)
    H.set_clover(CSW, m0)
    del U_big
    kern = dict(transfer)
    for name, code, prec in [("dslash_clover_fp32", B.MG_KERNEL_DSLASH_CLOVER, B.MG_FP32),
                             ("dslash_xpay_fp32", B.MG_KERNEL_DSLASH_XPAY, B.MG_FP32),
                             ("dr_fp32", B.MG_KERNEL_DR, B.MG_FP32),
                             ("dslash_clover_fp64", B.MG_KERNEL_DSLASH_CLOVER, B.MG_FP64)]:
        ms_k, by = B.mg_benchmark_kernel(H.ctx, code, prec, warmup=10, iters=50)
        kern[name] = {"ms": ms_k, "bytes": by, "gbs": by / ms_k / 1e6}
    if not args.no_extra:
        # multi-RHS D_r (links and clover read once per site for all rhs)
        for nrhs in MRHS:
            ms_k, by = B.mg_benchmark_kernel_nrhs(H.ctx, B.MG_KERNEL_DR, B.MG_FP32, nrhs, warmup=3, iters=10)
            kern[f"dr_fp32_nrhs{nrhs}"] = {"ms": ms_k, "bytes": by, "gbs": by / ms_k / 1e6, "ms_per_rhs": ms_k / nrhs}
    H.close()
    # CUDA-core FMA peaks of this GPU (denominators of the ALU-bound kernels)
    peaks = {"fp64_fma_tflops": B.mg_benchmark_fma(dev, B.MG_FP64), "fp32_fma_tflops": B.mg_benchmark_fma(dev, B.MG_FP32)}
    kern["dslash_clover_fp64"]["tflops"] = kern["dslash_clover_fp64"]["bytes"] / 2112.0 * DSLASH_FLOPS_PER_SITE / \
        kern["dslash_clover_fp64"]["ms"] / 1e9
    kern["dslash_clover_fp64"]["frac_of_fp64_fma_peak"] = kern["dslash_clover_fp64"]["tflops"] / peaks["fp64_fma_tflops"]

    # the GPU's solve of the CPU sample's configuration (8^4, setup with the same passes)
    small = None
    if not args.no_cpu:
        Us = I.make_gauge(CPU_DIMS, EPS, APE, ALPHA, GAUGE_SEED)
        T = Solver(CPU_DIMS, device=dev, stream=stream.cuda_stream)
        T.load_gauge(Us)
        T.set_clover(CSW, m0)
        T.set_params(seed=NULLVEC_SEED, maxit_fine=2000, setup_iters=CPU_SETUP_ITERS, **MG)
        T.setup()
        es = torch.from_numpy(I.gaussian_source(CPU_DIMS, SOURCE_SEED)).to(f"cuda:{dev}")
        ps = torch.zeros_like(es)
        T.solve(es, TOL, B.MG_MODE_MG, out=ps)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        T.solve(es, TOL, B.MG_MODE_MG, out=ps)
        e1.record(stream)
        torch.cuda.synchronize()
        small = e0.elapsed_time(e1)
        T.close()
    return dict(ms=ms, times=times, info=last, setup_ms=setup_ms, sinfo=sinfo, e2e_ms=e2e_ms, nbytes=nbytes,
                eo=eo, kern=kern, clocks=clk, launches=launches // max(1, args.steps), extra=extra, coarse=coarse,
                peaks=peaks, small_ms=small)


def run_extras(args, S, U, eta, flush, stream, dev) -> dict:
    """The batching, storage and differentiation rows on the same workload:
    a block solve of BATCH_RHS right-hand sides against the same sources solved
    one at a time, an FP16-storage solve, a differentiated solve (forward
    solve, adjoint solve, link derivative), and a solve of the anisotropic
    operator on the same field."""
    import torch
    from paper_1011_2775_gb300 import binding as B
    from paper_1011_2775_gb300 import inputs as I
    from paper_1011_2775_gb300.autograd import dirac_solve
    from paper_1011_2775_gb300.solver import Solver

    out = {}

    def timed(fn):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), res

    # ---- the same solve with coarse tolerance 0.3 (setup kept) and with the
    #      original single-system coarsest kernel
    e_d = torch.from_numpy(eta).to(f"cuda:{dev}")
    p_d = torch.zeros_like(e_d)
    alt = {}
    for name, kw in (("tol_0.3", dict(tol_coarse=ALT_COARSE_TOL)), ("single_system_kernel", dict(coarse_impl=1)),
                     ("outer_fp64_products", dict(outer_prec=B.MG_FP64)), ("level_timing", dict(level_timing=1))):
        S.set_params(**kw)
        S.solve(e_d, TOL, B.MG_MODE_MG, out=p_d)
        t_p, (_, qi) = timed(lambda: S.solve(e_d, TOL, B.MG_MODE_MG, out=p_d))
        alt[name] = {"ms": t_p, "outer_iterations": qi.outer_iterations, "coarse_iterations": qi.coarse_iterations[1],
                     "true_residual": qi.true_residual}
        if name == "level_timing":   # GPU ms inside the level-0 cycles and the level-1 coarse solves
            alt[name]["level_ms"] = [qi.level_ms[0], qi.level_ms[1]]
        S.set_params(tol_coarse=MG["tol_coarse"], coarse_impl=0, outer_prec=B.MG_FP32, level_timing=0)
    out["coarse_tolerance"] = alt
    del e_d, p_d

    # ---- batched right-hand sides (12 Gaussian sources, the point-source count of one propagator)
    etas = torch.from_numpy(I.gaussian_source(DIMS, SOURCE_SEED + 10, nrhs=BATCH_RHS)).to(f"cuda:{dev}")
    psis = torch.zeros_like(etas)
    S.set_params(rhs_block=BATCH_RHS)
    S.solve(etas, TOL, B.MG_MODE_MG, out=psis)   # warm-up (allocations, autotuning)
    t_blk, (_, bi) = timed(lambda: S.solve(etas, TOL, B.MG_MODE_MG, out=psis))
    S.set_params(rhs_block=1)
    t_seq, (_, si) = timed(lambda: S.solve(etas, TOL, B.MG_MODE_MG, out=psis))
    S.set_params(rhs_block=16)
    out["batched"] = {"nrhs": BATCH_RHS, "block_ms": t_blk, "sequential_ms": t_seq,
                      "block_ms_per_rhs": t_blk / BATCH_RHS, "sequential_ms_per_rhs": t_seq / BATCH_RHS,
                      "speedup": t_seq / t_blk, "block_outer_iterations": bi.outer_iterations,
                      "sequential_outer_iterations": si.outer_iterations,
                      "true_residual_max": max(bi.true_residual, si.true_residual)}
    del etas, psis

    # ---- differentiated solve: L = Re<chi, D^{-1} eta>, grads w.r.t. eta and U
    eta_d = torch.from_numpy(eta).to(f"cuda:{dev}").requires_grad_(True)
    U_d = torch.from_numpy(U).to(f"cuda:{dev}").requires_grad_(True)
    chi_d = torch.from_numpy(I.gaussian_source(DIMS, SOURCE_SEED + 20)).to(f"cuda:{dev}")
    S.load_gauge(U_d)                              # the same field; the setup must be redone after a load
    S.set_clover(CSW, args.mass)
    S.setup()
    t_fwd, psi = timed(lambda: dirac_solve(S, eta_d, U_d, tol=TOL))
    loss = torch.sum(torch.conj(chi_d) * psi).real
    t_bwd, _ = timed(lambda: loss.backward())
    lam = eta_d.grad.detach()
    t_force, f64 = timed(lambda: S.force(lam, psi.detach(), kind=B.MG_FORCE_SU3))
    t_force32, f32 = timed(lambda: S.force(lam, psi.detach(), kind=B.MG_FORCE_SU3 | B.MG_FORCE_FP32))
    out["gradient"] = {"forward_ms": t_fwd, "backward_ms": t_bwd, "backward_over_forward": t_bwd / t_fwd,
                       "force_ms": t_force, "force_fp32_ms": t_force32,
                       "force_fp32_rel_err": float((f32 - f64).abs().max() / f64.abs().max()), "what": "backward = adjoint MG solve through gamma_5 D gamma_5 + "
                                                   "FP64 hop and clover link derivative"}
    del eta_d, U_d, chi_d, psi, lam, loss, f64, f32

    # ---- the 2-level cycle replayed as a CUDA graph (default) against direct launches
    e_g = torch.from_numpy(eta).to(f"cuda:{dev}")
    p_g = torch.zeros_like(e_g)
    tg = {}
    for flag in (0, 1):
        S.set_params(cuda_graphs=flag)
        S.solve(e_g, TOL, B.MG_MODE_MG, out=p_g)     # warm-up (and capture)
        tg[flag] = statistics.median(timed(lambda: S.solve(e_g, TOL, B.MG_MODE_MG, out=p_g))[0] for _ in range(3))
    out["cuda_graph"] = {"graph_ms": tg[1], "direct_launch_ms": tg[0], "speedup": tg[0] / tg[1]}
    del e_g, p_g

    # ---- the mass sweep of the workload: MG-GCR, and plain EO-GCR and mixed-precision BiCGStab
    #      capped at SWEEP_EO_CAP iterations
    sweep = []
    for m0 in MASSES:
        Q = Solver(DIMS, device=dev, stream=stream.cuda_stream)
        Q.load_gauge(U)
        Q.set_clover(CSW, m0)
        Q.set_params(seed=NULLVEC_SEED, maxit_fine=2000, **MG)
        Q.setup()
        e_d = torch.from_numpy(eta).to(f"cuda:{dev}")
        p_d = torch.zeros_like(e_d)
        Q.solve(e_d, TOL, B.MG_MODE_MG, out=p_d)
        t_mg, (_, mi) = timed(lambda: Q.solve(e_d, TOL, B.MG_MODE_MG, out=p_d))
        Q.set_params(maxit_fine=SWEEP_EO_CAP)
        t_eo, (st, ei) = timed(lambda: B.mg_solve(Q.ctx, p_d, e_d, 1, TOL, B.MG_MODE_EO_GCR, allow_not_converged=True))
        B.mg_solve(Q.ctx, p_d, e_d, 1, 1e-2, B.MG_MODE_BICGSTAB_MP, allow_not_converged=True)   # buffers
        t_bi, (sb, bi) = timed(lambda: B.mg_solve(Q.ctx, p_d, e_d, 1, TOL, B.MG_MODE_BICGSTAB_MP,
                                                  allow_not_converged=True))
        sweep.append({"m0": m0, "mg_ms": t_mg, "mg_outer_iterations": mi.outer_iterations,
                      "mg_true_residual": mi.true_residual, "eo_gcr_ms": t_eo, "eo_gcr_iterations": ei.outer_iterations,
                      "eo_gcr_true_residual": ei.true_residual, "eo_gcr_converged": st == B.MG_OK,
                      "bicgstab_mixed_ms": t_bi, "bicgstab_mixed_iterations": bi.outer_iterations,
                      "bicgstab_mixed_true_residual": bi.true_residual, "bicgstab_mixed_converged": sb == B.MG_OK})
        Q.close()
    out["mass_sweep"] = sweep

    # ---- setup reuse: rebuild for the next mass of the sweep from the current null vectors, and
    #      the setup effort (inverse-iteration passes) against the solve it buys
    reuse = {}
    Q = Solver(DIMS, device=dev, stream=stream.cuda_stream)
    Q.load_gauge(U)
    Q.set_clover(CSW, MASSES[-1])
    Q.set_params(seed=NULLVEC_SEED, maxit_fine=2000, **MG)
    Q.setup()
    e_d = torch.from_numpy(eta).to(f"cuda:{dev}")
    p_d = torch.zeros_like(e_d)
    ui = Q.update_mass(MASSES[-2])
    Q.solve(e_d, TOL, B.MG_MODE_MG, out=p_d)
    t_u, (_, qi) = timed(lambda: Q.solve(e_d, TOL, B.MG_MODE_MG, out=p_d))
    reuse["update_mass"] = {"from_m0": MASSES[-1], "to_m0": MASSES[-2], "rebuild_ms": ui.setup_ms, "solve_ms": t_u,
                            "outer_iterations": qi.outer_iterations, "true_residual": qi.true_residual}
    Q.close()
    effort = []
    for iters in (2, 5, 20):
        Q = Solver(DIMS, device=dev, stream=stream.cuda_stream)
        Q.load_gauge(U)
        Q.set_clover(CSW, MASSES[-1])
        Q.set_params(seed=NULLVEC_SEED, maxit_fine=2000, setup_iters=iters, **MG)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        si_ = Q.setup()
        t_setup = 1e3 * (time.perf_counter() - t0)
        Q.solve(e_d, TOL, B.MG_MODE_MG, out=p_d)
        t_s, (_, qi) = timed(lambda: Q.solve(e_d, TOL, B.MG_MODE_MG, out=p_d))
        effort.append({"setup_iters": iters, "setup_passes": si_.passes[0], "setup_ms": t_setup, "solve_ms": t_s,
                       "outer_iterations": qi.outer_iterations})
        Q.close()
    # a weak (2 passes per vector) and the default setup, each refined by one adaptive pass
    for iters in (2, None):
        Q = Solver(DIMS, device=dev, stream=stream.cuda_stream)
        Q.load_gauge(U)
        Q.set_clover(CSW, MASSES[-1])
        Q.set_params(seed=NULLVEC_SEED, maxit_fine=2000, **MG)
        if iters is not None:
            Q.set_params(setup_iters=iters)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Q.setup()
        ai = Q.adapt_setup(passes=1, relax=2)
        t_setup = 1e3 * (time.perf_counter() - t0)
        Q.solve(e_d, TOL, B.MG_MODE_MG, out=p_d)
        t_s, (_, qi) = timed(lambda: Q.solve(e_d, TOL, B.MG_MODE_MG, out=p_d))
        effort.append({"setup_iters": iters if iters is not None else "default", "adaptive_passes": 1,
                       "adaptive_relax": 2, "setup_ms": t_setup, "adaptive_ms": ai.setup_ms, "solve_ms": t_s,
                       "outer_iterations": qi.outer_iterations})
        Q.close()
    reuse["setup_effort"] = effort
    out["setup_reuse"] = reuse
    del e_d, p_d

    # ---- FP16 storage of P and the coarse links
    Q = Solver(DIMS, device=dev, stream=stream.cuda_stream)
    Q.load_gauge(U)
    Q.set_clover(CSW, args.mass)
    Q.set_params(seed=NULLVEC_SEED, maxit_fine=2000, storage=B.MG_STORE_FP16, **MG)
    Q.setup()
    e_d = torch.from_numpy(eta).to(f"cuda:{dev}")
    p_d = torch.zeros_like(e_d)
    Q.solve(e_d, TOL, B.MG_MODE_MG, out=p_d)
    ts = []
    for _ in range(3):
        t, (_, qi) = timed(lambda: Q.solve(e_d, TOL, B.MG_MODE_MG, out=p_d))
        ts.append(t)
    out["fp16_storage"] = {"ms": statistics.median(ts), "outer_iterations": qi.outer_iterations,
                           "coarse_iterations": qi.coarse_iterations[1], "true_residual": qi.true_residual}
    Q.close()

    # ---- the anisotropic operator on the same field: a lattice finer in t
    # (spatial hopping weights 0.3), csw_t apart from csw; informational, so a
    # failure is recorded instead of ending the run
    try:
        Q = Solver(DIMS, device=dev, stream=stream.cuda_stream)
        Q.load_gauge(U)
        Q.set_clover_aniso(ANISO_W, CSW, ANISO_CSW_T, ANISO_M0)
        Q.set_params(seed=NULLVEC_SEED, maxit_fine=2000, **MG)
        t0 = time.perf_counter()
        Q.setup()
        t_setup = 1e3 * (time.perf_counter() - t0)
        Q.solve(e_d, TOL, B.MG_MODE_MG, out=p_d, allow_not_converged=True)
        ts = []
        for _ in range(3):
            t, (_, qi) = timed(lambda: Q.solve(e_d, TOL, B.MG_MODE_MG, out=p_d, allow_not_converged=True))
            ts.append(t)
        out["anisotropic"] = {"weights": list(ANISO_W), "csw_s": CSW, "csw_t": ANISO_CSW_T, "m0": ANISO_M0,
                              "ms": statistics.median(ts), "setup_ms": t_setup, "outer_iterations": qi.outer_iterations,
                              "coarse_iterations": qi.coarse_iterations[1], "true_residual": qi.true_residual}
        Q.close()
    except Exception as exc:   # pragma: no cover - recorded in the bench line
        out["anisotropic"] = {"error": f"{type(exc).__name__}: {exc}"}
    t_k = time.perf_counter()
    out["krylov"] = run_krylov(dev, flush, stream)
    SECTIONS["krylov"] = time.perf_counter() - t_k
    return out


# The anisotropic extra: hopping weights (x, y, z, t), the clover coefficient
# of the planes containing t, and a mass above the critical one of these
# weights on the nearly free field (smallest Re lambda of D at m0 = 0 is 0.060
# on 4^3x8, of which 0.076 is the lowest antiperiodic momentum in t).
ANISO_W = (0.3, 0.3, 0.3, 1.0)
ANISO_CSW_T = 1.4
ANISO_M0 = 0.05

# The Krylov comparison (the paper's time-to-solution vs. mass, speedup vs.
# tolerance and error/residual axes) on a rougher ensemble of the same shape,
# eps = 1.0 + 5 APE, whose critical mass lies below -0.65: the masses swept
# toward it stay subcritical there, so the plain Krylov solvers converge.
KRYLOV_EPS = 1.0
KRYLOV_MASSES = (-0.35, -0.5, -0.65)
KRYLOV_MAXIT = 10000                 # iteration cap of the comparison solvers
KRYLOV_TOLS = (1e-6, 1e-8, 1e-10)
ERROR_TOLS = (1e-4, 1e-6, 1e-8, 1e-10)


def run_krylov(dev: int, flush, stream) -> dict:
    """MG-GCR against BiCGStab (FP64 and mixed precision), CGNR and EO-GCR per
    mass; MG against mixed-precision BiCGStab per tolerance at the lightest
    mass; and the error/residual ratio of MG and BiCGStab for a manufactured
    solution b = D x0 (x0 = an approximate solution for a point source)."""
    import numpy as np
    import torch
    from paper_1011_2775_gb300 import binding as B
    from paper_1011_2775_gb300 import inputs as I
    from paper_1011_2775_gb300.solver import Solver

    def timed(fn):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), res

    U = I.make_gauge(DIMS, KRYLOV_EPS, APE, ALPHA, GAUGE_SEED)
    eta_d = torch.from_numpy(I.gaussian_source(DIMS, SOURCE_SEED)).to(f"cuda:{dev}")
    psi_d = torch.zeros_like(eta_d)
    modes = [("mg", B.MG_MODE_MG), ("bicgstab", B.MG_MODE_BICGSTAB), ("bicgstab_mixed", B.MG_MODE_BICGSTAB_MP),
             ("cgnr", B.MG_MODE_CGNR), ("eo_gcr", B.MG_MODE_EO_GCR)]
    out = {"ensemble": f"{DIMS[0]}^3x{DIMS[3]}, eps={KRYLOV_EPS}+{APE} APE(alpha={ALPHA}), csw={CSW}",
           "iteration_cap": KRYLOV_MAXIT, "masses": []}

    def solve_row(S, mode, tol):
        S.solve(eta_d, 1e-2, mode, out=psi_d, allow_not_converged=True)     # buffers allocated outside the timing
        ms, (st, info) = timed(lambda: B.mg_solve(S.ctx, psi_d, eta_d, 1, tol, mode, allow_not_converged=True))
        return {"ms": ms, "iterations": info.outer_iterations, "converged": st == B.MG_OK,
                "true_residual": info.true_residual}

    S = None
    for m0 in KRYLOV_MASSES:
        S = Solver(DIMS, device=dev, stream=stream.cuda_stream)
        S.load_gauge(U)
        S.set_clover(CSW, m0)
        S.set_params(seed=NULLVEC_SEED, maxit_fine=KRYLOV_MAXIT, **MG)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.setup()
        row = {"m0": m0, "mg_setup_ms": 1e3 * (time.perf_counter() - t0)}
        for name, mode in modes:
            row[name] = solve_row(S, mode, TOL)
        out["masses"].append(row)
        if m0 != KRYLOV_MASSES[-1]:
            S.close()
    # speedup vs. requested tolerance at the lightest mass (S is still set up there)
    out["tolerance"] = []
    for tol in KRYLOV_TOLS:
        mg_r = solve_row(S, B.MG_MODE_MG, tol)
        bi_r = solve_row(S, B.MG_MODE_BICGSTAB_MP, tol)
        out["tolerance"].append({"tol": tol, "mg_ms": mg_r["ms"], "bicgstab_mixed_ms": bi_r["ms"],
                                 "speedup": bi_r["ms"] / mg_r["ms"], "mg_iterations": mg_r["iterations"],
                                 "bicgstab_mixed_iterations": bi_r["iterations"]})
    # error / residual with a manufactured solution
    p = I.point_source(DIMS, 0, (0, 0, 0, 0))
    x0, _ = S.solve(p, 1e-6, B.MG_MODE_MG)
    b = S.apply(B.MG_OP_D, x0, prec=B.MG_FP64)
    nb, nx = float(np.linalg.norm(b.ravel())), float(np.linalg.norm(x0.ravel()))
    out["error_vs_residual"] = []
    for tol in ERROR_TOLS:
        for name, mode in (("mg", B.MG_MODE_MG), ("bicgstab", B.MG_MODE_BICGSTAB)):
            x = np.zeros_like(b)
            st, info = B.mg_solve(S.ctx, x, b, 1, tol, mode, allow_not_converged=True)
            err = float(np.linalg.norm((x - x0).ravel()))
            res = info.true_residual * nb
            out["error_vs_residual"].append({"tol": tol, "solver": name, "residual": res, "error": err,
                                             "error_over_residual": err / res if res > 0 else None,
                                             "relative_error": err / nx})
    S.close()
    return out


# Batched sources on lattices of uneven size (the batching workload): 12 point
# sources on 32^3x64, 8 Gaussian sources each on 16^3x32 and 24^3x48, the same
# gauge construction, m0 = -0.3, 2-level MG with 4^4 blocks and Nv = 24.
MULTI = [((32, 32, 32, 64), "point", 12), ((16, 16, 16, 32), "gauss", 8), ((24, 24, 24, 48), "gauss", 8)]
MULTI_M0 = -0.3
SWEEP_EO_CAP = 2000                  # EO-GCR and BiCGStab iteration cap in the mass sweep

# The 3-level configuration: 24^3x64, same gauge construction, m0 = -0.35,
# 4^4 blocks (Nv = 24) then 2^4 blocks (Nv = 32) onto a 3^3x8 coarsest lattice
# (odd extent: no even-odd there), 16-bit storage of P and coarse links.
CONFIG3_DIMS = (24, 24, 24, 64)
CONFIG3_MG = dict(levels=3, blocks=[(4, 4, 4, 4), (2, 2, 2, 2)], nv=[24, 32])
# a rougher field whose critical mass lies near -0.75 (24^3x64: m0 = -0.75 no longer converges in 300 outer
# iterations), at a light subcritical mass: the regime of the paper's 3-level runs
ROUGH_EPS, ROUGH_M0 = 1.0, -0.7


def run_config3(dev: int, pre: dict | None = None) -> dict:
    """The 24^3x64 configuration: the 3-level solve with BF16 storage of P and
    the coarse links, the 2-level solve with BF16 and with FP32 storage, and
    the FP32 dslash on this lattice (467 MB per launch, beyond L2)."""
    import torch
    from paper_1011_2775_gb300 import binding as B
    from paper_1011_2775_gb300 import inputs as I
    from paper_1011_2775_gb300.solver import Solver

    stream = torch.cuda.current_stream(dev)
    pre = pre or {}

    def field(eps):
        spec = (CONFIG3_DIMS, eps, APE, ALPHA, 3001)
        return pre[spec] if spec in pre else I.make_gauge(*spec)

    fields = {EPS: field(EPS)}
    eta = torch.from_numpy(I.gaussian_source(CONFIG3_DIMS, 3002)).to(f"cuda:{dev}")
    psi = torch.zeros_like(eta)
    out = {"lattice": "24^3x64", "m0": -0.35, "mg": "3-level: 4^4 (Nv=24) then 2^4 (Nv=32), coarsest 3^3x8",
           "rough": f"the rough ensemble eps = {ROUGH_EPS} + 5 APE at m0 = {ROUGH_M0}, below its critical mass, "
                    "2 against 3 levels in FP32 storage"}
    runs = (("three_level_bf16", B.MG_STORE_BF16, CONFIG3_MG, EPS, -0.35),
            ("two_level_bf16", B.MG_STORE_BF16, MG, EPS, -0.35), ("two_level_fp32", B.MG_STORE_FP32, MG, EPS, -0.35),
            ("rough_three_level_fp32", B.MG_STORE_FP32, CONFIG3_MG, ROUGH_EPS, ROUGH_M0),
            ("rough_two_level_fp32", B.MG_STORE_FP32, MG, ROUGH_EPS, ROUGH_M0))
    for name, store, mg, eps, m0 in runs:
        if eps not in fields:
            fields[eps] = field(eps)
        U = fields[eps]
        S = Solver(CONFIG3_DIMS, device=dev, stream=stream.cuda_stream)
        S.load_gauge(U)
        S.set_clover(CSW, m0)
        S.set_params(seed=3003, maxit_fine=2000, storage=store, **mg)
        t0 = time.perf_counter()
        S.setup()
        setup_ms = 1e3 * (time.perf_counter() - t0)
        S.solve(eta, TOL, B.MG_MODE_MG, out=psi, allow_not_converged=True)
        ts = []
        for _ in range(1):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, info = S.solve(eta, TOL, B.MG_MODE_MG, out=psi, allow_not_converged=True)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        out[name] = {"solve_ms": min(ts), "setup_ms": setup_ms, "outer_iterations": info.outer_iterations,
                     "level1_iterations": info.coarse_iterations[1], "level2_iterations": info.coarse_iterations[2],
                     "true_residual": info.true_residual, "levels": mg["levels"], "eps": eps, "m0": m0}
        if name == "two_level_fp32":
            ms_k, by = B.mg_benchmark_kernel(S.ctx, B.MG_KERNEL_DSLASH_CLOVER, B.MG_FP32, warmup=10, iters=50)
            out["dslash_clover_fp32"] = {"ms": ms_k, "bytes": by, "gbs": by / ms_k / 1e6}
        S.close()
    return out


def run_multi(dev: int, sequential: bool = False, pre: dict | None = None) -> dict:
    """All 28 right-hand sides through mg_solve_batch (lock-step, shared coarsest
    launches) against each lattice's own block solve and against 28 solves one
    after another; every time is CUDA events on the one stream all contexts use."""
    import numpy as np
    import torch
    from paper_1011_2775_gb300 import binding as B
    from paper_1011_2775_gb300 import inputs as I
    from paper_1011_2775_gb300.solver import Solver, solve_batch

    stream = torch.cuda.current_stream(dev)
    solvers, etas, outs, setup_ms = [], [], [], []
    for k, (dims, kind, nrhs) in enumerate(MULTI):
        spec = (dims, EPS, APE, ALPHA, 4001 + 10 * k)
        U = pre.pop(spec) if pre and spec in pre else I.make_gauge(*spec)
        S = Solver(dims, device=dev, stream=stream.cuda_stream)
        S.load_gauge(U)
        del U
        S.set_clover(CSW, MULTI_M0)
        S.set_params(seed=4003 + 10 * k, maxit_fine=2000, **MG)
        t0 = time.perf_counter()
        S.setup()
        setup_ms.append(1e3 * (time.perf_counter() - t0))
        if kind == "point":
            e = np.stack([I.point_source(dims, a) for a in range(nrhs)])
        else:
            e = I.gaussian_source(dims, 4002 + 10 * k, nrhs=nrhs)
        etas.append(torch.from_numpy(e).to(f"cuda:{dev}"))
        outs.append(torch.zeros_like(etas[-1]))
        solvers.append(S)

    def timed(fn):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), res

    solve_batch(solvers, etas, TOL, outs)                        # warm-up (allocations, autotuning)
    t_all, (_, infos) = timed(lambda: solve_batch(solvers, etas, TOL, outs))
    t_lat = []
    for S, e, o in zip(solvers, etas, outs):
        t, _ = timed(lambda: S.solve(e, TOL, B.MG_MODE_MG, out=o))
        t_lat.append(t)
    t_seq = []
    if sequential:
        for S, e, o in zip(solvers, etas, outs):
            S.set_params(rhs_block=1)
            t, (_, si) = timed(lambda: S.solve(e, TOL, B.MG_MODE_MG, out=o))
            t_seq.append(t)
            S.set_params(rhs_block=16)
    out = {"lattices": [f"{d[0]}^3x{d[3]} x{n} {kind}" for d, kind, n in MULTI], "m0": MULTI_M0,
           "all_in_one_ms": t_all, "per_lattice_block_ms": t_lat, "one_at_a_time_ms": t_seq or None,
           "speedup_vs_one_at_a_time": sum(t_seq) / t_all if t_seq else None,
           "speedup_vs_per_lattice_blocks": sum(t_lat) / t_all,
           "outer_iterations": [i.outer_iterations for i in infos],
           "true_residual_max": max(i.true_residual for i in infos), "setup_ms": setup_ms}
    for S in solvers:
        S.close()
    return out


def run_extra_configs(args, dist, r: dict) -> None:
    """The multi-lattice batch and the 24^3x64 configuration, at N = 1 only
    (they are no part of the step), their gauge fields generated in parallel
    first; results go to r["extra"]."""
    do_multi, do_config3 = dist.world == 1 and not args.no_multi, dist.world == 1 and not args.no_config3
    pre = {}
    if do_multi or do_config3:
        t_f = time.perf_counter()
        pre = big_fields([sp for sp in extra_field_specs()
                          if (do_multi and sp[0] != CONFIG3_DIMS) or (do_config3 and sp[0] == CONFIG3_DIMS)])
        SECTIONS["extra_fields"] = time.perf_counter() - t_f
    if do_multi:
        t_m = time.perf_counter()
        r["extra"]["multi_lattice"] = run_multi(dist.local, args.multi_sequential, pre)
        SECTIONS["multi_lattice"] = time.perf_counter() - t_m
    if do_config3:
        t_c = time.perf_counter()
        r["extra"]["config3_24x64"] = run_config3(dist.local, pre)
        SECTIONS["config3"] = time.perf_counter() - t_c


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["mg", "reference"], default="mg")
    ap.add_argument("--mass", type=float, default=MASSES[-1])
    ap.add_argument("--no-eo", action="store_true", help="skip the plain EO-GCR comparison")
    ap.add_argument("--eo-maxit", type=int, default=5000)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--no-config3", action="store_true",
                    help="skip the 24^3x64 solves (2 and 3 levels, BF16 and FP32 storage)")
    ap.add_argument("--no-multi", action="store_true",
                    help="skip the batched sources on three lattices of uneven size")
    ap.add_argument("--ref-procs", type=int, default=0,
                    help="reference arm: host processes (default: one per core, at most 16)")
    ap.add_argument("--ref-dims", help=argparse.SUPPRESS)   # reference arm on another lattice (CPU tests)
    ap.add_argument("--multi-sequential", action="store_true",
                    help="also solve the 28 batched sources one at a time (about 30 s)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched, FP16-storage, gradient and multi-RHS D_r measurements")
    ap.add_argument("--profile-nrhs", type=int, default=PROFILE_MRHS,
                    help="right-hand sides per launch of --profile dslash_mrhs")
    ap.add_argument("--profile", choices=["solve", "block", "block_tc", "dslash", "dslash_mrhs", "coarse", "transfer"],
                    help="for ncu --profile-from-start off: bracket `steps` solves (after setup and warm-up), "
                         "`steps` block solves of the batched right-hand sides, or `steps` launches of the FP32 fused "
                         "dslash (HBM-size lattice; dslash_mrhs: its multi-RHS form), with cudaProfilerStart/Stop; "
                         "nothing else is run")
    args = ap.parse_args()
    if args.profile:
        profile_main(args)
        return
    args.warmup = max(args.warmup, 0)
    dist = Dist()
    hbm_peak, peak_kind = load_peaks()

    if args.impl == "reference":
        if dist.rank != 0:
            dist.close()
            return
        # every host process: the oracle's setup on CPU_DIMS, then warmup + steps
        # samples of CPU_STEP_ITERS outer iterations; a step's value is the
        # median over the processes, projected to one 16^3x32 solve
        n = host_cores(args.ref_procs)
        rdims = tuple(int(x) for x in args.ref_dims.split(",")) if args.ref_dims else CPU_DIMS
        res = oracle_pool([("steps", q, args.warmup + args.steps, rdims) for q in range(n)])
        vol = (DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3]) / (rdims[0] * rdims[1] * rdims[2] * rdims[3])
        steps = [1e3 * statistics.median(r["step_s"][i] for r in res) / CPU_STEP_ITERS * vol * REFERENCE_OUTER_PER_SOLVE / n
                 for i in range(args.warmup, args.warmup + args.steps)]
        value = statistics.mean(steps)
        sample = (f"{n} concurrent single-thread processes, each the oracle's MG-GCR on a "
                  f"{'x'.join(str(d) for d in rdims)} lattice of the same "
                  f"construction and parameters (4^4 blocks, Nv=24, setup {CPU_SETUP_ITERS} passes per vector, not "
                  f"timed); a step = {CPU_STEP_ITERS} outer iterations (fine and coarse work) in every process; "
                  f"projection: median seconds per outer iteration x {vol:.0f} (volume) x "
                  f"{REFERENCE_OUTER_PER_SOLVE} (outer iterations of the GPU solve) / {n} (processes)")
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": value, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload_name(args.mass)},
                "cpu_baseline": {"value": value, "unit": "ms", "cores": n, "kind": "oracle", "sample": sample},
                "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        dist.close()
        return

    r = run_gpu(args, dist)
    run_extra_configs(args, dist, r)
    info = r["info"]
    dr_per_solve = info.dslash_launches / 2.0
    c = r["coarse"]
    roof = {"kernel": "persistent coarsest-level GCR with links streamed through shared memory (k_coarse_gcr_stream, "
                      "with its site-local pre/post launches), 4^3x8 x Nc=48 coarse lattice of the step",
            "bound": "hbm", "achieved": c["bytes"] / c["ms"] / 1e6, "peak": hbm_peak, "unit": "GB/s",
            "frac": c["bytes"] / c["ms"] / 1e6 / hbm_peak,
            "traffic": (COARSE_TRAFFIC_BYTES if COARSE_TRAFFIC_BYTES and round(c["gcr_iterations"]) == COARSE_PROFILE_ITERS
                        else None),
            "peak_kind": peak_kind, "bytes_per_launch": c["bytes"], "ms_per_launch": c["ms"],
            "gcr_iterations_per_launch": c["gcr_iterations"], "share_of_step": c["share_of_step"],
            "floor": c["floor"],
            "note": "the 75.5 MB of links per iteration stay in the 129 MB L2; bytes are the links each GCR iteration "
                    "streams (folded odd-site links FP32 + even-site Y), per launch"}
    k = r["kern"]["dslash_clover_fp32"]
    roof_dslash = {"kernel": "fused hop + clover-inverse dslash, FP32, 32^3x64 (HBM-resident)", "bound": "hbm",
                   "achieved": k["gbs"], "peak": hbm_peak, "unit": "GB/s", "frac": k["gbs"] / hbm_peak,
                   "traffic": DSLASH_TRAFFIC_BYTES, "peak_kind": peak_kind, "bytes_per_launch": k["bytes"],
                   "ms_per_launch": k["ms"]}
    line = {"metric": METRIC, "value": r["ms"], "unit": "ms", "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": workload_name(args.mass), "lattice": "16x16x16x32", "m0": args.mass,
                       "mg": "2-level, 4^4 blocks, Nv=24, coarse GCR(64) tol 0.1, nu_post=4 MR",
                       "precision": "FP64 outer GCR(16) (FP64 vectors, orthogonalisation, updates and true residuals; "
                                    "FP32 D_r products of its directions), FP32 preconditioner",
                       "l2": "flushed before every solve",
                       "parallelism": f"replicas x{dist.world}"},
            "roofline": roof, "roofline_dslash": roof_dslash,
            "e2e": {"value": r["e2e_ms"], "unit": "ms", "h2d_bytes_per_step": r["nbytes"],
                    "d2h_bytes_per_step": r["nbytes"]},
            "gpu_launches": r["launches"], "clocks": r["clocks"],
            "solve": {"outer_iterations": info.outer_iterations, "coarse_iterations": info.coarse_iterations[1],
                      "true_residual": info.true_residual, "fine_dr_applications": dr_per_solve,
                      "step_ms": r["times"]},
            "setup_ms": r["setup_ms"], "setup_passes": r["sinfo"].passes[0], "peaks": dict(r["peaks"], hbm_gbs=hbm_peak),
            "eo_gcr": r["eo"], "kernels": r["kern"], **r["extra"]}
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu:
        t_b = time.perf_counter()
        line["cpu_baseline"] = cpu_baseline(info.outer_iterations, r["small_ms"])
        SECTIONS["cpu_baseline"] = time.perf_counter() - t_b
    line["bench_sections_s"] = SECTIONS
    if dist.rank == 0:
        print(json.dumps(line))
    dist.close()


if __name__ == "__main__":
    main()
