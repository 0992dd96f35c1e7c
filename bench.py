"""Benchmark: mixed-precision SAP-BiCGStab solve of D x = b to float64 true
residual 1e-10 on a 32^4 lattice, plus the float32 Dslash roofline and the
plain float32 SAP-BiCGStab time on the same GB300.

One step = one complete solve (import of b, defect-correction loop with
float16-storage SAP + float32 BiCGStab + float64 residuals, export of x) of
the 32^4 workload: eps = 0.3 gauge field, kappa = 0.125, c_SW = 1.0, one
Gaussian source, 4^4 domains, n_sap = 4, n_jac = 4.  Every step works on
inputs far larger than L2 (the float32 links and clover alone are 600 MB).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
With N > 1 (torchrun) every rank solves its own replica (weak scaling, no
collective on the data path); the timed region is bracketed by a barrier.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Dslash GB/s vs HBM roofline; SAP-BiCGStab time to FP64 resid 1e-10 vs plain FP32"
DIMS = (32, 32, 32, 32)
DOMAIN = (4, 4, 4, 4)
EPS, KAPPA, CSW = 0.3, 0.125, 1.0
N_SAP, N_JAC = 4, 4
GAUGE_SEED, SOURCE_SEED = 1001, 2001
WORKLOAD = ("32^4 lattice, periodic space / antiperiodic time, chiral basis, U = exp(i 0.3 H) "
            "(seeded), kappa 0.125, c_sw 1.0, one Gaussian source; float16-storage SAP "
            "(4^4 domains, n_sap 4, n_jac 4) + float32 BiCGStab + float64 defect correction "
            "to true residual 1e-10")
D_BYTES_PER_SITE = 96 + 96 + 4 * 72 + 288          # in + out spinor, 4 links (18 reals), clover
D_BYTES_PER_SITE_12 = 96 + 96 + 4 * 48 + 288       # the same with links as their first two rows (12 reals)


def d_bytes_per_site(tuning_lines, mode=0):
    """Algorithmic bytes per site of the float32 D that ran (the last tuned
    shape for the operator): the 12-real-link variants (shape names ending
    in 'c') read 48 bytes per link instead of 72."""
    key = f"dslash_f32_mode{mode}_nrhs1"
    for ln in tuning_lines:
        parts = ln.split()
        if len(parts) > 1 and (parts[0] == key or parts[0].startswith(key + "_")):
            return D_BYTES_PER_SITE_12 if parts[1].endswith("c") else D_BYTES_PER_SITE
    return D_BYTES_PER_SITE
D_FLOP_PER_SITE = 1824


def sap_bytes_per_launch(prec, sweep, colour):
    """Algorithmic bytes per site of the SAP half-sweep launch (sweep, colour)
    of one M_SAP (n_sap + 1 sweeps, two colours): read s (the float32 source
    in the first sweep), the domain's links and C_inv, and with a surface
    term the domain's halo (one float32 half spinor per hop that enters the
    domain: 2 per site for 4^4 domains, 96 B); write the halo of the other
    colour's domains (96 B, all but the last launch); then either the residual
    update (read b in float32, write s) or, in the last sweep, the float32
    result x."""
    sp = 96 if prec == "single" else 52
    link = 72 if prec == "single" else 36
    clov = 288 if prec == "single" else 144
    halo = 96
    last = sweep == N_SAP
    nb = (96 if sweep == 0 else sp) + 4 * link + clov
    if not (sweep == 0 and colour == 0):
        nb += halo                       # halo in
    if not (last and colour == 1):
        nb += halo                       # halo out
    nb += 96 if last else 96 + sp        # x out, or b in and s out
    return nb


def sap_bytes_per_site(prec):
    """sap_bytes_per_launch averaged over the launches of one M_SAP."""
    seq = [sap_bytes_per_launch(prec, sweep, colour) for sweep in range(N_SAP + 1) for colour in (0, 1)]
    return sum(seq) / len(seq)


def sap_flop_per_site():
    """Flop per site of one SAP half-sweep launch, averaged over the launches
    of one M_SAP, in the per-site constants of the paper's flop accounting for
    4^4 domains in the chiral basis (168 flop per hop in every direction,
    600 flop for C_inv and the axpy, 48 flop for the residual update):
    f_in = 600 + 8 * (3/4) * 168 = 1608 per A_cc application (n_jac Jacobi
    sweeps + one for the update), f_out = 2 * 168 + 600 * 15/16 = 898.5 for
    the surface term."""
    f_in = 600 + 8 * 0.75 * 168
    f_out = 2 * 168 + 600 * 15 / 16
    seq = []
    for sweep in range(N_SAP + 1):
        last = sweep == N_SAP
        for colour in (0, 1):
            has_surf = not (sweep == 0 and colour == 0)
            seq.append((f_out if has_surf else 0) + N_JAC * f_in + (0 if last else f_in + 48))
    return sum(seq) / len(seq)


# float32 peak of the CUDA cores: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2070 MHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle leg
# ---------------------------------------------------------------------------
# The oracle (float64 numpy, Algorithms 4 and 5 with the literal SAP of
# Algorithms 1-3) is timed on complete solves to true residual 1e-10 on an
# 8^4 lattice of the benchmark recipe (eps 0.3, kappa 0.125, c_SW 1.0, 4^4
# domains, n_sap 4, n_jac 4, inner tolerance 1e-5): one process per core,
# each single-threaded (BLAS and OpenMP pinned to one thread).  Its rate is
# converted to the benchmark's unit, 32^4 solves per second, by the volume
# ratio and by the number of A M_SAP applications of each solve (two per
# BiCGStab iteration, one M_SAP per outer step); the output marks that
# conversion as extrapolated and also gives the measured 8^4 rates.
DEFAULT_ITERS = {"inner": 8, "outer": 2}   # the 32^4 GPU solve's counts (inner tolerance 1e-5)
ORACLE_DIMS = (8, 8, 8, 8)
_ONE_THREAD_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
                   "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS")


def _oracle_solve_task(dims):
    """One complete oracle solve of the benchmark recipe on `dims` (runs in a
    single-threaded worker process).  Returns its wall time and counts."""
    from lattice_inputs import gaussian_spinor, random_su3_field
    from oracle import solvers
    from oracle.dirac import CloverWilson
    from oracle.gamma import gamma_chiral
    if dims is None:  # warm-up task: the imports only
        return None
    u = random_su3_field(dims, EPS, GAUGE_SEED)
    op = CloverWilson(u, KAPPA, CSW, gamma_chiral(), bc_t=-1, domain=DOMAIN)
    b = gaussian_spinor(dims, SOURCE_SEED)
    its = []

    def inner(p):
        x, _, it, _ = solvers.bicgstab_precdd(op, op.apply_cinv(solvers.to_double(p)), N_SAP, N_JAC, 1e-5, 1000)
        its.append(it)
        return x

    t0 = time.perf_counter()
    _, outer, ok, hist = solvers.dci(op, b, 1e-10, inner)
    return {"seconds": time.perf_counter() - t0, "inner": sum(its), "outer": outer, "converged": bool(ok),
            "true_resid": float(hist[-1]) if hist else 0.0}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_solves(n_solves, procs, warmup=0, dims=ORACLE_DIMS):
    """Run `warmup` untimed and then `n_solves` timed oracle solves on a pool
    of `procs` single-threaded worker processes (started with spawn, so that
    a CUDA context in this process is never forked).  Returns the wall time
    of the timed solves and their per-solve records."""
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in _ONE_THREAD_ENV}
    for k in _ONE_THREAD_ENV:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(procs) as pool:
            pool.map(_oracle_solve_task, [None] * procs, chunksize=1)      # imports, outside the clock
            if warmup:
                pool.map(_oracle_solve_task, [dims] * warmup, chunksize=1)
            t0 = time.perf_counter()
            recs = pool.map(_oracle_solve_task, [dims] * n_solves, chunksize=1)
            wall = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return wall, recs


def solve_cost_ratio(rec, iters):
    """Cost of one benchmark-size solve over one sampled oracle solve: the
    volume ratio times the ratio of A M_SAP applications (2 per BiCGStab
    iteration + 1 M_SAP per outer step)."""
    vol_ratio = float(np.prod(DIMS)) / float(np.prod(ORACLE_DIMS))
    apps_big = 2 * iters["inner"] + iters["outer"]
    apps_small = 2 * rec["inner"] + rec["outer"]
    return vol_ratio * apps_big / apps_small, vol_ratio, apps_big, apps_small


def oracle_baseline(iters=None, procs=None, n_solves=None, warmup=0, one_thread_solves=1):
    """cpu_baseline: the oracle timed on the host cores.  All cores: `procs`
    concurrent single-threaded solves (default: one per host core); one
    thread: `one_thread_solves` solves on a pool of one (median)."""
    iters = iters or DEFAULT_ITERS
    cores = host_cores()
    procs = procs or cores
    n_solves = n_solves or procs
    wall, recs = oracle_solves(n_solves, procs, warmup)
    rate8 = n_solves / wall
    one = None
    if one_thread_solves:
        _, recs1 = oracle_solves(one_thread_solves, 1)
        one = statistics.median(r["seconds"] for r in recs1)
    ratio, vol_ratio, apps_big, apps_small = solve_cost_ratio(recs[0], iters)
    value = rate8 / ratio
    per_solve = statistics.median(r["seconds"] for r in recs)
    return {
        "value": value,
        "unit": "solves/s",
        "cores": procs,
        "host_cores": cores,
        "threads_per_process": 1,
        "kind": "oracle",
        "extrapolated": True,
        "sample": (f"{n_solves} complete float64 oracle solves (Algorithm 4 around Algorithm 5 with the literal SAP, "
                   f"n_sap {N_SAP}, n_jac {N_JAC}, 4^4 domains, inner tol 1e-5) to true residual 1e-10 on an "
                   f"8^4 lattice of the same recipe, {procs} single-threaded processes at once; converted to "
                   f"32^4 solves by the volume ratio {vol_ratio:.0f} and the A*M_SAP count ratio "
                   f"{apps_big}/{apps_small}"),
        "measured": {
            "lattice": list(ORACLE_DIMS),
            "solves": n_solves,
            "wall_s": wall,
            "solves_per_s_all_cores": rate8,
            "median_s_per_solve_all_cores": per_solve,
            "s_per_solve_one_thread": one,
            "one_thread_solves": one_thread_solves,
            "inner_iterations": recs[0]["inner"],
            "outer_steps": recs[0]["outer"],
            "true_resid": max(r["true_resid"] for r in recs),
            "all_converged": all(r["converged"] for r in recs),
        },
        "per_32x4_solve_s_all_cores": 1.0 / value,
    }


def run_reference(args):
    """Reference arm: the oracle itself, on the host cores.  Each step is one
    complete 8^4 oracle solve; the K timed steps run on a pool of
    min(K, cores) single-threaded processes, so ms_per_step is the measured
    wall time per solve of that pool.  `value` is in the benchmark's unit
    (32^4 solves/s), converted from the measured rate as stated in the line."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    procs = max(1, min(args.steps, host_cores()))
    t0 = time.perf_counter()
    cpu = oracle_baseline(procs=procs, n_solves=args.steps, warmup=args.warmup,
                          one_thread_solves=1 if procs > 1 else 0)
    elapsed = time.perf_counter() - t0
    m = cpu["measured"]
    if m["s_per_solve_one_thread"] is None:
        m["s_per_solve_one_thread"] = m["median_s_per_solve_all_cores"]
    value = cpu["value"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * m["wall_s"] / args.steps,
        "ms_per_step_is": "measured wall time per sampled 8^4 oracle solve on the process pool",
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "extrapolated": True,
        "config": {"workload": WORKLOAD, "lattice": list(DIMS), "parallelism": "replicas",
                   "sample_lattice": list(ORACLE_DIMS)},
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": elapsed,
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
def run_kernel_case(args):
    """Small profiling case: one kernel family applied REPS times on an L^4
    lattice of the benchmark recipe (for ncu captures; prints nothing timed)."""
    import torch
    from lattice_inputs import gaussian_spinor, random_su3_field
    from paper_2109_10687_gb300 import binding as B
    from paper_2109_10687_gb300.lattice import Lattice
    torch.cuda.set_device(0)
    dims = tuple(int(v) for v in args.dims.split(",")) if args.dims else (args.lattice,) * 4
    # the numpy generator: the profiling case avoids torch's linear algebra,
    # whose library a profiler's environment may not load
    lat = Lattice(dims, DOMAIN, -1, "chiral", "cuda:0").setup(random_su3_field(dims, EPS, GAUGE_SEED), KAPPA, CSW)
    if args.sap_domain:
        B.qcd_set_sap_domain(lat.ctx, [int(v) for v in args.sap_domain.split(",")])
    b = torch.view_as_real(torch.from_numpy(gaussian_spinor(dims, SOURCE_SEED))).cuda().contiguous()
    prec = B.PREC_DOUBLE if args.kernel == "dslash64" else B.PREC_SINGLE
    if args.shape is not None:
        B.qcd_set_sap_shape(lat.ctx, args.shape)
    nrhs = args.nrhs
    a = lat.field("double" if prec == B.PREC_DOUBLE else "single", nrhs)
    o = lat.field("double" if prec == B.PREC_DOUBLE else "single", nrhs)
    B.qcd_import_spinor(lat.ctx, a, b.expand((nrhs,) + tuple(b.shape)).contiguous() if nrhs > 1 else b, prec, nrhs)
    for _ in range(args.reps):
        if args.kernel == "solve_df":
            # the float16 solve with the double-float residual (its D kernel is
            # the one of interest); the source is a's float32 copy, any field will do
            P = B.qcd_solve_params_default()
            P.sap_prec = B.PREC_HALF
            P.inner_tol = 1e-5
            P.residual_prec = 0
            x = torch.zeros_like(b)
            B.qcd_solve(lat.ctx, x, b, 1, P)
        elif args.kernel.startswith("sap"):
            sp = {"sap16": B.PREC_HALF, "sap16g": B.PREC_HALF_GAUGE}.get(args.kernel, B.PREC_SINGLE)
            B.qcd_sap_apply_nrhs(lat.ctx, o, a, nrhs, N_SAP, N_JAC, sp, 0)
        else:
            B.qcd_apply_D(lat.ctx, o, a, prec, nrhs=nrhs)
    torch.cuda.synchronize()
    print(f"kernel case {args.kernel} on {dims}, {nrhs} right-hand sides: {args.reps} applications done")
    print(B.qcd_tuning_report(lat.ctx).strip())
    lat.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-48", action="store_true", help="skip the 48^4 batched comparison")
    ap.add_argument("--no-ragged", action="store_true", help="skip the ragged 32-lattice batch comparison")
    ap.add_argument("--no-n2", action="store_true", help="skip the paper-parameter (16x6x4x3 domains) rates")
    ap.add_argument("--no-grad", action="store_true", help="skip the 16^4 and 32^4 gradients")
    ap.add_argument("--no-64", action="store_true", help="skip the 64^4 operator and solves")
    ap.add_argument("--kernel", choices=["sap16", "sap16g", "sap32", "dslash", "dslash64", "solve_df"], default=None,
                    help="profiling case: set up the workload and run only REPS applications of one kernel")
    ap.add_argument("--lattice", type=int, default=32, help="lattice extent of the profiling case")
    ap.add_argument("--dims", default=None, help="lattice extents Lx,Ly,Lz,Lt of the profiling case")
    ap.add_argument("--sap-domain", default=None, help="SAP domain extents of the profiling case (qcd_set_sap_domain)")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--nrhs", type=int, default=1, help="right-hand sides of the profiling case")
    ap.add_argument("--shape", type=int, default=None, help="fix the SAP block-kernel shape of the profiling case")
    ap.add_argument("--config", default="c2", choices=["c1", "c2", "c3", "c4", "c5", "c5ragged", "n2", "cpu"],
                    help="c2 (default) is the benchmark line; the others measure the other workloads")
    args = ap.parse_args()
    if args.config != "c2":
        import bench_configs
        bench_configs.run(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.kernel:
        run_kernel_case(args)
        return

    import torch
    import torch.distributed as dist

    from paper_2109_10687_gb300 import replicas

    world, rank, local = replicas.rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from lattice_inputs import gaussian_spinor, random_su3_field
    from paper_2109_10687_gb300 import binding as B
    from paper_2109_10687_gb300 import build as _build
    from paper_2109_10687_gb300.lattice import Lattice

    _build.build()
    dev = torch.device("cuda", local)
    gauge_seed, source_seed = replicas.replica_seeds(GAUGE_SEED, SOURCE_SEED, rank)
    u = random_su3_field(DIMS, EPS, gauge_seed)
    b_np = gaussian_spinor(DIMS, source_seed)
    lat = Lattice(DIMS, DOMAIN, -1, "chiral", dev).setup(u, KAPPA, CSW)
    del u
    b_dev = torch.view_as_real(torch.from_numpy(b_np)).to(dev).contiguous()
    x_dev = torch.zeros_like(b_dev)

    def params(sap_prec, graph=2):
        p = B.qcd_solve_params_default()
        p.tol, p.n_sap, p.n_jac = 1e-10, N_SAP, N_JAC
        p.sap_prec = {"half": B.PREC_HALF, "half_gauge": B.PREC_HALF_GAUGE, "single": B.PREC_SINGLE}[sap_prec]
        # 1e-5 is the faster inner tolerance for both preconditioner precisions
        # at this workload (fewer inner iterations, still two outer steps)
        p.inner_tol = 1e-5
        p.max_inner = 1000
        p.use_graph = graph
        return p

    P_MIX = params("half")
    P_F32 = params("single")

    def barrier():
        replicas.barrier(world)
        torch.cuda.synchronize()

    def solve(p, xb=x_dev, bb=b_dev):
        rc, info = B.qcd_solve(lat.ctx, xb, bb, 1, p)
        return info

    def f64_resid(xb=x_dev, bb=b_dev):
        """|b - D x| / |b| of a solution with the native float64 D (outside
        every timed region): the check beside the double-float residual the
        solve stops on."""
        xi = lat.field("double")
        yi = lat.field("double")
        B.qcd_import_spinor(lat.ctx, xi, xb, B.PREC_DOUBLE)
        B.qcd_apply_D(lat.ctx, yi, xi, B.PREC_DOUBLE)
        y = torch.empty_like(bb)
        B.qcd_export_spinor(lat.ctx, y, yi, B.PREC_DOUBLE)
        return float(torch.linalg.vector_norm(bb - y) / torch.linalg.vector_norm(bb))

    # warm-up
    for _ in range(args.warmup):
        info = solve(P_MIX)
    # timed region: K full solves in the production setting (inner loop as
    # one CUDA graph with a conditional while node), CUDA events on the
    # launching stream, barrier + synchronize on both sides, nvidia-smi
    # clocks sampled throughout
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    smi_index = vis.split(",")[local] if vis else str(local)
    clocks = ClockSampler(smi_index)
    clocks.start()
    launches0 = B.qcd_launch_count(lat.ctx)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    infos = []
    for _ in range(args.steps):
        infos.append(solve(P_MIX))
    ev1.record()
    barrier()
    launches = B.qcd_launch_count(lat.ctx) - launches0
    resid_f64_check = f64_resid()
    elapsed = ev0.elapsed_time(ev1) / 1000.0
    elapsed = replicas.max_over_ranks(elapsed, world, device=dev)
    value = replicas.job_throughput(world, args.steps, elapsed)
    ms_per_step = 1000.0 * elapsed / args.steps
    graph_ms = ms_per_step

    # second timed region, same K solves with every launch bracketed by CUDA
    # events (kernels launched one by one): device time per kernel class and
    # the dominant kernel's average launch duration for the roofline
    for kc in range(5):
        B.qcd_profile_read(lat.ctx, kc, reset=True)
    P_PROF = params("half", graph=0)
    B.qcd_profile_enable(lat.ctx, True)
    barrier()
    # NVTX range: lets a kernel-list profiler select exactly these launches
    torch.cuda.nvtx.range_push("profiled_pass")
    tp = time.perf_counter()
    for _ in range(args.steps):
        solve(P_PROF)
    barrier()
    torch.cuda.nvtx.range_pop()
    prof_ms = 1000.0 * (time.perf_counter() - tp) / args.steps
    B.qcd_profile_enable(lat.ctx, False)
    clk = clocks.stop()
    prof = {kc: B.qcd_profile_read(lat.ctx, kc, reset=True) for kc in range(5)}

    # plain float32 SAP-BiCGStab (same defect correction), the comparison arm
    solve(P_F32)
    barrier()
    tf = time.perf_counter()
    nf = max(1, args.steps // 2)
    for _ in range(nf):
        info_f32 = solve(P_F32)
    barrier()
    f32_ms = 1000.0 * (time.perf_counter() - tf) / nf
    # the SAP variant with float16 links and C_inv but float32 vectors
    P_HG = params("half_gauge")
    solve(P_HG)
    barrier()
    th = time.perf_counter()
    for _ in range(nf):
        info_hg = solve(P_HG)
    barrier()
    hg_ms = 1000.0 * (time.perf_counter() - th) / nf
    # the same float16 SAP-BiCGStab inner solve under a flexible GMRES(4) outer iteration
    P_FG = params("half")
    P_FG.outer_restart = 4
    solve(P_FG)
    barrier()
    tg = time.perf_counter()
    for _ in range(nf):
        info_fg = solve(P_FG)
    barrier()
    fg_ms = 1000.0 * (time.perf_counter() - tg) / nf
    # the same solve with the residual of Algorithm 4 in native float64
    # instead of double-float arithmetic on the float32 pipes
    P_DF = params("half")
    P_DF.residual_prec = 1
    solve(P_DF)
    barrier()
    td = time.perf_counter()
    for _ in range(nf):
        info_df = solve(P_DF)
    barrier()
    df_ms = 1000.0 * (time.perf_counter() - td) / nf

    # Dslash: float32 D on the 32^4 field, CUDA events on the launching stream
    a32 = lat.field("single")
    o32 = lat.field("single")
    B.qcd_import_spinor(lat.ctx, a32, b_dev, B.PREC_SINGLE)
    for _ in range(5):
        B.qcd_apply_D(lat.ctx, o32, a32, B.PREC_SINGLE)
    nrep = 50
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(nrep):
        B.qcd_apply_D(lat.ctx, o32, a32, B.PREC_SINGLE)
    e1.record()
    torch.cuda.synchronize()
    d_ms = e0.elapsed_time(e1) / nrep
    vol = int(np.prod(DIMS))
    peak, peak_kind = measured_peaks()
    d_bytes = d_bytes_per_site(B.qcd_tuning_report(lat.ctx).strip().splitlines())
    d_gbs = d_bytes * vol / (d_ms * 1e-3) / 1e9
    d_gflops = D_FLOP_PER_SITE * vol / (d_ms * 1e-3) / 1e9

    # end to end through the public call with host buffers (pinned)
    b_host = torch.from_numpy(b_np.view(np.float64).reshape(b_dev.shape)).pin_memory()
    x_host = torch.zeros_like(b_host).pin_memory()
    barrier()
    te = time.perf_counter()
    ne = max(1, args.steps // 2)
    for _ in range(ne):
        rc, _ = B.qcd_solve(lat.ctx, x_host, b_host, 1, P_MIX)
    barrier()
    e2e_s = (time.perf_counter() - te) / ne
    e2e_s = replicas.max_over_ranks(e2e_s, world, device=dev)
    e2e_value = replicas.job_throughput(world, 1, e2e_s)

    tuning = B.qcd_tuning_report(lat.ctx).strip().splitlines()
    # float32 FMA throughput measured on this device (outside every timed region)
    fma_tflops = B.qcd_measure_fp32_peak(lat.ctx)

    # dominant kernel by device time in the timed region
    sap_n, sap_ms = prof[B.KC_SAP_BLOCK]
    total_ms = sum(v[1] for v in prof.values())
    sap_avg_ms = sap_ms / max(1, sap_n)
    sap_bytes = sap_bytes_per_site("half") * vol / 2
    sap_gbs = sap_bytes / (sap_avg_ms * 1e-3) / 1e9
    sap_tflops = sap_flop_per_site() * (vol / 2) / (sap_avg_ms * 1e-3) / 1e12
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "sap_block_traffic.json")
    if os.path.exists(tfile):
        with open(tfile) as fh:
            traffic = json.load(fh).get("bytes_per_launch_32x4")

    inner = int(np.median([i.inner_iters for i in infos]))
    outer = int(np.median([i.outer_iters for i in infos]))
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "precision": {"sap_storage": "f16", "krylov": "f32",
                      "correction": "double-float (2 x f32, ~48 bits) residual and x; the returned x "
                                    "re-checked with the native float64 D, true_resid_float64_check"},
        "config": {"workload": WORKLOAD, "lattice": list(DIMS), "domain": list(DOMAIN), "n_sap": N_SAP,
                   "n_jac": N_JAC, "tol": 1e-10, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (links + clover + vectors > 1 GB)"},
        "time_to_solution_ms": ms_per_step,
        "iterations": {"inner": inner, "outer": outer},
        "true_resid": max(i.true_resid for i in infos),
        "true_resid_float64_check": resid_f64_check,
        "plain_fp32": {"time_to_solution_ms": f32_ms, "inner": info_f32.inner_iters, "outer": info_f32.outer_iters,
                       "true_resid": info_f32.true_resid, "speedup_of_mixed": f32_ms / graph_ms},
        "variants_ms": {"f16_all_graph_loop": graph_ms, "f16_links_clover_f32_vectors_graph_loop": hg_ms,
                        "f32_graph_loop": f32_ms, "f16_all_no_graph_events_per_launch": prof_ms,
                        "f16_all_graph_loop_fgmres4_outer": fg_ms,
                        "f16_all_graph_loop_native_float64_residual": df_ms},
        "fgmres4_outer": {"inner": info_fg.inner_iters, "outer": info_fg.outer_iters, "true_resid": info_fg.true_resid},
        "native_float64_residual": {"inner": info_df.inner_iters, "outer": info_df.outer_iters,
                                    "true_resid": info_df.true_resid},
        "dslash": {"kernel": "dslash_kernel<float, D>", "ms": d_ms, "gbs": d_gbs, "gflops": d_gflops,
                   "bytes_per_site": d_bytes, "flop_per_site": D_FLOP_PER_SITE,
                   "frac_of_hbm": d_gbs / peak, "peak_gbs": peak, "peak_kind": peak_kind},
        "roofline": {"kernel": "sap_staged_kernel<float16 storage>", "bound": "alu", "achieved": sap_tflops,
                     "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": sap_tflops / FP32_PEAK_TFLOPS,
                     "traffic": traffic, "flop_per_site": sap_flop_per_site(), "sites_per_launch": vol // 2,
                     "avg_launch_ms": sap_avg_ms, "share_of_device_time": sap_ms / total_ms if total_ms else None,
                     "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
                     "measured_fp32_fma_tflops": fma_tflops,
                     "frac_of_measured_fma": sap_tflops / fma_tflops if fma_tflops else None,
                     "hbm_view": {"bytes_per_site": sap_bytes_per_site("half"), "achieved_gbs": sap_gbs,
                                  "frac_of_measured": sap_gbs / peak}},
        "kernel_classes_ms": {name: prof[k][1] for k, name in
                              ((B.KC_DSLASH, "dslash_A"), (B.KC_SAP_BLOCK, "sap_block"), (B.KC_BLAS, "blas"),
                               (B.KC_DOUBLE, "float64"), (B.KC_OTHER, "other"))},
        "clocks": clk,
        "tuning": tuning,
        "gpu_launches": int(launches),
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": int(b_host.numel() * 8),
                "d2h_bytes_per_step": int(x_host.numel() * 8)},
    }
    lat.close()
    del b_dev, x_dev, a32, o32, b_host, x_host
    torch.cuda.empty_cache()
    if not args.no_48:
        # the 48^4 batched target: 12 point sources solved in one batched
        # mixed-precision solve, against 12 sequential mixed and 12 sequential
        # plain float32 solves (outside the headline's timed region)
        import bench_configs
        barrier()
        line["batched_48x4_12_point_sources"] = bench_configs.batched_48x4_12_point_sources(reps=1)
        barrier()
    if not args.no_n2:
        # the paper's parameters (n_sap 4, n_jac 2) on its own 16x6x4x3 SAP
        # domains, per BiCGStab iteration, against Table 2's A64FX node
        import bench_configs
        line["paper_parameters_n2"] = bench_configs.n2_paper_domains(float32=False)
        barrier()
    if not args.no_ragged:
        # the ragged batch of 32 lattices (8^4..16^4) in shared launches, against
        # the same lattices as concurrent and as sequential solves
        import bench_configs
        line["ragged_batch_32"] = bench_configs.ragged_batch(reps=3, precs=("half",), dslash=False)
        barrier()
    if not args.no_grad:
        # gradients of Re(eta^dag D^-1 b) with respect to b and U at 16^4 and 32^4
        import bench_configs
        g4 = bench_configs.c4(argparse.Namespace(steps=5))
        line["gradient_16x4_32x4"] = dict(g4["results"], workload=g4["config"]["workload"])
        barrier()
    if not args.no_64:
        # 64^4: the float32 D's GB/s and the mixed against the plain float32 solve
        import bench_configs
        g5 = bench_configs.c5(argparse.Namespace(steps=2))
        line["lattice_64x4"] = dict(g5["results"], workload=g5["config"]["workload"])
        barrier()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_baseline(iters={"inner": inner, "outer": outer})
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
