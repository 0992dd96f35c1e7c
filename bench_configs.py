"""The other workloads of the solver, one JSON line each (``bench.py --config``).

c1        8^4, eps 0.3, kappa 0.12, c_sw 1.0: float32 SAP-BiCGStab to relative
          residual 1e-6 (the small solve).
c3        48^4, eps 0.25, kappa 0.125, c_sw 1.1: the 12 spin-colour point
          sources at the origin solved together (SAP with float16 links and
          C_inv + float32 BiCGStab + float64 correction to 1e-10, the inner
          loop one CUDA graph with a conditional while node)
          against 12 sequential plain float32 solves.
c4        16^4 and 32^4, eps 0.3, kappa 0.12, c_sw 1.0: gradients of
          Re(eta^dag D^-1 b) with respect to b and U (two solves + force
          kernels), and at 32^4 one solve for comparison.
c5        64^4, eps 0.2, kappa 0.126, c_sw 1.1: float32 Dslash roofline and the
          mixed-precision solve to 1e-10.
c5ragged  32 lattices with extents drawn from {8, 16} per direction,
          kappa ~ U[0.115, 0.125], seeds 5000 + i: the batched operator in one
          launch (GB/s) and the batched solve to 1e-10.
All times are CUDA-event or synchronised wall times on one GPU; inputs are
seeded and synthetic.
"""

import json
import os
import time

import numpy as np
import torch

from bench import D_BYTES_PER_SITE, D_FLOP_PER_SITE, ClockSampler, d_bytes_per_site, measured_peaks


def _smi_index():
    """nvidia-smi index of cuda:0 (the first visible device)."""
    import os
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    return vis.split(",")[0] if vis else "0"


def _lat(dims, eps, kappa, csw, seed, domain=(4, 4, 4, 4)):
    from lattice_inputs import random_su3_field, random_su3_field_fast
    from paper_2109_10687_gb300.lattice import Lattice
    vol = int(np.prod(dims))
    u = random_su3_field(dims, eps, seed) if vol <= 65536 else random_su3_field_fast(dims, eps, seed, "cuda")
    lat = Lattice(dims, domain, -1, "chiral", "cuda:0").setup(u, kappa, csw)
    return lat


def _params(sap_prec="half_gauge", tol=1e-10, graph=2):
    from paper_2109_10687_gb300 import binding as B
    p = B.qcd_solve_params_default()
    p.tol = tol
    p.sap_prec = {"half": B.PREC_HALF, "half_gauge": B.PREC_HALF_GAUGE, "single": B.PREC_SINGLE}[sap_prec]
    p.inner_tol = 1e-5
    p.max_inner = 2000
    p.use_graph = graph
    return p


def _timed(fn, reps):
    torch.cuda.synchronize()
    t = time.perf_counter()
    out = None
    for _ in range(reps):
        out = fn()
    torch.cuda.synchronize()
    return (time.perf_counter() - t) / reps, out


def _dslash_gbs(lat, b_dev, nrep=20):
    from paper_2109_10687_gb300 import binding as B
    a, o = lat.field("single"), lat.field("single")
    B.qcd_import_spinor(lat.ctx, a, b_dev, B.PREC_SINGLE)
    for _ in range(3):
        B.qcd_apply_D(lat.ctx, o, a, B.PREC_SINGLE)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(nrep):
        B.qcd_apply_D(lat.ctx, o, a, B.PREC_SINGLE)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / nrep
    vol = int(np.prod(lat.dims))
    peak, kind = measured_peaks()
    nbytes = d_bytes_per_site(B.qcd_tuning_report(lat.ctx).strip().splitlines())
    gbs = nbytes * vol / (ms * 1e-3) / 1e9
    return {"ms": ms, "gbs": gbs, "bytes_per_site": nbytes, "gflops": D_FLOP_PER_SITE * vol / (ms * 1e-3) / 1e9,
            "frac_of_hbm": gbs / peak, "peak_gbs": peak, "peak_kind": kind}


def c1(args):
    from lattice_inputs import gaussian_spinor
    from paper_2109_10687_gb300 import binding as B
    dims = (8, 8, 8, 8)
    lat = _lat(dims, 0.3, 0.12, 1.0, 1001)
    b = torch.view_as_real(torch.from_numpy(gaussian_spinor(dims, 2001))).cuda().contiguous()
    x = torch.zeros_like(b)
    res = {}
    for name, p in (("plain_f32", _params("single", 1e-6, 0)), ("plain_f32_graph_loop", _params("single", 1e-6, 2)),
                    ("mixed_f16_gauge_graph_loop", _params("half_gauge", 1e-6, 2))):
        for _ in range(3):
            B.qcd_solve(lat.ctx, x, b, 1, p)
        t, (rc, info) = _timed(lambda: B.qcd_solve(lat.ctx, x, b, 1, p), max(3, args.steps))
        res[name] = {"ms": 1e3 * t, "inner": info.inner_iters, "outer": info.outer_iters,
                     "true_resid": info.true_resid}
    return {"config": {"workload": "8^4, eps 0.3, kappa 0.12, c_sw 1.0, one Gaussian source, 4^4 domains, "
                                   "n_sap 4, n_jac 4, FP32 SAP-BiCGStab to relative residual 1e-6"},
            "metric": "time to relative residual 1e-6", "unit": "ms", "results": res}


def per_rhs_resid(lat, x, b, nrhs):
    """|b_i - D x_i| / |b_i| for each right-hand side, with the library's
    float64 D (canonical device fields in, one right-hand side at a time)."""
    from paper_2109_10687_gb300 import binding as B
    xi, dxi = lat.field("double"), lat.field("double")
    out = []
    for i in range(nrhs):
        B.qcd_import_spinor(lat.ctx, xi, x[i].contiguous(), B.PREC_DOUBLE)
        B.qcd_apply_D(lat.ctx, dxi, xi, B.PREC_DOUBLE)
        dx = torch.empty_like(b[i])
        B.qcd_export_spinor(lat.ctx, dx, dxi, B.PREC_DOUBLE)
        out.append(float(torch.linalg.vector_norm(b[i] - dx) / torch.linalg.vector_norm(b[i])))
    del xi, dxi
    return out


def batched_48x4_12_point_sources(reps=1, f32_vectors=False):
    """48^4, eps 0.25, kappa 0.125, c_SW 1.1, the 12 spin-colour point sources
    at the origin, to float64 true residual 1e-10, three ways on one GPU:
    one batched mixed-precision solve (float16-storage SAP, float32
    BiCGStab, float64 defect correction; all right-hand sides through every
    launch, the inner loop one graph), 12 sequential mixed-precision solves
    (the same precision without batching), and 12 sequential plain float32
    solves (float32 SAP; the comparison arm).  The ratio of the first two is
    the batching gain, of the last two the precision gain."""
    from lattice_inputs import point_source
    from paper_2109_10687_gb300 import binding as B
    dims = (48, 48, 48, 48)
    t_setup = time.perf_counter()
    lat = _lat(dims, 0.25, 0.125, 1.1, 1301)
    srcs = np.stack([point_source(dims, c, s) for c in range(3) for s in range(4)])
    b = torch.view_as_real(torch.from_numpy(srcs)).cuda().contiguous()
    del srcs
    x = torch.zeros_like(b)
    t_setup = time.perf_counter() - t_setup
    out = {}
    clk = ClockSampler(_smi_index())
    clk.start()
    B.qcd_solve(lat.ctx, x, b, 12, _params("half"))        # warm: allocations, tuning, graph
    t_batch, (rc, info) = _timed(lambda: B.qcd_solve(lat.ctx, x, b, 12, _params("half")), reps)
    res = per_rhs_resid(lat, x, b, 12)
    out["batched_mixed"] = {"s": t_batch, "inner": info.inner_iters, "outer": info.outer_iters,
                            "true_resid": info.true_resid, "true_resid_per_rhs": res, "status": rc,
                            "sap_storage": "f16 links, C_inv, vectors"}
    if f32_vectors:
        x.zero_()
        B.qcd_solve(lat.ctx, x, b, 12, _params("half_gauge"))
        t_h, (rc_h, info_h) = _timed(lambda: B.qcd_solve(lat.ctx, x, b, 12, _params("half_gauge")), reps)
        out["batched_mixed_f32_vectors"] = {"s": t_h, "inner": info_h.inner_iters, "outer": info_h.outer_iters,
                                            "true_resid": info_h.true_resid, "status": rc_h}
    b1 = [b[i].contiguous() for i in range(12)]
    x1 = [torch.zeros_like(b1[0]) for _ in range(12)]
    for name, prec in (("sequential_mixed", "half"), ("sequential_plain_f32", "single")):
        B.qcd_solve(lat.ctx, x1[0], b1[0], 1, _params(prec))    # warm
        per = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(12):
            rc_i, inf = B.qcd_solve(lat.ctx, x1[i], b1[i], 1, _params(prec))
            per.append({"inner": inf.inner_iters, "outer": inf.outer_iters, "true_resid": inf.true_resid,
                        "status": rc_i})
        torch.cuda.synchronize()
        out[name] = {"s": time.perf_counter() - t0, "inner_total": sum(q["inner"] for q in per),
                     "true_resid": max(q["true_resid"] for q in per), "per_rhs": per}
    out["speedup_vs_plain_f32"] = out["sequential_plain_f32"]["s"] / t_batch
    out["batching_gain"] = out["sequential_mixed"]["s"] / t_batch
    out["precision_gain"] = out["sequential_plain_f32"]["s"] / out["sequential_mixed"]["s"]
    out["faster_than_plain_f32"] = bool(t_batch < out["sequential_plain_f32"]["s"])
    out["setup_s"] = t_setup
    out["clocks"] = clk.stop()
    out["tuning"] = [ln for ln in B.qcd_tuning_report(lat.ctx).splitlines() if ln.startswith("sap_staged")]
    lat.close()
    return out


def c3(args):
    out = batched_48x4_12_point_sources(reps=1, f32_vectors=True)
    return {"config": {"workload": "48^4, eps 0.25, kappa 0.125, c_sw 1.1, 12 spin-colour point sources at the "
                                   "origin; batched float16-storage SAP + float32 BiCGStab + float64 "
                                   "correction to 1e-10 (device-side graph loop) vs 12 sequential mixed and "
                                   "12 sequential plain float32 solves (also with the graph loop)"},
            "metric": "time to FP64 residual 1e-10 for 12 right-hand sides", "unit": "s", "results": out}


def c4(args):
    from lattice_inputs import gaussian_spinor
    from paper_2109_10687_gb300 import binding as B
    dims = (16, 16, 16, 16)
    lat = _lat(dims, 0.3, 0.12, 1.0, 1401)
    eta = torch.view_as_real(torch.from_numpy(gaussian_spinor(dims, 3001))).cuda().contiguous()
    b = torch.view_as_real(torch.from_numpy(gaussian_spinor(dims, 3002))).cuda().contiguous()
    gb = torch.zeros_like(b)
    gu = torch.zeros(lat.site_shape + (4, 3, 3, 2), dtype=torch.float64, device="cuda")
    p = _params("half_gauge")
    B.qcd_grad(lat.ctx, eta, b, gb, gu, project=1, params=p)
    t, _ = _timed(lambda: B.qcd_grad(lat.ctx, eta, b, gb, gu, project=1, params=p), max(3, args.steps))
    res = {"ms": 1e3 * t}
    lat.close()
    # the same gradient at 32^4, where the device work dominates; a single
    # solve with the same parameters shows how much of it the two solves take
    dims = (32, 32, 32, 32)
    lat = _lat(dims, 0.3, 0.12, 1.0, 1401)
    eta = torch.view_as_real(torch.from_numpy(gaussian_spinor(dims, 3001))).cuda().contiguous()
    b = torch.view_as_real(torch.from_numpy(gaussian_spinor(dims, 3002))).cuda().contiguous()
    gb = torch.zeros_like(b)
    gu = torch.zeros(lat.site_shape + (4, 3, 3, 2), dtype=torch.float64, device="cuda")
    B.qcd_grad(lat.ctx, eta, b, gb, gu, project=1, params=p)
    t32, _ = _timed(lambda: B.qcd_grad(lat.ctx, eta, b, gb, gu, project=1, params=p), 3)
    x = torch.zeros_like(b)
    B.qcd_solve(lat.ctx, x, b, 1, p)
    ts, _ = _timed(lambda: B.qcd_solve(lat.ctx, x, b, 1, p), 3)
    res["ms_32x4"] = 1e3 * t32
    res["one_solve_ms_32x4"] = 1e3 * ts
    res["beyond_two_solves_ms_32x4"] = 1e3 * (t32 - 2 * ts)
    lat.close()
    return {"config": {"workload": "16^4 and 32^4, eps 0.3, kappa 0.12, c_sw 1.0: gradients of Re(eta^dag D^-1 b) "
                                   "wrt b and U (su(3)-projected), two mixed-precision solves + force kernels"},
            "metric": "time per gradient", "unit": "ms", "results": res}


def c5(args):
    from lattice_inputs import gaussian_spinor
    from paper_2109_10687_gb300 import binding as B
    dims = (64, 64, 64, 64)
    lat = _lat(dims, 0.2, 0.126, 1.1, 1501)
    b = torch.view_as_real(torch.from_numpy(gaussian_spinor(dims, 2501))).cuda().contiguous()
    clk = ClockSampler(_smi_index())
    clk.start()
    d = _dslash_gbs(lat, b)
    x = torch.zeros_like(b)
    B.qcd_solve(lat.ctx, x, b, 1, _params("half_gauge"))
    t, (rc, info) = _timed(lambda: B.qcd_solve(lat.ctx, x, b, 1, _params("half_gauge")), 2)
    check = per_rhs_resid(lat, x.unsqueeze(0), b.unsqueeze(0), 1)[0]
    B.qcd_solve(lat.ctx, x, b, 1, _params("single"))  # first use: the float32 shapes are tuned here
    tf, (rcf, infof) = _timed(lambda: B.qcd_solve(lat.ctx, x, b, 1, _params("single")), 1)
    out = {"config": {"workload": "64^4, eps 0.2, kappa 0.126, c_sw 1.1, one Gaussian source"},
           "metric": "Dslash GB/s; time to FP64 residual 1e-10", "unit": "GB/s; s",
           "results": {"dslash": d, "mixed_solve_s": t, "inner": info.inner_iters, "outer": info.outer_iters,
                       "true_resid": info.true_resid, "true_resid_float64_check": check, "plain_f32_solve_s": tf,
                       "plain_inner": infof.inner_iters, "speedup_of_mixed": tf / t, "clocks": clk.stop()}}
    lat.close()
    return out


def ragged_batch(reps=3, precs=("half", "half_gauge"), dslash=True):
    """32 lattices with extents drawn from {8, 16} per direction (seed 5000),
    kappa ~ U[0.115, 0.125], eps 0.3, c_SW 1.0, one Gaussian source each
    (seed 7000 + i), to float64 true residual 1e-10: the solve in shared
    launches, the same batch as 32 concurrent solves (one host thread and
    stream each) and as 32 solves one after the other; and the batched
    operator in one launch."""
    from lattice_inputs import gaussian_spinor
    from paper_2109_10687_gb300 import binding as B
    rng = np.random.default_rng(5000)
    lats, bs, ins, outs, vols = [], [], [], [], []
    for i in range(32):
        dims = tuple(int(v) for v in rng.choice([8, 16], size=4))
        kappa = float(rng.uniform(0.115, 0.125))
        lat = _lat(dims, 0.3, kappa, 1.0, 5000 + i)
        b = torch.view_as_real(torch.from_numpy(gaussian_spinor(dims, 7000 + i))).cuda().contiguous()
        lats.append(lat)
        bs.append(b)
        vols.append(int(np.prod(dims)))
    bt = B.qcd_batch_create([l.ctx for l in lats])
    res = {"sites": sum(vols)}
    if dslash:
        for lat, b in zip(lats, bs):
            a = lat.field("single")
            B.qcd_import_spinor(lat.ctx, a, b, B.PREC_SINGLE)
            ins.append(a)
            outs.append(lat.field("single"))
        for _ in range(3):
            B.qcd_batch_apply_D(bt, outs, ins)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        nrep = 20
        for _ in range(nrep):
            B.qcd_batch_apply_D(bt, outs, ins)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / nrep
        peak, kind = measured_peaks()
        # bytes of the link format the lattices' operators use (12 or 18 reals)
        nbytes = sum((D_BYTES_PER_SITE - 4 * 24 if B.qcd_link_format(l.ctx) == 12 else D_BYTES_PER_SITE) * v
                     for l, v in zip(lats, vols))
        gbs = nbytes / (ms * 1e-3) / 1e9
        res["dslash_batched"] = {"ms": ms, "gbs": gbs, "frac_of_hbm": gbs / peak, "peak_kind": kind}
    xs = [torch.zeros_like(b) for b in bs]
    solves = {}
    for prec in precs:
        # shared launches: every SAP half-sweep, operator and BLAS-1 step of an
        # iteration one launch over the 32 lattices, the inner loop one graph
        B.qcd_batch_set_shared(bt, True)
        B.qcd_batch_solve(bt, xs, bs, _params(prec))
        n0 = B.qcd_launch_count(lats[0].ctx)
        t, (rc, infos) = _timed(lambda: B.qcd_batch_solve(bt, xs, bs, _params(prec)), reps)
        launches = (B.qcd_launch_count(lats[0].ctx) - n0) / reps
        # the same batch as 32 concurrent solves (one host thread and stream each)
        B.qcd_batch_set_shared(bt, False)
        B.qcd_batch_solve(bt, xs, bs, _params(prec))
        tc, (rcc, infosc) = _timed(lambda: B.qcd_batch_solve(bt, xs, bs, _params(prec)), reps)
        B.qcd_batch_set_shared(bt, True)
        # and as 32 solves one after the other
        ones = [torch.zeros_like(b) for b in bs]
        for lat, x1, b1 in zip(lats, ones, bs):
            B.qcd_solve(lat.ctx, x1, b1, 1, _params(prec))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            for lat, x1, b1 in zip(lats, ones, bs):
                B.qcd_solve(lat.ctx, x1, b1, 1, _params(prec))
        torch.cuda.synchronize()
        ts = (time.perf_counter() - t0) / reps
        solves[prec] = {
            "shared_launches_s": t, "status": rc, "worst_true_resid": max(i.true_resid for i in infos),
            "inner_per_lattice": [i.inner_iters for i in infos], "outer_per_lattice": [i.outer_iters for i in infos],
            "launches_per_batch_solve": launches,
            "concurrent_threads_s": tc, "concurrent_worst_true_resid": max(i.true_resid for i in infosc),
            "sequential_s": ts, "speedup_vs_sequential": ts / t, "speedup_vs_concurrent": tc / t}
    res["batched_solve"] = solves
    B.qcd_batch_destroy(bt)
    for lat in lats:
        lat.close()
    return res


def c5ragged(args):
    res = ragged_batch(reps=max(3, args.steps))
    return {"config": {"workload": "ragged batch of 32 lattices, extents from {8, 16} per direction, eps 0.3, "
                                   "kappa ~ U[0.115, 0.125], c_sw 1.0, seeds 5000 + i", "sites": res["sites"]},
            "metric": "batched Dslash GB/s (one launch); batched solve time to 1e-10", "unit": "GB/s; s",
            "results": res}


# Per-site flop of one SAP-BiCGStab iteration in the paper's accounting
# (Sec. 4; reproduces its Tables 2-3): 168 flop per hop (156 for a temporal
# hop in the paper's basis, 168 in the chiral basis used here), 600 per C_inv
# apply with the axpy, 48 per residual update.
def _paper_flop_per_site_iter(domain, n_sap, n_jac, hops=(168, 168, 168, 168)):
    f_in = 600 + sum(2 * (1 - 1 / d) * h for d, h in zip(domain, hops))
    inner = vol = 1
    for d in domain:
        inner *= max(d - 2, 0)
        vol *= d
    f_out = sum(2 / d * h for d, h in zip(domain, hops)) + 600 * (1 - inner / vol)
    return 2 * (n_sap + 1) * (f_in + n_jac * (f_in + 48) + f_out) + 96 * n_sap + 48 + 1008


# One A64FX node's site-iterations per second for the paper's SAP domain
# shapes: Table 2 times 500 iterations on a process block of two domains
# (the block's extent in x is twice the domain's); a node runs 4 processes.
def _a64fx_node_rate(domain):
    table2 = {(16, 6, 4, 3): 0.334867, (16, 6, 4, 6): 0.515010}  # seconds for 500 iterations
    block_sites = 2 * int(np.prod(domain))
    return 4 * block_sites * 500 / table2[domain]


def _n2_rate(lat, dims, prec, flop, flop_paper_basis=None, n_sap=4, n_jac=2, node_rate=1.38e7):
    """ms per BiCGStab iteration from the difference of two fixed-length solves
    (10 and 30 iterations, one outer step, graph loop)."""
    from lattice_inputs import gaussian_spinor
    from paper_2109_10687_gb300 import binding as B
    vol = int(np.prod(dims))
    b = torch.view_as_real(torch.from_numpy(gaussian_spinor(dims, 2001))).cuda().contiguous()
    x = torch.zeros_like(b)
    times = {}
    for iters in (10, 30):
        p = _params(prec, 1e-30, 2)
        p.n_sap, p.n_jac = n_sap, n_jac
        p.inner_tol, p.max_inner, p.max_outer = 1e-30, iters, 1
        B.qcd_solve(lat.ctx, x, b, 1, p, raise_on_error=False)
        t, (rc, info) = _timed(lambda: B.qcd_solve(lat.ctx, x, b, 1, p, raise_on_error=False), 3)
        times[iters] = (t, info.inner_iters)
    (t1, i1), (t2, i2) = times[10], times[30]
    t_iter = (t2 - t1) / max(1, i2 - i1)
    r = {"lattice": list(dims), "ms_per_iteration": 1e3 * t_iter, "iterations": [i1, i2],
         "site_iterations_per_s": vol / t_iter, "flop_per_site_iteration": flop,
         "tflops_paper_accounting": flop * vol / t_iter / 1e12,
         "a64fx_node_site_iterations_per_s": node_rate, "vs_a64fx_node_site_iterations": vol / t_iter / node_rate}
    if flop_paper_basis is not None:
        r["flop_per_site_iteration_paper_basis"] = flop_paper_basis
        r["tflops_paper_accounting_paper_basis"] = flop_paper_basis * vol / t_iter / 1e12
    return r


def n2_paper_domains(float32=True):
    """The paper's parameters (n_sap 4, n_jac 2) on 64x24x32x24 with its own
    16x6x4x3 SAP domains (float16 links and C_inv on the cluster kernel; and
    float32 on the one-CTA kernel), its 16x6x4x6 domains and 4^4 domains,
    against one A64FX node (Table 2's row for the same domains; 4^4 against
    its first row, 1.38e7 site-iterations/s)."""
    from paper_2109_10687_gb300 import binding as B
    n_sap, n_jac = 4, 2
    out = {}
    dims = (64, 24, 32, 24)
    lat = _lat(dims, 0.3, 0.125, 1.0, 1001, (4, 4, 4, 4))
    out["float32_domains_4x4x4x4"] = _n2_rate(lat, dims, "single", _paper_flop_per_site_iter((4, 4, 4, 4), n_sap, n_jac))
    paper = (16, 6, 4, 3)
    B.qcd_set_sap_domain(lat.ctx, paper)
    # chiral basis (168 flop for every hop, what the kernels compute) and the
    # paper's basis (156 for a temporal hop), which reproduces Tables 2-3
    fl, fl_paper = (_paper_flop_per_site_iter(paper, n_sap, n_jac),
                    _paper_flop_per_site_iter(paper, n_sap, n_jac, hops=(168, 168, 168, 156)))
    out["float16_gauge_domains_16x6x4x3"] = _n2_rate(lat, dims, "half_gauge", fl, fl_paper,
                                                     node_rate=_a64fx_node_rate(paper))
    if float32:
        out["float32_domains_16x6x4x3"] = _n2_rate(lat, dims, "single", fl, fl_paper,
                                                   node_rate=_a64fx_node_rate(paper))
    # Table 2's fastest row: 16x6x4x6 domains (six time slices per cluster)
    paper6 = (16, 6, 4, 6)
    B.qcd_set_sap_domain(lat.ctx, paper6)
    out["float16_gauge_domains_16x6x4x6"] = _n2_rate(
        lat, dims, "half_gauge", _paper_flop_per_site_iter(paper6, n_sap, n_jac),
        _paper_flop_per_site_iter(paper6, n_sap, n_jac, hops=(168, 168, 168, 156)), node_rate=_a64fx_node_rate(paper6))
    out["tuning"] = [ln for ln in B.qcd_tuning_report(lat.ctx).splitlines() if ln.startswith("sap_general")]
    lat.close()
    return out


def n2(args):
    """The paper's algorithm parameters (n_sap 4, n_jac 2): BiCGStab iterations
    per second and the rate in the paper's flop accounting.  Paper, one A64FX
    node (4 processes): 1.38e7 site-iterations/s, 0.83 TFLOPS (Table 2, first
    row, 32x6x4x3 per process = two 16x6x4x3 domains).  Measured on 32^4 with
    4^4 domains (the shared-memory block kernel), and on 64x24x32x24 with the
    paper's own 16x6x4x3 domains and with 4^4 domains."""
    out = {}
    dims, domain, n_sap, n_jac = (32, 32, 32, 32), (4, 4, 4, 4), 4, 2
    flop = _paper_flop_per_site_iter(domain, n_sap, n_jac)
    lat = _lat(dims, 0.3, 0.125, 1.0, 1001, domain)
    for name, prec in (("float32", "single"), ("float16_storage", "half")):
        out[name] = _n2_rate(lat, dims, prec, flop)
    lat.close()
    for k, v in n2_paper_domains().items():
        out["64x24x32x24_" + k] = v
    return {"config": {"workload": "eps 0.3, kappa 0.125, c_sw 1.0; SAP-BiCGStab with the paper's n_sap 4, n_jac 2: "
                                   "32^4 on 4^4 domains; 64x24x32x24 on the paper's 16x6x4x3 domains and on 4^4 "
                                   "domains; fixed iteration counts (graph loop)"},
            "metric": "BiCGStab iterations: site-iterations/s and TFLOPS in the paper's flop accounting",
            "unit": "site-iterations/s", "results": out}


def _oracle_cpu_task(job):
    """One single-threaded oracle timing job (runs in a spawned worker):
    ("D", dims) times one float64 D apply, ("iter", dims) one SAP-BiCGStab
    iteration (two A M_SAP applications, n_sap 4, n_jac 4, 4^4 domains),
    both after building the operator outside the clock."""
    from lattice_inputs import gaussian_spinor, random_su3_field
    from oracle import sap
    from oracle.dirac import CloverWilson
    from oracle.gamma import gamma_chiral
    if job is None:
        return None
    kind, dims = job
    op = CloverWilson(random_su3_field(dims, 0.3, 1001), 0.125, 1.0, gamma_chiral(), bc_t=-1, domain=(4, 4, 4, 4))
    x = gaussian_spinor(dims, 2001)
    if kind == "D":
        op.D(x)
        t0 = time.perf_counter()
        op.D(x)
        return time.perf_counter() - t0
    t0 = time.perf_counter()
    y = sap.am_sap(op, x, 4, 4)
    sap.am_sap(op, y, 4, 4)
    return time.perf_counter() - t0


def _oracle_pool(jobs, procs):
    """Run oracle timing jobs on `procs` single-threaded spawned workers;
    returns (wall seconds, per-job results)."""
    import multiprocessing as mp
    import bench as bn
    saved = {k: os.environ.get(k) for k in bn._ONE_THREAD_ENV}
    for k in bn._ONE_THREAD_ENV:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(procs) as pool:
            pool.map(_oracle_cpu_task, [None] * procs, chunksize=1)
            t0 = time.perf_counter()
            res = pool.map(_oracle_cpu_task, jobs, chunksize=1)
            return time.perf_counter() - t0, res
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def cpu(args):
    """The float64 oracle timed on the host cores, each worker process one
    thread (numpy's elementwise work is single-threaded, so all cores means
    one independent job per core):
    - D apply at 8^4, 16^4 and 32^4 on one thread, and one 16^4 apply per
      core at once; bytes counted as the float32 D's 768 B per site doubled
      for float64 (1536 B), 1824 flop per site;
    - the 8^4 solve of the main benchmark's recipe (Algorithm 4 around
      Algorithm 5 to 1e-10) on one thread and one per core at once;
    - one SAP-BiCGStab iteration at 16^4 on one thread.  Solves at 16^4 and
      above take the oracle tens of minutes (an A M_SAP application costs
      about 20 s at 16^4), so their per-iteration times at 32^4, 48^4 and
      64^4 are extrapolated by volume from the 16^4 figure and labelled so."""
    import bench as bn
    cores = bn.host_cores()
    out = {"host_cores": cores, "threads_per_process": 1}
    apply = {}
    for L in (8, 16, 32):
        _, (t,) = _oracle_pool([("D", (L,) * 4)], 1)
        v = L ** 4
        apply[f"{L}^4_one_thread"] = {"s": t, "gsites_per_s": v / t / 1e9, "gbs": 1536 * v / t / 1e9,
                                      "gflops": 1824 * v / t / 1e9}
    _, ts = _oracle_pool([("D", (16,) * 4)] * cores, cores)
    v = 16 ** 4
    agg = sum(v / t for t in ts)
    apply["16^4_all_cores"] = {"processes": cores, "gsites_per_s": agg / 1e9, "gbs": 1536 * agg / 1e9,
                               "gflops": 1824 * agg / 1e9}
    out["D_apply_f64"] = apply
    wall1, (rec,) = bn.oracle_solves(1, 1, 0, bn.ORACLE_DIMS)
    wallc, recs = bn.oracle_solves(cores, cores, 0, bn.ORACLE_DIMS)
    out["solve_8^4_to_1e-10"] = {"one_thread_s": wall1, "inner": rec["inner"], "outer": rec["outer"],
                                 "true_resid": rec["true_resid"], "all_cores_solves_per_s": cores / wallc,
                                 "all_converged": all(r["converged"] for r in recs + [rec])}
    _, (ti,) = _oracle_pool([("iter", (16,) * 4)], 1)
    per_site = ti / 16 ** 4
    out["sap_bicgstab_iteration_one_thread"] = {
        "16^4_s": ti,
        "extrapolated_by_volume_s": {f"{L}^4": per_site * L ** 4 for L in (32, 48, 64)}}
    return {"config": {"workload": "float64 oracle (numpy) on the host cores: D apply at 8^4, 16^4, 32^4; "
                                   "8^4 solves to 1e-10; one SAP-BiCGStab iteration at 16^4 "
                                   "(eps 0.3, kappa 0.125, c_sw 1.0, n_sap 4, n_jac 4, 4^4 domains)"},
            "metric": "oracle rates", "unit": "mixed (see keys)", "results": out}


def run(args):
    if args.config != "cpu":
        torch.cuda.set_device(0)
    fn = {"c1": c1, "c3": c3, "c4": c4, "c5": c5, "c5ragged": c5ragged, "n2": n2, "cpu": cpu}[args.config]
    line = fn(args)
    line["name"] = args.config
    print(json.dumps(line))
