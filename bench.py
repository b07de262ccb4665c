"""Benchmark of the RPIM global stiffness assembly on GB300.

Workload: the 129 x 17 x 17 cantilever (37,281 field nodes, 298,248 Gauss
points, support radius 2.5h, multiquadric alpha_c = 4, q = 1.03), FP64,
seeded synthetic node cloud. One step is the whole assembly path of Sec. 2's
first stage on device-resident inputs: rpim_build_pattern (Gauss points,
cell list, supports, node incidence, BSR pattern) + rpim_assemble (shape
functions, B^T D B, deterministic reduction) + rpim_add_point_loads. The
penalty stage and the PCG solve are timed once after the timed steps and
reported under "solve" (full solves/s). "batched" compares one batched
pattern + assembly + batched PCG over blocks of the 512-block workload with
the same blocks run one by one through the plain entry points.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank assembles its own replica (weak scaling, no data
exchange; timing is max over ranks). Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

import gen

METRIC = "RPIM assembly Gauss-pts/s, % of FP64/HBM roofline; batched vs per-instance"
UNIT = "Gauss-pts/s"
WORKLOAD = ("cantilever 129x17x17 (37,281 nodes, 298,248 Gauss points), interior jitter 0.2h, "
            "alpha_s 2.5, MQ alpha_c 4.0 q 1.03, E 1e4 nu 0.3, FP64")


def _hbm_peak():
    """Measured copy bandwidth of this GPU pool (GB/s), else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured copy bandwidth, MEASURED_PEAKS.json (of measured)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback copy bandwidth 6.8 TB/s (of fallback)"


HBM_PEAK, HBM_SRC = _hbm_peak()


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# --------------------------------------------------------------------------- flop model
def shape_flops(n):
    """Algorithmic flops of one point's shape functions (moment matrix with one
    kernel evaluation per pair counted as one flop, LU of the (n+4) system,
    four solves, right-hand sides)."""
    n = np.asarray(n, dtype=np.float64)
    N = n + 4
    return 2 * N**3 / 3 + 8 * N**2 + 5 * n * (n - 1) + 16 * n


def pair_flops(n):
    """Algorithmic flops of one point's B^T D B contributions (45 per pair of
    the upper triangle, diagonal included)."""
    n = np.asarray(n, dtype=np.float64)
    return 22.5 * n * (n + 1)


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "power_w_max": max(pw), "samples": len(sm)}


# --------------------------------------------------------------------------- traffic record
def _traffic_for(kernel, source):
    """DRAM bytes of `kernel` per step (all its launches in one step) from the
    committed ncu summary, if the kernel's source is unchanged since the
    counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    sha = hashlib.sha256(open(source, "rb").read()).hexdigest()[:16]
    for line in open(path):
        kv = dict(tok.split("=", 1) for tok in line.split() if "=" in tok)
        if kv.get("kernel") == kernel and kv.get("source_sha256") == sha:
            try:
                return float(kv["dram_bytes_per_step"])
            except (KeyError, ValueError):
                return None
    return None


# --------------------------------------------------------------------------- ranks
def max_over_ranks(x, dist, device):
    """The largest value of a per-rank host float over all ranks (the
    slowest replica sets the time); the value itself with one rank."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms):
    """Units processed by all ranks per second, every rank doing
    `units_per_rank` in `ms` milliseconds (weak scaling: replicas)."""
    return world * units_per_rank / (ms / 1e3)


# --------------------------------------------------------------------------- CPU baseline
def _spread(n, m):
    """Every k-th of n items, m of them (a sample spread evenly over the
    workload, interior and boundary points in their proportions)."""
    k = max(1, n // max(1, m))
    return slice(0, k * min(m, n), k), k


def cpu_baseline(p, budget_s=15.0):
    """The oracle (FP64, OpenMP over points on all host cores) on M Gauss
    points spread evenly over the workload, M sized to about `budget_s`
    seconds; and the same oracle on one thread on a smaller spread sample."""
    import oracle
    oracle.build()
    cores = _cores()
    oracle.set_threads(cores)
    pts, wj = oracle.gauss_points(p.cell_lo, p.cell_hi)

    def run(m):
        sel, k = _spread(len(pts), m)
        t0 = time.perf_counter()
        oracle.assemble(p.xyz, pts[sel], wj[sel], p.E[sel], p.nu[sel], p.alpha_s, p.alpha_c, p.q, p.h)
        return time.perf_counter() - t0, len(pts[sel]), k

    m0 = 1024
    t0, _, _ = run(m0)
    m = int(min(len(pts), max(m0, m0 * budget_s / max(t0, 1e-3))))
    dt, m, k = run(m)
    oracle.set_threads(1)
    dt1, m1, k1 = run(max(256, m // (2 * cores)))
    oracle.set_threads(cores)
    return {"value": m / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "every %d-th of the %d Gauss points of the workload (%d, %.1f%%), f64 oracle, OpenMP %d "
                      "threads, %.1f s" % (k, len(pts), m, 100.0 * m / len(pts), cores, dt),
            "single_thread": {"value": m1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": "every %d-th Gauss point (%d), f64 oracle, 1 thread, %.1f s" % (k1, m1, dt1)}}


# --------------------------------------------------------------------------- reference arm
def run_reference(args, rank):
    if rank != 0:
        return
    p = gen.cantilever_config()
    import oracle
    oracle.build()
    cores = _cores()
    oracle.set_threads(cores)
    pts, wj = oracle.gauss_points(p.cell_lo, p.cell_hi)

    def step(m):
        sel, _ = _spread(len(pts), m)
        t0 = time.perf_counter()
        oracle.assemble(p.xyz, pts[sel], wj[sel], p.E[sel], p.nu[sel], p.alpha_s, p.alpha_c, p.q, p.h)
        return time.perf_counter() - t0

    # size each step to about 4 s of host work
    t = step(1024)
    m = int(min(len(pts), max(1024, 1024 * 4.0 / max(t, 1e-3))))
    for _ in range(args.warmup):
        step(m)
    times = [step(m) for _ in range(args.steps)]
    ms = 1e3 * sum(times) / len(times)
    value = m / (ms / 1e3)
    sample = ("%d of the %d Gauss points of the workload per step, spread evenly (every %d-th), f64 oracle, "
              "OpenMP %d threads" % (len(pts[_spread(len(pts), m)[0]]), len(pts), _spread(len(pts), m)[1], cores))
    out = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample_points": m},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# --------------------------------------------------------------------------- stages 2 and 3
def _solve(pat, p, E, nu, lxyz, lf, tt, stream, peak_gflops, fixed_iters=0):
    """Penalty (alpha = 1e8 max diag K) and Jacobi-PCG to 1e-10, timed once
    with CUDA events; the assembly that feeds it is not timed."""
    import torch
    K, f = pat.assemble(E, nu)
    pat.add_point_loads(lxyz, lf, f)
    dofs, vals = tt(p.fixed_dofs, torch.int64), tt(p.fixed_vals)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    alpha = pat.apply_penalty(K, f, dofs, vals)
    if fixed_iters > 0:   # a fixed number of iterations (profiling runs)
        u, iters, relres = pat.solve_pcg(K, f, rtol=0.0, max_iter=fixed_iters, check=False)
    else:
        u, iters, relres = pat.solve_pcg(K, f, rtol=1e-10, max_iter=200000)
    s1.record(stream)
    torch.cuda.synchronize()
    solve_ms = s0.elapsed_time(s1)
    tip = int(np.nonzero(np.all(np.abs(p.nominal - [8.0, 0.5, 0.5]) < 1e-9, axis=1))[0][0])
    nnzb = pat.nnz_blocks
    # per-kernel times of the iteration: 256 more iterations with event timing
    import paper_1802_04256_gb300 as R
    R.rpim_profile_read(reset=True)
    R.rpim_profile_enable(True)
    pat.solve_pcg(K, f, u.clone(), rtol=0.0, max_iter=256, check=False)
    R.rpim_profile_enable(False)
    prof = R.rpim_profile_read(reset=True)
    spmv_bytes = nnzb * (72 + 4) + p.n_nodes * (8 + 24 + 24)
    roof = None
    if "pcg_spmv" in prof:
        # 9 FMA per 3x3 block: on this chip the FP64 time of a product
        # (18 nnzb / DFMA peak) exceeds its HBM time (bytes / copy bandwidth)
        c, tot = prof["pcg_spmv"]
        t = tot / c / 1e3
        t_alu, t_hbm = 18 * nnzb / (peak_gflops * 1e9), spmv_bytes / (HBM_PEAK * 1e9)
        if t_alu >= t_hbm:
            ach = 18 * nnzb / t / 1e12
            roof = {"bound": "alu", "achieved": ach, "peak": peak_gflops / 1e3, "unit": "TFLOP/s",
                    "frac": ach * 1e3 / peak_gflops, "peak_source": "FP64 DFMA throughput measured in this run"}
        else:
            ach = spmv_bytes / t / 1e9
            roof = {"bound": "hbm", "achieved": ach, "peak": HBM_PEAK, "unit": "GB/s", "frac": ach / HBM_PEAK,
                    "peak_source": HBM_SRC}
        roof.update({"kernel": "pcg_spmv", "algorithmic_bytes_per_launch": spmv_bytes,
                     "algorithmic_flops_per_launch": 18 * nnzb, "hbm_GBps": spmv_bytes / t / 1e9,
                     "hbm_frac": spmv_bytes / t / 1e9 / HBM_PEAK, "avg_launch_ms": tot / c})
    out = {"pcg_iterations": iters, "relres": relres, "ms": solve_ms, "solves_per_s": 1e3 / solve_ms,
           "ms_per_iteration": solve_ms / max(iters, 1), "penalty_alpha": alpha,
           "tip_deflection": -u[3 * tip + 2].item(), "timoshenko": 0.20700,
           "spmv_algorithmic_bytes": spmv_bytes, "spmv_flops": 18 * nnzb, "spmv_roofline": roof,
           "iteration_kernel_ms": {k: round(v[1] / v[0], 4) for k, v in prof.items()}}
    del K, f, u
    pat.free()
    return out


# --------------------------------------------------------------------------- MLS variant
def _mls(p, xyz, lo, hi, E, nu, lxyz, lf, stream, peak_gflops, steps=3):
    """The same assembly step with MLS shape functions (linear basis,
    cubic-spline weight; the variant Sec. 4 plans): rpim_build_pattern +
    rpim_pattern_set_shape(MLS) + rpim_assemble + rpim_add_point_loads,
    device-resident inputs, CUDA events on the launching stream, per-kernel
    device times from the library's own event timing."""
    import torch
    import paper_1802_04256_gb300 as R

    def step():
        pat = R.Pattern(xyz, lo, hi, p.alpha_s, p.alpha_c, p.q, p.h, shape="mls")
        K, f = pat.assemble(E, nu)
        pat.add_point_loads(lxyz, lf, f)
        pat.free()

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    R.rpim_profile_read(reset=True)
    R.rpim_profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    R.rpim_profile_enable(False)
    prof = R.rpim_profile_read(reset=True)
    ms = e0.elapsed_time(e1) / steps
    pat = R.Pattern(xyz, lo, hi, p.alpha_s, p.alpha_c, p.q, p.h)
    nsup = np.diff(pat.points()[2].cpu().numpy())
    pat.free()
    roof = None
    if "row" in prof:
        nl, tot = prof["row"]
        ach = pair_flops(nsup).sum() / (tot / steps / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": "row", "achieved": ach, "peak": peak_gflops / 1e3, "unit": "TFLOP/s",
                "frac": ach * 1e3 / peak_gflops, "peak_source": "FP64 DFMA throughput measured in this run"}
    return {"step": "rpim_build_pattern + rpim_pattern_set_shape(MLS) + rpim_assemble + rpim_add_point_loads",
            "workload": WORKLOAD.replace("MQ alpha_c 4.0 q 1.03", "MLS linear basis, cubic-spline weight"),
            "steps": steps, "ms_per_step": ms, "pts_per_s": p.n_points / (ms / 1e3),
            "kernel_ms_per_step": {k: round(v[1] / steps, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])},
            "roofline_row_kernel": roof}


# --------------------------------------------------------------------------- differentiable solve
def _backanalysis(dev, stream, rtol=1e-10):
    """One gradient of the back-analysis misfit L = 1/2 sum |u - u_obs|^2 at
    500 observed nodes with respect to the per-point E and nu of the
    64 x 32 x 32 block (524,288 points): forward = assembly + frozen penalty
    + PCG, backward = adjoint PCG + the per-point gradient kernel. Timed once
    with CUDA events after one untimed gradient."""
    import torch
    import paper_1802_04256_gb300 as R
    p = gen.backanalysis_config()
    tt = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    pat = R.Pattern.from_problem(p)
    f_ext = torch.zeros(3 * p.n_nodes, dtype=torch.float64, device=dev)
    pat.add_point_loads(tt(p.load_xyz), tt(p.load_force), f_ext)
    dofs, vals = tt(p.fixed_dofs, torch.int64), tt(p.fixed_vals)
    obs = tt(p.meta["obs_nodes"], torch.int64)
    E0, nu0 = tt(p.E), tt(p.nu)
    alpha = R.penalty_alpha(pat, E0, nu0)
    with torch.no_grad():   # observations: displacements of the hidden field
        u_obs = R.solve(pat, tt(p.meta["E_hidden"]), tt(p.meta["nu_hidden"]), f_ext, dofs, vals, alpha,
                        rtol=rtol).view(-1, 3)[obs].clone()

    def one():
        E = E0.clone().requires_grad_()
        nu = nu0.clone().requires_grad_()
        e0, e1, e2 = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        e0.record(stream)
        u = R.solve(pat, E, nu, f_ext, dofs, vals, alpha, rtol=rtol)
        loss = 0.5 * ((u.view(-1, 3)[obs] - u_obs) ** 2).sum()
        e1.record(stream)
        loss.backward()
        e2.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), e1.elapsed_time(e2), float(E.grad.abs().max()), float(nu.grad.abs().max())

    one()
    fwd, bwd, gE, gn = one()
    pat.free()
    return {"workload": "back-analysis block 64x32x32 (65,536 nodes, 524,288 points), log-normal E field, "
                        "500 observed nodes", "parameters": 2 * p.n_points, "rtol": rtol,
            "forward_ms": fwd, "backward_ms": bwd, "gradients_per_s": 1e3 / (fwd + bwd),
            "max_abs_dL_dE": gE, "max_abs_dL_dnu": gn,
            "step": "forward: rpim_assemble + rpim_apply_penalty_alpha + rpim_solve_pcg; "
                    "backward: rpim_solve_pcg (adjoint) + rpim_grad_material"}


# --------------------------------------------------------------------------- batched vs per-instance
def _batched(n_sel, dev, stream, reps=1, warm=1):
    """Blocks of the 512-instance batched workload (node counts log-uniform in
    500-20,000, alpha_s uniform in [2, 3.5]), every (512 / n_sel)-th one:
    one batched pattern + assembly + loads + per-instance penalty + batched
    PCG, against the same instances through the plain entry points one after
    another. Device-resident inputs; CUDA events on the launching stream."""
    import torch
    import paper_1802_04256_gb300 as R
    allp = gen.batched_configs()
    sel = allp[::max(1, len(allp) // n_sel)][:n_sel]
    tt = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    offs = np.concatenate([[0], np.cumsum([p.n_nodes for p in sel])])
    inst = [(p.n_nodes, p.alpha_s, p.h) for p in sel]
    cat = lambda name: np.concatenate([getattr(p, name) for p in sel])
    bx, blo, bhi, bE, bnu = tt(cat("xyz")), tt(cat("cell_lo")), tt(cat("cell_hi")), tt(cat("E")), tt(cat("nu"))
    blx, blf = tt(cat("load_xyz")), tt(cat("load_force"))
    bli = tt(np.concatenate([np.full(len(p.load_xyz), k, np.int32) for k, p in enumerate(sel)]), torch.int32)
    bdofs = tt(np.concatenate([p.fixed_dofs + 3 * offs[k] for k, p in enumerate(sel)]), torch.int64)
    bvals = tt(cat("fixed_vals"))
    single = [dict(x=tt(p.xyz), lo=tt(p.cell_lo), hi=tt(p.cell_hi), E=tt(p.E), nu=tt(p.nu), lx=tt(p.load_xyz),
                   lf=tt(p.load_force), dofs=tt(p.fixed_dofs, torch.int64), vals=tt(p.fixed_vals)) for p in sel]
    rtol = 1e-10

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    def b_assemble():
        pat = R.Pattern(bx, blo, bhi, None, sel[0].alpha_c, sel[0].q, None, instances=inst)
        K, f = pat.assemble(bE, bnu)
        pat.add_point_loads(blx, blf, f, inst=bli)
        return pat, K, f

    def b_solve(pat, K, f):
        pat.apply_penalty(K, f, bdofs, bvals)
        return pat.solve_pcg_batched(K, f, rtol=rtol, max_iter=500000)

    def s_assemble(p, d):
        pat = R.Pattern(d["x"], d["lo"], d["hi"], p.alpha_s, p.alpha_c, p.q, p.h)
        K, f = pat.assemble(d["E"], d["nu"])
        pat.add_point_loads(d["lx"], d["lf"], f)
        return pat, K, f

    def s_solve(pat, K, f, d):
        pat.apply_penalty(K, f, d["dofs"], d["vals"])
        return pat.solve_pcg(K, f, rtol=rtol, max_iter=500000)

    def run_batched():
        ta, (pat, K, f) = timed(b_assemble)
        ts, (u, its, rrs) = timed(lambda: b_solve(pat, K, f))
        pat.free()
        return ta, ts, u, its

    def run_single():
        ta = ts = 0.0
        us, its = [], []
        for p, d in zip(sel, single):
            a, (pat, K, f) = timed(lambda: s_assemble(p, d))
            s, (u, it, rr) = timed(lambda: s_solve(pat, K, f, d))
            pat.free()
            ta, ts = ta + a, ts + s
            us.append(u)
            its.append(it)
        return ta, ts, us, its

    # setup, untimed: tune the bucket bounds and the shape kernel's launch
    # shapes on this batch's support sizes (process-wide: both arms use them)
    tp = R.Pattern(bx, blo, bhi, None, sel[0].alpha_c, sel[0].q, None, instances=inst)
    bounds = tp.autotune_buckets(max_points=200000)
    tp.autotune(max_points=20000)
    tp.free()
    for _ in range(warm):
        run_batched()
        run_single()
    l0 = R.rpim_kernel_launches()
    bres = [run_batched() for _ in range(reps)]
    lb = (R.rpim_kernel_launches() - l0) / reps
    l0 = R.rpim_kernel_launches()
    sres = [run_single() for _ in range(reps)]
    ls = (R.rpim_kernel_launches() - l0) / reps
    ba, bs = min(r[0] for r in bres), min(r[1] for r in bres)
    sa, ss = min(r[0] for r in sres), min(r[1] for r in sres)
    ub, itb = bres[-1][2], bres[-1][3]
    us, its = sres[-1][2], sres[-1][3]
    du = max(float(torch.linalg.norm(ub[3 * offs[k]:3 * offs[k + 1]] - us[k]) / torch.linalg.norm(us[k]))
             for k in range(len(sel)))
    npts = int(sum(p.n_points for p in sel))

    # re-assembly with new material, patterns built beforehand (the repeated
    # assembly of a parameter study or a back-analysis): the batched pattern
    # replays its captured graph (one persistent shape launch over all
    # buckets); the per-instance arm calls rpim_assemble on each instance's
    # own pattern. Only the assembly calls are timed.
    pat = R.Pattern(bx, blo, bhi, None, sel[0].alpha_c, sel[0].q, None, instances=inst)
    Kb, fb = pat.assemble_graphed(bE, bnu)
    l0 = R.rpim_kernel_launches()
    rb = [timed(lambda: pat.assemble_graphed(bE, bnu, K=Kb, f=fb))[0] for _ in range(2)]
    lrb = (R.rpim_kernel_launches() - l0) / 2
    # per-kernel device times of one more assembly (plain launches while
    # timing is on) and the algorithmic flops of the batch's supports
    R.rpim_profile_read(reset=True)
    R.rpim_profile_enable(True)
    pat.assemble_graphed(bE, bnu, K=Kb, f=fb)
    R.rpim_profile_enable(False)
    kprof = R.rpim_profile_read(reset=True)
    nsup = np.diff(pat.points()[2].cpu().numpy())
    fl_shape, fl_pair = float(shape_flops(nsup).sum()), float(pair_flops(nsup).sum())
    pat.free()
    del Kb, fb
    rs, lrs = 0.0, 0
    for p, d in zip(sel, single):
        pt = R.Pattern(d["x"], d["lo"], d["hi"], p.alpha_s, p.alpha_c, p.q, p.h)
        K1, f1 = pt.assemble(d["E"], d["nu"])
        l0 = R.rpim_kernel_launches()
        rs += min(timed(lambda: pt.assemble(d["E"], d["nu"], K=K1, f=f1))[0] for _ in range(2))
        lrs += (R.rpim_kernel_launches() - l0) / 2
        pt.free()
        del K1, f1
    # the same per-instance re-assembly with the unbucketed kernel: one shape
    # launch per instance sized for that instance's largest support (every
    # point gets the largest point's shared-memory buffers and launch shape)
    ru = 0.0
    R.rpim_set_shape_schedule(False)
    for p, d in zip(sel, single):
        pt = R.Pattern(d["x"], d["lo"], d["hi"], p.alpha_s, p.alpha_c, p.q, p.h)
        R.rpim_pattern_set_buckets(pt.handle, [1 << 29])
        K1, f1 = pt.assemble(d["E"], d["nu"])
        ru += min(timed(lambda: pt.assemble(d["E"], d["nu"], K=K1, f=f1))[0] for _ in range(2))
        pt.free()
        del K1, f1
    R.rpim_set_shape_schedule(True)
    reasm = {"batched_graph_ms": min(rb), "per_instance_ms": rs, "speedup": rs / min(rb),
             "per_instance_unbucketed_ms": ru, "speedup_vs_unbucketed": ru / min(rb),
             "batched_pts_per_s": npts / (min(rb) / 1e3), "per_instance_pts_per_s": npts / (rs / 1e3),
             "kernel_launches": {"batched": lrb, "per_instance": lrs},
             "kernel_ms": {k: round(v[1] / v[0], 3) for k, v in sorted(kprof.items(), key=lambda kv: -kv[1][1])},
             "algorithmic_flops": {"shape": fl_shape, "pair": fl_pair},
             "assembly_tflops": (fl_shape + fl_pair) / (min(rb) / 1e3) / 1e12,
             "shape_tflops": fl_shape / (kprof["shape"][1] / 1e3) / 1e12 if "shape" in kprof else None,
             "support_sizes": {"min": int(nsup.min()), "max": int(nsup.max()), "mean": float(nsup.mean())},
             "step": "rpim_assemble_graphed on the batched pattern vs rpim_assemble per instance "
                     "(patterns built beforehand, not timed); unbucketed: one support-size bucket and one "
                     "shape launch per instance"}
    return {"instances": len(sel), "of": len(allp), "selection": "every %d-th block of the 512-block workload"
            % max(1, len(allp) // n_sel), "n_nodes": int(offs[-1]), "n_points": npts,
            "node_range": [int(min(p.n_nodes for p in sel)), int(max(p.n_nodes for p in sel))],
            "assembly": {"batched_ms": ba, "per_instance_ms": sa, "speedup": sa / ba,
                         "batched_pts_per_s": npts / (ba / 1e3), "per_instance_pts_per_s": npts / (sa / 1e3)},
            "solve": {"batched_ms": bs, "per_instance_ms": ss, "speedup": ss / bs, "rtol": rtol,
                      "iterations_max": int(max(itb)), "iterations_sum_per_instance": int(sum(its))},
            "end_to_end": {"batched_ms": ba + bs, "per_instance_ms": sa + ss, "speedup": (sa + ss) / (ba + bs)},
            "kernel_launches": {"batched": lb, "per_instance": ls},
            "reassembly": reasm, "bucket_bounds": bounds,
            "u_max_rel_diff_batched_vs_per_instance": du,
            "step": "build pattern + assemble + surface loads (assembly); penalty + Jacobi-PCG to 1e-10 (solve)"}


# --------------------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1802_04256_gb300 as R

    dist = None
    if world > 1:
        import torch.distributed as dist
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    R.lib()
    p = gen.cantilever_config()
    tt = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    xyz, lo, hi, E, nu = tt(p.xyz), tt(p.cell_lo), tt(p.cell_hi), tt(p.E), tt(p.nu)
    lxyz, lf = tt(p.load_xyz), tt(p.load_force)
    stream = torch.cuda.current_stream()

    def step():
        pat = R.Pattern(xyz, lo, hi, p.alpha_s, p.alpha_c, p.q, p.h)
        K, f = pat.assemble(E, nu)
        pat.add_point_loads(lxyz, lf, f)
        pat.free()
        return K, f

    def barrier():
        if dist is not None:
            dist.barrier()

    # setup, untimed: launch shapes of the shape kernel picked by the
    # autotuner on this workload's support-size buckets (results are bitwise
    # independent of the launch shape)
    tuned = bounds = None
    if not args.no_autotune:
        tp = R.Pattern(xyz, lo, hi, p.alpha_s, p.alpha_c, p.q, p.h)
        bounds = tp.autotune_buckets(max_points=100000)
        tuned = tp.autotune(max_points=20000)
        tp.free()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # FP64 peak of this GPU, measured warm (best of two best-of-5 runs)
    peak_gflops = max(R.rpim_probe_dfma(5), R.rpim_probe_dfma(5))

    # ---- timed region
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    idx = vis.split(",")[local_rank] if vis else str(local_rank)
    clocks = ClockSampler(idx)
    clocks.start()
    R.rpim_profile_read(reset=True)
    R.rpim_profile_enable(True)
    launches0 = R.rpim_kernel_launches()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = R.rpim_kernel_launches() - launches0
    R.rpim_profile_enable(False)
    prof = R.rpim_profile_read(reset=True)
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
    value = whole_job_rate(p.n_points, world, ms)

    # ---- roofline of the dominant kernel (largest device time)
    pat = R.Pattern(xyz, lo, hi, p.alpha_s, p.alpha_c, p.q, p.h)
    _, _, soff, _ = pat.points()
    nsup = np.diff(soff.cpu().numpy())
    kinds = {"shape": (shape_flops(nsup).sum(), "shape.cu"), "row": (pair_flops(nsup).sum(), "assemble.cu")}
    top = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None
    roof = None
    if top in kinds:
        # the shape kernel runs once per support-size bucket: the algorithmic
        # flops of one step (all points) over the kernel's device time per step
        flops, src = kinds[top]
        nl, tot = prof[top]
        step_ms = tot / args.steps
        ach = flops / (step_ms / 1e3) / 1e12
        peak = peak_gflops / 1e3
        roof = {"bound": "alu", "kernel": top, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": _traffic_for(top, os.path.join(ROOT, "paper_1802_04256_gb300", "csrc", src)),
                "peak_source": "FP64 DFMA throughput measured in this run (rpim_probe_dfma)",
                "algorithmic_flops_per_step": flops, "launches_per_step": nl / args.steps,
                "kernel_ms_per_step": step_ms, "avg_launch_ms": tot / nl}
    kernel_ms = {k: round(v[1] / args.steps, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    kernel_share = {k: round(v[1] / max(sum(x[1] for x in prof.values()), 1e-9), 4)
                    for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}

    # ---- stage 2 + 3 once: penalty and PCG (full solve)
    solve = None
    nnzb = pat.nnz_blocks
    if args.no_solve:
        pat.free()
    else:
        solve = _solve(pat, p, E, nu, lxyz, lf, tt, stream, peak_gflops, args.solve_iters)

    # ---- end to end through host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        host = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in
                dict(xyz=p.xyz, lo=p.cell_lo, hi=p.cell_hi, E=p.E, nu=p.nu, lx=p.load_xyz, lf=p.load_force).items()}
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        Kh = None
        # the device->host copy of a step's K and f runs on its own stream,
        # overlapped with the next step's assembly (pipelined as a caller
        # would run a stream of problems); record_stream keeps the caching
        # allocator from reusing K and f before their copy has finished
        copy_stream = torch.cuda.Stream(device=dev)

        def e2e_step():
            nonlocal Kh
            d = {k: v.to(dev, non_blocking=True) for k, v in host.items()}
            pat = R.Pattern(d["xyz"], d["lo"], d["hi"], p.alpha_s, p.alpha_c, p.q, p.h)
            K, f = pat.assemble(d["E"], d["nu"])
            pat.add_point_loads(d["lx"], d["lf"], f)
            if Kh is None:
                Kh = (torch.empty(K.shape, dtype=K.dtype, pin_memory=True),
                      torch.empty(f.shape, dtype=f.dtype, pin_memory=True))
            done = torch.cuda.Event()
            done.record(stream)
            copy_stream.wait_event(done)
            with torch.cuda.stream(copy_stream):
                Kh[0].copy_(K, non_blocking=True)
                Kh[1].copy_(f, non_blocking=True)
            K.record_stream(copy_stream)
            f.record_stream(copy_stream)
            pat.free()
            return K.numel() * 8 + f.numel() * 8

        e2e_step()
        torch.cuda.synchronize()
        n_e2e = max(2, min(args.steps, 5))
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d2h = 0
        for _ in range(n_e2e):
            d2h = e2e_step()
        torch.cuda.synchronize()
        barrier()
        e2e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0) / n_e2e, dist, dev)
        e2e = {"value": whole_job_rate(p.n_points, world, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms}

    mls = None
    if not args.no_mls:
        mls = _mls(p, xyz, lo, hi, E, nu, lxyz, lf, stream, peak_gflops)

    batched = None
    if args.batched_instances > 0:
        batched = _batched(args.batched_instances, dev, stream, warm=args.batched_warmup)
    grad = None
    if not args.no_grad:
        grad = _backanalysis(dev, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(p)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": WORKLOAD, "n_nodes": p.n_nodes, "n_points": p.n_points,
                          "step": "rpim_build_pattern + rpim_assemble + rpim_add_point_loads",
                          "l2": "working set larger than L2 (K %.2f GB, shape functions %.2f GB)"
                                % (nnzb * 72 / 1e9, nsup.sum() * 32 / 1e9),
                          "parallelism": "replicas" if world > 1 else "single GPU"},
               "roofline": roof, "kernel_ms_per_step": kernel_ms, "kernel_time_share": kernel_share,
               "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
               "solve": solve, "batched": batched, "backanalysis": grad, "mls": mls,
               "autotune": [{"max_support": a, "warps_per_point": g, "points_per_block": c} for a, g, c in tuned]
               if tuned else None, "bucket_bounds": bounds,
               "fp64_peak_gflops_measured": peak_gflops}
        print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true", help="skip the penalty + PCG measurement")
    ap.add_argument("--no-grad", action="store_true", help="skip the back-analysis gradient measurement")
    ap.add_argument("--no-mls", action="store_true", help="skip the MLS-variant assembly measurement")
    ap.add_argument("--batched-warmup", type=int, default=1,
                    help="untimed runs of each arm of the batched comparison before the timed one")
    ap.add_argument("--no-autotune", action="store_true", help="use the built-in launch shapes of the shape kernel")
    ap.add_argument("--solve-iters", type=int, default=0,
                    help="run the solve for exactly this many PCG iterations (profiling; 0 = to rtol 1e-10)")
    ap.add_argument("--batched-instances", type=int, default=32,
                    help="blocks of the 512-block batched workload in the batched vs per-instance "
                         "comparison (512 = all; 0 = skip)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
