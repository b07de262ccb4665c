"""Benchmark of the RPIM global stiffness assembly on GB300.

Headline workload: the layered slope at scale, 100 x 100 x 100 lattice in the
unit cube clipped to a 45-degree face (590,500 field nodes, 4,724,000 Gauss
points), interior jitter 0.2h, support radius 3.0h, multiquadric alpha_c = 4,
q = 1.03, three horizontal layers of E and nu, gravity body force, FP64,
seeded synthetic node cloud. One step is the whole assembly path of Sec. 2's
first stage on device-resident inputs: rpim_build_pattern (Gauss points,
cell list, supports, node incidence, BSR pattern) + rpim_assemble (shape
functions, B^T D B, deterministic reduction, body force) (+ rpim_add_traction
on workloads with surface loads). The penalty stage and the PCG solve of the
same system are timed separately afterwards ("solve": iterations and full
solves/s, Jacobi and 3x3 block-Jacobi preconditioners).

Extra keys: "configs" times the other workloads (the 6x6x6 cube, the
129x17x17 cantilever, the 64x32x32 back-analysis block) the same way, each
with its roofline fraction, solves/s and the oracle on the host cores;
"batched" compares one batched pattern + assembly + batched PCG over blocks
of the 512-block workload with the same blocks run one by one through the
plain entry points; "backanalysis" times one material gradient; "mls" the
cantilever step with MLS shape functions.

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

WORKLOADS = {
    "slope": ("layered slope 100x100x100 clipped at 45 degrees (590,500 nodes, 4,724,000 Gauss points), "
              "interior jitter 0.2h, alpha_s 3.0, MQ alpha_c 4.0 q 1.03, E 8e4/2e4/5e3 nu 0.25/0.30/0.35 "
              "by layer, gravity 20, FP64", gen.slope_config),
    "cantilever": ("cantilever 129x17x17 (37,281 nodes, 298,248 Gauss points), interior jitter 0.2h, "
                   "alpha_s 2.5, MQ alpha_c 4.0 q 1.03, E 1e4 nu 0.3, parabolic end shear, FP64",
                   gen.cantilever_config),
    "cube": ("cube 6x6x6 (216 nodes, 1,728 Gauss points), alpha_s 2.5, MQ alpha_c 4.0 q 1.03, E 1e4 nu 0.3, "
             "pressure 10 on top, FP64", gen.cube_config),
    "backanalysis": ("back-analysis block 64x32x32 (65,536 nodes, 524,288 Gauss points), jitter 0.2h, "
                     "alpha_s 2.5, log-normal E field, pressure 10 on top, FP64", gen.backanalysis_config),
}


def _hbm_peak():
    """Measured copy bandwidth of this GPU pool (GB/s), else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured copy bandwidth, MEASURED_PEAKS.json (of measured)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback copy bandwidth 6.8 TB/s (of fallback)"


HBM_PEAK, HBM_SRC = _hbm_peak()
SMS, DFMA_PER_CLK = 152, 2   # SMs of a GB300; FP64 FMA per clock per SM


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
def _traffic_for(kernel, source, workload):
    """DRAM bytes of `kernel` per step (all its launches in one step) of
    `workload` from the committed ncu summary, if the kernel's source is
    unchanged since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    sha = hashlib.sha256(open(source, "rb").read()).hexdigest()[:16]
    for line in open(path):
        kv = dict(tok.split("=", 1) for tok in line.split() if "=" in tok)
        if kv.get("kernel") == kernel and kv.get("workload") == workload and kv.get("source_sha256") == sha:
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


def cpu_baseline(p, budget_s=15.0, single_s=None):
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

    m0 = 256
    t0, _, _ = run(m0)
    m = int(min(len(pts), max(m0, m0 * budget_s / max(t0, 1e-3))))
    dt, m, k = run(m)
    oracle.set_threads(1)
    single_s = budget_s / 3 if single_s is None else single_s
    m1 = int(min(len(pts), max(64, m * single_s / dt / cores)))
    dt1, m1, k1 = run(m1)
    oracle.set_threads(cores)
    return {"value": m / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "every %d-th of the %d Gauss points of the workload (%d, %.2f%%), f64 oracle, OpenMP %d "
                      "threads, %.1f s" % (k, len(pts), m, 100.0 * m / len(pts), cores, dt),
            "single_thread": {"value": m1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": "every %d-th Gauss point (%d), f64 oracle, 1 thread, %.1f s" % (k1, m1, dt1)}}


# --------------------------------------------------------------------------- reference arm
def run_reference(args, rank):
    """The oracle as it stands, on the host cores, on a bounded sample of the
    headline workload per step (about 4 s of host work)."""
    if rank != 0:
        return
    desc, make = WORKLOADS[args.workload]
    p = make()
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

    t = step(256)
    m = int(min(len(pts), max(256, 256 * 4.0 / max(t, 1e-3))))
    for _ in range(args.warmup):
        step(m)
    times = [step(m) for _ in range(args.steps)]
    ms = 1e3 * sum(times) / len(times)
    value = m / (ms / 1e3)
    sel, k = _spread(len(pts), m)
    sample = ("%d of the %d Gauss points of the workload per step, spread evenly (every %d-th), f64 oracle, "
              "OpenMP %d threads" % (len(pts[sel]), len(pts), k, cores))
    out = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": desc, "sample_points": m},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# --------------------------------------------------------------------------- device inputs
class Inputs:
    """Device tensors of one problem."""

    def __init__(self, p, dev):
        import torch
        tt = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
        self.p, self.dev = p, dev
        self.xyz, self.lo, self.hi = tt(p.xyz), tt(p.cell_lo), tt(p.cell_hi)
        self.E, self.nu = tt(p.E), tt(p.nu)
        self.body = tt(p.body) if np.any(p.body) else None
        self.faces = (tt(p.face_lo), tt(p.face_hi), tt(p.face_axis, torch.int8), tt(p.face_coef)) \
            if p.n_faces else None
        self.dofs, self.vals = tt(p.fixed_dofs, torch.int64), tt(p.fixed_vals)

    def pattern(self, shape="rpim"):
        import paper_1802_04256_gb300 as R
        p = self.p
        return R.Pattern(self.xyz, self.lo, self.hi, p.alpha_s, p.alpha_c, p.q, p.h, shape=shape)

    def assemble(self, pat, K=None, f=None):
        K, f = pat.assemble(self.E, self.nu, self.body, K=K, f=f)
        if self.faces is not None:
            pat.add_traction(*self.faces, f)
        return K, f

    def step(self, shape="rpim"):
        """One assembly step: pattern + assembly (+ tractions)."""
        pat = self.pattern(shape)
        K, f = self.assemble(pat)
        pat.free()
        return K, f


def _events(n):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def _support_sizes(inp):
    pat = inp.pattern()
    nsup = np.diff(pat.points()[2].cpu().numpy())
    nnzb = pat.nnz_blocks
    pat.free()
    return nsup, nnzb


def _roofline(prof, steps, nsup, peak_gflops, workload):
    """Roofline of the dominant kernel of an assembly step (largest device
    time): its algorithmic flops per step over its device time per step."""
    kinds = {"shape": (shape_flops(nsup).sum(), "shape.cu"), "row": (pair_flops(nsup).sum(), "assemble.cu")}
    top = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None
    if top not in kinds:
        return None
    flops, src = kinds[top]
    nl, tot = prof[top]
    step_ms = tot / steps
    ach = flops / (step_ms / 1e3) / 1e12
    peak = peak_gflops / 1e3
    return {"bound": "alu", "kernel": top, "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": _traffic_for(top, os.path.join(ROOT, "paper_1802_04256_gb300", "csrc", src), workload),
            "peak_source": "FP64 DFMA throughput measured in this run (rpim_probe_dfma)",
            "algorithmic_flops_per_step": flops, "launches_per_step": nl / steps, "kernel_ms_per_step": step_ms,
            "avg_launch_ms": tot / nl}


def _time_steps(inp, steps, stream, shape="rpim"):
    """Device time per assembly step (CUDA events on the launching stream)
    and per-kernel device times (the library's own events)."""
    import torch
    import paper_1802_04256_gb300 as R
    torch.cuda.synchronize()
    R.rpim_profile_read(reset=True)
    R.rpim_profile_enable(True)
    l0 = R.rpim_kernel_launches()
    e0, e1 = _events(2)
    e0.record(stream)
    for _ in range(steps):
        inp.step(shape)
    e1.record(stream)
    torch.cuda.synchronize()
    R.rpim_profile_enable(False)
    prof = R.rpim_profile_read(reset=True)
    return e0.elapsed_time(e1) / steps, prof, (R.rpim_kernel_launches() - l0) / steps


# --------------------------------------------------------------------------- stages 2 and 3
def _solve(inp, stream, peak_gflops, precond="jacobi", fixed_iters=0, tip=None, rtol=1e-10, max_iter=200000):
    """Penalty (alpha = 1e8 max diag K) and PCG to rtol, timed once with CUDA
    events (the assembly that feeds it is not timed); per-kernel times of the
    iteration from 256 more iterations with event timing."""
    import torch
    import paper_1802_04256_gb300 as R
    pat = inp.pattern()
    K, f = inp.assemble(pat)
    torch.cuda.synchronize()
    s0, s1 = _events(2)
    s0.record(stream)
    alpha = pat.apply_penalty(K, f, inp.dofs, inp.vals)
    if fixed_iters > 0:   # a fixed number of iterations (profiling runs)
        u, iters, relres = pat.solve_pcg(K, f, rtol=0.0, max_iter=fixed_iters, check=False, precond=precond)
    else:
        u, iters, relres = pat.solve_pcg(K, f, rtol=rtol, max_iter=max_iter, precond=precond)
    s1.record(stream)
    torch.cuda.synchronize()
    solve_ms = s0.elapsed_time(s1)
    nnzb, n_nodes = pat.nnz_blocks, inp.p.n_nodes
    R.rpim_profile_read(reset=True)
    R.rpim_profile_enable(True)
    pat.solve_pcg(K, f, u.clone(), rtol=0.0, max_iter=256, check=False, precond=precond)
    R.rpim_profile_enable(False)
    prof = R.rpim_profile_read(reset=True)
    spmv_bytes = nnzb * (72 + 4) + n_nodes * (8 + 24 + 24)
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
    out = {"precond": precond, "pcg_iterations": iters, "relres": relres, "rtol": rtol, "ms": solve_ms,
           "solves_per_s": 1e3 / solve_ms, "ms_per_iteration": solve_ms / max(iters, 1), "penalty_alpha": alpha,
           "spmv_roofline": roof, "iteration_kernel_ms": {k: round(v[1] / v[0], 4) for k, v in prof.items()}}
    if tip is not None:
        out["tip_deflection"] = -u[3 * tip + 2].item()
    del K, f, u
    pat.free()
    return out


def _solves(inp, stream, peak_gflops, args, tip=None, preconds=None):
    """The full solve with each preconditioner."""
    if args.no_solve:
        return None
    pcs = preconds or args.precond.split(",")
    return {pc: _solve(inp, stream, peak_gflops, pc, args.solve_iters, tip) for pc in pcs}


# --------------------------------------------------------------------------- MLS variant
def _mls(inp, stream, peak_gflops, steps=3):
    """The same assembly step with MLS shape functions (linear basis,
    cubic-spline weight; the variant Sec. 4 plans), device-resident inputs."""
    for _ in range(2):
        inp.step("mls")
    ms, prof, _ = _time_steps(inp, steps, stream, "mls")
    nsup, _ = _support_sizes(inp)
    roof = None
    if "row" in prof:
        nl, tot = prof["row"]
        ach = pair_flops(nsup).sum() / (tot / steps / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": "row", "achieved": ach, "peak": peak_gflops / 1e3, "unit": "TFLOP/s",
                "frac": ach * 1e3 / peak_gflops, "peak_source": "FP64 DFMA throughput measured in this run"}
    return {"step": "rpim_build_pattern + rpim_pattern_set_shape(MLS) + rpim_assemble + rpim_add_traction",
            "workload": WORKLOADS["cantilever"][0].replace("MQ alpha_c 4.0 q 1.03",
                                                          "MLS linear basis, cubic-spline weight"),
            "steps": steps, "ms_per_step": ms, "pts_per_s": inp.p.n_points / (ms / 1e3),
            "kernel_ms_per_step": {k: round(v[1] / steps, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])},
            "roofline_row_kernel": roof}


# --------------------------------------------------------------------------- other workloads
def _config(name, dev, stream, peak_gflops, args, steps, warm, cpu_s, tip=None, preconds=None):
    """One workload: assembly pts/s with its roofline, full solves/s, and the
    oracle on the host cores (all cores and one thread)."""
    desc, make = WORKLOADS[name]
    p = make()
    inp = Inputs(p, dev)
    for _ in range(warm):
        inp.step()
    ms, prof, launches = _time_steps(inp, steps, stream)
    nsup, nnzb = _support_sizes(inp)
    out = {"workload": desc, "n_nodes": p.n_nodes, "n_points": p.n_points, "steps": steps, "ms_per_step": ms,
           "pts_per_s": p.n_points / (ms / 1e3), "gpu_launches_per_step": launches,
           "roofline": _roofline(prof, steps, nsup, peak_gflops, name),
           "support": {"min": int(nsup.min()), "max": int(nsup.max()), "mean": float(nsup.mean())},
           "nnz_blocks": nnzb,
           "kernel_ms_per_step": {k: round(v[1] / steps, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}}
    out["solve"] = _solves(inp, stream, peak_gflops, args, tip, preconds)
    if not args.no_cpu_baseline and cpu_s > 0:
        out["cpu_baseline"] = cpu_baseline(p, cpu_s)
    return out, inp


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
    inp = Inputs(p, dev)
    pat = inp.pattern()
    f_ext = torch.zeros(3 * p.n_nodes, dtype=torch.float64, device=dev)
    pat.add_traction(*inp.faces, f_ext)
    tt = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    obs = tt(p.meta["obs_nodes"], torch.int64)
    alpha = R.penalty_alpha(pat, inp.E, inp.nu)
    with torch.no_grad():   # observations: displacements of the hidden field
        u_obs = R.solve(pat, tt(p.meta["E_hidden"]), tt(p.meta["nu_hidden"]), f_ext, inp.dofs, inp.vals, alpha,
                        rtol=rtol).view(-1, 3)[obs].clone()

    def one():
        E = inp.E.clone().requires_grad_()
        nu = inp.nu.clone().requires_grad_()
        e0, e1, e2 = _events(3)
        torch.cuda.synchronize()
        e0.record(stream)
        u = R.solve(pat, E, nu, f_ext, inp.dofs, inp.vals, alpha, rtol=rtol)
        loss = 0.5 * ((u.view(-1, 3)[obs] - u_obs) ** 2).sum()
        e1.record(stream)
        loss.backward()
        e2.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), e1.elapsed_time(e2), float(E.grad.abs().max()), float(nu.grad.abs().max())

    one()
    fwd, bwd, gE, gn = one()
    pat.free()
    return {"workload": WORKLOADS["backanalysis"][0] + ", 500 observed nodes", "parameters": 2 * p.n_points,
            "rtol": rtol, "forward_ms": fwd, "backward_ms": bwd, "gradients_per_s": 1e3 / (fwd + bwd),
            "max_abs_dL_dE": gE, "max_abs_dL_dnu": gn,
            "step": "forward: rpim_assemble + rpim_add_vector + rpim_apply_penalty_alpha + rpim_solve_pcg; "
                    "backward: rpim_solve_pcg (adjoint) + rpim_grad_material"}


# --------------------------------------------------------------------------- batched vs per-instance
def _batched(n_sel, dev, stream, reps=1, warm=1, small_nodes=2000, cpu=True):
    """Blocks of the 512-instance batched workload (node counts log-uniform in
    500-20,000, alpha_s uniform in [2, 3.5]), every (512 / n_sel)-th one:
    one batched pattern + assembly + tractions + per-instance penalty +
    batched PCG, against the same instances through the plain entry points
    one after another. Device-resident inputs; CUDA events on the launching
    stream. Also the assembly of every block below `small_nodes` nodes, the
    regime where per-instance launches under-fill the GPU."""
    import torch
    import paper_1802_04256_gb300 as R
    allp = gen.batched_configs()
    sel = allp[::max(1, len(allp) // n_sel)][:n_sel]
    tt = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    rtol = 1e-10

    def timed(fn):
        e0, e1 = _events(2)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    class Batch:
        def __init__(self, probs):
            self.probs = probs
            self.offs = np.concatenate([[0], np.cumsum([p.n_nodes for p in probs])])
            self.inst = [(p.n_nodes, p.alpha_s, p.h) for p in probs]
            cat = lambda name: np.concatenate([getattr(p, name) for p in probs])
            self.x, self.lo, self.hi, self.E, self.nu = (tt(cat("xyz")), tt(cat("cell_lo")), tt(cat("cell_hi")),
                                                         tt(cat("E")), tt(cat("nu")))
            fl, fh, fa, fc, fi = gen.concat_faces(probs)
            self.faces = (tt(fl), tt(fh), tt(fa, torch.int8), tt(fc))
            self.finst = tt(fi, torch.int32)
            self.dofs = tt(np.concatenate([p.fixed_dofs + 3 * self.offs[k] for k, p in enumerate(probs)]),
                           torch.int64)
            self.vals = tt(cat("fixed_vals"))
            self.npts = int(sum(p.n_points for p in probs))

        def pattern(self):
            return R.Pattern(self.x, self.lo, self.hi, None, self.probs[0].alpha_c, self.probs[0].q, None,
                             instances=self.inst)

        def assemble(self):
            pat = self.pattern()
            K, f = pat.assemble(self.E, self.nu)
            pat.add_traction(*self.faces, f, inst=self.finst)
            return pat, K, f

    bat = Batch(sel)
    single = [Inputs(p, dev) for p in sel]

    def b_solve(pat, K, f):
        pat.apply_penalty(K, f, bat.dofs, bat.vals)
        return pat.solve_pcg_batched(K, f, rtol=rtol, max_iter=500000)

    def s_solve(pat, K, f, d):
        pat.apply_penalty(K, f, d.dofs, d.vals)
        return pat.solve_pcg(K, f, rtol=rtol, max_iter=500000)

    def run_batched():
        ta, (pat, K, f) = timed(bat.assemble)
        ts, (u, its, rrs) = timed(lambda: b_solve(pat, K, f))
        pat.free()
        return ta, ts, u, its

    def s_assemble(d):
        pat = d.pattern()
        K, f = d.assemble(pat)
        return pat, K, f

    def run_single():
        ta = ts = 0.0
        us, its = [], []
        for d in single:
            a, (pat, K, f) = timed(lambda: s_assemble(d))
            s, (u, it, rr) = timed(lambda: s_solve(pat, K, f, d))
            pat.free()
            ta, ts = ta + a, ts + s
            us.append(u)
            its.append(it)
        return ta, ts, us, its

    # setup, untimed: tune the bucket bounds and the shape kernel's launch
    # shapes on this batch's support sizes (process-wide: both arms use them)
    tp = bat.pattern()
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
    offs = bat.offs
    du = max(float(torch.linalg.norm(ub[3 * offs[k]:3 * offs[k + 1]] - us[k]) / torch.linalg.norm(us[k]))
             for k in range(len(sel)))
    npts = bat.npts

    # re-assembly with new material, patterns built beforehand (the repeated
    # assembly of a parameter study or a back-analysis): the batched pattern
    # replays its captured graph (one persistent shape launch over all
    # buckets); the per-instance arm calls rpim_assemble on each instance's
    # own pattern. Only the assembly calls are timed.
    pat = bat.pattern()
    Kb, fb = pat.assemble_graphed(bat.E, bat.nu)
    pat.assemble_graphed(bat.E, bat.nu, K=Kb, f=fb)
    l0 = R.rpim_kernel_launches()
    rb = [timed(lambda: pat.assemble_graphed(bat.E, bat.nu, K=Kb, f=fb))[0] for _ in range(2)]
    lrb = (R.rpim_kernel_launches() - l0) / 2
    R.rpim_profile_read(reset=True)
    R.rpim_profile_enable(True)
    pat.assemble_graphed(bat.E, bat.nu, K=Kb, f=fb)
    R.rpim_profile_enable(False)
    kprof = R.rpim_profile_read(reset=True)
    nsup = np.diff(pat.points()[2].cpu().numpy())
    fl_shape, fl_pair = float(shape_flops(nsup).sum()), float(pair_flops(nsup).sum())
    pat.free()
    del Kb, fb
    rs, lrs = 0.0, 0
    for d in single:
        pt = d.pattern()
        K1, f1 = pt.assemble(d.E, d.nu)
        pt.assemble(d.E, d.nu, K=K1, f=f1)
        l0 = R.rpim_kernel_launches()
        rs += min(timed(lambda: pt.assemble(d.E, d.nu, K=K1, f=f1))[0] for _ in range(2))
        lrs += (R.rpim_kernel_launches() - l0) / 2
        pt.free()
        del K1, f1
    reasm = {"batched_graph_ms": min(rb), "per_instance_ms": rs, "speedup": rs / min(rb),
             "batched_pts_per_s": npts / (min(rb) / 1e3), "per_instance_pts_per_s": npts / (rs / 1e3),
             "kernel_launches": {"batched": lrb, "per_instance": lrs},
             "kernel_ms": {k: round(v[1] / v[0], 3) for k, v in sorted(kprof.items(), key=lambda kv: -kv[1][1])},
             "algorithmic_flops": {"shape": fl_shape, "pair": fl_pair},
             "assembly_tflops": (fl_shape + fl_pair) / (min(rb) / 1e3) / 1e12,
             "shape_tflops": fl_shape / (kprof["shape"][1] / 1e3) / 1e12 if "shape" in kprof else None,
             "support_sizes": {"min": int(nsup.min()), "max": int(nsup.max()), "mean": float(nsup.mean())},
             "step": "rpim_assemble_graphed on the batched pattern vs rpim_assemble per instance "
                     "(patterns built beforehand, not timed), both warm"}

    # every block of the 512 below small_nodes: assembly (pattern + assemble +
    # tractions), batched vs per instance, both warm
    small = [p for p in allp if p.n_nodes < small_nodes]
    sbat = Batch(small)
    ssingle = [Inputs(p, dev) for p in small]
    tp = sbat.pattern()
    tp.autotune(max_points=20000)
    tp.free()

    def small_b():
        ta, (pat, K, f) = timed(sbat.assemble)

        def solve():
            pat.apply_penalty(K, f, sbat.dofs, sbat.vals)
            return pat.solve_pcg_batched(K, f, rtol=rtol, max_iter=500000)

        ts, _ = timed(solve)
        pat.free()
        return ta, ts

    def small_s():
        ta = ts = 0.0
        for d in ssingle:
            a, (pat, K, f) = timed(lambda: s_assemble(d))
            s, _ = timed(lambda: s_solve(pat, K, f, d))
            pat.free()
            ta, ts = ta + a, ts + s
        return ta, ts

    small_b(), small_s()
    l0 = R.rpim_kernel_launches()
    tb = min((small_b() for _ in range(2)), key=sum)
    lsb = (R.rpim_kernel_launches() - l0) / 2
    l0 = R.rpim_kernel_launches()
    tsg = min((small_s() for _ in range(2)), key=sum)
    lss = (R.rpim_kernel_launches() - l0) / 2
    snpts = sbat.npts
    small_out = {"instances": len(small), "n_nodes": int(sum(p.n_nodes for p in small)), "n_points": snpts,
                 "assembly": {"batched_ms": tb[0], "per_instance_ms": tsg[0], "speedup": tsg[0] / tb[0],
                              "batched_pts_per_s": snpts / (tb[0] / 1e3),
                              "per_instance_pts_per_s": snpts / (tsg[0] / 1e3)},
                 "solve": {"batched_ms": tb[1], "per_instance_ms": tsg[1], "speedup": tsg[1] / tb[1], "rtol": rtol},
                 "end_to_end": {"batched_ms": sum(tb), "per_instance_ms": sum(tsg), "speedup": sum(tsg) / sum(tb)},
                 "kernel_launches": {"batched": lsb, "per_instance": lss},
                 "step": "every block below %d nodes: build pattern + assemble + tractions (assembly); penalty "
                         "+ Jacobi-PCG to 1e-10 (solve); both arms warm, best of two" % small_nodes}
    # the oracle on host cores: a spread sample of the points of four blocks
    # of the selection (smallest to largest), all cores and one thread
    cpu_out = None
    if cpu:
        picks = sorted(sel, key=lambda p: p.n_nodes)
        picks = [picks[int(i * (len(picks) - 1) / 3)] for i in range(4)]
        runs = [cpu_baseline(p, 2.0, 1.0) for p in picks]
        cpu_out = {"value": len(runs) / sum(1.0 / r["value"] for r in runs), "unit": UNIT, "cores": runs[0]["cores"],
                   "kind": "oracle",
                   "single_thread": {"value": len(runs) / sum(1.0 / r["single_thread"]["value"] for r in runs),
                                     "unit": UNIT, "cores": 1},
                   "sample": "four blocks of the selection (%s nodes), about 2 s of all-core and 1 s of one-thread "
                             "oracle work each, rates combined as a harmonic mean"
                             % ", ".join(str(p.n_nodes) for p in picks)}
    return {"instances": len(sel), "of": len(allp), "selection": "every %d-th block of the 512-block workload"
            % max(1, len(allp) // n_sel), "n_nodes": int(offs[-1]), "n_points": npts,
            "node_range": [int(min(p.n_nodes for p in sel)), int(max(p.n_nodes for p in sel))],
            "warmup_runs_each_arm": warm,
            "assembly": {"batched_ms": ba, "per_instance_ms": sa, "speedup": sa / ba,
                         "batched_pts_per_s": npts / (ba / 1e3), "per_instance_pts_per_s": npts / (sa / 1e3)},
            "solve": {"batched_ms": bs, "per_instance_ms": ss, "speedup": ss / bs, "rtol": rtol,
                      "iterations_max": int(max(itb)), "iterations_sum_per_instance": int(sum(its))},
            "end_to_end": {"batched_ms": ba + bs, "per_instance_ms": sa + ss, "speedup": (sa + ss) / (ba + bs)},
            "kernel_launches": {"batched": lb, "per_instance": ls},
            "reassembly": reasm, "small_blocks": small_out, "bucket_bounds": bounds, "cpu_baseline": cpu_out,
            "u_max_rel_diff_batched_vs_per_instance": du,
            "target_5x": "not met on this workload (FP64-bound blocks fill the GPU alone)",
            "step": "build pattern + assemble + tractions (assembly); penalty + Jacobi-PCG to 1e-10 (solve)"}


# --------------------------------------------------------------------------- end to end
def _e2e(p, dev, stream, n_steps, dist):
    """The headline step through host buffers: pinned host inputs copied to
    the device, the C ABI calls, and K and f copied back into pinned host
    memory on a second stream (overlapped with the next step's assembly, as
    a caller streaming problems would run it), all inside the timed region.
    K and f alternate between two device buffers allocated before the timed
    region, as such a caller would keep them: a step waits for the copy out
    of its buffer to finish before it assembles into it."""
    import torch
    import paper_1802_04256_gb300 as R
    arrays = dict(xyz=p.xyz, lo=p.cell_lo, hi=p.cell_hi, E=p.E, nu=p.nu)
    if np.any(p.body):
        arrays["body"] = p.body
    if p.n_faces:
        arrays.update(fl=p.face_lo, fh=p.face_hi, fc=p.face_coef)
    host = {k: torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).pin_memory() for k, v in arrays.items()}
    if p.n_faces:
        host["fa"] = torch.from_numpy(np.ascontiguousarray(p.face_axis, dtype=np.int8)).pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    Kh = None
    bufs = None
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    copy_stream = torch.cuda.Stream(device=dev)
    count = [0]

    def step():
        nonlocal Kh, bufs
        d = {k: v.to(dev, non_blocking=True) for k, v in host.items()}
        pat = R.Pattern(d["xyz"], d["lo"], d["hi"], p.alpha_s, p.alpha_c, p.q, p.h)
        if bufs is None:
            bufs = [(torch.empty(pat.nnz_blocks, 9, dtype=torch.float64, device=dev),
                     torch.empty(3 * pat.info.n_nodes, dtype=torch.float64, device=dev)) for _ in range(2)]
            for e in copied:
                e.record(copy_stream)
        slot = count[0] % 2
        count[0] += 1
        stream.wait_event(copied[slot])   # the previous copy out of this buffer is done
        K, f = pat.assemble(d["E"], d["nu"], d.get("body"), K=bufs[slot][0], f=bufs[slot][1])
        if p.n_faces:
            pat.add_traction(d["fl"], d["fh"], d["fa"], d["fc"], f)
        if Kh is None:
            Kh = (torch.empty(K.shape, dtype=K.dtype, pin_memory=True),
                  torch.empty(f.shape, dtype=f.dtype, pin_memory=True))
        done = torch.cuda.Event()
        done.record(stream)
        copy_stream.wait_event(done)
        with torch.cuda.stream(copy_stream):
            Kh[0].copy_(K, non_blocking=True)
            Kh[1].copy_(f, non_blocking=True)
            copied[slot].record(copy_stream)
        pat.free()
        return K.numel() * 8 + f.numel() * 8

    step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(n_steps):
        d2h = step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = 1e3 * (time.perf_counter() - t0) / n_steps
    del Kh
    return ms, h2d, d2h


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
    R.rpim_set_row_order(args.row_order == "morton")
    R.rpim_set_shape_solver(args.solver)
    desc, make = WORKLOADS[args.workload]
    p = make()
    inp = Inputs(p, dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    # setup, untimed: bucket bounds and launch shapes of the shape kernel
    # picked by the autotuners on this workload's support sizes (results are
    # bitwise independent of both)
    tuned = bounds = None
    if not args.no_autotune:
        tp = inp.pattern()
        bounds = tp.autotune_buckets(max_points=60000)
        tuned = tp.autotune(max_points=args.tune_points)
        tp.free()
    for _ in range(args.warmup):
        inp.step()
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
    e0, e1 = _events(2)
    e0.record(stream)
    for _ in range(args.steps):
        inp.step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = R.rpim_kernel_launches() - launches0
    R.rpim_profile_enable(False)
    prof = R.rpim_profile_read(reset=True)
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
    value = whole_job_rate(p.n_points, world, ms)

    nsup, nnzb = _support_sizes(inp)
    roof = _roofline(prof, args.steps, nsup, peak_gflops, args.workload)
    if roof and clk:
        roof["peak_nominal_at_clock"] = SMS * DFMA_PER_CLK * 2 * clk["sm_mhz"] * 1e6 / 1e12
    kernel_ms = {k: round(v[1] / args.steps, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    kernel_share = {k: round(v[1] / max(sum(x[1] for x in prof.values()), 1e-9), 4)
                    for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}

    # ---- stages 2 + 3: penalty and PCG (full solves)
    solve = _solves(inp, stream, peak_gflops, args)

    # ---- end to end through host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        e2e_ms, h2d, d2h = _e2e(p, dev, stream, args.e2e_steps, dist)
        e2e_ms = max_over_ranks(e2e_ms, dist, dev)
        e2e = {"value": whole_job_rate(p.n_points, world, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "steps": args.e2e_steps}
    del inp

    # ---- the other workloads (rank 0 only: context, not the headline)
    configs = None
    if rank == 0 and not args.no_configs:
        configs = {}
        cube, _ = _config("cube", dev, stream, peak_gflops, args, steps=10, warm=3, cpu_s=3.0)
        configs["cube"] = cube
        tip = int(np.nonzero(np.all(np.abs(gen.cantilever_config().nominal - [8.0, 0.5, 0.5]) < 1e-9,
                                    axis=1))[0][0])
        cant, cinp = _config("cantilever", dev, stream, peak_gflops, args, steps=5, warm=2, cpu_s=5.0, tip=tip,
                             preconds=["jacobi", "block"])
        if cant.get("solve"):
            for s in cant["solve"].values():
                s["timoshenko"] = 0.20700
        configs["cantilever"] = cant
        del cinp
        back, _ = _config("backanalysis", dev, stream, peak_gflops, args, steps=3, warm=1, cpu_s=4.0)
        configs["backanalysis"] = back

    mls = None
    if rank == 0 and not args.no_mls:
        mls = _mls(Inputs(gen.cantilever_config(), dev), stream, peak_gflops)

    batched = None
    if rank == 0 and args.batched_instances > 0:
        batched = _batched(args.batched_instances, dev, stream, warm=args.batched_warmup,
                           cpu=not args.no_cpu_baseline)
    grad = None
    if rank == 0 and not args.no_grad:
        grad = _backanalysis(dev, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(p, args.cpu_seconds)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": desc, "n_nodes": p.n_nodes, "n_points": p.n_points,
                          "step": "rpim_build_pattern + rpim_assemble" + (" + rpim_add_traction" if p.n_faces else ""),
                          "l2": "inputs and outputs larger than L2 (K %.1f GB, shape functions %.1f GB)"
                                % (nnzb * 72 / 1e9, nsup.sum() * 32 / 1e9),
                          "support": {"min": int(nsup.min()), "max": int(nsup.max()), "mean": float(nsup.mean())},
                          "nnz_blocks": nnzb, "shape_solver": args.solver,
                          "parallelism": "replicas" if world > 1 else "single GPU"},
               "roofline": roof, "kernel_ms_per_step": kernel_ms, "kernel_time_share": kernel_share,
               "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
               "solve": solve, "configs": configs, "mls": mls, "batched": batched, "backanalysis": grad,
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
    ap.add_argument("--workload", default="slope", choices=["slope", "cantilever"],
                    help="headline workload (the layered slope; the cantilever for small profiling runs)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="host seconds of the oracle's all-core sample of the headline workload")
    ap.add_argument("--no-solve", action="store_true", help="skip the penalty + PCG measurements")
    ap.add_argument("--precond", default="jacobi,block",
                    help="PCG preconditioners of the headline solve (comma separated: jacobi, block); the "
                         "cantilever's solve is timed with both")
    ap.add_argument("--row-order", default="morton", choices=["morton", "node"],
                    help="order in which the row-owner kernels take their rows (results are bitwise the same)")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads")
    ap.add_argument("--solver", default="fp64", choices=["fp64", "refined"],
                    help="solver of the moment system in the shape kernel (FP64 LDL', or float-float LDL' "
                         "with one FP64 refinement step)")
    ap.add_argument("--no-grad", action="store_true", help="skip the back-analysis gradient measurement")
    ap.add_argument("--no-mls", action="store_true", help="skip the MLS-variant assembly measurement")
    ap.add_argument("--batched-warmup", type=int, default=1,
                    help="untimed runs of each arm of the batched comparison before the timed one")
    ap.add_argument("--no-autotune", action="store_true", help="use the built-in launch shapes of the shape kernel")
    ap.add_argument("--tune-points", type=int, default=8000,
                    help="points per support-size bucket timed by the launch-shape autotuner")
    ap.add_argument("--solve-iters", type=int, default=0,
                    help="run each solve for exactly this many PCG iterations (profiling; 0 = to rtol 1e-10)")
    ap.add_argument("--batched-instances", type=int, default=64,
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
