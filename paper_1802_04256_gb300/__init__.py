"""GB300 (sm_103a) RPIM stiffness assembly -- Python binding of librpim.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``librpim.so`` behind the C ABI declared in ``include/rpim.h``.
PyTorch provides device memory and streams. The functions ``rpim_*`` mirror
the C entry points one to one; :class:`Pattern` is a thin convenience wrapper.

There is no CPU fallback: if the library is missing or no CUDA device is
present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librpim.so")

RPIM_MAX_SUPPORT = 216
STATUS = {0: "OK", 1: "E_ARG", 2: "E_CUDA", 3: "E_OOM", 4: "E_SUPPORT", 5: "E_SINGULAR",
          6: "E_NOCONV", 7: "E_NONFINITE", 8: "E_TIMEOUT"}

EXPORTED = [
    "rpim_build_pattern", "rpim_pattern_free", "rpim_pattern_get_info", "rpim_pattern_csr",
    "rpim_pattern_points", "rpim_pattern_copy_csr", "rpim_pattern_copy_points", "rpim_assemble",
    "rpim_shape_functions", "rpim_add_point_loads", "rpim_apply_penalty_bc", "rpim_solve_pcg",
    "rpim_stress", "rpim_stress_noalloc", "rpim_last_error", "rpim_version",
    "rpim_apply_penalty_alpha", "rpim_grad_material", "rpim_build_pattern_batched",
    "rpim_add_point_loads_batched", "rpim_apply_penalty_bc_batched", "rpim_stress_batched",
    "rpim_solve_pcg_batched", "rpim_autotune_shape", "rpim_autotune_reset",
    "rpim_autotune_set", "rpim_probe_dfma", "rpim_probe_dmma", "rpim_probe_fp64_mixed",
    "rpim_kernel_launches", "rpim_profile_enable", "rpim_profile_read", "rpim_kernel_series_info",
    "rpim_pattern_set_shape", "rpim_pattern_get_shape", "rpim_assemble_graphed", "rpim_pattern_set_buckets",
    "rpim_pattern_get_buckets", "rpim_autotune_buckets", "rpim_set_shape_schedule",
    "rpim_device_allocations", "rpim_pool_used_bytes", "rpim_add_traction", "rpim_add_traction_batched",
    "rpim_add_vector", "rpim_pattern_set_precond", "rpim_pattern_get_precond", "rpim_set_row_order",
    "rpim_pattern_copy_row_order", "rpim_probe_recip", "rpim_set_shape_solver", "rpim_get_shape_solver",
]

SHAPE_KINDS = {"rpim": 0, "mls": 1, "shepard": 2}
PRECONDS = {"jacobi": 0, "block": 1}


class RpimError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__("%s: RPIM_%s (%d): %s" % (where, STATUS.get(status, "?"), status, msg))
        self.status = status


class Params(C.Structure):
    _fields_ = [("alpha_s", C.c_double), ("alpha_c", C.c_double), ("q", C.c_double),
                ("h", C.c_double), ("gauss_order", C.c_int32)]


class Instance(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("alpha_s", C.c_double), ("h", C.c_double)]


class PatternInfo(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_points", C.c_int64), ("n_entries", C.c_int64),
                ("nnz_blocks", C.c_int64), ("max_support", C.c_int32), ("min_support", C.c_int32),
                ("max_row", C.c_int32), ("device", C.c_int32)]


_lib = None


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile librpim.so in-tree (nvcc, sm_103a)."""
    from . import _compile
    return _compile.build(force=force, verbose=verbose)


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("librpim.so is not built (call paper_1802_04256_gb300.build())")
    L = C.CDLL(LIB_PATH)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    sig = {
        "rpim_build_pattern": [i64, vp, vp, vp, C.POINTER(Params), vp, C.POINTER(vp), C.POINTER(i64)],
        "rpim_pattern_free": [vp],
        "rpim_pattern_get_info": [vp, C.POINTER(PatternInfo)],
        "rpim_pattern_csr": [vp, C.POINTER(vp), C.POINTER(vp)],
        "rpim_pattern_points": [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp)],
        "rpim_pattern_copy_csr": [vp, vp, vp, vp],
        "rpim_pattern_copy_points": [vp, vp, vp, vp, vp, vp],
        "rpim_assemble": [vp, vp, vp, vp, vp, vp, vp],
        "rpim_shape_functions": [vp, vp, vp],
        "rpim_add_point_loads": [vp, i64, vp, vp, vp, vp],
        "rpim_apply_penalty_bc": [vp, vp, vp, i64, vp, vp, dbl, C.POINTER(dbl), vp],
        "rpim_solve_pcg": [vp, vp, vp, vp, dbl, i32, C.POINTER(i32), C.POINTER(dbl), vp],
        "rpim_stress": [vp, vp, i64, vp, vp, vp, vp, vp],
        "rpim_stress_noalloc": [vp, vp, i64, vp, vp, vp, vp, vp],
        "rpim_apply_penalty_alpha": [vp, vp, vp, i64, vp, vp, dbl, vp],
        "rpim_grad_material": [vp, vp, vp, vp, vp, vp, vp, vp],
        "rpim_build_pattern_batched": [i32, C.POINTER(Instance), vp, vp, vp, dbl, dbl, i32, vp, C.POINTER(vp),
                                       C.POINTER(i64)],
        "rpim_add_point_loads_batched": [vp, i64, vp, vp, vp, vp, vp],
        "rpim_apply_penalty_bc_batched": [vp, vp, vp, i64, vp, vp, dbl, C.POINTER(dbl), vp],
        "rpim_stress_batched": [vp, vp, i64, vp, vp, vp, vp, vp, vp],
        "rpim_solve_pcg_batched": [vp, vp, vp, vp, dbl, i32, C.POINTER(i32), C.POINTER(dbl), vp],
        "rpim_autotune_shape": [vp, i64, C.POINTER(i32), C.POINTER(i32), vp],
        "rpim_autotune_reset": [],
        "rpim_autotune_set": [i32, i32, i32],
        "rpim_probe_dfma": [i32, C.POINTER(dbl)],
        "rpim_probe_dmma": [i32, C.POINTER(dbl)],
        "rpim_probe_fp64_mixed": [i32, C.POINTER(dbl)],
        "rpim_profile_enable": [i32],
        "rpim_profile_read": [C.c_char_p, i64, i32],
        "rpim_kernel_series_info": [dbl, dbl, dbl, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32),
                                    C.POINTER(dbl)],
        "rpim_pattern_set_shape": [vp, i32],
        "rpim_assemble_graphed": [vp, vp, vp, vp, vp, vp, vp],
        "rpim_pattern_set_buckets": [vp, i32, C.POINTER(i32), vp],
        "rpim_pattern_get_buckets": [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i64), i32],
        "rpim_autotune_buckets": [vp, i64, C.POINTER(i32), C.POINTER(i32), vp],
        "rpim_set_shape_schedule": [i32],
        "rpim_set_shape_solver": [i32],
        "rpim_get_shape_solver": [C.POINTER(i32)],
        "rpim_pattern_get_shape": [vp, C.POINTER(i32)],
        "rpim_pool_used_bytes": [C.POINTER(i64)],
        "rpim_add_traction": [vp, i64, vp, vp, vp, vp, vp, vp],
        "rpim_add_traction_batched": [vp, i64, vp, vp, vp, vp, vp, vp, vp],
        "rpim_add_vector": [vp, vp, vp, vp],
        "rpim_pattern_set_precond": [vp, i32],
        "rpim_pattern_get_precond": [vp, C.POINTER(i32)],
        "rpim_set_row_order": [i32],
        "rpim_pattern_copy_row_order": [vp, vp, vp],
        "rpim_probe_recip": [i64, vp, vp, vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.rpim_kernel_launches.restype = C.c_int64
    L.rpim_device_allocations.restype = C.c_int64
    L.rpim_last_error.restype = C.c_char_p
    L.rpim_version.restype = C.c_char_p
    _lib = L
    return L


def _check(st, where):
    if st != 0:
        raise RpimError(st, where, lib().rpim_last_error().decode(errors="replace"))


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _dev(t, dtype):
    if t.dtype != dtype:
        raise TypeError("expected %s, got %s" % (dtype, t.dtype))
    return _ptr(t)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


# --------------------------------------------------------------------------- C entry points
def rpim_build_pattern(xyz, cell_lo, cell_hi, params: Params, stream=None):
    h = C.c_void_p()
    nnz = C.c_int64(0)
    st = lib().rpim_build_pattern(xyz.shape[0], _dev(xyz, torch.float64), _dev(cell_lo, torch.float64),
                                  _dev(cell_hi, torch.float64), C.byref(params), _stream(stream),
                                  C.byref(h), C.byref(nnz))
    _check(st, "rpim_build_pattern")
    return h, nnz.value


def rpim_build_pattern_batched(instances, xyz, cell_lo, cell_hi, alpha_c, q, stream=None):
    """instances: sequence of (n_nodes, alpha_s, h); nodes are consecutive."""
    arr = (Instance * len(instances))(*[Instance(int(n), float(a), float(h)) for n, a, h in instances])
    hnd = C.c_void_p()
    nnz = C.c_int64(0)
    st = lib().rpim_build_pattern_batched(len(instances), arr, _dev(xyz, torch.float64), _dev(cell_lo, torch.float64),
                                          _dev(cell_hi, torch.float64), alpha_c, q, 2, _stream(stream),
                                          C.byref(hnd), C.byref(nnz))
    _check(st, "rpim_build_pattern_batched")
    return hnd, nnz.value


def rpim_add_point_loads_batched(handle, xyz, force, inst, f, stream=None):
    _check(lib().rpim_add_point_loads_batched(handle, xyz.shape[0], _dev(xyz, torch.float64),
                                              _dev(force, torch.float64), _dev(inst, torch.int32),
                                              _dev(f, torch.float64), _stream(stream)), "rpim_add_point_loads_batched")


def rpim_apply_penalty_bc_batched(handle, n_inst, K_vals, f, dofs, values, penalty_scale=1e8, stream=None):
    a = (C.c_double * n_inst)()
    _check(lib().rpim_apply_penalty_bc_batched(handle, _dev(K_vals, torch.float64), _dev(f, torch.float64),
                                               dofs.shape[0], _dev(dofs, torch.int64), _dev(values, torch.float64),
                                               penalty_scale, a, _stream(stream)), "rpim_apply_penalty_bc_batched")
    return list(a)


def rpim_stress_batched(handle, u, xyz, inst, E, nu, sigma, stream=None):
    _check(lib().rpim_stress_batched(handle, _dev(u, torch.float64), xyz.shape[0], _dev(xyz, torch.float64),
                                     _dev(inst, torch.int32), _dev(E, torch.float64), _dev(nu, torch.float64),
                                     _dev(sigma, torch.float64), _stream(stream)), "rpim_stress_batched")


def rpim_pattern_set_shape(handle, kind):
    """kind: "rpim", "mls" or "shepard" (or the integer of rpim_shape_kind)."""
    k = SHAPE_KINDS[kind] if isinstance(kind, str) else int(kind)
    _check(lib().rpim_pattern_set_shape(handle, k), "rpim_pattern_set_shape")


def rpim_pattern_get_shape(handle) -> str:
    k = C.c_int32(0)
    _check(lib().rpim_pattern_get_shape(handle, C.byref(k)), "rpim_pattern_get_shape")
    return {v: n for n, v in SHAPE_KINDS.items()}[k.value]


def rpim_pattern_set_precond(handle, kind):
    """kind: "jacobi" or "block" (3x3 block Jacobi), or the integer of rpim_precond_kind."""
    k = PRECONDS[kind] if isinstance(kind, str) else int(kind)
    _check(lib().rpim_pattern_set_precond(handle, k), "rpim_pattern_set_precond")


def rpim_pattern_get_precond(handle) -> str:
    k = C.c_int32(0)
    _check(lib().rpim_pattern_get_precond(handle, C.byref(k)), "rpim_pattern_get_precond")
    return {v: n for n, v in PRECONDS.items()}[k.value]


def rpim_pattern_free(handle):
    lib().rpim_pattern_free(handle)


def rpim_pattern_get_info(handle) -> PatternInfo:
    info = PatternInfo()
    _check(lib().rpim_pattern_get_info(handle, C.byref(info)), "rpim_pattern_get_info")
    return info


def rpim_pattern_copy_csr(handle, rowptr, cols, stream=None):
    _check(lib().rpim_pattern_copy_csr(handle, _dev(rowptr, torch.int64), _dev(cols, torch.int32),
                                       _stream(stream)), "rpim_pattern_copy_csr")


def rpim_pattern_copy_points(handle, xyz, wj, soff, sidx, stream=None):
    _check(lib().rpim_pattern_copy_points(handle, _ptr(xyz), _ptr(wj), _ptr(soff), _ptr(sidx),
                                          _stream(stream)), "rpim_pattern_copy_points")


def rpim_assemble(handle, E, nu, body, K_vals, f, stream=None):
    _check(lib().rpim_assemble(handle, _dev(E, torch.float64), _dev(nu, torch.float64),
                               None if body is None else _dev(body, torch.float64),
                               _dev(K_vals, torch.float64), _dev(f, torch.float64), _stream(stream)),
           "rpim_assemble")


def rpim_assemble_graphed(handle, E, nu, body, K_vals, f, stream=None):
    _check(lib().rpim_assemble_graphed(handle, _dev(E, torch.float64), _dev(nu, torch.float64),
                                       None if body is None else _dev(body, torch.float64),
                                       _dev(K_vals, torch.float64), _dev(f, torch.float64), _stream(stream)),
           "rpim_assemble_graphed")


def rpim_pattern_set_buckets(handle, bounds, stream=None):
    arr = (C.c_int32 * len(bounds))(*[int(b) for b in bounds])
    _check(lib().rpim_pattern_set_buckets(handle, len(bounds), arr, _stream(stream)), "rpim_pattern_set_buckets")


def rpim_pattern_get_buckets(handle):
    """[(upper bound, largest support, points)] of every bucket."""
    nb = C.c_int32(0)
    b, m, c = (C.c_int32 * 64)(), (C.c_int32 * 64)(), (C.c_int64 * 64)()
    _check(lib().rpim_pattern_get_buckets(handle, C.byref(nb), b, m, c, 64), "rpim_pattern_get_buckets")
    return [(b[i], m[i], c[i]) for i in range(min(nb.value, 64))]


def rpim_autotune_buckets(handle, max_points=200000, stream=None):
    """Picks the bucket bounds (see include/rpim.h); returns them."""
    b = (C.c_int32 * 32)()
    n = C.c_int32(0)
    _check(lib().rpim_autotune_buckets(handle, max_points, b, C.byref(n), _stream(stream)), "rpim_autotune_buckets")
    return list(b[:n.value])


def rpim_set_shape_schedule(persistent: bool):
    _check(lib().rpim_set_shape_schedule(1 if persistent else 0), "rpim_set_shape_schedule")


SOLVERS = {"fp64": 0, "refined": 1}


def rpim_set_shape_solver(solver: str):
    """Solver of the reduced moment system in the RPIM shape kernel: "fp64"
    (FP64 LDL', the default) or "refined" (float-float LDL' with one FP64
    refinement step)."""
    _check(lib().rpim_set_shape_solver(SOLVERS[solver]), "rpim_set_shape_solver")


def rpim_get_shape_solver() -> str:
    v = C.c_int32(0)
    _check(lib().rpim_get_shape_solver(C.byref(v)), "rpim_get_shape_solver")
    return {b: a for a, b in SOLVERS.items()}[v.value]


def rpim_set_row_order(morton: bool):
    """Rows of the row-owner kernels in Morton order (True) or node order."""
    _check(lib().rpim_set_row_order(1 if morton else 0), "rpim_set_row_order")


def rpim_pattern_copy_row_order(handle, order, stream=None):
    _check(lib().rpim_pattern_copy_row_order(handle, _dev(order, torch.int32), _stream(stream)),
           "rpim_pattern_copy_row_order")


def rpim_shape_functions(handle, phi, stream=None):
    _check(lib().rpim_shape_functions(handle, _dev(phi, torch.float64), _stream(stream)),
           "rpim_shape_functions")


def rpim_add_point_loads(handle, xyz, force, f, stream=None):
    _check(lib().rpim_add_point_loads(handle, xyz.shape[0], _dev(xyz, torch.float64),
                                      _dev(force, torch.float64), _dev(f, torch.float64),
                                      _stream(stream)), "rpim_add_point_loads")


def rpim_add_traction(handle, face_lo, face_hi, face_axis, coef, f, stream=None):
    _check(lib().rpim_add_traction(handle, face_lo.shape[0], _dev(face_lo, torch.float64),
                                   _dev(face_hi, torch.float64), _dev(face_axis, torch.int8),
                                   _dev(coef, torch.float64), _dev(f, torch.float64), _stream(stream)),
           "rpim_add_traction")


def rpim_add_traction_batched(handle, face_lo, face_hi, face_axis, coef, inst, f, stream=None):
    _check(lib().rpim_add_traction_batched(handle, face_lo.shape[0], _dev(face_lo, torch.float64),
                                           _dev(face_hi, torch.float64), _dev(face_axis, torch.int8),
                                           _dev(coef, torch.float64), _dev(inst, torch.int32),
                                           _dev(f, torch.float64), _stream(stream)), "rpim_add_traction_batched")


def rpim_add_vector(handle, x, f, stream=None):
    _check(lib().rpim_add_vector(handle, _dev(x, torch.float64), _dev(f, torch.float64), _stream(stream)),
           "rpim_add_vector")


def rpim_apply_penalty_bc(handle, K_vals, f, dofs, values, penalty_scale=1e8, stream=None):
    a = C.c_double(0)
    _check(lib().rpim_apply_penalty_bc(handle, _dev(K_vals, torch.float64), _dev(f, torch.float64),
                                       dofs.shape[0], _dev(dofs, torch.int64),
                                       _dev(values, torch.float64), penalty_scale, C.byref(a),
                                       _stream(stream)), "rpim_apply_penalty_bc")
    return a.value


def rpim_apply_penalty_alpha(handle, K_vals, f, dofs, values, alpha, stream=None):
    _check(lib().rpim_apply_penalty_alpha(handle, _dev(K_vals, torch.float64), _dev(f, torch.float64),
                                          dofs.shape[0], _dev(dofs, torch.int64), _dev(values, torch.float64),
                                          alpha, _stream(stream)), "rpim_apply_penalty_alpha")


def rpim_grad_material(handle, u, lam, E, nu, dE, dnu, stream=None):
    _check(lib().rpim_grad_material(handle, _dev(u, torch.float64), _dev(lam, torch.float64),
                                    _dev(E, torch.float64), _dev(nu, torch.float64), _dev(dE, torch.float64),
                                    _dev(dnu, torch.float64), _stream(stream)), "rpim_grad_material")


def rpim_solve_pcg(handle, K_vals, f, u, rtol=1e-10, max_iter=100000, stream=None, check=True):
    it = C.c_int32(0)
    rr = C.c_double(0)
    st = lib().rpim_solve_pcg(handle, _dev(K_vals, torch.float64), _dev(f, torch.float64),
                              _dev(u, torch.float64), rtol, max_iter, C.byref(it), C.byref(rr),
                              _stream(stream))
    if check:
        _check(st, "rpim_solve_pcg")
    return it.value, rr.value, st


def rpim_solve_pcg_batched(handle, n_inst, K_vals, f, u, rtol=1e-10, max_iter=100000, stream=None, check=True):
    """Returns (iterations per instance, relative residual per instance, status)."""
    it = (C.c_int32 * n_inst)()
    rr = (C.c_double * n_inst)()
    st = lib().rpim_solve_pcg_batched(handle, _dev(K_vals, torch.float64), _dev(f, torch.float64),
                                      _dev(u, torch.float64), rtol, max_iter, it, rr, _stream(stream))
    if check:
        _check(st, "rpim_solve_pcg_batched")
    return list(it), list(rr), st


def rpim_autotune_shape(handle, max_points=20000, stream=None):
    """Tunes the shape kernel's launch shape per support-size bucket of the
    pattern; returns [(largest support, warps per point, points per block)]."""
    table = (C.c_int32 * 48)()
    n = C.c_int32(0)
    _check(lib().rpim_autotune_shape(handle, max_points, table, C.byref(n), _stream(stream)), "rpim_autotune_shape")
    return [tuple(table[3 * i:3 * i + 3]) for i in range(min(n.value, 16))]


def rpim_autotune_set(max_support, warps_per_point, points_per_block):
    _check(lib().rpim_autotune_set(max_support, warps_per_point, points_per_block), "rpim_autotune_set")


def rpim_autotune_reset():
    _check(lib().rpim_autotune_reset(), "rpim_autotune_reset")


def rpim_stress(handle, u, xyz, E, nu, sigma, stream=None):
    _check(lib().rpim_stress(handle, _dev(u, torch.float64), xyz.shape[0], _dev(xyz, torch.float64),
                             _dev(E, torch.float64), _dev(nu, torch.float64),
                             _dev(sigma, torch.float64), _stream(stream)), "rpim_stress")


def rpim_probe_dfma(repeats=5) -> float:
    """Measured FP64 FMA-pipe throughput of the current device, GFLOP/s."""
    g = C.c_double(0)
    _check(lib().rpim_probe_dfma(repeats, C.byref(g)), "rpim_probe_dfma")
    return g.value


def rpim_probe_fp64_mixed(repeats=5) -> float:
    g = C.c_double(0)
    _check(lib().rpim_probe_fp64_mixed(repeats, C.byref(g)), "rpim_probe_fp64_mixed")
    return g.value


def rpim_probe_dmma(repeats=5) -> float:
    """Measured FP64 tensor-core (mma.sync m8n8k4) throughput, GFLOP/s."""
    g = C.c_double(0)
    _check(lib().rpim_probe_dmma(repeats, C.byref(g)), "rpim_probe_dmma")
    return g.value


def rpim_probe_recip(d, stream=None):
    """The shape kernel's reciprocal of every entry of d (device, float64)."""
    r = torch.empty_like(d)
    _check(lib().rpim_probe_recip(d.numel(), _dev(d, torch.float64), _dev(r, torch.float64), _stream(stream)),
           "rpim_probe_recip")
    return r


def rpim_kernel_series_info(alpha_c=4.0, alpha_s=2.5, q=1.03):
    """(pieces, degree, fp64_terms, max_err) of the kernel series (host only)."""
    p, d, h = C.c_int32(0), C.c_int32(0), C.c_int32(0)
    e = C.c_double(0)
    st = lib().rpim_kernel_series_info(alpha_c, alpha_s, q, C.byref(p), C.byref(d), C.byref(h), C.byref(e))
    _check(st, "rpim_kernel_series_info")
    return p.value, d.value, h.value, e.value


def rpim_kernel_launches() -> int:
    """Kernels launched by the library since it was loaded."""
    return int(lib().rpim_kernel_launches())


def rpim_device_allocations() -> int:
    """Device-memory allocations the library has requested since it was loaded."""
    return int(lib().rpim_device_allocations())


def rpim_pool_used_bytes() -> int:
    """Bytes in use from the current device's default stream-ordered pool."""
    b = C.c_int64(0)
    _check(lib().rpim_pool_used_bytes(C.byref(b)), "rpim_pool_used_bytes")
    return b.value


def rpim_profile_enable(on: bool = True) -> None:
    _check(lib().rpim_profile_enable(1 if on else 0), "rpim_profile_enable")


def rpim_profile_read(reset: bool = True) -> dict:
    """Per-kernel {name: (launches, total_ms)} gathered while timing was on."""
    import json
    buf = C.create_string_buffer(1 << 16)
    _check(lib().rpim_profile_read(buf, len(buf), 1 if reset else 0), "rpim_profile_read")
    return {k: (v[0], v[1]) for k, v in json.loads(buf.value.decode()).items()}


def rpim_stress_noalloc(handle, u, xyz, E, nu, sigma, stream=None):
    """rpim_stress with its scratch in the library's fixed device array
    (no allocation; at most 2048 points per call; calls must not overlap)."""
    _check(lib().rpim_stress_noalloc(handle, _dev(u, torch.float64), xyz.shape[0], _dev(xyz, torch.float64),
                                     _dev(E, torch.float64), _dev(nu, torch.float64),
                                     _dev(sigma, torch.float64), _stream(stream)), "rpim_stress_noalloc")


def rpim_version() -> str:
    return lib().rpim_version().decode()


# --------------------------------------------------------------------------- convenience
class Pattern:
    """Owns an ``rpim_pattern``: integration points, supports and the BSR
    pattern of K for one node cloud."""

    def __init__(self, xyz, cell_lo, cell_hi, alpha_s, alpha_c, q, h, stream=None, instances=None, shape="rpim"):
        self.device = xyz.device
        if instances is None:
            self.params = Params(alpha_s, alpha_c, q, h, 2)
            self.handle, self.nnz_blocks = rpim_build_pattern(xyz, cell_lo, cell_hi, self.params, stream)
            self.n_inst = 1
        else:
            self.params = None
            self.handle, self.nnz_blocks = rpim_build_pattern_batched(instances, xyz, cell_lo, cell_hi, alpha_c, q,
                                                                      stream)
            self.n_inst = len(instances)
        self.info = rpim_pattern_get_info(self.handle)
        if shape != "rpim":
            rpim_pattern_set_shape(self.handle, shape)

    def set_precond(self, kind):
        """Preconditioner of the later PCG solves: "jacobi" or "block"."""
        rpim_pattern_set_precond(self.handle, kind)

    def set_shape(self, kind):
        """Shape functions of the later stages: "rpim", "mls" or "shepard"."""
        rpim_pattern_set_shape(self.handle, kind)

    @property
    def shape(self):
        return rpim_pattern_get_shape(self.handle)

    @classmethod
    def batched(cls, problems, device="cuda", stream=None):
        """One pattern for a list of gen.Problem instances (concatenated in
        order); returns (pattern, node offsets)."""
        xyz = np.concatenate([p.xyz for p in problems])
        lo = np.concatenate([p.cell_lo for p in problems])
        hi = np.concatenate([p.cell_hi for p in problems])
        t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=device).contiguous()
        inst = [(p.n_nodes, p.alpha_s, p.h) for p in problems]
        offs = np.concatenate([[0], np.cumsum([p.n_nodes for p in problems])])
        return cls(t(xyz), t(lo), t(hi), None, problems[0].alpha_c, problems[0].q, None, stream, inst), offs

    @classmethod
    def from_problem(cls, p, device="cuda", stream=None, shape="rpim"):
        t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=device).contiguous()
        return cls(t(p.xyz), t(p.cell_lo), t(p.cell_hi), p.alpha_s, p.alpha_c, p.q, p.h, stream, shape=shape)

    def free(self):
        if self.handle:
            rpim_pattern_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def csr(self, stream=None):
        rowptr = torch.empty(self.info.n_nodes + 1, dtype=torch.int64, device=self.device)
        cols = torch.empty(max(self.nnz_blocks, 1), dtype=torch.int32, device=self.device)
        rpim_pattern_copy_csr(self.handle, rowptr, cols, stream)
        return rowptr, cols[: self.nnz_blocks]

    def row_order(self, stream=None):
        """The pattern's Morton row order (a permutation of the nodes)."""
        order = torch.empty(self.info.n_nodes, dtype=torch.int32, device=self.device)
        rpim_pattern_copy_row_order(self.handle, order, stream)
        return order

    def points(self, stream=None):
        i = self.info
        xyz = torch.empty(i.n_points, 3, dtype=torch.float64, device=self.device)
        wj = torch.empty(i.n_points, dtype=torch.float64, device=self.device)
        soff = torch.empty(i.n_points + 1, dtype=torch.int64, device=self.device)
        sidx = torch.empty(max(i.n_entries, 1), dtype=torch.int32, device=self.device)
        rpim_pattern_copy_points(self.handle, xyz, wj, soff, sidx, stream)
        return xyz, wj, soff, sidx[: i.n_entries]

    def shape_functions(self, stream=None):
        phi = torch.empty(self.info.n_entries, 4, dtype=torch.float64, device=self.device)
        rpim_shape_functions(self.handle, phi, stream)
        return phi

    def assemble(self, E, nu, body=None, K=None, f=None, stream=None):
        if K is None:
            K = torch.empty(self.nnz_blocks, 9, dtype=torch.float64, device=self.device)
        if f is None:
            f = torch.empty(3 * self.info.n_nodes, dtype=torch.float64, device=self.device)
        rpim_assemble(self.handle, E, nu, body, K, f, stream)
        return K, f

    def assemble_graphed(self, E, nu, body=None, K=None, f=None, stream=None):
        """assemble() replayed from the pattern's captured CUDA graph (the
        output buffers must stay the same between calls to reuse it)."""
        if K is None:
            K = torch.empty(self.nnz_blocks, 9, dtype=torch.float64, device=self.device)
        if f is None:
            f = torch.empty(3 * self.info.n_nodes, dtype=torch.float64, device=self.device)
        rpim_assemble_graphed(self.handle, E, nu, body, K, f, stream)
        return K, f

    def autotune_buckets(self, max_points=200000, stream=None):
        return rpim_autotune_buckets(self.handle, max_points, stream)

    def buckets(self):
        return rpim_pattern_get_buckets(self.handle)

    def add_point_loads(self, xyz, force, f, stream=None, inst=None):
        if inst is None:
            rpim_add_point_loads(self.handle, xyz, force, f, stream)
        else:
            rpim_add_point_loads_batched(self.handle, xyz, force, inst, f, stream)
        return f

    def add_traction(self, face_lo, face_hi, face_axis, coef, f, stream=None, inst=None):
        """f += the tractions of the faces (see rpim_add_traction); coef
        [n_faces, 3, 6]; inst: instance of every face (batched patterns)."""
        if inst is None:
            rpim_add_traction(self.handle, face_lo, face_hi, face_axis, coef, f, stream)
        else:
            rpim_add_traction_batched(self.handle, face_lo, face_hi, face_axis, coef, inst, f, stream)
        return f

    def apply_penalty(self, K, f, dofs, values, scale=1e8, stream=None):
        """alpha (a list of one alpha per instance for batched patterns)."""
        if self.n_inst > 1:
            return rpim_apply_penalty_bc_batched(self.handle, self.n_inst, K, f, dofs, values, scale, stream)
        return rpim_apply_penalty_bc(self.handle, K, f, dofs, values, scale, stream)

    def solve_pcg(self, K, f, u=None, rtol=1e-10, max_iter=100000, stream=None, check=True, precond=None):
        """PCG solve (u holds the initial guess); precond "jacobi" or "block"
        sets the pattern's preconditioner first (None: keep it)."""
        if precond is not None:
            rpim_pattern_set_precond(self.handle, precond)
        if u is None:
            u = torch.zeros(3 * self.info.n_nodes, dtype=torch.float64, device=self.device)
        it, rr, st = rpim_solve_pcg(self.handle, K, f, u, rtol, max_iter, stream, check)
        return u, it, rr

    def autotune(self, max_points=20000, stream=None):
        return rpim_autotune_shape(self.handle, max_points, stream)

    def solve_pcg_batched(self, K, f, u=None, rtol=1e-10, max_iter=100000, stream=None, check=True, precond=None):
        """Per-instance PCG: (u, iterations per instance, residual per instance)."""
        if precond is not None:
            rpim_pattern_set_precond(self.handle, precond)
        if u is None:
            u = torch.zeros(3 * self.info.n_nodes, dtype=torch.float64, device=self.device)
        it, rr, st = rpim_solve_pcg_batched(self.handle, self.n_inst, K, f, u, rtol, max_iter, stream, check)
        return u, it, rr

    def stress(self, u, xyz, E, nu, stream=None, inst=None):
        sig = torch.empty(xyz.shape[0], 6, dtype=torch.float64, device=self.device)
        if inst is None:
            rpim_stress(self.handle, u, xyz, E, nu, sig, stream)
        else:
            rpim_stress_batched(self.handle, u, xyz, inst, E, nu, sig, stream)
        return sig


# --------------------------------------------------------------------------- differentiable solve
class _Solve(torch.autograd.Function):
    """u(E, nu) for K(E, nu) u = f with a frozen penalty; backward by the
    adjoint K lam = dL/du (same K, K symmetric) and rpim_grad_material."""

    @staticmethod
    def forward(ctx, E, nu, pattern, f_ext, dofs, values, alpha, rtol, max_iter):
        E = E.detach().contiguous()
        nu = nu.detach().contiguous()
        K, f = pattern.assemble(E, nu)
        rpim_add_vector(pattern.handle, f_ext.contiguous(), f)
        rpim_apply_penalty_alpha(pattern.handle, K, f, dofs, values, alpha)
        u = torch.zeros(3 * pattern.info.n_nodes, dtype=torch.float64, device=E.device)
        it, rr, st = rpim_solve_pcg(pattern.handle, K, f, u, rtol, max_iter)
        ctx.pattern, ctx.K, ctx.rtol, ctx.max_iter = pattern, K, rtol, max_iter
        ctx.save_for_backward(E, nu, u)
        ctx.pcg = (it, rr)
        return u

    @staticmethod
    def backward(ctx, gu):
        E, nu, u = ctx.saved_tensors
        lam = torch.zeros_like(u)
        rpim_solve_pcg(ctx.pattern.handle, ctx.K, gu.contiguous(), lam, ctx.rtol, ctx.max_iter)
        dE = torch.empty_like(E)
        dnu = torch.empty_like(nu)
        rpim_grad_material(ctx.pattern.handle, u, lam, E, nu, dE, dnu)
        return dE, dnu, None, None, None, None, None, None, None


def penalty_alpha(pattern, E, nu, scale=1e8):
    """alpha = scale * max_i K_ii of K(E, nu): the value to freeze for a
    back-analysis."""
    K, f = pattern.assemble(E, nu)
    dofs = torch.zeros(0, dtype=torch.int64, device=K.device)
    vals = torch.zeros(0, dtype=torch.float64, device=K.device)
    return rpim_apply_penalty_bc(pattern.handle, K, f, dofs, vals, scale)


def solve(pattern, E, nu, f_ext, fixed_dofs, fixed_values, alpha, rtol=1e-12, max_iter=200000):
    """Displacements u(E, nu) with gradients with respect to the per-point
    Young's modulus E and Poisson's ratio nu (torch.autograd).

    f_ext: surface loads (device, 3*n_nodes, material independent, e.g.
    from rpim_add_traction once), added by rpim_add_vector to the
    body-force vector of every assembly;
    alpha: the frozen penalty (see penalty_alpha)."""
    return _Solve.apply(E, nu, pattern, f_ext, fixed_dofs, fixed_values, alpha, rtol, max_iter)
