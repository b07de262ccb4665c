"""ctypes front end of the RPIM oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers. The product path never
imports this package. Two builds exist: ``f64`` (every step in double) and
``ld`` (every step after the integration points in long double: 80-bit x87
on x86-64, IEEE binary128 on AArch64), which measures the FP64 floor.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIBS = {"f64": os.path.join(HERE, "liboracle_f64.so"), "ld": os.path.join(HERE, "liboracle_ld.so")}

MAX_SUPPORT = 4096


def build(force: bool = False) -> None:
    """Compile both oracle builds with gcc (no fused multiply-add contraction)."""
    for kind, out in LIBS.items():
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
            continue
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
               SRC, "-o", out + ".tmp", "-lm"]
        if kind == "ld":
            cmd.insert(1, "-DORC_LONG")
        subprocess.run(cmd, check=True)
        os.replace(out + ".tmp", out)


_libs: dict = {}


def register(kind: str, path: str) -> None:
    """Make another build of oracle.c (e.g. a test's deliberately broken
    copy) available under ``kind``."""
    LIBS[kind] = path
    _libs.pop(kind, None)

_P = np.ctypeslib.ndpointer
_D = _P(dtype=np.float64, flags="C_CONTIGUOUS")
_I64 = _P(dtype=np.int64, flags="C_CONTIGUOUS")
_I32 = _P(dtype=np.int32, flags="C_CONTIGUOUS")


def lib(kind: str = "f64"):
    if kind in _libs:
        return _libs[kind]
    if not os.path.exists(LIBS[kind]):
        build()
    L = C.CDLL(LIBS[kind])
    i64, i32, dbl, vp = C.c_int64, C.c_int, C.c_double, C.c_void_p
    L.orc_real_bytes.restype = i32
    L.orc_set_threads.argtypes = [i32]
    L.orc_gauss_points.argtypes = [i64, _D, _D, _D, _D]
    L.orc_support.argtypes = [i64, _D, _D, dbl, _I32, i64]
    L.orc_support.restype = i64
    L.orc_support_radius2.argtypes = [dbl, dbl]
    L.orc_support_radius2.restype = dbl
    L.orc_shape.argtypes = [_D, _I32, i32, _D, dbl, dbl, dbl, _D]
    L.orc_shape.restype = i32
    L.orc_shape_mls.argtypes = [_D, _I32, i32, _D, dbl, dbl, _D]
    L.orc_shape_mls.restype = i32
    L.orc_shape_shepard.argtypes = [_D, _I32, i32, _D, dbl, dbl, _D]
    L.orc_shape_shepard.restype = i32
    L.orc_set_shape.argtypes = [i32]
    L.orc_get_shape.restype = i32
    L.orc_assemble.argtypes = [i64, _D, i64, _D, _D, _D, _D, vp, dbl, dbl, dbl, dbl, i32, vp]
    L.orc_assemble.restype = vp
    L.orc_free.argtypes = [vp]
    for fn in ("orc_status",):
        getattr(L, fn).argtypes = [vp]
        getattr(L, fn).restype = i32
    for fn in ("orc_bad_point", "orc_nnzb", "orc_support_total"):
        getattr(L, fn).argtypes = [vp]
        getattr(L, fn).restype = i64
    L.orc_copy_csr.argtypes = [vp, _I64, _I32, _D, _D]
    L.orc_copy_support.argtypes = [vp, _I64, _I32]
    L.orc_point_loads.argtypes = [i64, _D, i64, _D, _D, dbl, dbl, dbl, dbl, i32, _D]
    L.orc_point_loads.restype = i32
    L.orc_traction.argtypes = [i64, _D, i64, _D, _D, _P(dtype=np.int8, flags="C_CONTIGUOUS"), _D, dbl, dbl,
                               dbl, dbl, i32, _D]
    L.orc_traction.restype = i32
    L.orc_penalty.argtypes = [i64, _I64, _I32, _D, _D, i64, _I64, _D, dbl, C.POINTER(dbl)]
    L.orc_penalty.restype = i32
    L.orc_pcg.argtypes = [i64, _I64, _I32, _D, _D, _D, dbl, i32, C.POINTER(i32), C.POINTER(dbl), i32]
    L.orc_pcg.restype = i32
    L.orc_stress.argtypes = [i64, _D, _D, i64, _D, _D, _D, dbl, dbl, dbl, dbl, i32, _D]
    L.orc_stress.restype = i32
    L.orc_grad_material.argtypes = [i64, _D, i64, _D, _D, _D, _D, _D, _D, dbl, dbl, dbl, dbl, i32, _D, _D]
    L.orc_grad_material.restype = i32
    _libs[kind] = L
    return L


def _c(a, dt=np.float64):
    return np.ascontiguousarray(a, dtype=dt)


class OracleError(RuntimeError):
    def __init__(self, status, what=""):
        super().__init__("oracle status %d %s" % (status, what))
        self.status = status


def set_threads(t: int, kind: str = "f64") -> None:
    lib(kind).orc_set_threads(int(t))


SHAPES = {"rpim": 0, "mls": 1, "shepard": 2}


class shape_kind:
    """Context manager selecting the shape functions of every assembly-level
    oracle function (assemble, point_loads, stress, grad_material, and the
    *_problem helpers) in every registered build:
    ``with oracle.shape_kind("mls"): ...``"""

    def __init__(self, name: str):
        self.code = SHAPES[name]

    def __enter__(self):
        self.saved = {k: lib(k).orc_get_shape() for k in LIBS}
        for k in LIBS:
            lib(k).orc_set_shape(self.code)
        return self

    def __exit__(self, *exc):
        for k, v in self.saved.items():
            lib(k).orc_set_shape(v)
        return False


def gauss_points(cell_lo, cell_hi, kind="f64"):
    lo, hi = _c(cell_lo), _c(cell_hi)
    n = lo.shape[0]
    pts = np.zeros((8 * n, 3))
    wj = np.zeros(8 * n)
    lib(kind).orc_gauss_points(n, lo, hi, pts, wj)
    return pts, wj


def support_radius2(alpha_s, h, kind="f64"):
    return lib(kind).orc_support_radius2(alpha_s, h)


def support(xyz, x, rs2, kind="f64"):
    xyz = _c(xyz)
    out = np.zeros(MAX_SUPPORT, np.int32)
    c = lib(kind).orc_support(xyz.shape[0], xyz, _c(x), rs2, out, MAX_SUPPORT)
    if c > MAX_SUPPORT:
        raise OracleError(4, "support too large")
    return out[:c].copy()


def shape(xyz, supp, x, h, alpha_c=4.0, q=1.03, kind="f64"):
    """phi, dphi/dx, dphi/dy, dphi/dz at x: array (4, n)."""
    supp = _c(supp, np.int32)
    n = len(supp)
    out = np.zeros(4 * n)
    st = lib(kind).orc_shape(_c(xyz), supp, n, _c(x), h, alpha_c, q, out)
    if st:
        raise OracleError(st, "shape")
    return out.reshape(4, n)


class Model:
    """Assembled K (3x3-block CSR) and body-force vector."""

    def __init__(self, n_nodes, rowptr, cols, vals, f, soff, sidx):
        self.n_nodes, self.rowptr, self.cols, self.vals, self.f = n_nodes, rowptr, cols, vals, f
        self.soff, self.sidx = soff, sidx

    def dense(self):
        n = self.n_nodes
        K = np.zeros((3 * n, 3 * n))
        for I in range(n):
            for t in range(self.rowptr[I], self.rowptr[I + 1]):
                J = self.cols[t]
                K[3 * I:3 * I + 3, 3 * J:3 * J + 3] = self.vals[t].reshape(3, 3)
        return K

    def matvec(self, x):
        x = np.asarray(x).reshape(-1, 3)
        rows = np.repeat(np.arange(self.n_nodes), np.diff(self.rowptr))
        y = np.einsum("tab,tb->ta", self.vals.reshape(-1, 3, 3), x[self.cols])
        out = np.zeros((self.n_nodes, 3))
        np.add.at(out, rows, y)
        return out.ravel()



def shape_mls(xyz, supp, x, h, alpha_s, kind="f64"):
    """MLS shape functions (linear basis, cubic-spline weight of radius
    alpha_s h) at x: array [4, n] (phi, dphi/dx, dphi/dy, dphi/dz)."""
    xyz, s = _c(xyz), _c(supp, np.int32)
    out = np.zeros(4 * len(s))
    st = lib(kind).orc_shape_mls(xyz, s, len(s), _c(x), h, alpha_s, out)
    if st != 0:
        raise OracleError(st, "shape_mls")
    return out.reshape(4, len(s))


def shape_shepard(xyz, supp, x, h, alpha_s, kind="f64"):
    """Shepard shape functions (constant basis, the same cubic-spline weight)
    at x: array [4, n] (phi, dphi/dx, dphi/dy, dphi/dz)."""
    xyz, s = _c(xyz), _c(supp, np.int32)
    out = np.zeros(4 * len(s))
    st = lib(kind).orc_shape_shepard(xyz, s, len(s), _c(x), h, alpha_s, out)
    if st != 0:
        raise OracleError(st, "shape_shepard")
    return out.reshape(4, len(s))

def assemble(xyz, pts, wj, E, nu, alpha_s, alpha_c, q, h, body=None, kind="f64",
             max_support=MAX_SUPPORT, rows=None):
    """Assemble K and f over the given integration points (ascending order);
    with `rows` (node ids), only those rows of K and entries of f are formed
    (the others are zero)."""
    L = lib(kind)
    xyz = _c(xyz)
    pts = _c(pts)
    bodyp = None
    if body is not None:
        bb = _c(body)
        bodyp = bb.ctypes.data_as(C.c_void_p)
    maskp = None
    if rows is not None:
        mask = np.zeros(xyz.shape[0], np.uint8)
        mask[np.asarray(rows, np.int64)] = 1
        maskp = mask.ctypes.data_as(C.c_void_p)
    h_ = L.orc_assemble(xyz.shape[0], xyz, pts.shape[0], pts, _c(wj), _c(E), _c(nu), bodyp,
                        alpha_s, alpha_c, q, h, max_support, maskp)
    if not h_:
        raise OracleError(3, "allocation")
    try:
        st = L.orc_status(h_)
        if st:
            raise OracleError(st, "assemble (point %d)" % L.orc_bad_point(h_))
        n = xyz.shape[0]
        nnzb = L.orc_nnzb(h_)
        rowptr = np.zeros(n + 1, np.int64)
        cols = np.zeros(nnzb, np.int32)
        vals = np.zeros(9 * nnzb)
        f = np.zeros(3 * n)
        L.orc_copy_csr(h_, rowptr, cols, vals, f)
        tot = L.orc_support_total(h_)
        soff = np.zeros(pts.shape[0] + 1, np.int64)
        sidx = np.zeros(max(tot, 1), np.int32)
        L.orc_copy_support(h_, soff, sidx)
        return Model(n, rowptr, cols, vals.reshape(-1, 9), f, soff, sidx[:tot])
    finally:
        L.orc_free(h_)


def assemble_problem(p, kind="f64", with_loads=True):
    """Gauss points, K, f (body force + surface tractions) for a gen.Problem."""
    pts, wj = gauss_points(p.cell_lo, p.cell_hi, kind)
    m = assemble(p.xyz, pts, wj, p.E, p.nu, p.alpha_s, p.alpha_c, p.q, p.h,
                 body=p.body if np.any(p.body) else None, kind=kind)
    if with_loads and p.n_faces:
        traction(p.xyz, p.face_lo, p.face_hi, p.face_axis, p.face_coef, p.alpha_s, p.alpha_c, p.q, p.h,
                 m.f, kind)
    m.pts, m.wj = pts, wj
    return m


def traction(xyz, face_lo, face_hi, face_axis, face_coef, alpha_s, alpha_c, q, h, f, kind="f64"):
    """f += the tractions of the faces (2x2 Gauss-Legendre per face rectangle)."""
    xyz = _c(xyz)
    assert f.dtype == np.float64 and f.flags.c_contiguous
    st = lib(kind).orc_traction(xyz.shape[0], xyz, len(face_lo), _c(face_lo), _c(face_hi),
                                _c(face_axis, np.int8), _c(face_coef), alpha_s, alpha_c, q, h, MAX_SUPPORT, f)
    if st:
        raise OracleError(st, "traction")
    return f


def point_loads(xyz, pts, force, alpha_s, alpha_c, q, h, f, kind="f64"):
    xyz, pts = _c(xyz), _c(pts)
    assert f.dtype == np.float64 and f.flags.c_contiguous
    st = lib(kind).orc_point_loads(xyz.shape[0], xyz, pts.shape[0], pts, _c(force), alpha_s,
                                   alpha_c, q, h, MAX_SUPPORT, f)
    if st:
        raise OracleError(st, "point loads")
    return f


def penalty(n_nodes, rowptr, cols, vals, f, dofs, values, scale=1e8, kind="f64"):
    """Apply the penalty in place on (vals, f); returns alpha."""
    a = C.c_double(0)
    st = lib(kind).orc_penalty(n_nodes, _c(rowptr, np.int64), _c(cols, np.int32), vals, f,
                               len(dofs), _c(dofs, np.int64), _c(values), scale, C.byref(a))
    if st:
        raise OracleError(st, "penalty")
    return a.value


def pcg(n_nodes, rowptr, cols, vals, f, u0=None, rtol=1e-10, max_iter=100000, kind="f64", precond="jacobi"):
    """PCG with the Jacobi or the 3x3 block-Jacobi ("block") preconditioner:
    (u, iterations, relative residual, status)."""
    u = np.zeros(3 * n_nodes) if u0 is None else _c(u0).copy()
    it = C.c_int(0)
    rr = C.c_double(0)
    st = lib(kind).orc_pcg(n_nodes, _c(rowptr, np.int64), _c(cols, np.int32), _c(vals), _c(f), u,
                           rtol, max_iter, C.byref(it), C.byref(rr), {"jacobi": 0, "block": 1}[precond])
    return u, it.value, rr.value, st


def stress(xyz, u, pts, E, nu, alpha_s, alpha_c, q, h, kind="f64"):
    xyz, pts = _c(xyz), _c(pts)
    sig = np.zeros((pts.shape[0], 6))
    st = lib(kind).orc_stress(xyz.shape[0], xyz, _c(u), pts.shape[0], pts, _c(E), _c(nu),
                              alpha_s, alpha_c, q, h, MAX_SUPPORT, sig)
    if st:
        raise OracleError(st, "stress")
    return sig


def grad_material(xyz, pts, wj, E, nu, u, lam, alpha_s, alpha_c, q, h, kind="f64"):
    """Per point (dL/dE, dL/dnu) = -w eps(lam)^T dD/dtheta eps(u)."""
    xyz, pts = _c(xyz), _c(pts)
    dE = np.zeros(pts.shape[0])
    dnu = np.zeros(pts.shape[0])
    st = lib(kind).orc_grad_material(xyz.shape[0], xyz, pts.shape[0], pts, _c(wj), _c(E), _c(nu), _c(u),
                                     _c(lam), alpha_s, alpha_c, q, h, MAX_SUPPORT, dE, dnu)
    if st:
        raise OracleError(st, "grad_material")
    return dE, dnu


def solve_problem(p, kind="f64", rtol=1e-10, scale=1e8, max_iter=200000):
    """Assemble, apply the penalty, solve: returns (model, u, iters, relres, alpha)."""
    m = assemble_problem(p, kind)
    vals = m.vals.ravel().copy()
    f = m.f.copy()
    alpha = penalty(p.n_nodes, m.rowptr, m.cols, vals, f, p.fixed_dofs, p.fixed_vals, scale, kind)
    u, it, rr, st = pcg(p.n_nodes, m.rowptr, m.cols, vals, f, rtol=rtol, max_iter=max_iter, kind=kind)
    if st:
        raise OracleError(st, "pcg (%d iterations, relres %.3e)" % (it, rr))
    return m, u, it, rr, alpha
