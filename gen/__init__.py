"""Seeded synthetic inputs for RPIM stiffness assembly.

This module is shared by the CUDA path, the oracle, the tests and the
benchmark. It describes *problems* (node clouds, the background cell each node
owns, material fields, displacement constraints and applied loads) and holds
none of the RPIM arithmetic: no support search, no shape functions, no
quadrature of the stiffness matrix.

The workloads follow the verification examples of the paper: a cube under
load or gravity (Sec. 3.1), a cantilever beam (Sec. 3.2, without the crack)
and a simplified slope discretised by regular or irregular nodes (Sec. 3.3).
Field nodes sit on a regular lattice; irregular clouds jitter the interior
nodes. Each node owns the lattice cell centred on its nominal (unjittered)
position, clipped to the domain, so the cells tile the domain exactly.

Random numbers come from a counter-based SplitMix64 stream (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), so an
input is a pure function of (seed, stream, index) on every platform.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem", "splitmix64", "uniform", "normal", "lattice_problem", "cube_config",
    "cantilever_config", "gravity_column", "slope_config", "batched_configs",
    "backanalysis_config", "config", "concat_faces",
]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """n outputs of SplitMix64 at counters start..start+n-1 of (seed, stream)."""
    with np.errstate(over="ignore"):
        base = (np.uint64(seed & 0xFFFFFFFF) << np.uint64(32)) ^ np.uint64(stream & 0xFFFFFFFF)
        x = base * _GOLDEN + (np.arange(start, start + n, dtype=np.uint64) + np.uint64(1)) * _GOLDEN
        z = (x ^ (x >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """n doubles uniform in [lo, hi) from the top 53 bits of SplitMix64."""
    u = (splitmix64(seed, stream, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normal deviates by the Box-Muller transform of two streams."""
    u1 = uniform(seed, stream, n)
    u2 = uniform(seed, stream + 0x5151, n)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


@dataclass
class Problem:
    """One linear-elastic RPIM problem on a node cloud.

    Node ``i`` sits at ``xyz[i]`` and owns the box ``[cell_lo[i], cell_hi[i]]``.
    Volume integration points are numbered ``8*i + l`` (``l = a + 2b + 4c`` for the
    2x2x2 rule of cell ``i``); ``E`` and ``nu`` are given per integration point in
    that numbering. ``fixed_dofs`` (DOF ``3*node + axis``) are held at
    ``fixed_vals`` by the penalty method. Surface tractions act on the
    rectangles ``[face_lo[k], face_hi[k]]`` (planar: ``face_lo == face_hi``
    along the normal axis ``face_axis[k]``); component ``c`` of the traction
    on face ``k`` is the polynomial
    ``sum_j face_coef[k, c, j] * m_j(u, v)``, ``m = (1, u, v, u^2, u v, v^2)``,
    in the global coordinates ``u < v`` of the face's two tangent axes (in
    ascending axis order). How a face is integrated is left to the library
    and to the oracle.
    """
    name: str
    xyz: np.ndarray
    cell_lo: np.ndarray
    cell_hi: np.ndarray
    alpha_s: float
    alpha_c: float
    q: float
    h: float
    E: np.ndarray
    nu: np.ndarray
    body: np.ndarray = field(default_factory=lambda: np.zeros(3))
    fixed_dofs: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    fixed_vals: np.ndarray = field(default_factory=lambda: np.zeros(0))
    face_lo: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    face_hi: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    face_axis: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int8))
    face_coef: np.ndarray = field(default_factory=lambda: np.zeros((0, 3, 6)))
    extent: tuple = (1.0, 1.0, 1.0)
    shape: tuple = (0, 0, 0)
    nominal: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_points(self) -> int:
        return 8 * self.n_nodes

    @property
    def n_faces(self) -> int:
        return int(self.face_lo.shape[0])

    @property
    def volume(self) -> float:
        return float(np.prod(self.cell_hi - self.cell_lo, axis=1).sum())


def lattice_problem(name, shape, extent, jitter=0.0, seed=0, keep=None):
    """Nodes on an ``nx x ny x nz`` lattice spanning ``[0, extent]``.

    ``jitter`` is the amplitude, in units of the per-axis spacing, of a uniform
    perturbation applied to every node that lies on no face of the box.
    ``keep`` optionally filters nominal positions (e.g. a slope profile).
    Node numbering is x fastest, then y, then z.
    """
    nx, ny, nz = shape
    Lx, Ly, Lz = extent
    hx, hy, hz = Lx / (nx - 1), Ly / (ny - 1), Lz / (nz - 1)
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ijk = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], 1)
    nom = ijk * np.array([hx, hy, hz])
    # exact face coordinates for boundary lattice planes
    for a, (n, L) in enumerate(zip(shape, extent)):
        nom[ijk[:, a] == n - 1, a] = L
    sel = np.ones(len(nom), bool) if keep is None else keep(nom, ijk)
    ijk, nom = ijk[sel], nom[sel]
    spacing = np.array([hx, hy, hz])
    lo = np.maximum(nom - 0.5 * spacing, 0.0)
    hi = np.minimum(nom + 0.5 * spacing, np.array(extent))
    xyz = nom.copy()
    if jitter > 0.0:
        interior = np.all((ijk > 0) & (ijk < np.array(shape) - 1), axis=1)
        m = len(nom)
        d = np.stack([uniform(seed, 10 + a, m, -jitter, jitter) for a in range(3)], 1) * spacing
        xyz[interior] += d[interior]
    return ijk, nom, xyz, lo, hi, spacing


def _faces(nom, spacing, extent, ijk, shape, axis, side, coef):
    """The face rectangles of the node cells on one box face: the cell of each
    node on the face, clipped to the domain, flattened onto the face plane.
    ``coef`` (3 x 6) is the traction polynomial of every one of them (see
    :class:`Problem`)."""
    n_ax = shape[axis]
    on = ijk[:, axis] == (n_ax - 1 if side else 0)
    c = nom[on]
    lo = np.maximum(c - 0.5 * spacing, 0.0)
    hi = np.minimum(c + 0.5 * spacing, np.array(extent))
    lo[:, axis] = hi[:, axis] = extent[axis] if side else 0.0
    m = len(c)
    return (lo, hi, np.full(m, axis, np.int8),
            np.broadcast_to(np.asarray(coef, np.float64), (m, 3, 6)).copy())


def _pressure(p):
    """Traction polynomial of a uniform pressure p on a top face (inward
    normal: -z)."""
    c = np.zeros((3, 6))
    c[2, 0] = -p
    return c


def _fix_face(ijk, shape, axis, side, comps=(0, 1, 2)):
    n_ax = shape[axis]
    nodes = np.nonzero(ijk[:, axis] == (n_ax - 1 if side else 0))[0]
    return np.sort(np.concatenate([3 * nodes + c for c in comps]).astype(np.int64))


def _material(n_nodes, E, nu):
    return np.full(8 * n_nodes, float(E)), np.full(8 * n_nodes, float(nu))


def cube_config(n=6, seed=0, jitter=0.0, pressure=10.0, E=1.0e4, nu=0.3):
    """Tiny cube: ``n^3`` nodes in the unit cube, base fixed, pressure on top.

    The 6x6x6 default (h = 0.2, 1,728 integration points) is the smallest
    workload; it mirrors the cubic domain of the first verification example
    (Sec. 3.1) with a surface pressure instead of gravity.
    """
    shape = (n, n, n)
    ext = (1.0, 1.0, 1.0)
    ijk, nom, xyz, lo, hi, sp = lattice_problem("cube", shape, ext, jitter, seed)
    Ev, nuv = _material(len(xyz), E, nu)
    fixed = _fix_face(ijk, shape, 2, 0)
    fl, fh, fa, fc = _faces(nom, sp, ext, ijk, shape, 2, 1, _pressure(pressure))
    return Problem("cube%d" % n, xyz, lo, hi, 2.5, 4.0, 1.03, float(sp.max()), Ev, nuv,
                   np.zeros(3), fixed, np.zeros(len(fixed)), fl, fh, fa, fc, ext, shape, nom,
                   {"pressure": pressure, "E": E, "nu": nu})


def cantilever_config(shape=(129, 17, 17), length=8.0, seed=1, jitter=0.2, P=1.0,
                      E=1.0e4, nu=0.3):
    """Cantilever ``length x 1 x 1`` clamped at x = 0, parabolic shear at x = L.

    The shear traction ``t_z = -(3P/2A)(1 - 4(z - 1/2)^2)`` (A = 1) sums to a
    total load P along -z. Interior nodes are jittered by up to
    ``jitter`` times the spacing. Default: 37,281 nodes, h = 1/16.
    """
    ext = (length, 1.0, 1.0)
    ijk, nom, xyz, lo, hi, sp = lattice_problem("cantilever", shape, ext, jitter, seed)
    Ev, nuv = _material(len(xyz), E, nu)
    fixed = _fix_face(ijk, shape, 0, 0)
    # t_z = -(3P/2)(1 - 4(z - 1/2)^2) = -6P z + 6P z^2 on the face x = L,
    # whose tangent coordinates are (u, v) = (y, z)
    shear = np.zeros((3, 6))
    shear[2, 2] = -6.0 * P
    shear[2, 5] = 6.0 * P
    fl, fh, fa, fc = _faces(nom, sp, ext, ijk, shape, 0, 1, shear)
    return Problem("cantilever", xyz, lo, hi, 2.5, 4.0, 1.03, float(sp.max()), Ev, nuv,
                   np.zeros(3), fixed, np.zeros(len(fixed)), fl, fh, fa, fc, ext, shape, nom,
                   {"P": P, "E": E, "nu": nu, "L": length, "D": 1.0})


def gravity_column(shape=(5, 5, 9), height=2.0, width=1.0, gamma=20.0, E=1.0e4, nu=0.3,
                   seed=0, jitter=0.0):
    """Column under self weight: base fixed, lateral faces on rollers.

    The closed-form vertical stress at depth d below the top is -gamma*d
    (the first verification example, Sec. 3.1, compares the bottom stress of a
    cube under gravity with rho*g*H).
    """
    ext = (width, width, height)
    ijk, nom, xyz, lo, hi, sp = lattice_problem("column", shape, ext, jitter, seed)
    Ev, nuv = _material(len(xyz), E, nu)
    fixed = np.concatenate([
        _fix_face(ijk, shape, 2, 0),
        _fix_face(ijk, shape, 0, 0, (0,)), _fix_face(ijk, shape, 0, 1, (0,)),
        _fix_face(ijk, shape, 1, 0, (1,)), _fix_face(ijk, shape, 1, 1, (1,)),
    ])
    fixed = np.unique(fixed)
    return Problem("column", xyz, lo, hi, 2.5, 4.0, 1.03, float(sp.max()), Ev, nuv,
                   np.array([0.0, 0.0, -gamma]), fixed, np.zeros(len(fixed)),
                   extent=ext, shape=shape, nominal=nom,
                   meta={"gamma": gamma, "H": height, "E": E, "nu": nu})


def slope_config(n=100, seed=2, jitter=0.2, gamma=20.0):
    """Layered slope in the unit cube (the simplified slope of Sec. 3.3).

    Nodes whose nominal position satisfies z <= min(1, 1.1 - x) are kept
    (a 45 degree face). Three horizontal layers by the owning node's nominal z
    (thirds, stiffest at depth): E = 8e4/2e4/5e3, nu = 0.25/0.30/0.35. Gravity
    loads the body; the base is fixed and the four lateral box faces are on
    rollers.
    """
    shape = (n, n, n)
    ext = (1.0, 1.0, 1.0)
    keep = lambda nom, ijk: nom[:, 2] <= np.minimum(1.0, 1.1 - nom[:, 0]) + 1e-12
    ijk, nom, xyz, lo, hi, sp = lattice_problem("slope", shape, ext, jitter, seed, keep)
    layer = np.minimum((nom[:, 2] * 3.0).astype(int), 2)
    Etab = np.array([8.0e4, 2.0e4, 5.0e3])
    nutab = np.array([0.25, 0.30, 0.35])
    Ev = np.repeat(Etab[layer], 8)
    nuv = np.repeat(nutab[layer], 8)
    fixed = np.unique(np.concatenate([
        _fix_face(ijk, shape, 2, 0),
        _fix_face(ijk, shape, 0, 0, (0,)), _fix_face(ijk, shape, 0, 1, (0,)),
        _fix_face(ijk, shape, 1, 0, (1,)), _fix_face(ijk, shape, 1, 1, (1,)),
    ]))
    return Problem("slope", xyz, lo, hi, 3.0, 4.0, 1.03, float(sp.max()), Ev, nuv,
                   np.array([0.0, 0.0, -gamma]), fixed, np.zeros(len(fixed)),
                   extent=ext, shape=shape, nominal=nom, meta={"gamma": gamma})


def batched_configs(count=512, seed=3, lo_nodes=500, hi_nodes=20000):
    """Independent rectangular blocks of uneven size and support.

    Node count log-uniform in [lo_nodes, hi_nodes], aspect a ~ U[1, 4] for an
    ``a x 1 x 1`` block, alpha_s ~ U[2.0, 3.5], E log-uniform in [1e3, 1e5],
    nu ~ U[0.2, 0.4], base fixed, top pressure ~ U[1, 100].
    """
    tgt = np.exp(uniform(seed, 1, count, np.log(lo_nodes), np.log(hi_nodes)))
    asp = uniform(seed, 2, count, 1.0, 4.0)
    als = uniform(seed, 3, count, 2.0, 3.5)
    Es = np.exp(uniform(seed, 4, count, np.log(1.0e3), np.log(1.0e5)))
    nus = uniform(seed, 5, count, 0.2, 0.4)
    prs = uniform(seed, 6, count, 1.0, 100.0)
    out = []
    for k in range(count):
        ny = max(4, int(round((tgt[k] / asp[k]) ** (1.0 / 3.0))))
        nx = int(round(asp[k] * (ny - 1))) + 1
        shape = (nx, ny, ny)
        ext = ((nx - 1) / (ny - 1), 1.0, 1.0)
        ijk, nom, xyz, lo, hi, sp = lattice_problem("block", shape, ext, 0.2, seed * 100003 + k)
        Ev, nuv = _material(len(xyz), Es[k], nus[k])
        fixed = _fix_face(ijk, shape, 2, 0)
        p = prs[k]
        fl, fh, fa, fc = _faces(nom, sp, ext, ijk, shape, 2, 1, _pressure(p))
        out.append(Problem("block%d" % k, xyz, lo, hi, float(als[k]), 4.0, 1.03, float(sp.max()),
                           Ev, nuv, np.zeros(3), fixed, np.zeros(len(fixed)), fl, fh, fa, fc, ext, shape,
                           nom, {"E": Es[k], "nu": nus[k], "pressure": p}))
    return out


def _ar1_field(seed, stream, dims, steps, ell):
    """Zero-mean unit-variance Gaussian field with separable exponential
    correlation exp(-|dx|/l - |dy|/l - |dz|/l) on a tensor lattice, generated
    exactly by first-order autoregressive filtering along each axis
    (``steps[a]`` holds the gaps between successive lattice coordinates)."""
    f = normal(seed, stream, int(np.prod(dims))).reshape(dims[2], dims[1], dims[0])
    for a, ax in ((0, 2), (1, 1), (2, 0)):
        rho = np.exp(-np.asarray(steps[a]) / ell)
        f = np.moveaxis(f, ax, 0).copy()
        for i in range(1, f.shape[0]):
            r = rho[i - 1]
            f[i] = r * f[i - 1] + np.sqrt(1.0 - r * r) * f[i]
        f = np.moveaxis(f, 0, ax)
    return f


def backanalysis_config(shape=(64, 32, 32), seed=4, hidden_seed=1004, n_obs=500):
    """Block 2 x 1 x 1 with a log-normal Young's modulus field per
    integration point (median 2e4, sigma 0.5, correlation length 0.2) and
    nu = 0.3 + 0.05 N(0,1) clipped to [0.2, 0.45]; base fixed, pressure 10 on
    top. ``meta`` carries the hidden field used to make observations at
    ``n_obs`` random nodes."""
    ext = (2.0, 1.0, 1.0)
    ijk, nom, xyz, lo, hi, sp = lattice_problem("backanalysis", shape, ext, 0.2, seed)
    nx, ny, nz = shape

    def fields(sd):
        # integration-point lattice: 2 points per node cell per axis
        steps = []
        for a, n in enumerate(shape):
            coords = []
            for i in range(n):
                c = i * sp[a]
                clo, chi = max(c - 0.5 * sp[a], 0.0), min(c + 0.5 * sp[a], ext[a])
                m, hw = 0.5 * (clo + chi), 0.5 * (chi - clo)
                coords += [m - hw / np.sqrt(3.0), m + hw / np.sqrt(3.0)]
            steps.append(np.diff(np.array(coords)))
        g = _ar1_field(sd, 40, (2 * nx, 2 * ny, 2 * nz), steps, 0.2)  # [z][y][x]
        E = 2.0e4 * np.exp(0.5 * g)
        nu = np.clip(0.3 + 0.05 * normal(sd, 41, g.size).reshape(g.shape), 0.2, 0.45)
        # reorder lattice (2ix+a, 2iy+b, 2iz+c) -> point 8*node + a + 2b + 4c
        Ep = E.reshape(nz, 2, ny, 2, nx, 2).transpose(0, 2, 4, 5, 3, 1).reshape(-1, 8)
        nup = nu.reshape(nz, 2, ny, 2, nx, 2).transpose(0, 2, 4, 5, 3, 1).reshape(-1, 8)
        return Ep.ravel().copy(), nup.ravel().copy()

    Ev, nuv = fields(seed)
    Eh, nuh = fields(hidden_seed)
    fixed = _fix_face(ijk, shape, 2, 0)
    fl, fh, fa, fc = _faces(nom, sp, ext, ijk, shape, 2, 1, _pressure(10.0))
    obs = np.sort((splitmix64(seed, 42, n_obs) % np.uint64(len(xyz))).astype(np.int64))
    obs = np.unique(obs)
    return Problem("backanalysis", xyz, lo, hi, 2.5, 4.0, 1.03, float(sp.max()), Ev, nuv,
                   np.zeros(3), fixed, np.zeros(len(fixed)), fl, fh, fa, fc, ext, shape, nom,
                   {"E_hidden": Eh, "nu_hidden": nuh, "obs_nodes": obs})


def config(i: int, **kw):
    """Workload ``i`` of the five reference workloads (0 tiny cube, 1 cantilever,
    2 layered slope, 3 batched blocks, 4 back-analysis block)."""
    return [cube_config, cantilever_config, slope_config, batched_configs,
            backanalysis_config][i](**kw)


def concat_faces(problems):
    """Faces of several problems concatenated (lo, hi, axis, coef, instance
    of every face), for a batched pattern of those problems in that order."""
    cat = lambda name: np.concatenate([getattr(p, name) for p in problems])
    inst = np.concatenate([np.full(p.n_faces, k, np.int32) for k, p in enumerate(problems)])
    return cat("face_lo"), cat("face_hi"), cat("face_axis").astype(np.int8), cat("face_coef"), inst
