"""Pins of the RPIM oracle against facts fixed by the mathematics.

Each test checks the oracle (``oracle/oracle.c``) against something other than
itself: closed forms (quadrature of cubics, Timoshenko's cantilever deflection,
the weight carried by a column), identities that exact RPIM shape functions
satisfy (partition of unity, linear reproduction, the Kronecker property,
reproduction of any constrained RBF combination), special cases that reduce to
textbook formulas (barycentric interpolation from four nodes), brute force,
and an extended-precision rerun. A plausible slip anywhere in the oracle (a
dropped term, a wrong sign, index or factor, a transposed operand) breaks at
least one of them; ``test_oracle_mutations.py`` plants such slips to show it.
"""
import mpmath as mp
import numpy as np
import pytest

import gen
import oracle

KINDS = ["f64", "ld"]


def _extended(kind):
    """Whether build `kind` computes in extended precision: the "ld" build
    only (every other build, the planted-mistake copies included, is FP64
    and is held to the FP64 tolerances)."""
    return kind == "ld"


@pytest.fixture(scope="module")
def cube_j():
    return gen.cube_config(jitter=0.2, seed=7)


def _points(p):
    return oracle.gauss_points(p.cell_lo, p.cell_hi)


# ---------------------------------------------------------------- quadrature
def test_gauss_rule_integrates_cubics_exactly(cube_j):
    """2x2x2 Gauss-Legendre on the node cells integrates any polynomial of
    degree <= 3 per axis exactly over the domain (cells tile the box)."""
    pts, wj = _points(cube_j)
    x, y, z = pts.T
    f = x**3 + 2 * x**2 * y - y * z**3 + x * y * z + 5.0
    exact = 1 / 4 + 2 * (1 / 3) * (1 / 2) - (1 / 2) * (1 / 4) + 1 / 8 + 5.0
    assert abs(np.dot(wj, f) - exact) < 1e-14
    assert abs(wj.sum() - 1.0) < 1e-15


def test_gauss_points_of_rectangular_cells():
    p = gen.cantilever_config(shape=(9, 3, 3), length=2.0, jitter=0.0)
    pts, wj = _points(p)
    assert abs(wj.sum() - 2.0) < 1e-14
    # every point lies inside its own cell
    c = np.repeat(np.arange(p.n_nodes), 8)
    assert np.all(pts >= p.cell_lo[c]) and np.all(pts <= p.cell_hi[c])


# ---------------------------------------------------------------- support
def test_support_matches_brute_force(cube_j):
    p = cube_j
    pts, _ = _points(p)
    rs2 = oracle.support_radius2(p.alpha_s, p.h)
    assert rs2 == pytest.approx((2.5 * 0.2) ** 2, rel=1e-15)
    for g in range(0, len(pts), 37):
        s = oracle.support(p.xyz, pts[g], rs2)
        d2 = ((p.xyz - pts[g]) ** 2).sum(1)
        sure_in = set(np.nonzero(d2 < rs2 * (1 - 1e-12))[0])
        maybe = set(np.nonzero(d2 <= rs2 * (1 + 1e-12))[0])
        assert sure_in <= set(s) <= maybe
        assert np.all(np.diff(s) > 0)


# ---------------------------------------------------------------- shape functions
def _some_points(p, stride=61):
    pts, _ = _points(p)
    return pts[::stride]


@pytest.mark.parametrize("kind", KINDS)
def test_partition_of_unity_and_linear_reproduction(cube_j, kind):
    p = cube_j
    rs2 = oracle.support_radius2(p.alpha_s, p.h)
    for x in _some_points(p):
        s = oracle.support(p.xyz, x, rs2)
        ph = oracle.shape(p.xyz, s, x, p.h, kind=kind)
        X = p.xyz[s]
        assert abs(ph[0].sum() - 1.0) < 1e-10
        assert np.abs(ph[0] @ X - x).max() < 1e-10
        for k in range(3):
            assert abs(ph[1 + k].sum()) < 1e-10 / p.h
            assert np.abs(ph[1 + k] @ X - np.eye(3)[k]).max() < 1e-10


@pytest.mark.parametrize("kind", KINDS)
def test_kronecker_delta_at_nodes(cube_j, kind):
    p = cube_j
    rs2 = oracle.support_radius2(p.alpha_s, p.h)
    for j in np.linspace(0, p.n_nodes - 1, 7).astype(int):
        x = p.xyz[j]
        s = oracle.support(p.xyz, x, rs2)
        ph = oracle.shape(p.xyz, s, x, p.h, kind=kind)
        e = (s == j).astype(float)
        assert np.abs(ph[0] - e).max() < (1e-13 if _extended(kind) else 1e-10)


def _mq(r2, c2, q):
    return (r2 + c2) ** q


@pytest.mark.parametrize("kind", KINDS)
def test_reproduces_constrained_rbf_combinations(cube_j, kind):
    """Any f(y) = sum_j c_j R(|y - x_j|/h) with sum_j c_j p(x_j) = 0 lies in
    the RPIM interpolation space, so sum_i phi_i(x) f(x_i) = f(x) and the same
    for the gradient. f and grad f are evaluated independently in 40-digit
    arithmetic (gradient by numerical differentiation)."""
    p = cube_j
    mp.mp.dps = 40
    rs2 = oracle.support_radius2(p.alpha_s, p.h)
    rng = np.random.default_rng(3)
    tol = 1e-10 if _extended(kind) else 2e-7
    for x in _some_points(p, 211):
        s = oracle.support(p.xyz, x, rs2)
        X = p.xyz[s]
        P = np.concatenate([np.ones((len(s), 1)), X], 1)
        c = rng.standard_normal(len(s))
        c -= P @ np.linalg.lstsq(P, c, rcond=None)[0]
        cm = [mp.mpf(float(v)) for v in c]
        Xm = [[mp.mpf(float(v)) for v in row] for row in X]
        hm, c2, qm = mp.mpf(p.h), mp.mpf(p.alpha_c) ** 2, mp.mpf(p.q)

        def f(y):
            return sum(cj * _mq(sum((y[k] - xj[k]) ** 2 for k in range(3)) / hm**2, c2, qm)
                       for cj, xj in zip(cm, Xm))

        fx = [float(f(row)) for row in Xm]
        xm = [mp.mpf(float(v)) for v in x]
        ph = oracle.shape(p.xyz, s, x, p.h, kind=kind)
        scale = sum(abs(v) for v in fx) / len(fx)
        assert abs(ph[0] @ fx - float(f(xm))) < tol * scale * 10
        for k in range(3):
            g = mp.diff(lambda t: f([xm[a] + (t if a == k else 0) for a in range(3)]), 0)
            assert abs(ph[1 + k] @ fx - float(g)) < tol * scale * 10 / p.h


@pytest.mark.parametrize("kind", KINDS)
def test_gradients_match_central_differences(cube_j, kind):
    p = cube_j
    rs2 = oracle.support_radius2(p.alpha_s, p.h)
    d = 1e-5 * p.h
    for x in _some_points(p, 173):
        s = oracle.support(p.xyz, x, rs2)
        ph = oracle.shape(p.xyz, s, x, p.h, kind=kind)
        for k in range(3):
            e = np.eye(3)[k] * d
            fd = (oracle.shape(p.xyz, s, x + e, p.h, kind=kind)[0] -
                  oracle.shape(p.xyz, s, x - e, p.h, kind=kind)[0]) / (2 * d)
            tol = 1e-6 if _extended(kind) else 1e-3
            assert np.abs(fd - ph[1 + k]).max() < tol / p.h


@pytest.mark.parametrize("kind", KINDS)
def test_four_nodes_reduce_to_barycentric_interpolation(kind):
    """With n = m = 4 the polynomial constraints fix phi completely: the shape
    functions are the barycentric coordinates of x in the tetrahedron and the
    gradients are constant, whatever the radial basis."""
    xyz = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.2, 0.9, 0.1], [0.1, 0.2, 1.1]])
    x = np.array([0.3, 0.25, 0.2])
    s = np.arange(4, dtype=np.int32)
    ph = oracle.shape(xyz, s, x, 0.5, kind=kind)
    A = np.vstack([np.ones(4), xyz.T])
    lam = np.linalg.solve(A, np.concatenate([[1.0], x]))
    grads = np.linalg.inv(A)[:, 1:]
    assert np.abs(ph[0] - lam).max() < 1e-12
    assert np.abs(ph[1:].T - grads).max() < 1e-11


def test_fp64_floor_against_extended_precision(cube_j):
    """The plain FP64 solve of the MQ moment matrix (alpha_c = 4, q = 1.03)
    loses about log10(cond G) ~ 9-10 digits: it agrees with the
    extended-precision oracle only to a few 1e-9 (h units)."""
    p = cube_j
    rs2 = oracle.support_radius2(p.alpha_s, p.h)
    worst = 0.0
    for x in _some_points(p, 97):
        s = oracle.support(p.xyz, x, rs2)
        a = oracle.shape(p.xyz, s, x, p.h, kind="f64")
        b = oracle.shape(p.xyz, s, x, p.h, kind="ld")
        worst = max(worst, np.abs(a - b).max() * p.h)
    assert worst < 5e-8


# ---------------------------------------------------------------- stiffness
@pytest.fixture(scope="module", params=KINDS)
def cube_model(request, cube_j):
    return oracle.assemble_problem(cube_j, request.param)


def _strain_fields(xyz):
    """Six displacement fields with unit engineering strain in Voigt order."""
    out = []
    for k in range(6):
        A = np.zeros((3, 3))
        if k < 3:
            A[k, k] = 1.0
        else:
            a, b = [(1, 2), (0, 2), (0, 1)][k - 3]
            A[a, b] = A[b, a] = 0.5
        out.append(((xyz @ A.T).ravel(), A))
    return out


def test_K_symmetric(cube_model):
    K = cube_model.dense()
    assert np.abs(K - K.T).max() <= 1e-14 * np.abs(K).max()


def test_K_rigid_body_modes(cube_model, cube_j):
    K = cube_model.dense()
    X = cube_j.xyz
    modes = [np.tile(np.eye(3)[k], len(X)) for k in range(3)]
    for k in range(3):
        w = np.eye(3)[k]
        modes.append(np.cross(w, X).ravel())
    kf = np.linalg.norm(K)
    for u in modes:
        assert np.linalg.norm(K @ u) / (kf * np.linalg.norm(u)) < 1e-10


def test_K_energy_of_linear_fields(cube_model, cube_j):
    """For u = A x, B u is the constant strain of A at every point, so
    u_a^T K u_b = V (lambda tr e_a tr e_b + 2 mu e_a : e_b): pins D, B and the
    quadrature weights through Hooke's law in tensor form."""
    K = cube_model.dense()
    E, nu = 1.0e4, 0.3
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    fields = _strain_fields(cube_j.xyz)
    V = cube_j.volume
    for ua, Aa in fields:
        for ub, Ab in fields:
            want = V * (lam * np.trace(Aa) * np.trace(Ab) + 2 * mu * np.sum(Aa * Ab))
            assert abs(ua @ K @ ub - want) < 1e-9 * (lam + 2 * mu) * V


@pytest.mark.parametrize("kind", KINDS)
def test_stress_of_linear_fields_is_hookes_law(cube_j, kind):
    """RPIM reproduces linear fields, so for u = A x the strain at every point
    is the constant strain eps = (A + A^T)/2 and the stress is Hooke's law in
    tensor form, sigma = lambda tr(eps) I + 2 mu eps, exactly (up to the
    rounding of the reproduction). Checked for all six Voigt components
    (xx, yy, zz, yz, xz, xy) of the six unit strains and of a rigid rotation
    (zero stress), with E and nu drawn per point so that a stress computed
    with another point's material, a swapped Voigt slot or a dropped shear
    term fails."""
    p = cube_j
    pts = _points(p)[0][::29]
    E = gen.uniform(7, 60, len(pts), 5e3, 2e4)
    nu = gen.uniform(7, 61, len(pts), 0.2, 0.4)
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    W = np.array([[0.0, -0.3, 0.2], [0.3, 0.0, -0.7], [-0.2, 0.7, 0.0]])
    cases = [A for _, A in _strain_fields(p.xyz)] + [W]
    voigt = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    for A in cases:
        u = (p.xyz @ A.T).ravel()
        sig = oracle.stress(p.xyz, u, pts, E, nu, p.alpha_s, p.alpha_c, p.q, p.h, kind)
        eps = 0.5 * (A + A.T)
        want = np.zeros((len(pts), 6))
        for c, (i, j) in enumerate(voigt):
            want[:, c] = lam * np.trace(eps) * (i == j) + 2 * mu * eps[i, j]
        assert np.abs(sig - want).max() <= 1e-12 * (lam + 2 * mu).max()


def test_K_positive_diagonal(cube_model):
    K = cube_model.dense()
    assert np.all(np.diag(K) > 0)


def test_K_ld_matches_f64_to_fp64_floor(cube_j):
    a = oracle.assemble_problem(cube_j, "f64")
    b = oracle.assemble_problem(cube_j, "ld")
    assert np.array_equal(a.rowptr, b.rowptr) and np.array_equal(a.cols, b.cols)
    assert np.abs(a.vals - b.vals).max() / np.abs(b.vals).max() < 2e-8


def test_body_force_moments():
    """f_I = sum_g phi_I b w: sum_I f_I = b V (partition of unity) and
    sum_I f_I x_I = b (first moment of the domain)."""
    p = gen.gravity_column(shape=(4, 4, 6), height=1.0, width=0.6, gamma=3.0)
    m = oracle.assemble_problem(p)
    F = m.f.reshape(-1, 3)
    V = p.volume
    assert np.abs(F.sum(0) - p.body * V).max() < 1e-12 * 3.0 * V
    mom = F[:, 2] @ p.xyz
    centroid = np.array([0.3, 0.3, 0.5])
    assert np.abs(mom - (-3.0) * V * centroid).max() < 1e-10


def test_point_loads_force_and_moment(cube_j):
    """f_I = sum_p phi_I(x_p) F_p: the nodal forces carry the applied
    resultant (partition of unity) and moment (linear reproduction)."""
    p = cube_j
    rng = np.random.default_rng(5)
    x = rng.uniform(0.05, 0.95, size=(30, 3))
    F = rng.standard_normal((30, 3))
    f = np.zeros(3 * p.n_nodes)
    oracle.point_loads(p.xyz, x, F, p.alpha_s, p.alpha_c, p.q, p.h, f)
    Fn = f.reshape(-1, 3)
    assert np.abs(Fn.sum(0) - F.sum(0)).max() < 1e-10
    assert np.abs(np.cross(p.xyz, Fn).sum(0) - np.cross(x, F).sum(0)).max() < 1e-10


def _traction_faces():
    """Faces normal to each axis, on the boundary of the unit cube, with
    seeded quadratic traction polynomials (every coefficient set)."""
    lo, hi, ax = [], [], []
    for a, side in ((0, 1.0), (1, 0.0), (2, 1.0), (0, 0.0)):
        for r in ((0.0, 0.6, 0.2, 0.9), (0.4, 1.0, 0.0, 0.5)):
            l, h = np.zeros(3), np.zeros(3)
            l[a] = h[a] = side
            u, v = [b for b in range(3) if b != a]
            l[u], h[u], l[v], h[v] = r
            lo.append(l)
            hi.append(h)
            ax.append(a)
    coef = gen.uniform(3, 77, 8 * 18, -4.0, 4.0).reshape(8, 3, 6)
    return np.array(lo), np.array(hi), np.array(ax, np.int8), coef


def _exact_face_loads(lo, hi, ax, coef):
    """Resultant and moment about the origin of polynomial tractions over
    face rectangles, from the closed-form integrals of monomials."""
    R = np.zeros(3)
    M = np.zeros(3)
    for l, h, a, c in zip(lo, hi, ax, coef):
        u, v = [b for b in range(3) if b != a]
        I = lambda k, b: (h[b] ** (k + 1) - l[b] ** (k + 1)) / (k + 1)

        def integral(du, dv):   # of u^du v^dv times each traction monomial
            e = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]
            return np.array([I(du + i, u) * I(dv + j, v) for i, j in e])

        R += c @ integral(0, 0)
        # x = (plane, u, v) components; moment = integral of x cross t
        xint = {a: l[a] * integral(0, 0), u: integral(1, 0), v: integral(0, 1)}
        for i in range(3):
            j, k = (i + 1) % 3, (i + 2) % 3
            M[i] += c[k] @ xint[j] - c[j] @ xint[k]
    return R, M


@pytest.mark.parametrize("kind", KINDS)
def test_traction_resultant_and_moment_are_the_exact_integrals(cube_j, kind):
    """The 2x2 Gauss rule integrates the (quadratic) traction times 1 and
    times a coordinate exactly, and RPIM reproduces constants and linear
    fields, so the nodal forces carry exactly the resultant and the moment of
    the traction over the faces: pins the face points, weights, the tangent
    axes and the polynomial of the oracle's face quadrature."""
    p = cube_j
    lo, hi, ax, coef = _traction_faces()
    f = np.zeros(3 * p.n_nodes)
    oracle.traction(p.xyz, lo, hi, ax, coef, p.alpha_s, p.alpha_c, p.q, p.h, f, kind)
    Fn = f.reshape(-1, 3)
    R, M = _exact_face_loads(lo, hi, ax, coef)
    assert np.abs(Fn.sum(0) - R).max() < 1e-10 * np.abs(R).max()
    assert np.abs(np.cross(p.xyz, Fn).sum(0) - M).max() < 1e-10 * np.abs(M).max()


def test_cantilever_shear_sums_to_the_tip_load():
    """The problem's parabolic end shear integrates to -P along z."""
    p = gen.cantilever_config(shape=(17, 5, 5))
    f = np.zeros(3 * p.n_nodes)
    oracle.traction(p.xyz, p.face_lo, p.face_hi, p.face_axis, p.face_coef, p.alpha_s, p.alpha_c, p.q, p.h, f)
    assert np.abs(f.reshape(-1, 3).sum(0) - [0.0, 0.0, -1.0]).max() < 1e-12


# ---------------------------------------------------------------- penalty and solve
def test_penalty_adds_alpha_on_listed_dofs(cube_j):
    m = oracle.assemble_problem(cube_j)
    vals = m.vals.ravel().copy()
    f = m.f.copy()
    dofs = np.array([2, 5, 300], np.int64)
    vv = np.array([0.0, 0.5, -1.0])
    diag0 = np.diag(m.dense()).copy()
    a = oracle.penalty(cube_j.n_nodes, m.rowptr, m.cols, vals, f, dofs, vv, 1e8)
    assert a == 1e8 * diag0.max()
    m2 = oracle.Model(m.n_nodes, m.rowptr, m.cols, vals.reshape(-1, 9), f, None, None)
    d = np.diag(m2.dense()) - diag0
    want = np.zeros_like(d)
    want[dofs] = a
    assert np.array_equal(d, want)
    assert np.array_equal(f - m.f, np.where(np.isin(np.arange(len(f)), dofs), 0, 0) +
                          np.bincount(dofs, a * vv, len(f)))


def test_pcg_matches_dense_solve(cube_j):
    m = oracle.assemble_problem(cube_j)
    vals = m.vals.ravel().copy()
    f = m.f.copy()
    oracle.penalty(cube_j.n_nodes, m.rowptr, m.cols, vals, f, cube_j.fixed_dofs,
                   cube_j.fixed_vals, 1e8)
    u, it, rr, st = oracle.pcg(cube_j.n_nodes, m.rowptr, m.cols, vals, f, rtol=1e-13)
    assert st == 0 and rr <= 1e-13
    K = oracle.Model(m.n_nodes, m.rowptr, m.cols, vals.reshape(-1, 9), f, None, None).dense()
    ud = np.linalg.solve(K, f)
    assert np.linalg.norm(u - ud) / np.linalg.norm(ud) < 1e-8


@pytest.mark.parametrize("kind", KINDS)
def test_block_jacobi_pcg_is_exact_on_a_block_diagonal_matrix(cube_j, kind):
    """With K reduced to its 3x3 diagonal blocks, the block-Jacobi
    preconditioner is K^-1 itself: PCG converges in one iteration, to the
    block-by-block solution (while scalar Jacobi needs more)."""
    m = oracle.assemble_problem(cube_j)
    vals = m.vals.ravel().copy()
    f = m.f.copy()
    oracle.penalty(cube_j.n_nodes, m.rowptr, m.cols, vals, f, cube_j.fixed_dofs, cube_j.fixed_vals, 1e8)
    rows = np.repeat(np.arange(cube_j.n_nodes), np.diff(m.rowptr))
    diag = np.nonzero(m.cols == rows)[0]
    rowptr = np.arange(cube_j.n_nodes + 1, dtype=np.int64)
    cols = np.arange(cube_j.n_nodes, dtype=np.int32)
    bd = vals.reshape(-1, 9)[diag].ravel().copy()
    u, it, rr, st = oracle.pcg(cube_j.n_nodes, rowptr, cols, bd, f, rtol=1e-12, kind=kind, precond="block")
    assert st == 0 and it == 1
    want = np.concatenate([np.linalg.solve(b.reshape(3, 3), f[3 * I:3 * I + 3]) for I, b in enumerate(bd.reshape(-1, 9))])
    assert np.linalg.norm(u - want) <= 1e-12 * np.linalg.norm(want)
    u2, it2, rr2, st2 = oracle.pcg(cube_j.n_nodes, rowptr, cols, bd, f, rtol=1e-12, kind=kind)
    assert st2 == 0 and it2 > 1


def test_block_jacobi_pcg_matches_dense_solve(cube_j):
    m = oracle.assemble_problem(cube_j)
    vals = m.vals.ravel().copy()
    f = m.f.copy()
    oracle.penalty(cube_j.n_nodes, m.rowptr, m.cols, vals, f, cube_j.fixed_dofs, cube_j.fixed_vals, 1e8)
    u, it, rr, st = oracle.pcg(cube_j.n_nodes, m.rowptr, m.cols, vals, f, rtol=1e-13, precond="block")
    assert st == 0 and rr <= 1e-13
    K = oracle.Model(m.n_nodes, m.rowptr, m.cols, vals.reshape(-1, 9), f, None, None).dense()
    ud = np.linalg.solve(K, f)
    assert np.linalg.norm(u - ud) / np.linalg.norm(ud) < 1e-8


def test_cantilever_tip_deflection_timoshenko():
    """Tip deflection of the end-loaded cantilever against Timoshenko's
    closed form PL^3/(3EI) + (4 + 5 nu) P D^2 L / (24 E I) = 0.2070 for
    L = 8, D = 1, E = 1e4, nu = 0.3, P = 1 (coarse 33x5x5 cloud)."""
    oracle.set_threads(4)
    p = gen.cantilever_config(shape=(33, 5, 5))
    m, u, it, rr, a = oracle.solve_problem(p)
    I = 1.0 / 12.0
    ref = 1.0 * 8**3 / (3 * 1e4 * I) + (4 + 5 * 0.3) * 1.0 * 1.0 * 8 / (24 * 1e4 * I)
    tip = np.nonzero(np.all(np.abs(p.nominal - [8.0, 0.5, 0.5]) < 1e-9, axis=1))[0][0]
    assert abs(-u[3 * tip + 2] - ref) / ref < 0.02


def test_gravity_column_reaction_and_stress():
    """Column under self weight, base fixed, sides on rollers: the penalty
    reactions at the base carry exactly the weight gamma V, and the
    volume-average vertical stress is -gamma H / 2 (uniaxial strain)."""
    oracle.set_threads(4)
    gam, H = 20.0, 2.0
    p = gen.gravity_column(shape=(5, 5, 9), height=H, width=1.0, gamma=gam)
    m, u, it, rr, a = oracle.solve_problem(p, rtol=1e-12)
    base = p.fixed_dofs[(p.fixed_dofs % 3 == 2)]
    reaction = -a * u[base].sum()
    assert abs(reaction - gam * p.volume) < 1e-6 * gam * p.volume
    sig = oracle.stress(p.xyz, u, m.pts, p.E, p.nu, p.alpha_s, p.alpha_c, p.q, p.h)
    avg = np.dot(m.wj, sig[:, 2]) / m.wj.sum()
    assert abs(avg - (-gam * H / 2)) < 0.03 * gam * H / 2


def check_cube_symmetries(kind="f64", n=5):
    """The cube of the smallest workload without jitter (base fixed, uniform
    pressure on top, Sec. 3) is invariant under the reflections x -> 1 - x,
    y -> 1 - y and the exchange of x and y, and so is its exact discrete
    solution: u_x is odd and u_y, u_z even under the first reflection, the
    same with x and y exchanged under the second, and the exchange swaps u_x
    and u_y. Nothing in the oracle knows these symmetries, so a slip that
    treats one axis differently (a derivative index, a Gauss point, a
    traction axis) breaks them. The support radius is 2.4 h here: at 2.5 h
    some lattice nodes lie exactly on the radius of a Gauss point (squared
    offsets summing to 6 h^2 with cancelling sign terms), and the inclusive
    FP64 test then decides their membership by rounding, which the
    reflections do not preserve (the exchange does: it only reorders the
    sum's operands)."""
    p = gen.cube_config(n=n, jitter=0.0)
    p.alpha_s = 2.4
    m, u, it, rr, a = oracle.solve_problem(p, kind, rtol=1e-13)
    U = u.reshape(n, n, n, 3)   # [z][y][x][component]: node x + n (y + n z)
    scale = np.abs(U).max()
    rx = U[:, :, ::-1, :] * np.array([-1.0, 1.0, 1.0])
    ry = U[:, ::-1, :, :] * np.array([1.0, -1.0, 1.0])
    sw = U.transpose(0, 2, 1, 3)[..., [1, 0, 2]]
    for name, other in (("x -> 1 - x", rx), ("y -> 1 - y", ry), ("x <-> y", sw)):
        err = np.abs(U - other).max() / scale
        assert err < 1e-8, "%s: %.3e" % (name, err)


@pytest.mark.parametrize("kind", KINDS)
def test_cube_solution_has_the_symmetries_of_the_problem(kind):
    """Measured: 1e-10 of max|u| (f64), 1e-13 (extended)."""
    check_cube_symmetries(kind)


# ---------------------------------------------------------------- material gradient
def test_grad_material_is_the_derivative_of_the_point_stiffness():
    """dL/dtheta_g = -lam^T (dK_g/dtheta) u: compare with central differences
    of lam^T K_g(theta) u, K_g the contribution of point g alone (K_g is
    linear in E, so that difference is exact up to rounding)."""
    check_grad_material("f64")


def check_grad_material(kind):
    p = gen.cube_config(n=5, jitter=0.2, seed=13)
    pts, wj = oracle.gauss_points(p.cell_lo, p.cell_hi)
    rng = np.random.default_rng(4)
    u = rng.standard_normal(3 * p.n_nodes)
    lam = rng.standard_normal(3 * p.n_nodes)
    E = gen.uniform(13, 1, p.n_points, 5e3, 2e4)
    nu = gen.uniform(13, 2, p.n_points, 0.2, 0.4)
    dE, dnu = oracle.grad_material(p.xyz, pts, wj, E, nu, u, lam, p.alpha_s, p.alpha_c, p.q, p.h, kind)

    def form(g, Eg, nug):
        m = oracle.assemble(p.xyz, pts[[g]], wj[[g]], [Eg], [nug], p.alpha_s, p.alpha_c, p.q, p.h, kind="f64")
        return lam @ m.matvec(u)

    for g in (0, 311, 777):
        dEf = (form(g, E[g] * (1 + 1e-4), nu[g]) - form(g, E[g] * (1 - 1e-4), nu[g])) / (2e-4 * E[g])
        dnf = (form(g, E[g], nu[g] + 1e-5) - form(g, E[g], nu[g] - 1e-5)) / 2e-5
        assert abs(dE[g] + dEf) <= 1e-9 * abs(dEf) + 1e-15
        assert abs(dnu[g] + dnf) <= 1e-7 * abs(dnf) + 1e-12


def _dense_solve(p, pts, wj, E, nu, f_ext, alpha):
    m = oracle.assemble(p.xyz, pts, wj, E, nu, p.alpha_s, p.alpha_c, p.q, p.h)
    vals = m.vals.ravel().copy()
    f = m.f + f_ext
    oracle.penalty(p.n_nodes, m.rowptr, m.cols, vals, f, p.fixed_dofs, p.fixed_vals, -alpha)
    K = oracle.Model(m.n_nodes, m.rowptr, m.cols, vals.reshape(-1, 9), f, None, None).dense()
    return K, np.linalg.solve(K, f)


def test_adjoint_gradient_matches_finite_differences_of_the_loss():
    """L = 1/2 |u(theta) - u_obs|^2 with a frozen penalty: the adjoint
    gradient (K lam = u - u_obs, then grad_material) agrees with central
    differences of L (dense solves) for single parameters and along a random
    direction of all parameters."""
    p = gen.cube_config(n=5, jitter=0.2, seed=17)
    pts, wj = oracle.gauss_points(p.cell_lo, p.cell_hi)
    E = gen.uniform(17, 1, p.n_points, 5e3, 2e4)
    nu = gen.uniform(17, 2, p.n_points, 0.2, 0.4)
    f_ext = np.zeros(3 * p.n_nodes)
    oracle.traction(p.xyz, p.face_lo, p.face_hi, p.face_axis, p.face_coef, p.alpha_s, p.alpha_c, p.q, p.h, f_ext)
    alpha = 1e8 * 4e3
    K, u = _dense_solve(p, pts, wj, E, nu, f_ext, alpha)
    u_obs = u * (1 + 0.1 * np.sin(np.arange(len(u))))
    lam = np.linalg.solve(K, u - u_obs)
    dE, dnu = oracle.grad_material(p.xyz, pts, wj, E, nu, u, lam, p.alpha_s, p.alpha_c, p.q, p.h)

    def loss(E_, nu_):
        return 0.5 * np.sum((_dense_solve(p, pts, wj, E_, nu_, f_ext, alpha)[1] - u_obs) ** 2)

    for g in (5, 400):
        h = 1e-3 * E[g]
        Ep, Em = E.copy(), E.copy()
        Ep[g] += h
        Em[g] -= h
        fd = (loss(Ep, nu) - loss(Em, nu)) / (2 * h)
        assert abs(fd - dE[g]) <= 1e-5 * abs(dE[g])
    rng = np.random.default_rng(9)
    dirE = rng.standard_normal(len(E)) * E
    dirn = rng.standard_normal(len(nu)) * 0.01
    t = 1e-5
    fd = (loss(E + t * dirE, nu + t * dirn) - loss(E - t * dirE, nu - t * dirn)) / (2 * t)
    an = dE @ dirE + dnu @ dirn
    assert abs(fd - an) <= 1e-6 * abs(an)
