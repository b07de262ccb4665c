"""Pins of the oracle's MLS shape functions (the shape-function variant the
paper lists as future work, Sec. 4: moving least squares with the linear
basis and a cubic-spline weight on the RPIM support radius).

Against facts fixed by the mathematics, not by the oracle itself:
* MLS with a linear basis reproduces linear fields exactly: partition of
  unity, sum phi_i x_i = x, and the same for the derivatives;
* with exactly four nodes the fit is an interpolation whatever the weights:
  barycentric coordinates and their constant gradients;
* derivatives against central differences of phi (the weight is C1, so
  the difference quotient converges);
* an extended-precision rerun (the 4x4 moment matrix is well conditioned in
  local coordinates, so FP64 agrees to ~1e-13);
* K from MLS shape functions: symmetry, rigid-body modes, and the energy of
  linear fields (the patch test in energy form); stresses of linear fields
  by Hooke's law;
* planted mistakes in a copy of the oracle's MLS code break these pins.
"""
import os
import subprocess

import numpy as np
import pytest

import gen
import oracle

KINDS = ["f64", "ld"]


@pytest.fixture(scope="module")
def cube():
    return gen.cube_config(jitter=0.2, seed=7)


def _points(p, n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.02, 0.98, (n, 3))


def check_reproduction(p, kind):
    rs2 = oracle.support_radius2(p.alpha_s, p.h)
    for x in _points(p, 60, 1):
        s = oracle.support(p.xyz, x, rs2)
        ph = oracle.shape_mls(p.xyz, s, x, p.h, p.alpha_s, kind=kind)
        X = p.xyz[s]
        assert abs(ph[0].sum() - 1.0) < 1e-13
        assert np.abs(ph[0] @ X - x).max() < 1e-13
        assert np.abs(ph[1:].sum(1)).max() < 1e-11 / p.h
        assert np.abs(ph[1:] @ X - np.eye(3)).max() < 1e-12


def check_central_differences(p, kind):
    rs2 = oracle.support_radius2(p.alpha_s, p.h)
    d = 1e-6 * p.h
    for x in _points(p, 40, 2):
        s = oracle.support(p.xyz, x, rs2)
        ph = oracle.shape_mls(p.xyz, s, x, p.h, p.alpha_s, kind=kind)
        for k in range(3):
            e = np.eye(3)[k] * d
            fd = (oracle.shape_mls(p.xyz, s, x + e, p.h, p.alpha_s, kind=kind)[0] -
                  oracle.shape_mls(p.xyz, s, x - e, p.h, p.alpha_s, kind=kind)[0]) / (2 * d)
            assert np.abs(fd - ph[1 + k]).max() < 1e-6 / p.h


@pytest.mark.parametrize("kind", KINDS)
def test_partition_of_unity_and_linear_reproduction(cube, kind):
    check_reproduction(cube, kind)


@pytest.mark.parametrize("kind", KINDS)
def test_four_nodes_reduce_to_barycentric_interpolation(kind):
    xyz = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.2, 0.9, 0.1], [0.1, 0.2, 1.1]])
    x = np.array([0.3, 0.25, 0.2])
    s = np.arange(4, dtype=np.int32)
    ph = oracle.shape_mls(xyz, s, x, 0.5, 4.0, kind=kind)   # radius 2: every weight > 0
    A = np.vstack([np.ones(4), xyz.T])
    lam = np.linalg.solve(A, np.concatenate([[1.0], x]))
    grads = np.linalg.inv(A)[:, 1:]
    assert np.abs(ph[0] - lam).max() < 1e-13
    assert np.abs(ph[1:].T - grads).max() < 1e-12


@pytest.mark.parametrize("kind", KINDS)
def test_gradients_match_central_differences(cube, kind):
    check_central_differences(cube, kind)


def test_fp64_agrees_with_extended_precision(cube):
    rs2 = oracle.support_radius2(cube.alpha_s, cube.h)
    worst = 0.0
    for x in _points(cube, 50, 3):
        s = oracle.support(cube.xyz, x, rs2)
        a = oracle.shape_mls(cube.xyz, s, x, cube.h, cube.alpha_s, kind="f64")
        b = oracle.shape_mls(cube.xyz, s, x, cube.h, cube.alpha_s, kind="ld")
        worst = max(worst, np.abs(a - b).max() * cube.h)
    assert worst < 1e-12


def test_coplanar_support_is_singular():
    g = np.linspace(0.0, 1.0, 5)
    X, Y = np.meshgrid(g, g, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], 1)
    s = np.arange(len(xyz), dtype=np.int32)
    with pytest.raises(oracle.OracleError):
        oracle.shape_mls(xyz, s, np.array([0.5, 0.5, 0.0]), 0.25, 3.0)


def check_K(p, kind):
    with oracle.shape_kind("mls"):
        m = oracle.assemble_problem(p, kind)
    K = m.dense()
    kf = np.linalg.norm(K)
    assert np.abs(K - K.T).max() <= 1e-14 * np.abs(K).max()
    X = p.xyz
    modes = [np.tile(np.eye(3)[k], len(X)) for k in range(3)]
    modes += [np.cross(np.eye(3)[k], X).ravel() for k in range(3)]
    for u in modes:
        assert np.linalg.norm(K @ u) / (kf * np.linalg.norm(u)) < 1e-12
    E, nu = 1.0e4, 0.3
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    for a in range(6):
        for b in range(6):
            A = np.zeros((3, 3))
            B = np.zeros((3, 3))
            for M, k in ((A, a), (B, b)):
                if k < 3:
                    M[k, k] = 1.0
                else:
                    i, j = [(1, 2), (0, 2), (0, 1)][k - 3]
                    M[i, j] = M[j, i] = 0.5
            want = p.volume * (lam * np.trace(A) * np.trace(B) + 2 * mu * np.sum(A * B))
            got = (X @ A.T).ravel() @ K @ (X @ B.T).ravel()
            assert abs(got - want) < 1e-10 * (lam + 2 * mu) * p.volume


@pytest.mark.parametrize("kind", KINDS)
def test_K_symmetry_rigid_modes_and_energy(cube, kind):
    check_K(cube, kind)


@pytest.mark.parametrize("kind", KINDS)
def test_stress_of_linear_fields_is_hookes_law(cube, kind):
    """MLS with the linear basis reproduces u = A x and its gradient exactly,
    so the stress of such a field at any point is Hooke's law of the
    constant strain, as for RPIM: the same pin, with the stresses computed
    from MLS shape functions."""
    import test_oracle_pins as pins
    with oracle.shape_kind("mls"):
        pins.test_stress_of_linear_fields_is_hookes_law(cube, kind)


def test_shape_kind_selection_is_scoped(cube):
    with oracle.shape_kind("mls"):
        assert oracle.lib("f64").orc_get_shape() == 1
    assert oracle.lib("f64").orc_get_shape() == 0
    a = oracle.assemble_problem(cube, "f64")
    with oracle.shape_kind("mls"):
        b = oracle.assemble_problem(cube, "f64")
    assert np.abs(a.vals - b.vals).max() > 1e-3 * np.abs(a.vals).max()


# ------------------------------------------------------- planted mistakes
MUTANTS = {
    "spline_branch_sign": ("*dw = -4 + 8 * sb - 4 * sb * sb;", "*dw = 4 - 8 * sb + 4 * sb * sb;"),
    "spline_inner_coefficient": ("*w = (real)2 / 3 - 4 * sb * sb + 4 * sb * sb * sb;",
                                 "*w = (real)2 / 3 - 4 * sb * sb + 3 * sb * sb * sb;"),
    "weight_derivative_sign": ("dws * (-xi[3 * i + k]) / (as * hr * d)", "dws * (xi[3 * i + k]) / (as * hr * d)"),
    "dropped_dA_term": ("for (int c = 0; c < 4; c++) s -= dA[k][a][c] * gam[c];", ""),
    "dp_without_1_over_h": ("real s = (a == k + 1) ? 1 / hr : 0;", "real s = (a == k + 1) ? 1 : 0;"),
    "dropped_dw_term_in_dphi": ("= w[4 * i + 1 + k] * pg + w[4 * i] * pdg;", "= w[4 * i] * pdg;"),
}


@pytest.fixture(scope="module", params=sorted(MUTANTS))
def mutant(request, tmp_path_factory):
    name = request.param
    a, b = MUTANTS[name]
    with open(oracle.SRC) as fh:
        src = fh.read()
    assert src.count(a) == 1, name
    d = tmp_path_factory.mktemp(name)
    c = os.path.join(d, "m.c")
    with open(c, "w") as fh:
        fh.write(src.replace(a, b))
    so = os.path.join(d, "m.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", c, "-o", so, "-lm"],
                   check=True)
    kind = "mls_mut_" + name
    oracle.register(kind, so)
    return kind


def test_planted_mistake_breaks_a_pin(mutant, cube):
    failed = []
    for name, fn in (("reproduction", lambda: check_reproduction(cube, mutant)),
                     ("fd", lambda: check_central_differences(cube, mutant)),
                     ("K", lambda: check_K(cube, mutant))):
        try:
            fn()
        except (AssertionError, oracle.OracleError):
            failed.append(name)
    assert failed, "no pin caught the planted mistake"
