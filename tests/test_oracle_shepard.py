"""Pins of the oracle's Shepard shape functions (the other shape-function
variant Sec. 4 lists as future work): inverse-distance weighting with the
cubic-spline weight of the MLS variant, i.e. moving least squares with a
constant basis.

Against facts fixed by the mathematics, not by the oracle itself:
* two nodes at spline arguments 0 and 1/2: the weights are the spline's
  values 2/3 and 1/6, so phi = (4/5, 1/5); the spline's slope there is -1,
  which with r_s = 1/2 gives dphi/dx = -/+ 48/25 by the quotient rule
  worked by hand;
* partition of unity (exact for any weights) and hence zero gradient sums;
* no linear reproduction in general (what distinguishes it from MLS);
* derivatives against central differences;
* an extended-precision rerun;
* K: symmetric, rigid translations in its null space, rotations not;
* stresses: zero for a rigid translation, not Hooke's law for a stretch;
* planted mistakes in a copy of the oracle's Shepard code break these pins.
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


def _points(n, seed):
    return np.random.default_rng(seed).uniform(0.02, 0.98, (n, 3))


def check_two_nodes(kind):
    xyz = np.array([[0.3, 0.2, 0.1], [0.3 + 0.25, 0.2, 0.1]])   # r_s = 2 * 0.25 = 0.5: sb = 0 and 1/2
    ph = oracle.shape_shepard(xyz, np.arange(2, dtype=np.int32), xyz[0], 0.25, 2.0, kind=kind)
    assert np.abs(ph[0] - [0.8, 0.2]).max() < 1e-15
    # W = 5/6, dW/dx = dw_2/dx = -w'(1/2) / r_s = 2
    assert np.abs(ph[1] - [-1.92, 1.92]).max() < 1e-13
    assert np.abs(ph[2:]).max() < 1e-15


def check_partition(p, kind):
    rs2 = oracle.support_radius2(p.alpha_s, p.h)
    for x in _points(60, 1):
        s = oracle.support(p.xyz, x, rs2)
        ph = oracle.shape_shepard(p.xyz, s, x, p.h, p.alpha_s, kind=kind)
        assert abs(ph[0].sum() - 1.0) < 1e-14
        assert np.abs(ph[1:].sum(1)).max() < 1e-12 / p.h
        assert (ph[0] >= 0).all()


def check_central_differences(p, kind):
    rs2 = oracle.support_radius2(p.alpha_s, p.h)
    d = 1e-6 * p.h
    for x in _points(40, 2):
        s = oracle.support(p.xyz, x, rs2)
        ph = oracle.shape_shepard(p.xyz, s, x, p.h, p.alpha_s, kind=kind)
        for k in range(3):
            e = np.eye(3)[k] * d
            fd = (oracle.shape_shepard(p.xyz, s, x + e, p.h, p.alpha_s, kind=kind)[0] -
                  oracle.shape_shepard(p.xyz, s, x - e, p.h, p.alpha_s, kind=kind)[0]) / (2 * d)
            assert np.abs(fd - ph[1 + k]).max() < 1e-6 / p.h


def check_K(p, kind):
    with oracle.shape_kind("shepard"):
        m = oracle.assemble_problem(p, kind)
    K = m.dense()
    kf = np.linalg.norm(K)
    assert np.abs(K - K.T).max() <= 1e-14 * np.abs(K).max()
    for k in range(3):
        u = np.tile(np.eye(3)[k], p.n_nodes)
        assert np.linalg.norm(K @ u) / (kf * np.linalg.norm(u)) < 1e-13
    X = p.xyz - p.xyz.mean(0)
    rot = np.cross(np.eye(3)[2], X).ravel()
    assert np.linalg.norm(K @ rot) / (kf * np.linalg.norm(rot)) > 1e-4


@pytest.mark.parametrize("kind", KINDS)
def test_two_nodes_closed_form(kind):
    check_two_nodes(kind)


@pytest.mark.parametrize("kind", KINDS)
def test_partition_of_unity(cube, kind):
    check_partition(cube, kind)


def test_no_linear_reproduction(cube):
    rs2 = oracle.support_radius2(cube.alpha_s, cube.h)
    worst = 0.0
    for x in _points(20, 4):
        s = oracle.support(cube.xyz, x, rs2)
        ph = oracle.shape_shepard(cube.xyz, s, x, cube.h, cube.alpha_s)
        worst = max(worst, np.abs(ph[0] @ cube.xyz[s] - x).max())
    assert worst > 1e-3 * cube.h


@pytest.mark.parametrize("kind", KINDS)
def test_gradients_match_central_differences(cube, kind):
    check_central_differences(cube, kind)


def test_fp64_agrees_with_extended_precision(cube):
    rs2 = oracle.support_radius2(cube.alpha_s, cube.h)
    worst = 0.0
    for x in _points(50, 3):
        s = oracle.support(cube.xyz, x, rs2)
        a = oracle.shape_shepard(cube.xyz, s, x, cube.h, cube.alpha_s, kind="f64")
        b = oracle.shape_shepard(cube.xyz, s, x, cube.h, cube.alpha_s, kind="ld")
        worst = max(worst, np.abs(a - b).max() * cube.h)
    assert worst < 1e-14


def test_no_weight_is_singular():
    xyz = np.array([[0.0, 0.0, 0.0], [1.2, 0.0, 0.0]])
    with pytest.raises(oracle.OracleError):   # both nodes beyond the support radius 0.5
        oracle.shape_shepard(xyz, np.arange(2, dtype=np.int32), np.array([0.6, 0.0, 0.0]), 0.25, 2.0)


@pytest.mark.parametrize("kind", KINDS)
def test_stress_of_a_translation_is_zero_and_of_a_stretch_is_not_exact(cube, kind):
    """Shepard functions sum to one, so their gradients sum to zero and a
    rigid translation has zero strain and stress at every point (to
    rounding); they do not reproduce linear fields, so a uniform stretch
    does not give Hooke's law of its strain (what sets Shepard apart from
    MLS and RPIM)."""
    pts = cube.xyz[::7] * 0.9 + 0.05
    E = np.full(len(pts), 1.0e4)
    nu = np.full(len(pts), 0.3)
    lam = E[0] * nu[0] / ((1 + nu[0]) * (1 - 2 * nu[0]))
    with oracle.shape_kind("shepard"):
        t = np.tile([0.3, -0.2, 0.5], cube.n_nodes)
        sig = oracle.stress(cube.xyz, t, pts, E, nu, cube.alpha_s, cube.alpha_c, cube.q, cube.h, kind)
        assert np.abs(sig).max() < 1e-12 * lam   # measured 2e-15 (f64), 1e-18 (ld)
        u = (cube.xyz * [1.0e-3, 0.0, 0.0]).ravel()
        sig = oracle.stress(cube.xyz, u, pts, E, nu, cube.alpha_s, cube.alpha_c, cube.q, cube.h, kind)
    want_xx = (lam + E[0] / (1 + nu[0])) * 1.0e-3
    assert np.abs(sig[:, 0] - want_xx).max() > 1e-3 * want_xx   # measured 44%


@pytest.mark.parametrize("kind", KINDS)
def test_K_symmetric_translations_null_rotations_not(cube, kind):
    check_K(cube, kind)


# ------------------------------------------------------- planted mistakes
MUTANTS = {
    "quotient_rule_sign": ("(dw[k] - ph * dW[k]) / W;", "(dw[k] + ph * dW[k]) / W;"),
    "derivative_not_divided": ("(dw[k] - ph * dW[k]) / W;", "(dw[k] - ph * dW[k]);"),
    "dropped_weight_sum_gradient": ("for (int k = 0; k < 3; k++) dW[k] += dw[k];", ""),
    "unnormalised_phi": ("const real ph = wv / W;", "const real ph = wv;"),
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
    kind = "shepard_mut_" + name
    oracle.register(kind, so)
    return kind


def test_planted_mistake_breaks_a_pin(mutant, cube):
    failed = []
    for name, fn in (("two nodes", lambda: check_two_nodes(mutant)),
                     ("partition", lambda: check_partition(cube, mutant)),
                     ("fd", lambda: check_central_differences(cube, mutant)),
                     ("K", lambda: check_K(cube, mutant))):
        try:
            fn()
        except (AssertionError, oracle.OracleError):
            failed.append(name)
    assert failed, "no pin caught the planted mistake"
