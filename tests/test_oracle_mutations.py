"""Planted mistakes in the oracle must break a pin.

Each case compiles a copy of ``oracle/oracle.c`` with one plausible slip
(a dropped factor, a wrong exponent, sign or index, a missing quadrature
factor, a wrong diagonal offset, a swapped ratio) and runs the pins of
``test_oracle_pins.py`` against it; at least one must fail.
"""
import os
import subprocess

import numpy as np
import pytest

import gen
import oracle
import test_oracle_pins as pins

MUTANTS = {
    "drop_factor_2_in_dR": ("2 * qr * RPOW(r2 + c2, qr - 1)", "qr * RPOW(r2 + c2, qr - 1)"),
    "wrong_exponent_in_dR": ("2 * qr * RPOW(r2 + c2, qr - 1)", "2 * qr * RPOW(r2 + c2, qr)"),
    "wrong_sign_in_dR": ("dR * (0 - xi[3 * i + k])", "dR * (xi[3 * i + k])"),
    "RQ_with_wrong_exponent": ("G[(size_t)i * N + j] = RPOW(r2 + c2, qr);",
                               "G[(size_t)i * N + j] = RPOW(r2 + c2, qr - 1);"),
    "shear_modulus_doubled": ("D[3 + a][3 + a] = mu;", "D[3 + a][3 + a] = 2 * mu;"),
    "transposed_B_entry": ("B[4][0] = g[2]; B[4][2] = g[0];", "B[4][0] = g[0]; B[4][2] = g[2];"),
    "missing_weight_factor": ("wj[8 * i + l] = (half[0] * half[1]) * half[2];",
                              "wj[8 * i + l] = (half[0] * half[1]);"),
    "penalty_on_wrong_entry": ("vals[9 * slot + 4 * a] += alpha;", "vals[9 * slot + a] += alpha;"),
    "pcg_beta_inverted": ("real beta = rz_new / rz;", "real beta = rz / rz_new;"),
    "lambda_wrong": ("real lam = E * nu / ((1 + nu) * (1 - 2 * nu));",
                     "real lam = E * nu / ((1 + nu) * (1 - nu));"),
    "dmu_dnu_sign": ("real dmu = -E / (2 * (1 + nu) * (1 + nu));", "real dmu = E / (2 * (1 + nu) * (1 + nu));"),
    "dlam_dnu_term": ("real dlam = E * (1 + 2 * nu * nu)", "real dlam = E * (1 + nu * nu)"),
    "traction_full_extent_weight": ("const double w = hu * hv;", "const double w = 4 * hu * hv;"),
    "traction_tangent_axes_swapped": ("const double U = x[ua], V = x[va];", "const double U = x[va], V = x[ua];"),
    "traction_gauss_point_off": ("x[va] = mv + hv * ((pt & 2) ? GAUSS2 : -GAUSS2);",
                                 "x[va] = mv + hv * ((pt & 2) ? 0.5 : -0.5);"),
    "traction_v_offset_with_u_half_width": ("x[va] = mv + hv * ((pt & 2) ? GAUSS2 : -GAUSS2);",
                                            "x[va] = mv + hu * ((pt & 2) ? GAUSS2 : -GAUSS2);"),
    "block_precond_diagonal_only": ("for (int b = 0; b < 3; b++) s += dinv[9 * I + 3 * a + b] * r[3 * I + b];",
                                    "for (int b = 0; b < 3; b++) s += dinv[9 * I + 4 * a] * r[3 * I + a];"),
    "block_inverse_wrong_row_op": ("for (int j = 0; j < 6; j++) m[i][j] -= l * m[k][j];",
                                   "for (int j = 0; j < 3; j++) m[i][j] -= l * m[k][j];"),
    "stress_voigt_slots_swapped": ("sigma[6 * p + r] = (double)acc;",
                                   "sigma[6 * p + (r == 3 ? 5 : r == 5 ? 3 : r)] = (double)acc;"),
    "stress_material_of_first_point": ("elastic_D((real)E[p], (real)nu[p], D);\n        for (int r = 0; r < 6; r++) {",
                                       "elastic_D((real)E[0], (real)nu[0], D);\n        for (int r = 0; r < 6; r++) {"),
}


def _build(name, tmp_path_factory):
    a, b = MUTANTS[name]
    with open(oracle.SRC) as fh:
        src = fh.read()
    assert src.count(a) == 1, name
    d = tmp_path_factory.mktemp(name)
    c = os.path.join(d, "m.c")
    with open(c, "w") as fh:
        fh.write(src.replace(a, b))
    so = os.path.join(d, "m.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", c, "-o", so,
                    "-lm"], check=True)
    kind = "mut_" + name
    oracle.register(kind, so)
    return kind


def _pins(kind, cube):
    """Every pin run against build `kind`; yields (name, callable)."""
    yield "quadrature", lambda: _quad(kind, cube)
    yield "reproduction", lambda: pins.test_partition_of_unity_and_linear_reproduction(cube, kind)
    yield "kronecker", lambda: pins.test_kronecker_delta_at_nodes(cube, kind)
    yield "rbf", lambda: pins.test_reproduces_constrained_rbf_combinations(cube, kind)
    yield "fd", lambda: pins.test_gradients_match_central_differences(cube, kind)
    m = lambda: oracle.assemble_problem(cube, kind)
    yield "rigid", lambda: pins.test_K_rigid_body_modes(m(), cube)
    yield "energy", lambda: pins.test_K_energy_of_linear_fields(m(), cube)
    yield "penalty", lambda: _penalty(kind, cube)
    yield "grad", lambda: pins.check_grad_material(kind)
    yield "pcg", lambda: _pcg(kind, cube)
    yield "stress", lambda: pins.test_stress_of_linear_fields_is_hookes_law(cube, kind)
    yield "traction", lambda: pins.test_traction_resultant_and_moment_are_the_exact_integrals(cube, kind)
    yield "block_pcg", lambda: pins.test_block_jacobi_pcg_is_exact_on_a_block_diagonal_matrix(cube, kind)
    yield "symmetry", lambda: pins.check_cube_symmetries(kind)


def _quad(kind, cube):
    pts, wj = oracle.gauss_points(cube.cell_lo, cube.cell_hi, kind)
    assert abs(wj.sum() - cube.volume) < 1e-14


def _penalty(kind, cube):
    m = oracle.assemble_problem(cube, "f64")
    vals = m.vals.ravel().copy()
    f = m.f.copy()
    diag0 = np.diag(m.dense()).copy()
    a = oracle.penalty(cube.n_nodes, m.rowptr, m.cols, vals, f, np.array([5], np.int64),
                       np.array([0.0]), 1e8, kind)
    m2 = oracle.Model(m.n_nodes, m.rowptr, m.cols, vals.reshape(-1, 9), f, None, None)
    d = np.diag(m2.dense()) - diag0
    assert d[5] == a and np.count_nonzero(d) == 1


def _pcg(kind, cube):
    m = oracle.assemble_problem(cube, "f64")
    vals = m.vals.ravel().copy()
    f = m.f.copy()
    oracle.penalty(cube.n_nodes, m.rowptr, m.cols, vals, f, cube.fixed_dofs, cube.fixed_vals, 1e8)
    u, it, rr, st = oracle.pcg(cube.n_nodes, m.rowptr, m.cols, vals, f, rtol=1e-12,
                               max_iter=5000, kind=kind)
    K = oracle.Model(m.n_nodes, m.rowptr, m.cols, vals.reshape(-1, 9), f, None, None).dense()
    assert st == 0
    assert np.linalg.norm(K @ u - f) <= 1e-10 * np.linalg.norm(f)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path_factory):
    kind = _build(name, tmp_path_factory)
    cube = gen.cube_config(n=5, jitter=0.2, seed=11)
    caught = []
    for pin, fn in _pins(kind, cube):
        try:
            fn()
        except (AssertionError, oracle.OracleError):
            caught.append(pin)
    assert caught, "no pin catches %s" % name


def test_unmutated_oracle_passes_the_same_pins():
    cube = gen.cube_config(n=5, jitter=0.2, seed=11)
    for pin, fn in _pins("f64", cube):
        fn()
