"""The two solvers of the reduced moment system in the RPIM shape kernel.

The RPIM shape functions are the solution of the moment problem (Sec. 1);
the kernel reduces it to S a_r = rhs and solves that either by an FP64
L D L' factorisation or by a float-float factorisation followed by one step
of iterative refinement with the residual in FP64. Both are
held here to the extended-precision oracle at the same per-case tolerances
as the parity tests (twice the error measured for the FP64 factorisation),
on every parity case; the two must also agree with each other in K and be
deterministic.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1802_04256_gb300 as R
from gpu_util import t
from test_gpu_parity import FLOORS, MARGIN, PROBLEMS

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _restore_solver():
    before = R.rpim_get_shape_solver()
    yield
    R.rpim_set_shape_solver(before)


def _phi_error(p, pat, phi):
    xyz, wj, soff, sidx = [a.cpu().numpy() for a in pat.points()]
    scale = np.array([1.0, p.h, p.h, p.h])
    worst = 0.0
    for k in range(0, p.n_points, max(1, p.n_points // 60)):
        s = sidx[soff[k]:soff[k + 1]]
        mine = phi[soff[k]:soff[k + 1]].T * scale[:, None]
        ref = oracle.shape(p.xyz, s, xyz[k], p.h, p.alpha_c, p.q, "ld") * scale[:, None]
        worst = max(worst, np.abs(mine - ref).max())
    return worst


@pytest.mark.parametrize("name", sorted(PROBLEMS))
def test_both_solvers_vs_extended_oracle(name):
    p = PROBLEMS[name]()
    pat = R.Pattern.from_problem(p)
    E, nu = t(p.E), t(p.nu)
    err, K = {}, {}
    for solver in ("fp64", "refined"):
        R.rpim_set_shape_solver(solver)
        assert R.rpim_get_shape_solver() == solver
        phi = pat.shape_functions().cpu().numpy()
        err[solver] = _phi_error(p, pat, phi)
        K[solver], _ = pat.assemble(E, nu)
        torch.cuda.synchronize()
    kmax = K["fp64"].abs().max().item()
    dK = (K["fp64"] - K["refined"]).abs().max().item() / kmax
    tol = MARGIN * FLOORS[name][0]
    print("solver %s: phi |fp64 - ld| %.3e, |refined - ld| %.3e (tol %.1e); K |fp64 - refined| %.3e"
          % (name, err["fp64"], err["refined"], tol, dK))
    assert err["fp64"] < tol
    assert err["refined"] < tol
    # both are within the K floor of the extended oracle, hence of each other
    assert dK < 2 * MARGIN * FLOORS[name][1]
    # the refined path is deterministic
    K2, _ = pat.assemble(E, nu)
    assert torch.equal(K2, K["refined"])
    pat.free()


def test_solver_setter_rejects_unknown():
    assert R.lib().rpim_set_shape_solver(2) == 1
    assert R.lib().rpim_set_shape_solver(-1) == 1
    assert R.rpim_get_shape_solver() in ("fp64", "refined")
