"""Material gradients (back-analysis) on the GPU through the C ABI.

* rpim_grad_material against the oracle's formula on the same seeded
  displacement and adjoint fields (the per-point formula; relative to max|g|).
* The autograd solve against the oracle's adjoint gradient of
  L = 1/2 |u - u_obs|^2 on a small block (oracle: its own assembly, dense
  solve and gradient).
* Central finite differences along a random direction of all parameters,
  on the small block and on the 64 x 32 x 32 back-analysis block
  (524,288 parameters of each kind), Richardson-extrapolated from steps h and
  2h (truncation O(h^4)). The relative step is 1e-4 (small block) and 1e-3
  (full block) rather than 1e-6: at 1e-6 the change of L is ~1e-8 of L,
  which is the reproducibility of two iterative solves of the penalised
  system (measured: FD noise 2.6e-6 small, 2e-4 full at step 1e-6).
Tolerance: relative 1e-6 (the shape functions of the two paths differ by the
plain-FP64 floor, ~1e-9, and the solves are run to 1e-13).
"""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1802_04256_gb300 as R
from gpu_util import faces, t

pytestmark = pytest.mark.gpu

TOL = 1e-6


def _material(p, seed):
    return gen.uniform(seed, 1, p.n_points, 5e3, 2e4), gen.uniform(seed, 2, p.n_points, 0.2, 0.4)


def test_grad_kernel_matches_oracle_formula():
    p = gen.cube_config(jitter=0.2, seed=31)
    E, nu = _material(p, 31)
    rng = np.random.default_rng(31)
    u = rng.standard_normal(3 * p.n_nodes)
    lam = rng.standard_normal(3 * p.n_nodes)
    pat = R.Pattern.from_problem(p)
    dE = torch.empty(p.n_points, dtype=torch.float64, device="cuda")
    dnu = torch.empty_like(dE)
    R.rpim_grad_material(pat.handle, t(u), t(lam), t(E), t(nu), dE, dnu)
    pts, wj = oracle.gauss_points(p.cell_lo, p.cell_hi)
    oE, onu = oracle.grad_material(p.xyz, pts, wj, E, nu, u, lam, p.alpha_s, p.alpha_c, p.q, p.h)
    dE, dnu = dE.cpu().numpy(), dnu.cpu().numpy()
    print("grad kernel: dE rel %.2e, dnu rel %.2e" % (np.abs(dE - oE).max() / np.abs(oE).max(),
                                                      np.abs(dnu - onu).max() / np.abs(onu).max()))
    assert np.abs(dE - oE).max() <= TOL * np.abs(oE).max()
    assert np.abs(dnu - onu).max() <= TOL * np.abs(onu).max()


def _block():
    p = gen.backanalysis_config(shape=(9, 5, 5), n_obs=60)
    return p


def _gpu_setup(p):
    pat = R.Pattern.from_problem(p)
    f_ext = torch.zeros(3 * p.n_nodes, dtype=torch.float64, device="cuda")
    pat.add_traction(*faces(p), f_ext)
    alpha = 1e8 * 4e3
    return pat, f_ext, alpha


def test_autograd_gradient_matches_oracle_adjoint():
    p = _block()
    obs = p.meta["obs_nodes"]
    pat, f_ext, alpha = _gpu_setup(p)
    E = t(p.E).requires_grad_()
    nu = t(p.nu).requires_grad_()
    u = R.solve(pat, E, nu, f_ext, t(p.fixed_dofs, torch.int64), t(p.fixed_vals), alpha, rtol=1e-13)
    rng = np.random.default_rng(7)
    u_obs = torch.as_tensor(rng.normal(0.0, 1e-3, (len(obs), 3)), device="cuda")
    loss = 0.5 * ((u.view(-1, 3)[torch.as_tensor(obs, device="cuda")] - u_obs) ** 2).sum()
    loss.backward()
    # oracle: its own assembly, dense solve, adjoint and gradient
    pts, wj = oracle.gauss_points(p.cell_lo, p.cell_hi)
    fo = np.zeros(3 * p.n_nodes)
    oracle.traction(p.xyz, p.face_lo, p.face_hi, p.face_axis, p.face_coef, p.alpha_s, p.alpha_c, p.q, p.h, fo)
    m = oracle.assemble(p.xyz, pts, wj, p.E, p.nu, p.alpha_s, p.alpha_c, p.q, p.h)
    vals = m.vals.ravel().copy()
    f = m.f + fo
    oracle.penalty(p.n_nodes, m.rowptr, m.cols, vals, f, p.fixed_dofs, p.fixed_vals, -alpha)
    K = oracle.Model(m.n_nodes, m.rowptr, m.cols, vals.reshape(-1, 9), f, None, None).dense()
    uo = np.linalg.solve(K, f)
    g = np.zeros_like(uo).reshape(-1, 3)
    g[obs] = uo.reshape(-1, 3)[obs] - u_obs.cpu().numpy()
    lam = np.linalg.solve(K, g.ravel())
    oE, onu = oracle.grad_material(p.xyz, pts, wj, p.E, p.nu, uo, lam, p.alpha_s, p.alpha_c, p.q, p.h)
    gE, gn = E.grad.cpu().numpy(), nu.grad.cpu().numpy()
    rE = np.abs(gE - oE).max() / np.abs(oE).max()
    rn = np.abs(gn - onu).max() / np.abs(onu).max()
    print("autograd vs oracle adjoint: dE rel %.2e dnu rel %.2e" % (rE, rn))
    assert rE <= TOL and rn <= TOL


def _fd_directional(p, pat, f_ext, alpha, obs, u_obs, E, nu, dirE, dirn, step):
    dofs, vals = t(p.fixed_dofs, torch.int64), t(p.fixed_vals)

    def loss(Ev, nuv):
        with torch.no_grad():
            u = R.solve(pat, Ev, nuv, f_ext, dofs, vals, alpha, rtol=1e-14)
        return 0.5 * ((u.view(-1, 3)[obs] - u_obs) ** 2).sum().item()

    def central(h):
        return (loss(E + h * dirE, nu + h * dirn) - loss(E - h * dirE, nu - h * dirn)) / (2 * h)

    return (4.0 * central(step) - central(2.0 * step)) / 3.0


@pytest.mark.parametrize("full", [False, True])
def test_gradient_matches_central_differences_along_a_direction(full):
    p = gen.backanalysis_config() if full else _block()
    pat, f_ext, alpha = _gpu_setup(p)
    obs = torch.as_tensor(p.meta["obs_nodes"], device="cuda")
    E = t(p.E).requires_grad_()
    nu = t(p.nu).requires_grad_()
    u = R.solve(pat, E, nu, f_ext, t(p.fixed_dofs, torch.int64), t(p.fixed_vals), alpha, rtol=1e-14)
    gen_obs = np.random.default_rng(11).normal(0.0, 1e-3, (len(obs), 3))
    u_obs = torch.as_tensor(gen_obs, device="cuda")
    loss = 0.5 * ((u.view(-1, 3)[obs] - u_obs) ** 2).sum()
    loss.backward()
    rng = np.random.default_rng(12)
    dirE = t(rng.standard_normal(p.n_points)) * E.detach()
    dirn = t(rng.standard_normal(p.n_points)) * 0.01
    an = (E.grad * dirE).sum().item() + (nu.grad * dirn).sum().item()
    fd = _fd_directional(p, pat, f_ext, alpha, obs, u_obs, E.detach(), nu.detach(), dirE, dirn,
                         1e-3 if full else 1e-4)
    print("%s: directional derivative adjoint %.9e fd %.9e rel %.2e" % ("full" if full else "small", an, fd,
                                                                       abs(an - fd) / abs(an)))
    assert abs(an - fd) <= TOL * abs(an)


def test_per_parameter_central_differences_on_the_backanalysis_block():
    """32 single parameters of the 64 x 32 x 32 back-analysis block (16 of E,
    16 of nu, at seeded random integration points), each against a central
    difference of L = 1/2 |u[obs] - u_obs|^2 at a step large enough to rise
    above the solver's noise (at the relative step of 1e-6 the change of L is
    about 1e-12 of L, below what two FP64 solves resolve). K is linear in
    E_g and a single point's stiffness is about 1e-6 of K's, so the central
    difference over 0.5% of E_g carries a truncation error of about 2e-7 of
    the gradient (measured: 6.6e-7 at 1%, 1.7e-5 at 5%, the O(h^2) term). D
    is nonlinear in nu, so the nu differences (steps 2e-3 and 4e-3) are
    Richardson-extrapolated (truncation O(h^4)). Both solves of a difference
    start from the converged unperturbed solution (warm start) and run to a
    relative residual of 1e-14; L+ - L- is formed as 1/2 (a+ - a-) . (a+ + a-),
    a = u[obs] - u_obs, which avoids subtracting two nearly equal losses.
    Tolerance: per entry, 1e-6 of the largest gradient of its kind among the
    16 (the gradients' own scale, as in the other checks of this file)."""
    p = gen.backanalysis_config()
    pat = R.Pattern.from_problem(p)
    pat.set_precond("block")
    f_ext = torch.zeros(3 * p.n_nodes, dtype=torch.float64, device="cuda")
    pat.add_traction(*faces(p), f_ext)
    E0, nu0 = t(p.E), t(p.nu)
    alpha = R.penalty_alpha(pat, E0, nu0)
    dofs, vals = t(p.fixed_dofs, torch.int64), t(p.fixed_vals)
    obs = torch.as_tensor(p.meta["obs_nodes"], device="cuda")
    u_obs = torch.as_tensor(np.random.default_rng(21).normal(0.0, 1e-3, (len(obs), 3)), device="cuda")

    def solve(E, nu, u0):
        K, f = pat.assemble(E, nu)
        R.rpim_add_vector(pat.handle, f_ext, f)
        R.rpim_apply_penalty_alpha(pat.handle, K, f, dofs, vals, alpha)
        u = u0.clone()
        _, it, rr = pat.solve_pcg(K, f, u=u, rtol=1e-14, max_iter=400000, check=False)
        assert rr <= 1e-13, rr
        return u

    E = E0.clone().requires_grad_()
    nu = nu0.clone().requires_grad_()
    u = R.solve(pat, E, nu, f_ext, dofs, vals, alpha, rtol=1e-14)
    loss = 0.5 * ((u.view(-1, 3)[obs] - u_obs) ** 2).sum()
    loss.backward()
    gE, gnu = E.grad, nu.grad
    u0 = u.detach()
    rng = np.random.default_rng(33)
    picks = [("E", g) for g in rng.choice(p.n_points, 16, replace=False)] + \
            [("nu", g) for g in rng.choice(p.n_points, 16, replace=False)]
    def central(kind, g, step):
        us = []
        for sgn in (1.0, -1.0):
            Ep, nup = E0.clone(), nu0.clone()
            (Ep if kind == "E" else nup)[g] += sgn * step
            us.append(solve(Ep, nup, u0).view(-1, 3)[obs] - u_obs)
        return float(0.5 * ((us[0] - us[1]) * (us[0] + us[1])).sum()) / (2 * step)

    res = {"E": [], "nu": []}
    for kind, g in picks:
        g = int(g)
        if kind == "E":
            fd = central(kind, g, 5e-3 * float(E0[g]))
        else:
            fd = (4.0 * central(kind, g, 2e-3) - central(kind, g, 4e-3)) / 3.0
        an = float((gE if kind == "E" else gnu)[g])
        res[kind].append((g, an, fd))
    worst = 0.0
    for kind, rows in res.items():
        scale = max(abs(an) for _, an, _ in rows)
        for g, an, fd in rows:
            d = abs(fd - an) / scale
            worst = max(worst, d)
            print("%s[%d]: adjoint %.9e central difference %.9e, |diff| / max|g| %.2e, rel %.2e"
                  % (kind, g, an, fd, d, abs(fd - an) / abs(an)))
    print("32 parameters: worst |diff| / max|g| %.2e" % worst)
    assert worst <= 1e-6
    pat.free()
