"""Stress recovery under self weight (the first verification example of
Sec. 3.1: a block under gravity, base fixed, sides on rollers, whose vertical
stress is -gamma times the depth).

With rollers on the sides the exact solution is uniaxial strain:
sigma_zz = -gamma (H - z) and sigma_xx = sigma_yy = nu / (1 - nu) sigma_zz.
Checked on the GPU path at two resolutions: the base reactions carry the
weight, centre-line stresses approach the closed form as h halves, the
volume average of sigma_zz over all integration points is -gamma H / 2, and
the coarse column's stresses match the oracle's.
"""
import numpy as np
import pytest
import torch

import gen
import oracle
from gpu_util import GpuRun, t

pytestmark = pytest.mark.gpu

H, W, GAMMA = 3.0, 0.6, 20.0


def _column(shape):
    p = gen.gravity_column(shape=shape, height=H, width=W, gamma=GAMMA)
    g = GpuRun(p)
    u, it, rr, alpha, K, f = g.solve(rtol=1e-12)
    return p, g, u, alpha


@pytest.fixture(scope="module")
def columns():
    return {h: _column(s) for h, s in ((0.1, (7, 7, 31)), (0.05, (13, 13, 61)))}


def _centre_line(p, g, u, zs):
    pts = np.array([[W / 2, W / 2, z] for z in zs])
    E = np.full(len(pts), p.meta["E"])
    nu = np.full(len(pts), p.meta["nu"])
    return g.pat.stress(u, t(pts), t(E), t(nu)).cpu().numpy(), pts, E, nu


def test_base_reaction_equals_weight(columns):
    for h, (p, g, u, alpha) in columns.items():
        fd = torch.as_tensor(p.fixed_dofs, device="cuda")
        base = fd[fd % 3 == 2]
        reaction = float(alpha * u[base].sum())
        weight = -GAMMA * W * W * H
        print("h %.2f: base reaction %.9f, weight %.9f" % (h, reaction, weight))
        assert abs(reaction - weight) < 1e-8 * abs(weight)


def test_centre_line_stress_converges(columns):
    zs = np.linspace(0.5, 2.5, 9)
    ref = -GAMMA * (H - zs)
    err = {}
    for h, (p, g, u, alpha) in columns.items():
        s, _, _, _ = _centre_line(p, g, u, zs)
        err[h] = np.abs(s[:, 2] - ref).max() / (GAMMA * H)
        ratio = s[:, 0] / s[:, 2]
        print("h %.2f: max |szz - closed form| / (gamma H) = %.3e, sxx/szz in [%.4f, %.4f] (%.4f)"
              % (h, err[h], ratio.min(), ratio.max(), 0.3 / 0.7))
        assert np.abs(ratio - 0.3 / 0.7).max() < 0.05
    assert err[0.1] < 0.025
    assert err[0.05] < err[0.1]


def test_volume_average_stress_at_all_points(columns):
    """Stresses at every integration point of the fine column (stress
    recovery at scale); their weighted mean is -gamma H / 2."""
    p, g, u, alpha = columns[0.05]
    xyz, wj, soff, sidx = g.pat.points()
    n = xyz.shape[0]
    E = torch.full((n,), p.meta["E"], dtype=torch.float64, device="cuda")
    nu = torch.full((n,), p.meta["nu"], dtype=torch.float64, device="cuda")
    s = g.pat.stress(u, xyz, E, nu)
    mean = float((s[:, 2] * wj).sum() / wj.sum())
    print("%d points: mean szz %.6f vs %.6f" % (n, mean, -GAMMA * H / 2))
    assert abs(mean + GAMMA * H / 2) < 0.01 * GAMMA * H / 2


def test_coarse_column_stress_vs_oracle(columns):
    p, g, u, alpha = columns[0.1]
    zs = np.linspace(0.25, 2.75, 11)
    s, pts, E, nu = _centre_line(p, g, u, zs)
    mo, uo, ito, rro, ao = oracle.solve_problem(p, "f64", rtol=1e-12)
    so = oracle.stress(p.xyz, uo, pts, E, nu, p.alpha_s, p.alpha_c, p.q, p.h, "f64")
    d = np.abs(s - so).max() / np.abs(so).max()
    print("stress vs oracle pipeline: %.3e" % d)
    assert d < 1e-6
