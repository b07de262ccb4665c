"""The 129 x 17 x 17 cantilever (37,281 nodes, 298,248 integration points),
the workload the benchmark times, in the benchmark's launch configuration:
sampled shape functions and K rows against the oracle, exact invariants of
the whole K, and Timoshenko's tip deflection."""
import numpy as np
import pytest
import torch

import gen
import oracle
from gpu_util import GpuRun, bsr_matvec, t

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def beam():
    p = gen.cantilever_config()
    g = GpuRun(p)
    return p, g


def test_sampled_shape_functions_vs_extended_oracle(beam):
    p, g = beam
    phi = g.pat.shape_functions().cpu().numpy()
    xyz, wj, soff, sidx = [a.cpu().numpy() for a in g.pat.points()]
    rs2 = oracle.support_radius2(p.alpha_s, p.h)
    scale = np.array([1.0, p.h, p.h, p.h])
    rng = np.random.default_rng(5)
    worst = 0.0
    for k in rng.choice(p.n_points, 48, replace=False):
        s = oracle.support(p.xyz, xyz[k], rs2)
        assert np.array_equal(s, sidx[soff[k]:soff[k + 1]])
        ref = oracle.shape(p.xyz, s, xyz[k], p.h, p.alpha_c, p.q, "ld")
        worst = max(worst, np.abs((phi[soff[k]:soff[k + 1]].T - ref) * scale[:, None]).max())
    print("sampled phi vs extended oracle: %.3e" % worst)
    assert worst < 1e-9


def test_sampled_rows_vs_oracle(beam):
    """Row I of K only involves the points whose support holds I; assembling
    those points with the oracle reproduces row I exactly. Held to the
    extended oracle with the parity rule (1e-10 of max|K|: twice the worst
    row measured on the parity cases' cantilever, 33x5x5), and to the plain
    FP64 oracle within its own error plus that."""
    p, g = beam
    rowptr, cols = g.host_csr()
    K = g.host_K()
    kmax = np.abs(K).max()
    pts, wj = oracle.gauss_points(p.cell_lo, p.cell_hi)
    rs2 = oracle.support_radius2(p.alpha_s, p.h)
    worst = e64 = 0.0
    for I in (0, 18000, 37280, 9000):
        near = np.nonzero(((pts - p.xyz[I]) ** 2).sum(1) <= rs2 * 1.01)[0]
        sel = [k for k in near if I in oracle.support(p.xyz, pts[k], rs2)]
        rows = {}
        for kind in ("f64", "ld"):
            m = oracle.assemble(p.xyz, pts[sel], wj[sel], p.E[sel], p.nu[sel], p.alpha_s, p.alpha_c,
                                p.q, p.h, kind=kind, rows=[I])
            assert np.array_equal(m.cols[m.rowptr[I]:m.rowptr[I + 1]], cols[rowptr[I]:rowptr[I + 1]])
            rows[kind] = m.vals[m.rowptr[I]:m.rowptr[I + 1]]
        d = np.abs(rows["ld"] - K[rowptr[I]:rowptr[I + 1]]).max() / kmax
        e = np.abs(rows["ld"] - rows["f64"]).max() / kmax
        print("row %d: %d points, |gpu - ld| %.3e, |f64 - ld| %.3e" % (I, len(sel), d, e))
        worst, e64 = max(worst, d), max(e64, e)
    assert worst < 1e-10


def test_invariants_of_full_K(beam):
    p, g = beam
    rowptr, cols = g.host_csr()
    K = g.host_K()
    X = p.xyz
    kf = np.sqrt((K ** 2).sum())
    modes = [np.tile(np.eye(3)[k], len(X)) for k in range(3)]
    modes += [np.cross(np.eye(3)[k], X).ravel() for k in range(3)]
    for u in modes:
        r = np.linalg.norm(bsr_matvec(rowptr, cols, K, u)) / (kf * np.linalg.norm(u))
        assert r < 1e-10
    lam = 1e4 * 0.3 / (1.3 * 0.4)
    mu = 1e4 / 2.6
    for a, b in [(0, 0), (0, 1), (3, 3), (5, 2)]:
        A = np.zeros((3, 3))
        B = np.zeros((3, 3))
        for M, k in ((A, a), (B, b)):
            if k < 3:
                M[k, k] = 1.0
            else:
                i, j = [(1, 2), (0, 2), (0, 1)][k - 3]
                M[i, j] = M[j, i] = 0.5
        ua, ub = (X @ A.T).ravel(), (X @ B.T).ravel()
        want = 8.0 * (lam * np.trace(A) * np.trace(B) + 2 * mu * np.sum(A * B))
        got = ua @ bsr_matvec(rowptr, cols, K, ub)
        assert abs(got - want) < 1e-8 * (lam + 2 * mu) * 8.0


def test_timoshenko_tip_deflection(beam):
    p, g = beam
    u, it, rr, alpha, K, f = g.solve(rtol=1e-10)
    tip = np.nonzero(np.all(np.abs(p.nominal - [8.0, 0.5, 0.5]) < 1e-9, axis=1))[0][0]
    I = 1.0 / 12.0
    ref = 8.0**3 / (3 * 1e4 * I) + (4 + 5 * 0.3) * 8.0 / (24 * 1e4 * I)
    w = -u[3 * tip + 2].item()
    print("tip deflection %.6f vs Timoshenko %.6f (%.2f%%), %d PCG iterations" % (w, ref, 100 * (w - ref) / ref, it))
    assert abs(w - ref) / ref < 0.02
