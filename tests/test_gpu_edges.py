"""Edge cases of the path: supports at the size limit, zero-length calls and
the smallest clouds.

* Support radius 3.7h on a 7x7x7 jittered lattice: the largest supports (208
  nodes) run in the last support-size bucket with one point per block;
  shape functions are held to the extended oracle with the parity rule of
  test_gpu_parity.py, K to the FP64 oracle and the rigid-body modes.
* Radius 3.9h puts more than RPIM_MAX_SUPPORT (216) nodes in a support:
  the build reports RPIM_E_SUPPORT.
* Zero loads, zero stress points and zero constrained DOFs are no-ops.
* A 2x2x2 cloud (8 nodes, every support the whole cloud) assembles and
  matches the oracle.
"""
import numpy as np
import pytest
import torch

import gen
import oracle
from gpu_util import GpuRun, bsr_matvec, t

import paper_1802_04256_gb300 as R

pytestmark = pytest.mark.gpu

TOL_PHI_LD = 4.3e-9   # twice the error measured at the largest supports on a GB300 (2.1e-9, h units)


def _problem(alpha_s, shape=(7, 7, 7), seed=41):
    p = gen.lattice_problem("edge", shape, (1.0, 1.0, 1.0), 0.2, seed)
    ijk, nom, xyz, lo, hi, sp = p
    n = len(xyz)
    return gen.Problem("edge", xyz, lo, hi, alpha_s, 4.0, 1.03, float(sp.max()),
                       np.full(8 * n, 1e4), np.full(8 * n, 0.3))


def test_largest_supports_vs_extended_oracle():
    p = _problem(3.7)
    g = GpuRun(p)
    info = g.pat.info
    print("supports %d..%d of %d nodes" % (info.min_support, info.max_support, p.n_nodes))
    assert info.max_support > 180 and info.max_support <= 216
    xyz, wj, soff, sidx = [a.cpu().numpy() for a in g.pat.points()]
    phi = g.pat.shape_functions().cpu().numpy()
    scale = np.array([1.0, p.h, p.h, p.h])
    big = np.argsort(np.diff(soff))[-12:]     # the largest supports
    worst = e64 = 0.0
    for k in big:
        s = sidx[soff[k]:soff[k + 1]]
        mine = phi[soff[k]:soff[k + 1]].T * scale[:, None]
        ld = oracle.shape(p.xyz, s, xyz[k], p.h, p.alpha_c, p.q, "ld") * scale[:, None]
        f64 = oracle.shape(p.xyz, s, xyz[k], p.h, p.alpha_c, p.q, "f64") * scale[:, None]
        worst = max(worst, np.abs(mine - ld).max())
        e64 = max(e64, np.abs(f64 - ld).max())
    tol = TOL_PHI_LD
    print("phi at the largest supports: |gpu - ld| %.3e (tol %.1e), |f64 - ld| %.3e" % (worst, tol, e64))
    assert worst < tol
    # K: the extended oracle is too slow here on a host whose long double is
    # software binary128, so K is held to the FP64 oracle within its own
    # floor (measured against the extended oracle on x86-64: 2.6e-8 of
    # max|K| for this cloud) and to the rigid-body null modes
    m = oracle.assemble_problem(p, "f64")
    K = g.host_K()
    kmax = np.abs(m.vals).max()
    d64 = np.abs(K - m.vals).max() / kmax
    rowptr, cols = g.host_csr()
    kf = np.sqrt((K ** 2).sum())
    rb = 0.0
    for k in range(3):
        e = np.eye(3)[k]
        for u in (np.tile(e, p.n_nodes), np.cross(e, p.xyz).ravel()):
            rb = max(rb, np.linalg.norm(bsr_matvec(rowptr, cols, K, u)) / (kf * np.linalg.norm(u)))
    print("K: |gpu - f64| %.3e of max|K|, rigid-body residual %.2e" % (d64, rb))
    assert d64 < 1e-7
    assert rb < 1e-10


def test_support_over_the_limit_is_reported():
    p = _problem(3.9)
    with pytest.raises(R.RpimError) as e:
        R.Pattern.from_problem(p)
    assert e.value.status == 4   # RPIM_E_SUPPORT


def test_zero_length_calls_are_no_ops():
    p = gen.cube_config(n=5)
    g = GpuRun(p)
    f = g.f.clone()
    g.pat.add_point_loads(t(np.zeros((0, 3))), t(np.zeros((0, 3))), f)
    g.pat.add_traction(t(np.zeros((0, 3))), t(np.zeros((0, 3))), t(np.zeros(0, np.int8), torch.int8),
                       t(np.zeros((0, 3, 6))), f)
    assert torch.equal(f, g.f)
    s = g.pat.stress(torch.zeros_like(f), t(np.zeros((0, 3))), t(np.zeros(0)), t(np.zeros(0)))
    assert s.shape == (0, 6)
    K = g.K.clone()
    g.pat.apply_penalty(K, f, t(np.zeros(0), torch.int64), t(np.zeros(0)))
    assert torch.equal(K, g.K) and torch.equal(f, g.f)


def test_smallest_cloud():
    p = _problem(2.5, shape=(2, 2, 2))
    g = GpuRun(p)
    assert g.pat.info.max_support == 8 and g.pat.info.min_support == 8
    m = oracle.assemble_problem(p, "ld")
    d = np.abs(g.host_K() - m.vals).max() / np.abs(m.vals).max()
    print("8-node cloud: K rel %.3e" % d)
    assert d < 1e-10
