"""Error paths of the C ABI: each bad input comes back as a status code and
the pattern stays usable. Nothing here faults the GPU: every case is caught
by a host check or by the kernels' own range and degeneracy tests."""
import numpy as np
import pytest
import torch

import gen
import paper_1802_04256_gb300 as R
from gpu_util import GpuRun, t

pytestmark = pytest.mark.gpu


def _status(fn):
    with pytest.raises(R.RpimError) as e:
        fn()
    return e.value.status


def test_coplanar_cloud_is_singular():
    n = 6
    g = np.arange(n) * 0.2
    X = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2)
    xyz = np.concatenate([X, np.zeros((len(X), 1))], 1)
    lo = np.concatenate([np.maximum(X - 0.1, 0), np.zeros((len(X), 1))], 1)
    hi = np.concatenate([np.minimum(X + 0.1, 1.0), np.zeros((len(X), 1))], 1)
    pat = R.Pattern(t(xyz), t(lo), t(hi), 2.5, 4.0, 1.03, 0.2)
    E = t(np.full(8 * len(xyz), 1e4))
    nu = t(np.full(8 * len(xyz), 0.3))
    assert _status(lambda: pat.assemble(E, nu)) == 5


def test_support_too_small():
    p = gen.cube_config()
    assert _status(lambda: R.Pattern(t(p.xyz), t(p.cell_lo), t(p.cell_hi), 0.5, 4.0, 1.03, 0.2)) == 4


def test_bad_material_and_recovery():
    p = gen.cube_config(n=5)
    g = GpuRun(p)
    nu = g.nu.clone()
    nu[7] = 0.5
    assert _status(lambda: g.pat.assemble(g.E, nu)) == 1
    K, f = g.pat.assemble(g.E, g.nu)
    assert torch.equal(K, g.K)


def test_duplicate_and_out_of_range_dofs():
    p = gen.cube_config(n=5)
    g = GpuRun(p)
    K, f = g.K.clone(), g.f.clone()
    v = t(np.zeros(2))
    assert _status(lambda: g.pat.apply_penalty(K, f, t([5, 5], torch.int64), v)) == 1
    assert _status(lambda: g.pat.apply_penalty(K, f, t([5, 3 * p.n_nodes], torch.int64), v)) == 1


def test_pcg_reports_non_convergence():
    p = gen.cube_config(n=5)
    g = GpuRun(p)
    K, f = g.K.clone(), g.f.clone()
    g.pat.apply_penalty(K, f, t(p.fixed_dofs, torch.int64), t(p.fixed_vals))
    assert _status(lambda: g.pat.solve_pcg(K, f, max_iter=1)) == 6
    u, it, rr = g.pat.solve_pcg(K, f, rtol=1e-10)
    assert rr <= 1e-10


def test_non_finite_coordinate():
    p = gen.cube_config(n=5)
    xyz = p.xyz.copy()
    xyz[3, 1] = np.nan
    assert _status(lambda: R.Pattern(t(xyz), t(p.cell_lo), t(p.cell_hi), 2.5, 4.0, 1.03, 0.25)) == 7


def test_node_that_no_point_reaches_is_rejected_by_the_build():
    """A node whose coordinates lie far from every integration point (here
    moved out of the domain while its cell stays in place) appears in no
    support, so its row of K would be empty and K singular: the build reports
    RPIM_E_SUPPORT with the node's index, before any stage reads the row."""
    p = gen.cube_config(n=5)
    xyz = p.xyz.copy()
    xyz[0] = [3.0, 3.0, 3.0]
    with pytest.raises(R.RpimError) as e:
        R.Pattern(t(xyz), t(p.cell_lo), t(p.cell_hi), 2.5, 4.0, 1.03, 0.25)
    assert e.value.status == 4
    assert "index 0" in str(e.value)
    # the same cloud with the node in place builds and assembles
    g = GpuRun(p)
    assert g.pat.info.n_nodes == p.n_nodes
