"""The seeded input generators: their random stream and the workload recipes
(node counts, cells, jitter, loads and material fields of the five
workloads). No method arithmetic is involved; these fix the inputs every
parity test and benchmark line is computed on."""
import numpy as np
import pytest

import gen


def test_splitmix64_matches_the_published_sequence():
    # SplitMix64 (Steele, Lea and Flood 2014) from state 0: the reference
    # implementation's first outputs
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [int(v) for v in gen.splitmix64(0, 0, 4)] == want


def test_stream_is_counter_based():
    full = gen.splitmix64(7, 3, 100)
    assert np.array_equal(gen.splitmix64(7, 3, 40, start=60), full[60:])
    assert not np.array_equal(gen.splitmix64(7, 4, 100), full)
    assert not np.array_equal(gen.splitmix64(8, 3, 100), full)


def test_uniform_and_normal_moments():
    u = gen.uniform(11, 0, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / len(u))
    z = gen.normal(11, 1, 200000)
    assert abs(z.mean()) < 4 / np.sqrt(len(z))
    assert abs(z.var() - 1.0) < 4 * np.sqrt(2 / len(z))


def _check_cells_tile(p, volume):
    """Every node owns a box around its nominal position, and the boxes
    fill the domain's volume."""
    assert np.all(p.cell_hi > p.cell_lo)
    assert np.all((p.nominal >= p.cell_lo) & (p.nominal <= p.cell_hi))
    assert abs(p.volume - volume) < 1e-12 * volume


def _check_jitter(p, amp):
    """Face nodes on their faces, interior nodes within amp spacings of
    their nominal positions."""
    sp = np.array(p.extent) / (np.array(p.shape) - 1)
    d = np.abs(p.xyz - p.nominal) / sp
    assert d.max() <= amp + 1e-12
    ext = np.array(p.extent)
    on_face = np.isclose(p.nominal, 0.0) | np.isclose(p.nominal, ext)
    assert np.all(p.xyz[on_face] == p.nominal[on_face])


def _check_faces_tile(p, axis, plane, area):
    """Every face lies in the plane x_axis = plane, and the faces tile an area."""
    assert np.all(p.face_axis == axis)
    assert np.all(p.face_lo[:, axis] == plane) and np.all(p.face_hi[:, axis] == plane)
    ext = p.face_hi - p.face_lo
    ext[:, axis] = 1.0
    assert np.all(ext > 0)
    assert np.prod(ext, axis=1).sum() == pytest.approx(area, rel=1e-12)


def test_cube_workload():
    p = gen.cube_config()
    assert p.n_nodes == 216 and p.n_points == 1728
    assert p.h == pytest.approx(0.2) and p.alpha_s == 2.5 and p.alpha_c == 4.0 and p.q == 1.03
    _check_cells_tile(p, 1.0)
    # base fixed in all three directions; the pressure's resultant is 10 x area
    assert len(p.fixed_dofs) == 3 * 36
    # the pressure acts on the 36 top-face rectangles, which tile z = 1
    _check_faces_tile(p, 2, 1.0, 1.0)
    assert np.all(p.face_coef[:, 2, 0] == -10.0)
    assert np.count_nonzero(p.face_coef) == p.n_faces


def test_cantilever_workload():
    p = gen.cantilever_config()
    assert p.n_nodes == 129 * 17 * 17 == 37281 and p.n_points == 298248
    assert p.h == pytest.approx(1 / 16)
    _check_cells_tile(p, 8.0)
    _check_jitter(p, 0.2)
    # the parabolic shear t_z = -(3P/2)(1 - 4(z - 1/2)^2) = -6Pz + 6Pz^2 on
    # the end face x = 8, in the face coordinates (u, v) = (y, z)
    _check_faces_tile(p, 0, 8.0, 1.0)
    assert np.all(p.face_coef[:, 2, 2] == -6.0) and np.all(p.face_coef[:, 2, 5] == 6.0)
    assert np.count_nonzero(p.face_coef) == 2 * p.n_faces
    assert len(p.fixed_dofs) == 3 * 17 * 17


def test_slope_workload():
    p = gen.slope_config()
    assert p.n_nodes == 590500
    assert p.alpha_s == 3.0
    # three layers, stiffest at depth, gravity with unit weight 20
    z = np.repeat(p.nominal[:, 2], 8)
    assert set(np.unique(p.E)) == {5.0e3, 2.0e4, 8.0e4}
    assert p.E[z < 0.3].min() == 8.0e4 and p.E[z > 0.7].max() == 5.0e3
    assert p.body.tolist() == [0.0, 0.0, -20.0]
    _check_jitter(p, 0.2)


def test_batched_workload():
    ps = gen.batched_configs()
    assert len(ps) == 512
    n = np.array([p.n_nodes for p in ps])
    a = np.array([p.alpha_s for p in ps])
    assert n.sum() == 2774654 and n.min() >= 300 and n.max() <= 21000
    assert a.min() >= 2.0 and a.max() < 3.5
    E = np.array([p.meta["E"] for p in ps])
    assert E.min() >= 1e3 and E.max() <= 1e5
    for p in ps[::97]:
        _check_cells_tile(p, float(np.prod(p.extent)))
        _check_jitter(p, 0.2)
        _check_faces_tile(p, 2, 1.0, float(np.prod(p.extent[:2])))
        assert np.all(p.face_coef[:, 2, 0] == -p.meta["pressure"])


def test_backanalysis_workload():
    p = gen.backanalysis_config()
    assert p.n_nodes == 64 * 32 * 32 == 65536 and p.n_points == 524288
    logE = np.log(p.E)
    assert np.median(p.E) == pytest.approx(2.0e4, rel=0.15)
    assert logE.std() == pytest.approx(0.5, rel=0.2)
    assert p.nu.min() >= 0.2 and p.nu.max() <= 0.45
    obs = p.meta["obs_nodes"]
    assert 490 <= len(obs) <= 500 and obs.max() < p.n_nodes
    assert not np.array_equal(p.meta["E_hidden"], p.E)
    # correlation length 0.2: neighbouring integration points are strongly
    # correlated, points 1.0 apart nearly independent
    g = logE.reshape(32, 32, 64, 8)[:, :, :, 0]
    near = np.corrcoef(g[:, :, :-1].ravel(), g[:, :, 1:].ravel())[0, 1]
    far = np.corrcoef(g[:, :, :-32].ravel(), g[:, :, 32:].ravel())[0, 1]
    assert near > 0.7 and abs(far) < 0.1
