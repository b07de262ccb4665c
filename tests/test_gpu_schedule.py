"""Schedules of the RPIM shape kernel and the graphed assembly.

The shape functions of a point are computed by one group of threads with a
fixed formula, so every schedule must give the same bits: one persistent
launch over all support-size buckets or one launch per bucket, any bucket
bounds (set by hand or picked by the bucket autotuner), and the assembly
replayed from a captured CUDA graph against the plain entry point.
"""
import numpy as np
import pytest
import torch

import gen
import paper_1802_04256_gb300 as R
from gpu_util import t

pytestmark = pytest.mark.gpu


def _batch():
    """Blocks with support radii 2.0-3.5 h: supports from ~8 to ~190 nodes,
    so the points fall into many buckets."""
    allp = gen.batched_configs(count=512)
    sel = [p for p in allp if p.n_nodes < 1500][:6]
    return sel


@pytest.fixture(scope="module")
def batched():
    sel = _batch()
    pat, offs = R.Pattern.batched(sel)
    E = t(np.concatenate([p.E for p in sel]))
    nu = t(np.concatenate([p.nu for p in sel]))
    yield pat, E, nu
    R.rpim_set_shape_schedule(True)
    R.rpim_autotune_reset()
    pat.free()


def _phi(pat):
    phi = pat.shape_functions()
    torch.cuda.synchronize()
    return phi


def test_persistent_equals_per_bucket_launches(batched):
    pat, E, nu = batched
    assert len([b for b in pat.buckets() if b[2] > 0]) >= 4
    R.rpim_set_shape_schedule(False)
    ref = _phi(pat)
    R.rpim_set_shape_schedule(True)
    assert torch.equal(_phi(pat), ref)
    K1, f1 = pat.assemble(E, nu)
    R.rpim_set_shape_schedule(False)
    K0, f0 = pat.assemble(E, nu)
    R.rpim_set_shape_schedule(True)
    assert torch.equal(K0, K1) and torch.equal(f0, f1)


def test_bucket_bounds_change_nothing(batched):
    pat, E, nu = batched
    ref = _phi(pat)
    for bounds in ([16, 24, 32, 40, 48, 56, 64, 72, 80, 96, 112, 128, 144, 160, 176, 192], [100], [30, 200]):
        R.rpim_pattern_set_buckets(pat.handle, bounds)
        bk = pat.buckets()
        assert sum(c for _, _, c in bk) == pat.info.n_points
        assert all(m <= b for b, m, c in bk[:-1])
        assert torch.equal(_phi(pat), ref), bounds
    chosen = pat.autotune_buckets(max_points=20000)
    assert chosen == sorted(set(chosen)) and len(chosen) >= 1
    assert torch.equal(_phi(pat), ref)
    R.rpim_pattern_set_buckets(pat.handle, [40, 56, 72, 96, 128, 160])


def test_bad_bucket_bounds_are_rejected(batched):
    pat, E, nu = batched
    for bad in ([40, 40], [56, 40], [0], list(range(1, 40))):
        with pytest.raises(R.RpimError) as e:
            R.rpim_pattern_set_buckets(pat.handle, bad)
        assert e.value.status == 1
    assert R.lib().rpim_set_shape_schedule(2) == 1


def test_graphed_assembly_equals_plain(batched):
    pat, E, nu = batched
    K0, f0 = pat.assemble(E, nu)
    K = torch.empty_like(K0)
    f = torch.empty_like(f0)
    n0 = R.rpim_kernel_launches()
    pat.assemble_graphed(E, nu, K=K, f=f)
    assert torch.equal(K, K0) and torch.equal(f, f0)
    # new material in the same buffers: the replay must see the new values
    E2, nu2 = E * 1.7, nu.clone()
    nu2[::3] = 0.25
    Ka, fa = pat.assemble(E2, nu2)
    E.copy_(E2)
    nu.copy_(nu2)
    pat.assemble_graphed(E, nu, K=K, f=f)
    assert torch.equal(K, Ka) and torch.equal(f, fa)
    assert R.rpim_kernel_launches() > n0
    # a change of the launch plan recaptures
    R.rpim_pattern_set_buckets(pat.handle, [48, 96, 144])
    pat.assemble_graphed(E, nu, K=K, f=f)
    assert torch.equal(K, Ka)
    R.rpim_set_shape_schedule(False)
    pat.assemble_graphed(E, nu, K=K, f=f)
    R.rpim_set_shape_schedule(True)
    assert torch.equal(K, Ka)
    R.rpim_pattern_set_buckets(pat.handle, [40, 56, 72, 96, 128, 160])


def test_graphed_assembly_single_instance_and_errors():
    p = gen.cube_config(jitter=0.2, seed=3)
    pat = R.Pattern.from_problem(p)
    E, nu = t(p.E), t(p.nu)
    K0, f0 = pat.assemble(E, nu)
    K, f = pat.assemble_graphed(E, nu)
    assert torch.equal(K, K0) and torch.equal(f, f0)
    nu_bad = nu.clone()
    nu_bad[5] = 0.6
    with pytest.raises(R.RpimError) as e:
        pat.assemble_graphed(E, nu_bad, K=K, f=f)
    assert e.value.status == 1
    K2, f2 = pat.assemble_graphed(E, nu, K=K, f=f)
    assert torch.equal(K2, K0)
    pat.free()

