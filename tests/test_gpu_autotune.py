"""The shape kernel's launch shape (warps per point, points per block) is a
speed choice only: every shape function is computed by one thread with a
fixed formula, the pivot searches break ties by index, and the one
reduction runs in a fixed warp. These tests force several launch shapes and
require bitwise-identical shape functions and K, then run the autotuner and
require the same again."""
import numpy as np
import pytest
import torch

import gen
from gpu_util import t

import paper_1802_04256_gb300 as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    probs = gen.batched_configs(count=8, seed=6, lo_nodes=60, hi_nodes=2000)
    pat, offs = R.Pattern.batched(probs)
    E = t(np.concatenate([p.E for p in probs]))
    nu = t(np.concatenate([p.nu for p in probs]))
    yield probs, pat, E, nu
    R.rpim_autotune_reset()


def _supports(pat):
    xyz, wj, soff, sidx = pat.points()
    return np.diff(soff.cpu().numpy())


def test_forced_launch_shapes_give_identical_results(batch):
    probs, pat, E, nu = batch
    R.rpim_autotune_reset()
    phi0 = pat.shape_functions().clone()
    K0, f0 = pat.assemble(E, nu)
    nmax = int(_supports(pat).max())
    tried = 0
    # force the shape for every support size where it is admissible (the
    # others keep the built-in rule), so each pass mixes launch shapes
    for G, ppb in [(1, 4), (2, 3), (3, 2), (4, 1), (1, 8), (2, 5), (8, 1), (16, 2), (12, 1)]:
        R.rpim_autotune_reset()
        n_set = 0
        for nc in range(8, nmax + 1):
            try:
                R.rpim_autotune_set(nc, G, ppb)
                n_set += 1
            except R.RpimError:
                pass
        if n_set == 0:
            continue
        phi = pat.shape_functions()
        K, f = pat.assemble(E, nu)
        assert torch.equal(phi, phi0), (G, ppb)
        assert torch.equal(K, K0), (G, ppb)
        tried += 1
    assert tried >= 6
    R.rpim_autotune_reset()


def test_autotuner_picks_admissible_shapes_and_keeps_K(batch):
    probs, pat, E, nu = batch
    R.rpim_autotune_reset()
    K0, f0 = pat.assemble(E, nu)
    table = pat.autotune(max_points=4096)
    print("tuned (largest support, warps per point, points per block):", table)
    assert len(table) >= 2
    for nc, G, ppb in table:
        assert 1 <= G <= 16 and 1 <= ppb <= 15 and G * ppb * 32 <= 768
    K, f = pat.assemble(E, nu)
    assert torch.equal(K, K0)
    assert torch.equal(f, f0)
    R.rpim_autotune_reset()


def test_inadmissible_shape_rejected():
    with pytest.raises(R.RpimError):
        R.rpim_autotune_set(200, 4, 15)   # 1920 threads
    with pytest.raises(R.RpimError):
        R.rpim_autotune_set(60, 16, 2)    # 1024 threads: above the FP64 solver's 768
    with pytest.raises(R.RpimError):
        R.rpim_autotune_set(100, 17, 1)   # more warps than the argmax buffers hold
    with pytest.raises(R.RpimError):
        R.rpim_autotune_set(216, 1, 15)   # shared memory of 15 large points
