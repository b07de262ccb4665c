"""rpim_stress_noalloc: stress recovery that allocates no device memory.

It exists for callers that cannot allocate device memory while they run
(hosts that fix and account their device-memory budget at start-up, or loops
that keep other streams busy and cannot accept the device synchronisation
that cudaMalloc/cudaFree may imply). It keeps its per-call scratch in one
fixed device array of the library, so its results must equal those of
rpim_stress, call after call, whatever the previous call left in that array,
and neither the library's allocation count nor the bytes in use in the
device's stream-ordered pool may change across a call.
This file is collected last so that a run stopping at the first failure has
run every other test before it.
"""
import numpy as np
import pytest
import torch

import gen
import paper_1802_04256_gb300 as R
from gpu_util import GpuRun, t

pytestmark = pytest.mark.gpu

MAX_POINTS = 2048        # RPIM_NOALLOC_MAX_POINTS
MAX_ENTRIES = 262144     # RPIM_NOALLOC_MAX_ENTRIES


@pytest.fixture(scope="module")
def solved():
    p = gen.cube_config(jitter=0.2, seed=5)
    g = GpuRun(p)
    u, it, rr, alpha, K, f = g.solve(rtol=1e-12)
    return p, g, u


def _points(p, count, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.02, 0.98, size=(count, 3))


def _noalloc(pat, u, xyz, E, nu, out):
    """One allocation-free call; asserts that it allocated nothing."""
    torch.cuda.synchronize()
    a0, b0 = R.rpim_device_allocations(), R.rpim_pool_used_bytes()
    try:
        R.rpim_stress_noalloc(pat.handle, u, xyz, E, nu, out)
    finally:
        torch.cuda.synchronize()
        assert R.rpim_device_allocations() == a0, "the call requested device memory"
        assert R.rpim_pool_used_bytes() == b0, "pool bytes in use changed across the call"


def test_noalloc_stress_equals_stress_on_two_calls_in_a_row(solved):
    p, g, u = solved
    for call, (count, seed) in enumerate([(700, 1), (123, 2)]):
        xyz = t(_points(p, count, seed))
        E = t(np.full(count, 1.0e4))
        nu = t(np.full(count, 0.3))
        a0 = R.rpim_device_allocations()
        ref = g.pat.stress(u, xyz, E, nu)
        assert R.rpim_device_allocations() > a0   # the allocating variant is counted
        out = torch.full_like(ref, float("nan"))
        _noalloc(g.pat, u, xyz, E, nu, out)
        scale = ref.abs().max().item()
        assert torch.isfinite(out).all(), "call %d left non-finite values" % call
        assert (out - ref).abs().max().item() <= 1e-12 * scale, "call %d differs" % call


def test_noalloc_stress_rejects_calls_beyond_its_point_limit(solved):
    p, g, u = solved
    n = MAX_POINTS + 1
    xyz = t(_points(p, n, 3))
    E = t(np.full(n, 1.0e4))
    nu = t(np.full(n, 0.3))
    out = torch.zeros(n, 6, dtype=torch.float64, device="cuda")
    with pytest.raises(R.RpimError) as e:
        _noalloc(g.pat, u, xyz, E, nu, out)
    assert e.value.status == 1


def test_noalloc_stress_rejects_calls_beyond_its_entry_limit_then_recovers():
    """2,000 points whose supports hold about 144 nodes each (support radius
    4.2h on the 6x6x6 cube, about 288,000 entries in all) need more than
    RPIM_NOALLOC_MAX_ENTRIES support entries: the call returns RPIM_E_ARG
    after counting, writes nothing, and the next call within the limits
    equals rpim_stress."""
    p = gen.cube_config(jitter=0.2, seed=5)
    p.alpha_s = 4.2
    pat = R.Pattern.from_problem(p)   # stress recovery needs the pattern only
    u = t(np.sin(np.arange(3 * p.n_nodes) * 0.37) * 1e-3)
    n = 2000
    xyz = t(_points(p, n, 4))
    E = t(np.full(n, 1.0e4))
    nu = t(np.full(n, 0.3))
    out = torch.zeros(n, 6, dtype=torch.float64, device="cuda")
    with pytest.raises(R.RpimError) as e:
        _noalloc(pat, u, xyz, E, nu, out)
    assert e.value.status == 1
    assert "entries" in str(e.value)
    m = 300   # about 43,000 entries
    xs, Es, nus = xyz[:m].contiguous(), E[:m].contiguous(), nu[:m].contiguous()
    ref = pat.stress(u, xs, Es, nus)
    out = torch.full_like(ref, float("nan"))
    _noalloc(pat, u, xs, Es, nus, out)
    assert (out - ref).abs().max().item() <= 1e-12 * ref.abs().max().item()
    pat.free()
