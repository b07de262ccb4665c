"""rpim_stress_noalloc: stress recovery that allocates no device memory.

It exists for callers that cannot allocate device memory while they run
(hosts that fix and account their device-memory budget at start-up, or loops
that keep other streams busy and cannot accept the device synchronisation
that cudaMalloc/cudaFree may imply). It keeps its per-call scratch in one
fixed device array of the library, so its results must equal those of
rpim_stress, call after call, whatever the previous call left in that array.
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


@pytest.fixture(scope="module")
def solved():
    p = gen.cube_config(jitter=0.2, seed=5)
    g = GpuRun(p)
    u, it, rr, alpha, K, f = g.solve(rtol=1e-12)
    return p, g, u


def _points(p, count, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.02, 0.98, size=(count, 3))


def test_noalloc_stress_equals_stress_on_two_calls_in_a_row(solved):
    p, g, u = solved
    for call, (count, seed) in enumerate([(700, 1), (123, 2)]):
        xyz = t(_points(p, count, seed))
        E = t(np.full(count, 1.0e4))
        nu = t(np.full(count, 0.3))
        ref = g.pat.stress(u, xyz, E, nu)
        out = torch.full_like(ref, float("nan"))
        R.rpim_stress_noalloc(g.pat.handle, u, xyz, E, nu, out)
        torch.cuda.synchronize()
        scale = ref.abs().max().item()
        assert torch.isfinite(out).all(), "call %d left non-finite values" % call
        assert (out - ref).abs().max().item() <= 1e-12 * scale, "call %d differs" % call


def test_noalloc_stress_rejects_calls_beyond_its_limit(solved):
    p, g, u = solved
    n = 2049  # RPIM_NOALLOC_MAX_POINTS + 1
    xyz = t(_points(p, n, 3))
    E = t(np.full(n, 1.0e4))
    nu = t(np.full(n, 0.3))
    out = torch.zeros(n, 6, dtype=torch.float64, device="cuda")
    with pytest.raises(R.RpimError) as e:
        R.rpim_stress_noalloc(g.pat.handle, u, xyz, E, nu, out)
    assert e.value.status == 1
