"""The reciprocal the shape kernel takes of its LDL^T pivots and of the pivot
tetrahedron's determinant: two Newton-Raphson steps r <- r (2 - d r) from a
single-precision seed (a published method; the relative error squares at
every step). Against correctly rounded division 1/d it must be within one
ulp everywhere the kernel uses it: pivots of the reduced moment matrices
(1e-12 to 1e3 in the shape kernel's units), determinants of either sign,
and, for margin, all of [2^-126, 2^126] (where d and the single-precision
seed 1/d are normal numbers), with values next to powers of two where the
seed's truncation matters most.
"""
import numpy as np
import pytest
import torch

import gen
import paper_1802_04256_gb300 as R

pytestmark = pytest.mark.gpu


def _inputs():
    u = gen.uniform(12, 1, 200000, -12.0, 12.0)
    mid = 10.0 ** u                                      # pivots and determinants
    wide = np.exp2(gen.uniform(12, 2, 200000, -126.0, 126.0))
    k = np.arange(-126, 127, dtype=np.float64)
    twos = np.concatenate([np.exp2(k), np.nextafter(np.exp2(k), 0), np.nextafter(np.exp2(k), np.inf),
                           np.exp2(k) * 1.5, np.exp2(k) * (2 - 2.0 ** -30)])
    twos = twos[(twos >= 2.0 ** -126) & (twos <= 2.0 ** 126)]
    d = np.concatenate([mid, wide, twos])
    sign = np.where(gen.uniform(12, 3, len(d)) < 0.5, -1.0, 1.0)
    return d * sign


def test_recip_within_one_ulp_of_correctly_rounded_division():
    d = _inputs()
    r = R.rpim_probe_recip(torch.as_tensor(d, device="cuda")).cpu().numpy()
    want = 1.0 / d                                        # IEEE division, correctly rounded
    ulps = np.abs(r - want) / np.spacing(np.abs(want))
    print("recip: %d values, max %.3f ulp, %.4f%% not correctly rounded"
          % (len(d), ulps.max(), 100.0 * np.mean(r != want)))
    assert np.all(np.isfinite(r))
    assert ulps.max() <= 1.0
