"""The single-precision prefilter of the support search decides a candidate
only outside a band [q - m, q + m] around the squared support radius (in
squared cell edges) and leaves the band to the exact FP64 test. This checks,
on the CPU, that the margin m the library uses bounds the FP32 error: node
and point coordinates rounded to FP32 in cell edges from the grid origin,
differences and the sum of squares in FP32, against the exact FP64 test
((dx*dx + dy*dy) + dz*dz <= r_s^2, every operation rounded), on grids of up
to 2,000 cells per axis and candidates placed within a few ulps of the
radius. No GPU is involved; the GPU tests compare whole support sets with
the oracle's brute force."""
import numpy as np
import pytest


def margin(q, n_max):
    """The library's bound (pattern.cu, grid set-up), restated."""
    U = n_max + 2.0
    e24 = 2.0 ** -24
    W = 2.0002 * U + 2.01
    return 1.5 * (3.0 * e24 * (q + 12.2) + 6.0 * 2.01 * e24 * W + 3.0 * e24 * e24 * W * W + 1e-12)


def f32_fma(a, b, c):
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


CASES = [(60, 0.0625, 0.0), (400, 1.0, 1e3), (2000, 3e-3, -7.5), (2000, 50.0, 1e6)]


@pytest.mark.parametrize("n_cells,scale,offset", CASES)
def test_prefilter_never_contradicts_the_exact_test(n_cells, scale, offset, shrink=1.0):
    rng = np.random.default_rng(n_cells)
    rs = 2.5 * scale
    edge = rs * (1.0 + 1e-9)
    inv = 1.0 / edge
    lo = np.array([offset, offset * 0.5, -offset])
    q = rs * rs * inv * inv
    m = margin(q, n_cells) * shrink
    q32, m32 = np.float32(q), np.float32(m)
    qin, qout = np.float32(q32 - m32), np.float32(q32 + m32)
    bad = far_in_band = 0
    for _ in range(4000):
        # a point anywhere in the grid, a node at distance r_s (1 +- delta),
        # delta log-uniform in [1e-16, 0.2], in a random direction
        cell = rng.integers(1, n_cells - 2, 3)
        p = lo + (cell + rng.random(3)) * edge
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        delta = 10.0 ** rng.uniform(-16, -0.7)
        d = rs * (1.0 + rng.choice([-1, 1]) * delta)
        x = p + v * d
        dx = x - p
        exact = (dx[0] * dx[0] + dx[1] * dx[1]) + dx[2] * dx[2] <= rs * rs
        up = ((p - lo) * inv).astype(np.float32)
        un = ((x - lo) * inv).astype(np.float32)
        e = (un - up).astype(np.float32)
        d2 = f32_fma(e[2], e[2], f32_fma(e[1], e[1], np.float32(e[0] * e[0])))
        if d2 < qin:
            bad += not exact
        elif d2 > qout:
            bad += exact
        else:
            far_in_band += delta > 1e-2
    assert bad == 0
    # the band is narrow: a candidate more than 1% from the radius is always
    # decided in FP32 (the FP64 test only sees the thin shell around r_s)
    assert far_in_band == 0


def test_a_hundredfold_smaller_margin_is_caught():
    """The sample is fine enough to see the FP32 error: with the margin cut
    100-fold some candidate is decided against the exact test."""
    for args in CASES:
        with pytest.raises(AssertionError):
            test_prefilter_never_contradicts_the_exact_test(*args, shrink=0.01)
