"""The algorithmic work model behind the bench's roofline fractions.

The shape-function work of one point is textbook RPIM arithmetic (Sec. 1):
the moment matrix of the n support nodes plus the linear polynomial
(order N = n + 4, one flop per kernel evaluation), its LU factorisation and
four solves; the stiffness work is 45 flops per upper pair of support nodes
(B^T D B for isotropic D, diagonal included). The totals per point are
checked against independently tabulated values of the same model
(F(34) = 8.1e4, F(65) = 3.8e5, F(113) = 1.5e6, F(180) = 5.3e6, each to two
significant digits), and the parts against their closed forms.
"""
import numpy as np

import bench


def test_per_point_totals_match_the_tabulated_model():
    for n, ref in ((34, 8.1e4), (65, 3.8e5), (113, 1.5e6), (180, 5.3e6)):
        total = float(bench.shape_flops(n) + bench.pair_flops(n))
        assert abs(total - ref) <= 0.05 * ref, (n, total)


def test_parts_are_their_closed_forms():
    n = np.arange(4, 220)
    N = n + 4
    lu = 2 * N**3 / 3                    # LU of the order-N moment matrix
    solves = 8 * N**2                    # four forward/back substitutions
    matrix = 5 * n * (n - 1) + 16 * n    # kernel values and right-hand sides
    assert np.allclose(bench.shape_flops(n), lu + solves + matrix, rtol=0, atol=1e-6)
    assert np.allclose(bench.pair_flops(n), 45 * n * (n + 1) / 2, rtol=0, atol=1e-6)
