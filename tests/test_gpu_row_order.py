"""Morton row order of the row-owner kernels.

rpim_build_pattern computes Morton keys of the nodes' grid cells (instance
first) and sorts them with a stable radix sort; the pattern passes and the
row kernel then take their rows in that order. Every row is computed the same
way in either order, so the pattern, K and f must be bitwise those of node
order; the order itself must be a permutation whose Morton keys, recomputed
here on the host from the same uniform grid, never decrease, with ids
ascending among equal keys.
"""
import math

import numpy as np
import pytest
import torch

import gen
import paper_1802_04256_gb300 as R
from gpu_util import faces, t

pytestmark = pytest.mark.gpu


def _morton(cx, cy, cz):
    m = np.zeros(len(cx), np.uint64)
    for b in range(11):
        m |= ((cx >> b) & 1).astype(np.uint64) << np.uint64(3 * b)
        m |= ((cy >> b) & 1).astype(np.uint64) << np.uint64(3 * b + 1)
        if b < 10:
            m |= ((cz >> b) & 1).astype(np.uint64) << np.uint64(3 * b + 2)
    return m


def _host_keys(p):
    """Cell coordinates on the uniform grid the library builds (origin at
    the nodes' lower bounding corner, edge r_s (1 + 1e-9)), Morton-coded."""
    lo = p.xyz.min(0)
    span = p.xyz.max(0) - lo
    edge = math.sqrt((p.alpha_s * p.h) ** 2) * (1.0 + 1e-9)
    n = np.floor(span / edge).astype(np.int64) + 1
    assert np.all(n[:2] <= 2047) and n[2] <= 1023
    c = np.floor((p.xyz - lo) * (1.0 / edge))
    c = np.minimum(np.maximum(c, 0), n - 1).astype(np.int64)
    return _morton(c[:, 0], c[:, 1], c[:, 2])


@pytest.mark.parametrize("name", ["cube", "beam"])
def test_morton_row_order_is_sorted_and_results_are_bitwise_node_order(name):
    p = gen.cube_config(jitter=0.2, seed=7) if name == "cube" else gen.cantilever_config(shape=(49, 7, 7))
    E, nu = t(p.E), t(p.nu)
    out = {}
    for morton in (1, 0):
        R.rpim_set_row_order(bool(morton))
        try:
            pat = R.Pattern.from_problem(p)
            K, f = pat.assemble(E, nu)
            pat.add_traction(*faces(p), f)
            rowptr, cols = pat.csr()
            out[morton] = (K, f, rowptr, cols, pat.row_order().cpu().numpy())
            pat.free()
        finally:
            R.rpim_set_row_order(True)
    for a, b in zip(out[1][:4], out[0][:4]):
        assert torch.equal(a, b)
    order = out[1][4]
    assert np.array_equal(np.sort(order), np.arange(p.n_nodes))
    keys = _host_keys(p)[order]
    assert np.all(keys[1:] >= keys[:-1])
    same = keys[1:] == keys[:-1]
    assert np.all(order[1:][same] > order[:-1][same])


def test_batched_row_order_keeps_instances_together():
    probs = gen.batched_configs(count=5, seed=5, lo_nodes=60, hi_nodes=400)
    pat, offs = R.Pattern.batched(probs)
    order = pat.row_order().cpu().numpy()
    inst = np.searchsorted(offs, order, side="right") - 1
    assert np.array_equal(np.sort(order), np.arange(offs[-1]))
    assert np.all(np.diff(inst) >= 0)
    for k, p in enumerate(probs):
        mine = order[inst == k] - offs[k]
        keys = _host_keys(p)[mine]
        assert np.all(keys[1:] >= keys[:-1])
    pat.free()
