"""Pins of the oracle's joint central moments of orders 2..4 (coskewness and cokurtosis sums;
the joint-plot section compares mean, covariance, coskewness and cokurtosis of summaries with
the raw data) and of their pairwise merge up the hierarchy (Pebay 2008).

Pinned by numpy's einsum of the deviation tensors, a two-point closed form, vanishing odd
moments of point-symmetric data, shift invariance, and the invariant that merged cell records
equal the records computed directly over each component and band.
"""
from itertools import combinations_with_replacement as cwr

import numpy as np


def _tuples(m, q):
    return list(cwr(range(m), q))


def _direct(X):
    """X: (n, m) float64 -> (mean, m2, m3, m4) by einsum of the deviations."""
    mu = X.mean(0) if len(X) else np.zeros(X.shape[1])
    D = X - mu
    m = X.shape[1]
    T2 = np.einsum("ni,nj->ij", D, D)
    T3 = np.einsum("ni,nj,nk->ijk", D, D, D)
    T4 = np.einsum("ni,nj,nk,nl->ijkl", D, D, D, D)
    return (mu, np.array([T2[t] for t in _tuples(m, 2)]), np.array([T3[t] for t in _tuples(m, 3)]),
            np.array([T4[t] for t in _tuples(m, 4)]))


def test_ranges_match_einsum(orc):
    rng = np.random.default_rng(0)
    m, n = 4, 300
    aux = (rng.standard_normal((m, n)) * np.array([[1.0], [2.0], [0.5], [3.0]]) + 5).astype(np.float32)
    order = rng.permutation(n).astype(np.int32)
    off = np.array([0, 1, 2, 40, 40, 170, 300])  # includes an empty range and single voxels
    rec = orc.joint_moments(aux, order, off)
    for r in range(len(off) - 1):
        sel = order[off[r]:off[r + 1]]
        X = aux[:, sel].T.astype(np.float64)
        assert rec["count"][r] == len(sel)
        if len(sel) == 0:
            assert not rec["m2"][r].any() and not rec["m4"][r].any()
            continue
        mu, M2, M3, M4 = _direct(X)
        np.testing.assert_allclose(rec["mean"][r], mu, rtol=1e-13)
        for got, ref in ((rec["m2"][r], M2), (rec["m3"][r], M3), (rec["m4"][r], M4)):
            np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-9 * np.abs(ref).max())


def test_two_point_closed_form(orc):
    a = np.array([1.0, -2.0, 0.5], np.float32)
    b = np.array([3.0, 2.0, -1.5], np.float32)
    aux = np.stack([a, b], 1)  # (m, 2)
    rec = orc.joint_moments(aux, np.array([0, 1]), np.array([0, 2]))
    D = (b - a).astype(np.float64)
    for q, key, scale in ((2, "m2", 2 / 4), (4, "m4", 2 / 16)):
        want = [scale * np.prod(D[list(t)]) for t in _tuples(3, q)]
        np.testing.assert_allclose(rec[key][0], want, rtol=1e-15)
    assert np.all(np.abs(rec["m3"][0]) < 1e-12)


def test_point_symmetric_data_has_no_third_moments(orc):
    rng = np.random.default_rng(1)
    half = rng.integers(-8, 9, size=(3, 50)).astype(np.float32)
    c = np.array([[10.0], [-3.0], [0.25]], np.float32)
    aux = np.concatenate([c + half, c - half], 1)  # x and its mirror image about c
    rec = orc.joint_moments(aux, np.arange(100), np.array([0, 100]))
    assert np.all(rec["m3"][0] == 0.0)  # small integers: every sum is exact
    assert np.all(rec["m4"][0][[0, 9, 14]] > 0)  # the pure fourth moments of each variable


def test_shift_invariance(orc):
    rng = np.random.default_rng(2)
    base = rng.integers(-20, 21, size=(2, 64)).astype(np.float32)
    r0 = orc.joint_moments(base, np.arange(64), np.array([0, 64]))
    r1 = orc.joint_moments(base + np.float32(1000.0), np.arange(64), np.array([0, 64]))
    for k in ("m2", "m3", "m4"):
        np.testing.assert_allclose(r1[k], r0[k], rtol=1e-12, atol=1e-9)


def test_merge_equals_direct_over_the_union(orc):
    rng = np.random.default_rng(3)
    import scipy.ndimage as ndi
    shape = (9, 10, 11)
    f = ndi.gaussian_filter(rng.standard_normal(shape), 1.2).astype(np.float32)
    band = orc.classify(f, np.array([-0.1, 0.1], np.float32))
    comp, cb, cs, cf = orc.label_components(band)
    sp, sc, off, nc = orc.seed(comp, None, len(cb), 25, 8, 5)
    cell, dist = orc.assign(band, sp)
    m = 3
    aux = (rng.standard_normal((m,) + shape) * 2 + np.array([1, 50, -7]).reshape(3, 1, 1, 1)).astype(np.float32)
    lay = orc.layout(cell, sc, cb, aux)
    cells = orc.joint_moments(aux, lay["order"], lay["cell_off"])
    comps = orc.joint_merge(cells, off.astype(np.int64))
    direct_c = orc.joint_moments(aux, lay["order"], lay["comp_off"])
    band_first = np.searchsorted(cb, np.arange(4))
    bands = orc.joint_merge(comps, band_first.astype(np.int64))
    direct_b = orc.joint_moments(aux, lay["order"], lay["band_off"][:4])
    for got, ref in ((comps, direct_c), (bands, direct_b)):
        assert np.array_equal(got["count"], ref["count"])
        np.testing.assert_allclose(got["mean"], ref["mean"], rtol=1e-12, atol=1e-12)
        for k in ("m2", "m3", "m4"):
            scale = np.abs(ref[k]).max()
            np.testing.assert_allclose(got[k], ref[k], rtol=1e-9, atol=1e-10 * scale)
