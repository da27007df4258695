"""Pins of the oracle's per-cell statistics and hierarchy merge (Sec. 3.3 "Aggregation").

Per-cell statistics are pinned by numpy's own mean / var / min / max / cov on each cell
and by histogram bins of values away from bin edges; merges are pinned by the invariant
that merged cell statistics equal statistics computed directly over each component,
isoband and the volume.
"""
import numpy as np
import pytest


def _case(orc, seed=0, shape=(10, 12, 14), m=4):
    rng = np.random.default_rng(seed)
    import scipy.ndimage as ndi
    f = ndi.gaussian_filter(rng.standard_normal(shape), 1.2).astype(np.float32)
    band = orc.classify(f, np.array([-0.1, 0.1], np.float32))
    comp, cb, cs, cf = orc.label_components(band)
    sp, sc, off, nc = orc.seed(comp, None, len(cb), 25, 8, 3)
    cell, dist = orc.assign(band, sp)
    aux = rng.standard_normal((m,) + shape).astype(np.float32) * np.float32(3) + np.float32(100)
    aux[0] = f
    return band, comp, cb, sp, sc, cell, aux


def test_aggregate_matches_numpy(orc):
    band, comp, cb, sp, sc, cell, aux = _case(orc)
    m = aux.shape[0]
    st = orc.aggregate(cell, aux, len(sp), n_bins=16, cov=True)
    flat = cell.ravel()
    A = aux.reshape(m, -1).astype(np.float64)
    iu = np.triu_indices(m)
    for s in range(len(sp)):
        sel = flat == s
        n = int(sel.sum())
        assert st["count"][s] == n
        if n == 0:
            assert np.all(st["min"][s] == np.inf) and np.all(st["max"][s] == -np.inf)
            continue
        X = A[:, sel]
        np.testing.assert_allclose(st["mean"][s], X.mean(1), rtol=1e-13, atol=1e-12)
        np.testing.assert_allclose(st["m2"][s] / n, X.var(1), rtol=1e-10, atol=1e-12)
        assert np.array_equal(st["min"][s], aux.reshape(m, -1)[:, sel].min(1))
        assert np.array_equal(st["max"][s], aux.reshape(m, -1)[:, sel].max(1))
        C = np.cov(X, bias=True).reshape(m, m) * n
        np.testing.assert_allclose(st["comom"][s], C[iu], rtol=1e-9, atol=1e-9)
        assert st["hist"][s].sum(1).tolist() == [n] * m


def test_histogram_bins_away_from_edges(orc):
    cell = np.zeros((1, 1, 200), np.int32)
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, 200).astype(np.float32)
    x[0], x[1] = 0.0, 1.0  # range is exactly [0, 1]
    st = orc.aggregate(cell, x.reshape(1, 1, 1, 200), 1, n_bins=10)
    t = x.astype(np.float64) * 10
    ok = np.abs(t - np.round(t)) > 1e-4
    want = np.bincount(np.minimum(np.floor(t[ok]), 9).astype(int), minlength=10)
    # values next to an edge are excluded from the reference and removed from the counts
    got = st["hist"][0, 0].astype(np.int64)
    near = np.bincount(np.minimum(np.floor(t[~ok]), 9).astype(int), minlength=10)
    assert np.all(np.abs(got - want) <= near + np.roll(near, 1) + np.roll(near, -1))
    assert got.sum() == 200 and got[9] >= 1 and got[0] >= 1


def test_empty_cells_and_nonfinite(orc):
    cell = np.array([0, 0, 2, 2], np.int32).reshape(1, 1, 4)
    aux = np.array([1, 3, 5, 9], np.float32).reshape(1, 1, 1, 4)
    st = orc.aggregate(cell, aux, 3, n_bins=4)
    assert st["count"].tolist() == [2, 0, 2]
    assert st["mean"][:, 0].tolist() == [2.0, 0.0, 7.0] and st["m2"][:, 0].tolist() == [2.0, 0.0, 8.0]
    assert st["min"][1, 0] == np.inf and st["max"][1, 0] == -np.inf
    aux[0, 0, 0, 1] = np.nan
    with pytest.raises(orc.OracleError) as e:
        orc.aggregate(cell, aux, 3, n_bins=4)
    assert e.value.rc == -6


def test_merge_equals_direct(orc):
    band, comp, cb, sp, sc, cell, aux = _case(orc, seed=2)
    lo, hi, scale = orc.aux_range(cell, aux, 8)
    cells = orc.aggregate(cell, aux, len(sp), lo, scale, n_bins=8, cov=True)
    comps, bands, vol = orc.merge_hierarchy(cells, sc, cb, 3)
    direct_c = orc.aggregate(comp, aux, len(cb), lo, scale, n_bins=8, cov=True)
    bl = band.astype(np.int32)
    bl[band == 255] = -1
    direct_b = orc.aggregate(bl, aux, 3, lo, scale, n_bins=8, cov=True)
    direct_v = orc.aggregate(np.where(bl >= 0, 0, -1).astype(np.int32), aux, 1, lo, scale, n_bins=8, cov=True)
    for got, ref in ((comps, direct_c), (bands, direct_b), (vol, direct_v)):
        for k in ("count", "min", "max", "hist"):
            assert np.array_equal(got[k], ref[k]), k
        scale_m = np.maximum(np.abs(ref["mean"]), 1.0)
        assert np.all(np.abs(got["mean"] - ref["mean"]) <= 1e-12 * scale_m)
        assert np.all(np.abs(got["m2"] - ref["m2"]) <= 1e-10 * np.maximum(ref["m2"], 1.0))
        assert np.all(np.abs(got["comom"] - ref["comom"]) <= 1e-9 * np.maximum(np.abs(ref["comom"]), 1.0))
