"""Pins of the oracle's isoband classification and connected-component labelling.

Classification (Sec. 3.1, B_{a,b} = {v : a < f(v) <= b}) is pinned by numpy's
searchsorted (count of isovalues strictly below f) and by hand cases at the band edges.
Component labelling (Sec. 3.1, 6-adjacency) is pinned by an independent union-find, by
scipy.ndimage.label, and by the adjacency / connectivity invariants.
"""
import numpy as np
import pytest
import scipy.ndimage as ndi


def test_classify_matches_searchsorted(orc):
    rng = np.random.default_rng(0)
    f = rng.uniform(-1, 2, size=(7, 9, 11)).astype(np.float32)
    iso = np.array([-0.5, 0.0, 0.25, 1.0, 1.5], np.float32)
    band = orc.classify(f, iso)
    ref = np.searchsorted(iso, f, side="left")  # number of isovalues < f
    assert np.array_equal(band, ref.astype(np.uint8))


def test_classify_edges_nan_and_signed_zero(orc):
    iso = np.array([0.0, 1.0], np.float32)
    f = np.array([-1.0, -0.0, 0.0, 1e-30, 1.0, np.nextafter(np.float32(1), np.float32(2)), np.inf, -np.inf,
                  np.nan], np.float32).reshape(1, 1, -1)
    band = orc.classify(f, iso).ravel().tolist()
    # a < f <= b: a value equal to an isovalue belongs to the band below it; -0 == +0
    assert band == [0, 0, 0, 1, 1, 2, 2, 0, 255]


def test_classify_argument_errors(orc):
    f = np.zeros((2, 2, 2), np.float32)
    with pytest.raises(orc.OracleError) as e:
        orc.classify(f, np.array([0.5, 0.5], np.float32))
    assert e.value.rc == -2
    with pytest.raises(orc.OracleError):
        orc.classify(f, np.array([1.0, 0.5], np.float32))
    with pytest.raises(orc.OracleError):
        orc.classify(f, np.array([np.nan], np.float32))
    with pytest.raises(orc.OracleError):
        orc.classify(f, np.arange(255, dtype=np.float32))
    assert orc.classify(f + 300, np.arange(254, dtype=np.float32)).max() == 254
    assert orc.classify(f, np.zeros(0, np.float32)).max() == 0


def _uf_components(band):
    """Independent union-find over 6-neighbour pairs; canonical ids (band, min index)."""
    nz, ny, nx = band.shape
    n = band.size
    par = list(range(n))

    def find(a):
        while par[a] != a:
            par[a] = par[par[a]]
            a = par[a]
        return a

    b = band.ravel()
    for v in range(n):
        if b[v] == 255:
            continue
        x, y, z = v % nx, (v // nx) % ny, v // (nx * ny)
        for (ok, u) in ((x + 1 < nx, v + 1), (y + 1 < ny, v + nx), (z + 1 < nz, v + nx * ny)):
            if ok and b[u] == b[v]:
                ra, rb = find(v), find(u)
                if ra != rb:
                    par[max(ra, rb)] = min(ra, rb)
    roots = {}
    for v in range(n):
        if b[v] != 255:
            r = find(v)
            roots.setdefault(r, v)
    order = sorted(roots, key=lambda r: (b[r], roots[r]))
    rid = {r: i for i, r in enumerate(order)}
    out = np.full(n, -1, np.int64)
    for v in range(n):
        if b[v] != 255:
            out[v] = rid[find(v)]
    return out.reshape(band.shape)


@pytest.mark.parametrize("seed,shape,nb", [(0, (6, 7, 8), 3), (1, (5, 5, 5), 2), (2, (1, 9, 13), 4),
                                           (3, (8, 1, 1), 2), (4, (4, 6, 5), 5)])
def test_ccl_matches_union_find(orc, seed, shape, nb):
    rng = np.random.default_rng(seed)
    band = rng.integers(0, nb, size=shape).astype(np.uint8)
    band[rng.random(shape) < 0.05] = 255
    comp, cb, cs, cf = orc.label_components(band)
    ref = _uf_components(band)
    assert np.array_equal(comp, ref)
    # per-component tables
    flat = comp.ravel()
    for c in range(len(cb)):
        idx = np.flatnonzero(flat == c)
        assert cs[c] == len(idx) and cf[c] == idx.min() and cb[c] == band.ravel()[idx[0]]


def test_ccl_matches_scipy_partition(orc):
    rng = np.random.default_rng(7)
    f = rng.standard_normal((12, 12, 12)).astype(np.float32)
    f = ndi.gaussian_filter(f, 1.0).astype(np.float32)
    band = orc.classify(f, np.array([-0.1, 0.0, 0.1], np.float32))
    comp, cb, cs, cf = orc.label_components(band)
    six = ndi.generate_binary_structure(3, 1)
    total = 0
    for b in range(4):
        lab, k = ndi.label(band == b, structure=six)
        total += k
        for i in range(1, k + 1):
            ids = np.unique(comp[lab == i])
            assert len(ids) == 1 and cb[ids[0]] == b
    assert total == len(cb)
    # canonical order: (band, first index) strictly increasing
    keys = list(zip(cb.tolist(), cf.tolist()))
    assert keys == sorted(keys)


def test_ccl_capacity_reports_count(orc):
    band = np.zeros((2, 2, 2), np.uint8)
    band.ravel()[::2] = 1  # checkerboard along x only -> columns
    comp, cb, cs, cf = orc.label_components(band)
    with pytest.raises(orc.OracleError) as e:
        orc.label_components(band, max_comp=len(cb) - 1)
    assert e.value.rc == -3


def test_ccl_checkerboard_gives_single_voxel_components(orc):
    z, y, x = np.indices((4, 5, 6))
    band = ((x + y + z) % 2).astype(np.uint8)
    comp, cb, cs, cf = orc.label_components(band)
    assert len(cb) == band.size and np.all(cs == 1)
