"""The on-disk structured layout (Sec. 3.2 "Data Reduction and Structured Data Layout"):
summaries load first, then a band's / component's / cell's raw records are read through a
memory map of exactly their range."""
import numpy as np

from paper_2208_06970_b300 import store


def _case(orc, seed=5, shape=(10, 12, 14), m=3):
    rng = np.random.default_rng(seed)
    import scipy.ndimage as ndi
    f = ndi.gaussian_filter(rng.standard_normal(shape), 1.3).astype(np.float32)
    band = orc.classify(f, np.array([-0.15, 0.0, 0.15], np.float32))
    comp, cb, cs, cf = orc.label_components(band)
    sp, sc, off, nc = orc.seed(comp, None, len(cb), 30, 8, seed)
    cell, dist = orc.assign(band, sp)
    aux = rng.standard_normal((m,) + shape).astype(np.float32)
    return band, comp, cb, sp, sc, cell, aux


def test_roundtrip_and_selective_reads(orc, tmp_path):
    band, comp, cb, sp, sc, cell, aux = _case(orc)
    lay = orc.layout(cell, sc, cb, aux)
    cells = orc.aggregate(cell, aux, len(sp), n_bins=8)
    comps, bands, vol = orc.merge_hierarchy(cells, sc, cb, 4)
    path = str(tmp_path / "x.lsrvt")
    store.save(path, lay, len(sp), len(cb), stats=dict(cells=cells, comps=comps, bands=bands, volume=vol),
               meta=dict(isovalues=[-0.15, 0.0, 0.15]))
    st = store.open_store(path)
    assert st.meta["n_kept"] == lay["n_kept"] and st.meta["n_vars"] == 3
    assert st.meta["isovalues"] == [-0.15, 0.0, 0.15]
    s = st.summary("comps")
    assert np.array_equal(s["count"], comps["count"]) and np.array_equal(s["mean"], comps["mean"])
    assert np.array_equal(st.summary("cells")["hist"], cells["hist"])
    flat_comp, flat_band, flat_cell = comp.ravel(), band.ravel(), cell.ravel()
    A = aux.reshape(3, -1)
    for c in range(len(cb)):
        coords, vals = st.component(c)
        assert np.array_equal(np.sort(coords), np.nonzero(flat_comp == c)[0])
        assert np.array_equal(vals, A[:, coords])
    for b in range(4):
        coords, vals = st.band(b)
        assert set(coords.tolist()) == set(np.nonzero(flat_band == b)[0].tolist())
    for k in range(0, len(sp), max(1, len(sp) // 7)):
        coords, vals = st.cell(k)
        assert np.array_equal(coords, np.nonzero(flat_cell == k)[0])  # linear order inside a cell


def test_band_subset_file_is_smaller(orc, tmp_path):
    band, comp, cb, sp, sc, cell, aux = _case(orc, seed=6)
    full = orc.layout(cell, sc, cb, aux)
    sub = orc.layout(cell, sc, cb, aux, bands=[1])
    pf, ps = str(tmp_path / "f.lsrvt"), str(tmp_path / "s.lsrvt")
    store.save(pf, full, len(sp), len(cb))
    store.save(ps, sub, len(sp), len(cb))
    # r (m + 1) words of voxel records plus offsets: dropping bands drops their records
    r_full, r_sub = full["n_kept"], sub["n_kept"]
    assert r_sub < r_full
    assert store.file_bytes(pf) - store.file_bytes(ps) >= (r_full - r_sub) * 4 * (3 + 1) - 2 * 64 * 8
    st = store.open_store(ps)
    for b in (0, 2, 3):
        coords, vals = st.band(b)
        assert coords.size == 0
    coords, vals = st.band(1)
    assert np.array_equal(coords, sub["order"])
