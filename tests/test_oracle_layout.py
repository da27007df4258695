"""Pins of the oracle's structured data layout (Sec. 3.2 "Data Reduction and Structured Data
Layout", Fig. hierarchy: the kept data ordered by layer and connected component, each layer
and component contiguous and directly indexable).

The layout position of every voxel is recounted by brute force (the number of kept voxels
whose (band, component, cell, index) tuple is smaller: the definition of a stable sort, with
no sort call), every band / component / cell range is checked to hold exactly its kept voxels,
and the per-cell counts and means are tied to the oracle's own aggregate.
"""
import numpy as np


def _case(orc, seed=0, shape=(9, 11, 13), m=3, iso=(-0.1, 0.1)):
    rng = np.random.default_rng(seed)
    import scipy.ndimage as ndi
    f = ndi.gaussian_filter(rng.standard_normal(shape), 1.2).astype(np.float32)
    f[0, 0, :3] = np.nan  # not graph nodes: cell -1
    band = orc.classify(f, np.array(iso, np.float32))
    comp, cb, cs, cf = orc.label_components(band)
    sp, sc, off, nc = orc.seed(comp, None, len(cb), 20, 8, seed + 3)
    cell, dist = orc.assign(band, sp)
    aux = rng.standard_normal((m,) + shape).astype(np.float32) * np.float32(2) + np.float32(10)
    return band, comp, cb, sp, sc, cell, aux


def _brute_keep(cell, sc, cb, bands):
    flat = cell.ravel()
    out = []
    for v in range(flat.size):
        s = int(flat[v])
        if s < 0:
            continue
        b = int(cb[sc[s]])
        if bands is None or b in bands:
            out.append((b, int(sc[s]), s, v))
    return out


def test_positions_match_brute_force_rank(orc):
    band, comp, cb, sp, sc, cell, aux = _case(orc)
    lay = orc.layout(cell, sc, cb, aux)
    keys = _brute_keep(cell, sc, cb, None)
    assert lay["n_kept"] == len(keys)
    pos = {}
    for k in keys:  # rank = number of smaller tuples (no sort)
        pos[k[3]] = sum(1 for u in keys if u < k)
    want = np.empty(len(keys), np.int64)
    for v, p in pos.items():
        want[p] = v
    assert np.array_equal(lay["order"], want)
    A = aux.reshape(aux.shape[0], -1)
    assert np.array_equal(lay["values"], A[:, want])


def test_ranges_hold_exactly_their_voxels(orc):
    band, comp, cb, sp, sc, cell, aux = _case(orc, seed=1, iso=(-0.2, 0.0, 0.2))
    lay = orc.layout(cell, sc, cb, aux)
    order = lay["order"]
    flat_band, flat_comp, flat_cell = band.ravel(), comp.ravel(), cell.ravel()
    r = lay["n_kept"]
    assert lay["band_off"][256] == lay["comp_off"][-1] == lay["cell_off"][-1] == r
    for off in (lay["band_off"], lay["comp_off"], lay["cell_off"]):
        assert np.all(np.diff(off) >= 0) and off[0] == 0
    for b in range(255):  # 255 = not a node
        seg = order[lay["band_off"][b]:lay["band_off"][b + 1]]
        assert set(seg.tolist()) == set(np.nonzero(flat_band == b)[0].tolist())
    for c in range(len(cb)):
        seg = order[lay["comp_off"][c]:lay["comp_off"][c + 1]]
        assert set(seg.tolist()) == set(np.nonzero(flat_comp == c)[0].tolist())
    for s in range(len(sp)):
        seg = order[lay["cell_off"][s]:lay["cell_off"][s + 1]]
        assert set(seg.tolist()) == set(np.nonzero(flat_cell == s)[0].tolist())
        assert np.all(np.diff(seg) > 0)  # linear order inside a cell


def test_counts_and_means_agree_with_aggregate(orc):
    band, comp, cb, sp, sc, cell, aux = _case(orc, seed=2, m=4)
    lay = orc.layout(cell, sc, cb, aux)
    st = orc.aggregate(cell, aux, len(sp), n_bins=8)
    cnt = np.diff(lay["cell_off"])
    assert np.array_equal(cnt, st["count"])
    for s in range(len(sp)):
        if cnt[s]:
            seg = lay["values"][:, lay["cell_off"][s]:lay["cell_off"][s + 1]].astype(np.float64)
            np.testing.assert_allclose(seg.mean(1), st["mean"][s], rtol=1e-12)


def test_band_subsets(orc):
    band, comp, cb, sp, sc, cell, aux = _case(orc, seed=3, iso=(-0.2, 0.0, 0.2))
    none = orc.layout(cell, sc, cb, aux, bands=[])
    assert none["n_kept"] == 0 and not none["cell_off"].any() and not none["band_off"].any()
    full = orc.layout(cell, sc, cb, aux)
    assert full["n_kept"] == int((cell >= 0).sum())
    keep = [1, 3]
    sub = orc.layout(cell, sc, cb, aux, bands=keep)
    keys = _brute_keep(cell, sc, cb, set(keep))
    assert sub["n_kept"] == len(keys)
    assert np.array_equal(sub["order"], np.array([k[3] for k in sorted(keys)], np.int64))
    # an excluded band's components and cells are empty ranges at the right place
    for c in range(len(cb)):
        if int(cb[c]) not in keep:
            assert sub["comp_off"][c] == sub["comp_off"][c + 1]
    # the kept data is the full layout's band ranges, concatenated
    parts = [full["order"][full["band_off"][b]:full["band_off"][b + 1]] for b in keep]
    assert np.array_equal(sub["order"], np.concatenate(parts))


def test_order_does_not_depend_on_id_numbering(orc):
    # the oracle compares (band, component, cell, index) tuples: renumbering the cells of a
    # component reorders the cells inside it and nothing else
    band, comp, cb, sp, sc, cell, aux = _case(orc, seed=4)
    lay = orc.layout(cell, sc, cb, aux)
    S = len(sp)
    perm = np.arange(S)[::-1].copy()  # new id of old cell s
    sc2 = np.empty_like(sc)
    sc2[perm] = sc
    cell2 = np.where(cell >= 0, perm[np.maximum(cell, 0)], -1).astype(np.int32)
    lay2 = orc.layout(cell2, sc2, cb, aux)
    assert np.array_equal(lay["comp_off"], lay2["comp_off"])
    assert np.array_equal(lay["band_off"], lay2["band_off"])
    for c in range(len(cb)):
        a = lay["order"][lay["comp_off"][c]:lay["comp_off"][c + 1]]
        b = lay2["order"][lay2["comp_off"][c]:lay2["comp_off"][c + 1]]
        assert set(a.tolist()) == set(b.tolist())
    flat = cell.ravel()
    for s in range(S):
        k = int((flat == s).sum())  # the ranges are no longer in id order: start + count
        a = lay["order"][lay["cell_off"][s]:lay["cell_off"][s] + k]
        b = lay2["order"][lay2["cell_off"][perm[s]]:lay2["cell_off"][perm[s]] + k]
        assert np.array_equal(a, b)
