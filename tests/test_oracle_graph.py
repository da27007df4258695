"""Pins of the oracle's Voronoi site graph and geodesic site distances (the "Voronoi Cell Views"
section: site connectivity from region adjacency, shortest paths between adjacent sites inside a
component, and the distance ||x_i - x_j|| / gd(s_i, s_j)).

Edges are recounted by comparing shifted label volumes (no per-voxel loop shared with the
oracle); weights are checked with exact integer arithmetic; shortest paths against
Floyd-Warshall; path lengths against the straight-line lower bound.
"""
import numpy as np


def _case(orc, seed=0, shape=(10, 12, 14), P=30):
    rng = np.random.default_rng(seed)
    import scipy.ndimage as ndi
    f = ndi.gaussian_filter(rng.standard_normal(shape), 1.4).astype(np.float32)
    band = orc.classify(f, np.array([-0.1, 0.1], np.float32))
    comp, cb, cs, cf = orc.label_components(band)
    sp, sc, off, nc = orc.seed(comp, None, len(cb), P, 8, seed)
    cell, dist = orc.assign(band, sp)
    return band, comp, cb, sp, sc, cell


def _brute_edges(cell, band):
    pairs = set()
    for ax in range(3):
        a = np.moveaxis(cell, ax, 0)
        b = np.moveaxis(band, ax, 0)
        ca, cb_ = a[:-1].ravel(), a[1:].ravel()
        ba, bb = b[:-1].ravel(), b[1:].ravel()
        sel = (ca >= 0) & (cb_ >= 0) & (ca != cb_) & (ba == bb)
        for x, y in zip(ca[sel], cb_[sel]):
            pairs.add((min(x, y), max(x, y)))
    return sorted(pairs)


def test_edges_are_face_adjacent_cells_of_one_component(orc):
    band, comp, cb, sp, sc, cell = _case(orc)
    g = orc.site_graph(cell, band, sp)
    want = _brute_edges(cell, band)
    assert [tuple(e) for e in g["edges"].tolist()] == want
    assert np.all(sc[g["edges"][:, 0]] == sc[g["edges"][:, 1]])
    # the CSR holds each edge in both directions
    S = len(sp)
    deg = np.diff(g["off"])
    assert deg.sum() == 2 * len(want)
    for a in range(S):
        nbr = g["dst"][g["off"][a]:g["off"][a + 1]]
        assert np.all(np.diff(nbr) > 0)
        for b in nbr:
            assert a in g["dst"][g["off"][b]:g["off"][b + 1]]


def test_weights_are_ceiled_euclidean_lengths(orc):
    for d in [(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 1, 1), (3, 4, 0), (7, -5, 2), (-300, 250, 123), (1000, 1000, 1000)]:
        w = orc.site_weight(*d)
        D = d[0] ** 2 + d[1] ** 2 + d[2] ** 2
        v = D << 32
        assert (w - 1) ** 2 < v <= w ** 2 or (D == 0 and w == 0)


def test_shortest_paths_match_floyd_warshall(orc):
    band, comp, cb, sp, sc, cell = _case(orc, seed=1, P=20)
    g = orc.site_graph(cell, band, sp)
    S = len(sp)
    INF = np.iinfo(np.uint64).max
    M = np.full((S, S), np.inf)
    np.fill_diagonal(M, 0)
    for (a, b), w in zip(g["edges"], g["weight"]):
        M[a, b] = M[b, a] = float(w)
    for k in range(S):
        M = np.minimum(M, M[:, k:k + 1] + M[k:k + 1, :])
    for s in range(S):
        d = orc.site_sssp(g, s)
        want = np.where(np.isinf(M[s]), INF, M[s]).astype(np.float64)
        got = np.where(d == INF, np.inf, d.astype(np.float64))
        assert np.array_equal(np.isinf(got), np.isinf(M[s]))
        fin = ~np.isinf(got)
        assert np.array_equal(got[fin], want[fin])
        # reachable exactly within the source's component
        assert np.array_equal(fin, sc == sc[s])


def test_paths_are_no_shorter_than_straight_lines(orc):
    band, comp, cb, sp, sc, cell = _case(orc, seed=2, P=25)
    g = orc.site_graph(cell, band, sp)
    nx, ny = cell.shape[2], cell.shape[1]
    P = np.stack([sp % nx, (sp // nx) % ny, sp // (nx * ny)], 1).astype(np.float64)
    for s in range(0, len(sp), 3):
        d = orc.site_sssp(g, s)
        fin = d != np.iinfo(np.uint64).max
        eu = np.linalg.norm(P[fin] - P[s], axis=1) * 65536.0
        assert np.all(d[fin].astype(np.float64) >= eu - 1e-6)
        # the paper's distance ||x_i - x_j|| / gd lies in (0, 1] between distinct connected sites
        other = fin.copy()
        other[s] = False
        if other.any():
            ratio = np.linalg.norm(P[other] - P[s], axis=1) * 65536.0 / d[other].astype(np.float64)
            assert np.all((ratio > 0) & (ratio <= 1.0 + 1e-12))
