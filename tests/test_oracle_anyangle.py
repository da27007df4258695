"""Pins of the oracle's any-angle tessellation (Sec. 3.2 region growing: each voxel weighs
the paths (v, P_w) and (v, P_src(w)) of its neighbours w, the latter only with a clear ray;
synchronous rounds until nothing changes) and of the Lloyd loop built on it (Eq. 2 with phi
following the src chain).

What pins it, independently of the oracle's code:
- one site in a box (convex for the ray traversal): every length is the straight segment,
  d(v) = ceil(2^16 |x_v - x_s|) (exact integer square roots here), src(v) = s, and the
  rounds equal the Chebyshev radius + 1 (the wave advances one voxel per round);
- a 1-D line: d = 2^16 times the distance to the nearest site, lower id on ties;
- any volume: ceil-Euclidean <= d <= the chamfer geodesic of the pinned `assign` (the direct
  neighbour paths are the chamfer edges), and d >= the brute-force shortest path of the
  visibility graph (every straight segment in band) on tiny grids;
- src chains: consistent lengths, same site, ending at the voxel's own site;
- one Lloyd step in a box equals the rounded centroid of each cell (numpy sums).
"""
import math

import numpy as np
import pytest

W = 65536


def ceil_len(dx, dy, dz):
    v = (dx * dx + dy * dy + dz * dz) << 32
    r = math.isqrt(v)
    return r if r * r == v else r + 1


def coords(i, shape):
    nz, ny, nx = shape
    return i % nx, (i // nx) % ny, i // (nx * ny)


def _blob_case(orc, seed, shape=(9, 11, 13), P=24):
    import scipy.ndimage as ndi
    rng = np.random.default_rng(seed)
    f = ndi.gaussian_filter(rng.standard_normal(shape), 1.3).astype(np.float32)
    f.ravel()[rng.integers(0, f.size, f.size // 40)] = np.nan
    band = orc.classify(f, np.array([-0.15, 0.1], np.float32))
    comp, cb, cs, cf = orc.label_components(band)
    sp, sc, off, nc = orc.seed(comp, None, len(cb), P, 4, seed)
    return band, comp, sp, sc


@pytest.mark.parametrize("shape,site", [((9, 10, 11), (5, 4, 3)), ((7, 1, 13), (0, 0, 6)), ((6, 8, 5), (4, 7, 5))])
def test_single_site_box_is_straight_line_distance(orc, shape, site):
    nz, ny, nx = shape
    band = np.zeros(shape, np.uint8)
    p = site[0] + nx * (site[1] + ny * site[2])
    cell, dist, src, rounds = orc.anyangle_assign(band, np.array([p], np.int32))
    assert np.all(cell == 0)
    for i in range(band.size):
        x, y, z = coords(i, shape)
        assert int(dist.ravel()[i]) == ceil_len(x - site[0], y - site[1], z - site[2])
        assert src.ravel()[i] == p
    cheb = max(max(site[0], nx - 1 - site[0]), max(site[1], ny - 1 - site[1]), max(site[2], nz - 1 - site[2]))
    assert rounds == cheb + 1


def test_box_inside_other_band(orc):
    # a box of band 1 inside band 0 with one site: closed form inside, band 0 unreached
    shape = (10, 9, 12)
    band = np.zeros(shape, np.uint8)
    band[2:8, 1:7, 3:10] = 1
    s = (5, 2, 4)
    p = s[0] + 12 * (s[1] + 9 * s[2])
    cell, dist, src, rounds = orc.anyangle_assign(band, np.array([p], np.int32))
    for i in range(band.size):
        x, y, z = coords(i, shape)
        if band.ravel()[i] == 1:
            assert int(dist.ravel()[i]) == ceil_len(x - s[0], y - s[1], z - s[2])
            assert cell.ravel()[i] == 0
        else:
            assert cell.ravel()[i] == -1 and dist.ravel()[i] == 0xFFFFFFFF and src.ravel()[i] == -1


def test_line_is_nearest_site(orc):
    n = 40
    band = np.zeros((n, 1, 1), np.uint8)
    band[17, 0, 0] = 255  # an invalid voxel splits the line
    sites = np.array([30, 3, 12, 8, 35, 22], np.int32)  # ids not in position order; 8/12 and 30/35 leave ties
    cell, dist, src, rounds = orc.anyangle_assign(band, sites)
    for i in range(n):
        if i == 17:
            assert cell[i, 0, 0] == -1
            continue
        same_side = [(abs(i - int(p)), k) for k, p in enumerate(sites) if (p < 17) == (i < 17)]
        dmin, kmin = min(same_side)
        assert dist[i, 0, 0] == dmin * W
        assert cell[i, 0, 0] == kmin


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bounds_chamfer_and_euclid(orc, seed):
    band, comp, sp, sc = _blob_case(orc, seed)
    cell, dist, src, rounds = orc.anyangle_assign(band, sp)
    ccell, cdist = orc.assign(band, sp)
    reached = cell >= 0
    assert np.array_equal(reached, ccell >= 0)
    assert np.all(dist[reached].astype(np.int64) <= cdist[reached].astype(np.int64))
    assert np.any(dist[reached] < cdist[reached])  # shortcuts do happen
    shape = band.shape
    for i in np.flatnonzero(reached.ravel()):
        s = int(cell.ravel()[i])
        x, y, z = coords(i, shape)
        px, py, pz = coords(int(sp[s]), shape)
        assert int(dist.ravel()[i]) >= ceil_len(x - px, y - py, z - pz)
        assert sc[s] == comp.ravel()[i]  # the cell stays in the voxel's component


@pytest.mark.parametrize("seed", [3, 4])
def test_src_chains(orc, seed):
    band, comp, sp, sc = _blob_case(orc, seed)
    cell, dist, src, rounds = orc.anyangle_assign(band, sp)
    shape = band.shape
    c, d, q = cell.ravel(), dist.ravel().astype(np.int64), src.ravel()
    for i in np.flatnonzero(c >= 0):
        v = int(i)
        steps = 0
        while d[v] > 0:
            u = int(q[v])
            assert c[u] == c[i]
            a, b = coords(v, shape), coords(u, shape)
            assert d[v] == d[u] + ceil_len(a[0] - b[0], a[1] - b[1], a[2] - b[2])
            v = u
            steps += 1
            assert steps <= band.size
        assert v == sp[c[i]] and q[v] == v


def _visibility_sssp(orc, band, sources):
    """Dijkstra over every pair of same-band voxels joined by a clear ray, lengths
    ceil(2^16 |.|): the shortest any-angle path any schedule could find (a chamfer edge is a
    clear ray too: the traversal of a diagonal step stays in the box it spans)."""
    import heapq
    shape = band.shape
    n = band.size
    flat = band.ravel()
    valid = [i for i in range(n) if flat[i] != 255]
    best = {}
    h = []
    for p in sources:
        best[int(p)] = 0
        heapq.heappush(h, (0, int(p)))
    done = set()
    while h:
        dv, v = heapq.heappop(h)
        if v in done:
            continue
        done.add(v)
        a = coords(v, shape)
        for u in valid:
            if u in done or flat[u] != flat[v]:
                continue
            b = coords(u, shape)
            if not orc.los(band, u, v):  # the segment u -> v, walked from u
                continue
            nd = dv + ceil_len(a[0] - b[0], a[1] - b[1], a[2] - b[2])
            if nd < best.get(u, 1 << 62):
                best[u] = nd
                heapq.heappush(h, (nd, u))
    out = np.full(n, -1, np.int64)
    for k, v in best.items():
        out[k] = v
    return out


def test_not_shorter_than_visibility_graph(orc):
    # a U-shaped slab: band 0 around a wall of band 1, one site at each end
    shape = (1, 12, 12)
    band = np.zeros(shape, np.uint8)
    band[0, 0:9, 5:7] = 1
    sites = np.array([2 + 12 * 1, 10 + 12 * 2], np.int32)
    cell, dist, src, rounds = orc.anyangle_assign(band, sites)
    vis = _visibility_sssp(orc, band, sites[:1])
    vis2 = _visibility_sssp(orc, band, sites[1:])
    lb = np.minimum(np.where(vis < 0, 1 << 62, vis), np.where(vis2 < 0, 1 << 62, vis2))
    flat = band.ravel()
    for i in range(band.size):
        if flat[i] == 0:
            assert int(dist.ravel()[i]) >= lb[i]
    # one site: behind the wall the path bends, so it is strictly longer than the segment
    c1, d1, s1, r1 = orc.anyangle_assign(band, sites[:1])
    i = 9 + 12 * 1
    assert int(d1.ravel()[i]) >= vis[i] > ceil_len(9 - 2, 1 - 1, 0)


def test_one_lloyd_step_in_a_box_is_the_rounded_centroid(orc):
    shape = (8, 9, 10)
    band = np.zeros(shape, np.uint8)
    rng = np.random.default_rng(5)
    sp = np.sort(rng.choice(band.size, 7, replace=False)).astype(np.int32)
    cell, dist, src, rounds = orc.anyangle_assign(band, sp)
    new, cell1, dist1, src1, trace, rr = orc.cvt_iterate_anyangle(band, None, sp, 1)
    z, y, x = np.indices(shape)
    for s in range(len(sp)):
        m = cell == s
        M = int(m.sum())
        if M == 0:
            assert new[s] == sp[s]
            continue
        t = [(2 * int(a[m].sum()) + M) // (2 * M) for a in (x, y, z)]
        assert new[s] == t[0] + shape[2] * (t[1] + shape[1] * t[2])
    assert rr[0] == rounds and rr[1] >= 1


def test_lloyd_invariants_on_blobs(orc):
    band, comp, sp, sc = _blob_case(orc, 7, shape=(8, 10, 12), P=20)
    q = np.random.default_rng(2).integers(1, 9, band.shape).astype(np.uint16)
    new, cell, dist, src, trace, rounds = orc.cvt_iterate_anyangle(band, q, sp, 3)
    cf = comp.ravel()
    assert np.all(cf[new] == sc)  # sites stay in their component
    ref_cell, ref_dist, ref_src, r2 = orc.anyangle_assign(band, new)
    assert np.array_equal(cell, ref_cell) and np.array_equal(dist, ref_dist) and np.array_equal(src, ref_src)
    assert rounds[-1] == r2
    assert np.all(trace[:, 0] >= 0)


def test_phi_follows_src_chain_behind_a_wall(orc):
    # a U-shaped slab and two sites on one side: voxels behind the wall have no line of sight,
    # so phi walks their src chain to the first node that sees the site (Eq. 2)
    shape = (2, 12, 13)
    band = np.zeros(shape, np.uint8)
    band[:, 0:9, 5:7] = 1
    sites = np.array([1 + 13 * 2, 3 + 13 * 6], np.int32)
    cell, dist, src, rounds = orc.anyangle_assign(band, sites)
    q = np.random.default_rng(3).integers(1, 5, shape).astype(np.uint16)
    new, st, diag = orc.update(band, q, cell, dist, sites, diagnostics=True, src=src)
    c, sr, qf = cell.ravel(), src.ravel(), q.ravel().astype(np.int64)
    sums = np.zeros((len(sites), 4), np.int64)
    hidden = 0
    for v in np.flatnonzero(c >= 0):
        s = int(c[v])
        u = int(v)
        steps = 0
        while not orc.los(band, u, int(sites[s])):
            u = int(sr[u])
            steps += 1
            assert steps <= band.size and c[u] == s
        hidden += u != v
        assert diag["phi"].ravel()[v] == u
        x, y, z = coords(u, shape)
        sums[s] += qf[v] * np.array([x, y, z, 1])
    assert hidden > 20
    assert np.array_equal(diag["sums"], sums)
    for s in range(len(sites)):
        t = [(2 * int(sums[s, k]) + int(sums[s, 3])) // (2 * int(sums[s, 3])) for k in range(3)]
        tp = t[0] + shape[2] * (t[1] + shape[1] * t[2])
        if orc.los(band, int(sites[s]), tp):  # the walk reaches an in-band target
            assert new[s] == tp


def test_symmetric_detour_takes_the_lower_source(orc):
    # a square pillar between the site and v: the detours left and right of it are mirror
    # images (the traversal's x-then-y tie rule is symmetric under x -> -x), so lengths are
    # mirror symmetric and v's two best sources tie in (length, site, d[src]); the lower voxel
    # index (the left side) wins
    n = 11
    band = np.zeros((1, n, n), np.uint8)
    band[0, 4:7, 4:7] = 1
    site = 5 + n * 1
    cell, dist, src, rounds = orc.anyangle_assign(band, np.array([site], np.int32))
    d2 = dist[0]
    assert np.array_equal(d2, d2[:, ::-1])
    v = 5 + n * 9
    sx, sy, sz = coords(int(src.ravel()[v]), band.shape)
    assert sx < 5
    m = (n - 1 - sx) + n * sy  # the mirrored source gives the same (length, site, d[src])
    assert dist.ravel()[m] == dist.ravel()[src.ravel()[v]]
