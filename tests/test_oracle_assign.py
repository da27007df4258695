"""Pins of the oracle's restricted geodesic Voronoi assignment (Eq. 1).

- brute force: an independent per-seed Dijkstra written here in Python, then the
  lexicographic minimum of (distance, site id) over seeds;
- closed form: on a box with one band the geodesic equals the 3D chamfer distance
  (a-b)W1 + (b-c)W2 + c W3 (a >= b >= c the sorted |delta|);
- hand case: a wall forces a detour;
- invariants: every voxel is assigned to a site of its own component; the Bellman
  certificate accepts the oracle's output and rejects perturbed outputs.
"""
import heapq
import itertools

import numpy as np
import pytest

W = {1: 65536, 2: 92682, 3: 113512}
OFFS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dx, dy, dz) != (0, 0, 0)]


def py_edge(band, x, y, z, dx, dy, dz):
    nz, ny, nx = band.shape
    if not (0 <= x + dx < nx and 0 <= y + dy < ny and 0 <= z + dz < nz):
        return False
    b = band[z, y, x]
    if b == 255:
        return False
    for ax in {0, dx}:
        for ay in {0, dy}:
            for az in {0, dz}:
                if band[z + az, y + ay, x + ax] != b:
                    return False
    return True


def py_sssp(band, src):
    nz, ny, nx = band.shape
    d = {src: 0}
    pq = [(0, src)]
    while pq:
        dv, v = heapq.heappop(pq)
        if dv != d.get(v):
            continue
        x, y, z = v % nx, (v // nx) % ny, v // (nx * ny)
        for dx, dy, dz in OFFS:
            if not py_edge(band, x, y, z, dx, dy, dz):
                continue
            u = (x + dx) + nx * ((y + dy) + ny * (z + dz))
            nd = dv + W[abs(dx) + abs(dy) + abs(dz)]
            if nd < d.get(u, 1 << 62):
                d[u] = nd
                heapq.heappush(pq, (nd, u))
    return d


def brute_assign(band, sites):
    n = band.size
    best = [(1 << 62, 1 << 30)] * n
    for s, p in enumerate(sites):
        for v, dv in py_sssp(band, int(p)).items():
            if (dv, s) < best[v]:
                best[v] = (dv, s)
    cell = np.array([s if d < (1 << 62) else -1 for d, s in best]).reshape(band.shape)
    dist = np.array([d if d < (1 << 62) else 0xFFFFFFFF for d, s in best], np.uint64).reshape(band.shape)
    return cell, dist


def chamfer(d):
    a, b, c = sorted(np.abs(d), reverse=True)
    return (a - b) * W[1] + (b - c) * W[2] + c * W[3]


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_assign_matches_per_seed_dijkstra(orc, seed):
    rng = np.random.default_rng(seed)
    shape = (6, 7, 8) if seed % 2 else (1, 10, 12)
    f = rng.standard_normal(shape).astype(np.float32)
    band = orc.classify(f, np.array([0.3], np.float32))
    band[rng.random(shape) < 0.03] = 255
    valid = np.flatnonzero(band.ravel() != 255)
    sites = rng.choice(valid, size=6, replace=False).astype(np.int32)
    sites = np.concatenate([sites, sites[:1]])  # a duplicate site: the higher id gets an empty cell
    cell, dist = orc.assign(band, sites)
    rc, rd = brute_assign(band, sites)
    assert np.array_equal(cell, rc)
    assert np.array_equal(dist.astype(np.uint64), rd)
    assert not np.any(cell == len(sites) - 1)


def test_assign_box_equals_chamfer_closed_form(orc):
    band = np.zeros((9, 9, 9), np.uint8)
    c0 = (4, 3, 5)  # x, y, z
    src = c0[0] + 9 * (c0[1] + 9 * c0[2])
    cell, dist = orc.assign(band, np.array([src], np.int32))
    for z, y, x in itertools.product(range(9), repeat=3):
        assert dist[z, y, x] == chamfer(np.array([x - c0[0], y - c0[1], z - c0[2]]))
    # the chamfer closed form is valid because of these inequalities
    assert W[1] + W[3] <= 2 * W[2] and W[3] <= W[1] + W[2] and W[2] <= 2 * W[1]


def test_assign_wall_detour(orc):
    # 2D slab (nz = 1): a wall of band 1 at x = 3 for y < 4 separates the site from (5, 0)
    band = np.zeros((1, 6, 7), np.uint8)
    band[0, :4, 3] = 1
    site = 0 + 7 * 0
    cell, dist = orc.assign(band, np.array([site], np.int32))
    # path: (0,0) -> diagonal up to (2,3)? no: (x=2,y=3) -> (3,4) needs box {(2,3),(3,3),(2,4),(3,4)} with (3,3) wall
    # so cross the gap row y = 4 through face moves: shortest is computed by brute force
    rc, rd = brute_assign(band, [site])
    assert np.array_equal(dist.astype(np.uint64), rd)
    assert dist[0, 0, 5] > chamfer(np.array([5, 0, 0]))  # longer than the straight line
    assert cell[0, 0, 3] == -1  # the wall is another component without a site


def test_assign_cells_stay_in_component(orc):
    rng = np.random.default_rng(5)
    f = rng.standard_normal((10, 11, 12)).astype(np.float32)
    band = orc.classify(f, np.array([-0.5, 0.5], np.float32))
    comp, cb, cs, cf = orc.label_components(band)
    sp, sc, off, nc = orc.seed(comp, None, len(cb), 20, 4, 1)
    cell, dist = orc.assign(band, sp)
    assert np.all(cell >= 0)
    assert np.array_equal(sc[cell], comp)
    assert orc.certify(band, sp, cell, dist) == 0
    bad = cell.copy()
    i = np.flatnonzero(cs[comp.ravel()] > 3)[0]
    other = np.flatnonzero(sc == comp.ravel()[i])
    bad.ravel()[i] = other[-1] if other[-1] != cell.ravel()[i] else other[0]
    if len(other) > 1:
        assert orc.certify(band, sp, bad, dist) >= 1
    d2 = dist.copy()
    d2.ravel()[i] += 1
    assert orc.certify(band, sp, cell, d2) >= 1
