"""Pins of the oracle's site update (Eq. 2) and Lloyd loop (Algorithm 1).

- line of sight: hand-walked Amanatides-Woo traversals, including simultaneous crossings;
- closed case: with one band the whole box is one component and every voxel sees its
  site, so LSRVT reduces to a plain discrete Lloyd with the chamfer closed form; an
  independent numpy implementation of that Lloyd must give the same site trajectory;
- single seed: the cell is the whole component;
- invariants on a contorted volume: phi(v) is a line-of-sight voxel on v's parent chain,
  sites never leave their component, displacement statistics agree with the sites;
- convergence shape: the mean displacement falls steeply as in the paper's Fig.
  "convergence".
"""
import math
import os

import numpy as np
import pytest

W1, W2, W3 = 65536, 92682, 113512
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def lin(x, y, z, nx, ny):
    return x + nx * (y + ny * z)


def test_los_hand_cases(orc):
    nx, ny, nz = 5, 4, 3
    band = np.zeros((nz, ny, nx), np.uint8)
    # (0,0,0) -> (1,1,0): simultaneous crossing, x steps first through (1,0,0)
    band[0, 0, 1] = 1
    assert not orc.los(band, lin(0, 0, 0, nx, ny), lin(1, 1, 0, nx, ny))
    band[0, 0, 1] = 0
    band[0, 1, 0] = 1  # (0,1,0) is not on the traversal
    assert orc.los(band, lin(0, 0, 0, nx, ny), lin(1, 1, 0, nx, ny))
    # walked from (1,1,0) toward (0,0,0) the x step comes first and enters (0,1,0)
    assert not orc.los(band, lin(1, 1, 0, nx, ny), lin(0, 0, 0, nx, ny))
    band[:] = 0
    # (0,0,0) -> (3,1,0): crossings x at 1/6, 3/6, 5/6, y at 1/2 -> x, x(tie, x first), y, x
    # visits (1,0) (2,0) (2,1) (3,1); (1,1) and (3,0) are not visited
    band[0, 1, 1] = 1
    band[0, 0, 3] = 1
    assert orc.los(band, lin(0, 0, 0, nx, ny), lin(3, 1, 0, nx, ny))
    band[0, 1, 2] = 1
    assert not orc.los(band, lin(0, 0, 0, nx, ny), lin(3, 1, 0, nx, ny))
    band[:] = 0
    # 3D: (0,0,0) -> (1,1,1) steps x, y, z: (1,0,0) (1,1,0) (1,1,1)
    band[1, 0, 0] = 1
    band[0, 1, 0] = 1
    assert orc.los(band, lin(0, 0, 0, nx, ny), lin(1, 1, 1, nx, ny))
    band[0, 1, 1] = 1
    assert not orc.los(band, lin(0, 0, 0, nx, ny), lin(1, 1, 1, nx, ny))
    assert orc.los(band, lin(2, 2, 2, nx, ny), lin(2, 2, 2, nx, ny))


def _box_lloyd(shape, sites, n_iters):
    """Independent plain discrete Lloyd on a box with chamfer distances (numpy)."""
    nz, ny, nx = shape
    z, y, x = np.indices(shape)
    coords = np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.int64)
    sites = np.array(sites, np.int64)
    traj = [sites.copy()]
    for _ in range(n_iters + 1):
        sc = np.stack([sites % nx, (sites // nx) % ny, sites // (nx * ny)], 1)
        d = np.abs(coords[:, None, :] - sc[None, :, :])
        d = -np.sort(-d, axis=2)
        D = (d[..., 0] - d[..., 1]) * W1 + (d[..., 1] - d[..., 2]) * W2 + d[..., 2] * W3
        # lexicographic (distance, id): argmin returns the first minimum = lowest id
        cell = np.argmin(D, axis=1)
        if len(traj) == n_iters + 1:
            return traj, cell.reshape(shape), D[np.arange(len(cell)), cell].reshape(shape)
        new = sites.copy()
        for s in range(len(sites)):
            m = cell == s
            M = int(m.sum())
            if M == 0:
                continue
            S = coords[m].sum(0)
            t = (2 * S + M) // (2 * M)  # round half up
            new[s] = t[0] + nx * (t[1] + ny * t[2])  # box is convex: the full move is allowed
        sites = new
        traj.append(sites.copy())


def test_constant_field_is_plain_lloyd(orc):
    shape = (9, 10, 12)
    f = np.full(shape, 0.5, np.float32)
    band = orc.classify(f, np.array([0.1, 0.9], np.float32))
    comp, cb, cs, cf = orc.label_components(band)
    assert len(cb) == 1 and cs[0] == band.size
    sp, sc, off, nc = orc.seed(comp, None, 1, 90, 4, 17)
    traj, rcell, rdist = _box_lloyd(shape, sp, 4)
    cur = sp.copy()
    for it in range(4):
        cell, dist = orc.assign(band, cur)
        new, _, diag = orc.update(band, None, cell, dist, cur, diagnostics=True)
        assert diag["los"].all()  # convex component: everything in line of sight
        assert np.array_equal(new, traj[it + 1])
        cur = new
    sp4, cell, dist, tr = orc.cvt_iterate(band, None, sp, 4)
    assert np.array_equal(sp4, traj[4])
    assert np.array_equal(cell, rcell) and np.array_equal(dist, rdist)


def test_single_seed_cell_is_component(orc):
    rng = np.random.default_rng(3)
    f = np.cumsum(rng.standard_normal((8, 9, 10)), axis=1).astype(np.float32)
    band = orc.classify(f, np.array([0.0], np.float32))
    comp, cb, cs, cf = orc.label_components(band)
    sp, sc, off, nc = orc.seed(comp, None, len(cb), 10 ** 9, 16, 2)
    assert len(sp) == len(cb)
    sp2, cell, dist, tr = orc.cvt_iterate(band, None, sp, 3)
    assert np.array_equal(cell, comp)


def test_update_invariants_contorted(orc):
    rng = np.random.default_rng(8)
    import scipy.ndimage as ndi
    f = ndi.gaussian_filter(rng.standard_normal((14, 16, 18)), 1.5).astype(np.float32)
    band = orc.classify(f, np.array([-0.05, 0.05], np.float32))
    comp, cb, cs, cf = orc.label_components(band)
    q = orc.saliency(f, 1)
    sp, sc, off, nc = orc.seed(comp, q, len(cb), 40, 8, 5)
    cell, dist = orc.assign(band, sp)
    new, (moved, sumsq, sumlen), diag = orc.update(band, q, cell, dist, sp, diagnostics=True)
    nz, ny, nx = band.shape
    par, losv, phi = diag["parent"].ravel(), diag["los"].ravel(), diag["phi"].ravel()
    flat_d, flat_c = dist.ravel(), cell.ravel()
    assert (~losv).sum() > 0  # the case exercises propagation to phi
    for v in np.flatnonzero(flat_c >= 0):
        # phi(v) is the first line-of-sight voxel on the parent chain of v
        u = v
        while not losv[u]:
            assert par[u] != u and flat_c[par[u]] == flat_c[u] and flat_d[par[u]] < flat_d[u]
            u = par[u]
        assert phi[v] == u
        assert orc.los(band, u, sp[flat_c[v]])
    # moment sums reproduce Eq. 2 from phi
    coords = np.stack(np.unravel_index(phi[flat_c >= 0], band.shape)[::-1], 1)
    w = q.ravel()[flat_c >= 0].astype(np.int64)
    S = np.zeros((len(sp), 4), np.int64)
    np.add.at(S, (flat_c[flat_c >= 0], 0), w * coords[:, 0])
    np.add.at(S, (flat_c[flat_c >= 0], 1), w * coords[:, 1])
    np.add.at(S, (flat_c[flat_c >= 0], 2), w * coords[:, 2])
    np.add.at(S, (flat_c[flat_c >= 0], 3), w)
    assert np.array_equal(S, diag["sums"])
    # sites never leave their component; statistics match the positions
    assert np.array_equal(comp.ravel()[new], sc)
    d = np.stack(np.unravel_index(new, band.shape), 1) - np.stack(np.unravel_index(sp, band.shape), 1)
    assert moved == int((new != sp).sum()) and sumsq == int((d * d).sum())
    # d_s in 16.16 fixed point rounded up: the least r with r^2 >= 2^32 |d|^2 (integer root)
    r = [math.isqrt((int(v) << 32) - 1) + 1 if v else 0 for v in (d * d).sum(1)]
    assert sumlen == sum(r)


def test_selected_update_matches_full(orc):
    # restricting the update to a subset of cells gives those cells' sites exactly the
    # positions and sums of the full update (the replay used for full-size volumes)
    rng = np.random.default_rng(9)
    import scipy.ndimage as ndi
    f = ndi.gaussian_filter(rng.standard_normal((14, 16, 18)), 1.5).astype(np.float32)
    band = orc.classify(f, np.array([-0.05, 0.05], np.float32))
    comp, cb, cs, cf = orc.label_components(band)
    q = orc.saliency(f, 1)
    sp, sc, off, nc = orc.seed(comp, q, len(cb), 40, 8, 5)
    cell, dist = orc.assign(band, sp)
    new, _, diag = orc.update(band, q, cell, dist, sp, diagnostics=True)
    sel = rng.choice(len(sp), size=len(sp) // 3, replace=False)
    got, sums = orc.update_selected(band, q, cell, dist, sp, sel)
    assert np.array_equal(got, new[sel]) and np.array_equal(sums, diag["sums"][sel])
    assert (new[sel] != sp[sel]).any()


def test_convergence_shape_like_paper(orc):
    import workloads
    ref = {}
    for line in open(os.path.join(GOLDEN, "fig_convergence_mean_ds.txt")):
        if not line.startswith("#"):
            vps, k, ds = line.split()
            ref[(int(vps), int(k))] = float(ds)
    # the paper's series drop by more than 4x from update 1 to update 10
    assert all(ref[(v, 10)] < ref[(v, 1)] / 4 for v in (7142, 3571, 1786))
    w = workloads.blobs_workload(side=40, seed=4)
    f = w["field"].numpy()
    band = orc.classify(f, w["iso"])
    comp, cb, cs, cf = orc.label_components(band)
    sp, sc, off, nc = orc.seed(comp, None, len(cb), 512, 16, 4)
    nz, ny, nx = band.shape
    ds = []
    cur = sp.copy()
    for it in range(10):
        cell, dist = orc.assign(band, cur)
        new, _ = orc.update(band, None, cell, dist, cur)
        a = np.stack(np.unravel_index(cur, band.shape), 1)
        b = np.stack(np.unravel_index(new, band.shape), 1)
        ds.append(np.sqrt(((a - b) ** 2).sum(1)).mean())
        cur = new
    assert ds[9] < ds[0] / 4


# --------------------------------------------------------------------------- hand cases
def _plane(rows):
    """A one-voxel-thick volume (nz = 1) from strings of band digits, row y = 0 first."""
    return np.array([[[int(c) for c in r] for r in rows]], np.uint8)


def test_clipped_move_axis_aligned_hand_case(orc):
    """Eq. 2: the site walks toward the target and stops at the last voxel of its band
    ("move only as far as possible before crossing the boundary").  Two rows, a one-voxel
    wall of band 1 at (3, 0); the band-0 site at (0, 0).  By hand (the walk from (x, 1) to
    the site crosses x, then x/y ties x first): the LOS voxels are (0..2, 0) and (0..5, 1);
    (4, 0), (5, 0), (6, 0) take phi = (4, 1) and (6, 1) takes (5, 1).  Weights 6000 at
    (2, 0) and 4000 at (6, 0) (1 elsewhere) give S = (28029, 4009), M = 10011, target
    (3, 0) = the wall, so the site walks (1, 0), (2, 0) and stops at (2, 0)."""
    band = _plane(["0001000", "0000000"])
    nz, ny, nx = band.shape
    sp = np.array([lin(0, 0, 0, nx, ny), lin(3, 0, 0, nx, ny)], np.int32)
    q = np.ones(band.shape, np.uint16)
    q[0, 0, 2] = 6000
    q[0, 0, 6] = 4000
    cell, dist = orc.assign(band, sp)
    new, st, diag = orc.update(band, q, cell, dist, sp, diagnostics=True)
    phi = diag["phi"][0]
    assert phi[0, 4] == phi[0, 5] == phi[0, 6] == lin(4, 1, 0, nx, ny) and phi[1, 6] == lin(5, 1, 0, nx, ny)
    assert list(diag["sums"][0]) == [28029, 4009, 0, 10011]
    assert new[0] == lin(2, 0, 0, nx, ny)  # not (0, 0) (no move), (1, 0) (one short) or (3, 0) (the wall)
    assert new[1] == sp[1]  # the one-voxel wall is its own cell
    assert st[0] == 1 and st[1] == 4 and st[2] == 2 * 65536


def test_clipped_move_diagonal_hand_case(orc):
    """A diagonal walk clipped after six steps.  Band 0 = the axes of an 11 x 11 plane (row
    y = 0 and column x = 0) plus the strip |x - y| <= 1 inside [0, 3]^2; every band-0 voxel
    sees the site at (0, 0), so phi(v) = v.  Weights 60000 at (10, 0) and (0, 10) give
    S = (600059, 600059), M = 120026, target (5, 5).  The walk from (0, 0) toward (5, 5)
    takes x first on each tie: (1, 0), (1, 1), (2, 1), (2, 2), (3, 2), (3, 3), then (4, 3) is
    band 1, so the site stops at (3, 3)."""
    rows = []
    for y in range(11):
        r = ""
        for x in range(11):
            inside = (x == 0 or y == 0 or (x <= 3 and y <= 3 and abs(x - y) <= 1))
            r += "0" if inside else "1"
        rows.append(r)
    band = _plane(rows)
    nz, ny, nx = band.shape
    sp = np.array([lin(0, 0, 0, nx, ny), lin(8, 8, 0, nx, ny)], np.int32)
    q = np.ones(band.shape, np.uint16)
    q[0, 0, 10] = 60000
    q[0, 10, 0] = 60000
    cell, dist = orc.assign(band, sp)
    new, st, diag = orc.update(band, q, cell, dist, sp, diagnostics=True)
    assert diag["los"][band == 0].all()
    assert list(diag["sums"][0]) == [600059, 600059, 0, 120026]
    assert new[0] == lin(3, 3, 0, nx, ny)  # not (0,0), (3,2) (one short) or (5,5) (band 1)


def test_parent_tie_order_hand_case(orc):
    """parent(v) is the FIRST neighbour in (dz, dy, dx) order with an edge, the same site and
    D(u) + w = D(v).  Two rows, wall of band 1 at (3, 1), the band-0 site at (0, 1).  The
    voxel (6, 1) has two tied shortest parents: (5, 0) (offset dy = -1, dx = -1: first) and
    (5, 1) (dy = 0, dx = -1); D = 4 W1 + 2 W2 through either (D(5, 0) = 4 W1 + W2 plus a
    diagonal, D(5, 1) = 3 W1 + 2 W2 plus a face).  (5, 0) sees the site, (5, 1)
    does not (its walk meets the wall; its own parent is (4, 0)), so phi(6, 1) = (5, 0) and
    S_x = 36 by hand; taking the last tied parent would give phi = (4, 0) and S_x = 35.
    The mirror image in y (site (0, 0), wall (3, 0)) puts the non-seeing parent first:
    there (6, 0) takes (5, 0), whose phi is (4, 1)."""
    band = _plane(["0000000", "0001000"])
    nz, ny, nx = band.shape
    sp = np.array([lin(0, 1, 0, nx, ny), lin(3, 1, 0, nx, ny)], np.int32)
    cell, dist = orc.assign(band, sp)
    assert dist[0, 1, 6] == 4 * W1 + 2 * W2 and dist[0, 0, 5] == 4 * W1 + W2 and dist[0, 1, 5] == 3 * W1 + 2 * W2
    new, st, diag = orc.update(band, None, cell, dist, sp, diagnostics=True)
    par, phi, los = diag["parent"][0], diag["phi"][0], diag["los"][0]
    assert los[0, 5] and not los[1, 5] and not los[1, 6]
    assert par[1, 6] == lin(5, 0, 0, nx, ny) and phi[1, 6] == lin(5, 0, 0, nx, ny)
    assert par[1, 5] == lin(4, 0, 0, nx, ny) and phi[1, 5] == lin(4, 0, 0, nx, ny)
    assert list(diag["sums"][0]) == [36, 3, 0, 13]
    # mirror image: the first tied parent does not see the site
    band2 = band[:, ::-1, :].copy()
    sp2 = np.array([lin(0, 0, 0, nx, ny), lin(3, 0, 0, nx, ny)], np.int32)
    cell2, dist2 = orc.assign(band2, sp2)
    new2, st2, diag2 = orc.update(band2, None, cell2, dist2, sp2, diagnostics=True)
    par2, phi2 = diag2["parent"][0], diag2["phi"][0]
    assert par2[0, 6] == lin(5, 0, 0, nx, ny) and phi2[0, 6] == lin(4, 1, 0, nx, ny)
    assert list(diag2["sums"][0]) == [35, 10, 0, 13]


def test_lattice_lloyd_energy_never_increases(orc):
    """The theorem behind Lloyd's method, on the integer lattice of a box with the Euclidean
    metric: nearest-site assignment and the move to the centroid rounded half up (a nearest
    lattice point to the centroid) can each only lower E = sum |v - site(v)|^2.  The
    rounding is the update's own (centroid_round), so a wrong rounding shows up here."""
    rng = np.random.default_rng(21)
    for shape, k in (((6, 9, 11), 7), ((1, 13, 17), 5), ((8, 8, 8), 12), ((1, 1, 40), 4)):
        n = shape[0] * shape[1] * shape[2]
        sp = rng.choice(n, size=k, replace=False).astype(np.int32)
        out, e = orc.lattice_lloyd(shape, sp, 12)
        assert np.all(np.diff(e) <= 0), e
        assert e[-1] < e[0]
        # E of the final sites, recomputed by brute force
        nz, ny, nx = shape
        z, y, x = np.indices(shape)
        P = np.stack([x.ravel(), y.ravel(), z.ravel()], 1)
        Sxyz = np.stack([out % nx, (out // nx) % ny, out // (nx * ny)], 1)
        d2 = ((P[:, None, :] - Sxyz[None, :, :]) ** 2).sum(2)
        assert e[-1] == int(d2.min(1).sum())


def test_lattice_lloyd_hand_case(orc):
    """One dimension, ten voxels, sites at 0 and 1: cells {0} and {1..9}, E0 = 1^2 + ... + 8^2;
    the second site moves to 45 / 9 = 5; then cells {0, 1, 2} and {3..9} (voxel 2 is nearer
    0 than 5); then the sites move to 3 / 3 = 1 and 42 / 7 = 6."""
    out, e = orc.lattice_lloyd((1, 1, 10), np.array([0, 1], np.int32), 2)
    assert e[0] == sum(d * d for d in range(1, 9))  # voxel 0 at its site, 2..9 at distance 1..8
    # after one step: site 0 at 0, site 1 at round(45/9) = 5; cells {0,1,2}, {3..9}
    e1 = (0 + 1 + 4) + sum((v - 5) ** 2 for v in range(3, 10))
    assert e[1] == e1
    # then site 0 at round(3/3) = 1, site 1 at round(42/7) = 6; cells {0..3}, {4..9}
    e2 = sum((v - 1) ** 2 for v in range(0, 4)) + sum((v - 6) ** 2 for v in range(4, 10))
    assert e[2] == e2 and list(out) == [1, 6]


def test_trace_records_energy_and_ds(orc):
    """The Lloyd trace: energy = sum m_v D(v)^2 over the iteration's assignment (exact
    integers) and sum ceil(2^16 |d|) over the moved sites, recomputed in Python integers from
    the oracle's pinned assign/update steps."""
    import scipy.ndimage as ndi
    rng = np.random.default_rng(5)
    f = ndi.gaussian_filter(rng.standard_normal((12, 14, 16)), 1.5).astype(np.float32)
    band = orc.classify(f, np.array([-0.05, 0.05], np.float32))
    comp, cb, cs, cf = orc.label_components(band)
    q = orc.saliency(f, 1)
    sp, sc, off, nc = orc.seed(comp, q, len(cb), 30, 8, 3)
    sp4, cell, dist, tr = orc.cvt_iterate(band, q, sp, 4)
    cols = orc.trace_columns(tr)
    cur = sp.copy()
    for it in range(4):
        c, d = orc.assign(band, cur)
        new, st = orc.update(band, q, c, d, cur)
        m = c.ravel() >= 0
        e = sum(int(w) * int(x) * int(x) for w, x in zip(q.ravel()[m], d.ravel()[m]))
        assert cols["energy"][it] == e == orc.energy(q, c, d)
        a = np.stack(np.unravel_index(cur, band.shape), 1)
        b = np.stack(np.unravel_index(new, band.shape), 1)
        dd = ((a - b) ** 2).sum(1)
        assert cols["moved"][it] == int((dd > 0).sum()) and cols["sumsq"][it] == int(dd.sum())
        assert cols["sum_ds_q16"][it] == sum(math.isqrt((int(v) << 32) - 1) + 1 for v in dd if v)
        cur = new
    assert np.array_equal(cur, sp4)
    assert any(cols["energy"][i + 1] < cols["energy"][i] for i in range(3))


def test_energy_exact_beyond_64_bits(orc):
    """The energy is kept in 128 bits: one site in the corner of a 40^3 box with the largest
    weight everywhere gives a sum above 2^64, recomputed here in Python integers."""
    band = np.zeros((40, 40, 40), np.uint8)
    q = np.full(band.shape, 65535, np.uint16)
    cell, dist = orc.assign(band, np.array([0], np.int32))
    e = orc.energy(q, cell, dist)
    ref = 65535 * sum(int(x) * int(x) for x in dist.ravel())
    assert e == ref and e > 1 << 64
