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
    new, (moved, sumsq), diag = orc.update(band, q, cell, dist, sp, diagnostics=True)
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
