"""The packed batch's exactness argument, checked on the oracle alone (no GPU): independent blocks
(Discussion "Block Based Distributed Parallelism") placed in one volume at least one voxel of
band 0xFF apart, with their sites renumbered block after block and moved by the block's
origin, give under Algorithm 1 (Eq. 1 assignment, Eq. 2 update) each block the cells,
distances and sites it gets alone, and a trace that is the sum of the blocks' traces.  A
control shows the gap is what makes it exact: two blocks of one band placed face to face
interact."""
import numpy as np
import pytest

import workloads
from paper_2208_06970_b300.runtime import pack_layout


def _energy(t):
    return ((int(t[4]) & (2 ** 64 - 1)) << 64) | (int(t[3]) & (2 ** 64 - 1))


def _pack(blocks, origins, ext, weighted):
    NX, NY, NZ = ext
    pband = np.full((NZ, NY, NX), 255, np.uint8)
    pq = np.zeros((NZ, NY, NX), np.uint16) if weighted else None
    psp, base = [], [0]
    for b, (x0, y0, z0) in zip(blocks, origins):
        nz, ny, nx = b["band"].shape
        pband[z0:z0 + nz, y0:y0 + ny, x0:x0 + nx] = b["band"]
        if weighted:
            pq[z0:z0 + nz, y0:y0 + ny, x0:x0 + nx] = b["q"]
        sp = b["sp"].astype(np.int64)
        x, y, z = sp % nx, (sp // nx) % ny, sp // (nx * ny)
        psp.append(((x + x0) + NX * ((y + y0) + NY * (z + z0))).astype(np.int32))
        base.append(base[-1] + len(sp))
    return pband, pq, np.concatenate(psp), base


def _run_and_compare(orc, blocks, origins, ext, weighted, n_iters):
    NX, NY, NZ = ext
    pband, pq, psp, base = _pack(blocks, origins, ext, weighted)
    sp2, cell, dist, trace = orc.cvt_iterate(pband, pq, psp, n_iters)
    sums = np.zeros((n_iters, 3), np.int64)
    energy = [0] * n_iters
    inside = np.zeros(pband.shape, bool)
    same = True
    for k, (b, (x0, y0, z0)) in enumerate(zip(blocks, origins)):
        nz, ny, nx = b["band"].shape
        spb, cellb, distb, trb = orc.cvt_iterate(b["band"], b["q"] if weighted else None, b["sp"], n_iters)
        sub = (slice(z0, z0 + nz), slice(y0, y0 + ny), slice(x0, x0 + nx))
        inside[sub] = True
        same &= np.array_equal(cell[sub], np.where(cellb >= 0, cellb + base[k], -1))
        same &= np.array_equal(dist[sub], distb)
        p = sp2[base[k]:base[k + 1]].astype(np.int64)
        X, Y, Z = p % NX, (p // NX) % NY, p // (NX * NY)
        same &= np.array_equal((X - x0) + nx * ((Y - y0) + ny * (Z - z0)), spb)
        sums += trb[:, :3]
        for it in range(n_iters):
            energy[it] += _energy(trb[it])
    trace_sum = np.array_equal(sums, trace[:, :3]) and energy == [_energy(trace[it]) for it in range(n_iters)]
    gaps_empty = bool(np.all(cell[~inside] == -1))
    return same, trace_sum, gaps_empty


@pytest.mark.parametrize("weighted", [False, True])
def test_packed_blocks_equal_blocks_alone(orc, weighted):
    dims = [(14, 11, 9), (9, 16, 12), (18, 7, 10), (8, 8, 8), (5, 13, 6)]
    blocks = []
    for k, (nx, ny, nz) in enumerate(dims):
        f = workloads.blob_field((nx, ny, nz), 40 + k, n_blobs=3).numpy()
        band = orc.classify(f, np.array([0.15, 0.35], np.float32))
        comp, cb, cs, cf = orc.label_components(band)
        q = orc.saliency(f, 1) if weighted else None
        sp, sc, off, _ = orc.seed(comp, q, len(cb), 48, strat_block=8, rng_seed=7 + k)
        blocks.append(dict(band=band, q=q, sp=sp))
    origins, ext = pack_layout(dims, gap=1, footprint=(40, 32))
    same, trace_sum, gaps_empty = _run_and_compare(orc, blocks, origins, ext, weighted, n_iters=3)
    assert same and trace_sum and gaps_empty


def test_blocks_face_to_face_interact(orc):
    # one band everywhere, one site per block near the shared face: without a gap the other
    # block's site takes voxels across the face, with one voxel of band 0xFF it cannot
    dims = [(8, 6, 6), (8, 6, 6)]
    blocks = []
    for k in range(2):
        band = np.zeros((6, 6, 8), np.uint8)
        x = 7 if k == 0 else 0
        blocks.append(dict(band=band, q=None, sp=np.array([x + 8 * (3 + 6 * 3)], np.int32)))
    touching = [(0, 0, 0), (8, 0, 0)]
    same, _, _ = _run_and_compare(orc, blocks, touching, (16, 6, 6), False, n_iters=1)
    assert not same
    apart = [(0, 0, 0), (9, 0, 0)]
    same, trace_sum, gaps_empty = _run_and_compare(orc, blocks, apart, (17, 6, 6), False, n_iters=1)
    assert same and trace_sum and gaps_empty
