"""Pins of the oracle's saliency weights and stratified seeding (Sec. 3.2, Eq. nc).

Weights: closed forms on linear fields (central differences are exact there).
Seeding: SplitMix64 published vectors; Eq. (nc) in its closed uniform-weight form; an
independent exact-fraction Hamilton apportionment; placement invariants.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_vectors(orc):
    for line in open(os.path.join(GOLDEN, "splitmix64_vectors.txt")):
        if line.startswith("#") or not line.strip():
            continue
        tok = line.split()
        state = int(tok[0], 0)
        for want in tok[1:]:
            assert orc.splitmix64(state) == int(want, 0)
            state = (state + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF


def test_saliency_linear_field_closed_form(orc):
    nz, ny, nx = 6, 7, 8
    z, y, x = np.indices((nz, ny, nx)).astype(np.float32)
    a, b, c = 0.5, 0.25, 1.0  # exactly representable; differences are exact
    f = (a * x + b * y + c * z).astype(np.float32)
    q = orc.saliency(f, 1).astype(np.int64)
    g_int = np.sqrt(a * a + b * b + c * c)
    assert np.all(q[1:-1, 1:-1, 1:-1] == 65535)  # interior: the maximum gradient
    # a voxel on the x = 0 face (interior in y, z): one-sided half difference a/2
    g = np.sqrt((a / 2) ** 2 + b * b + c * c)
    assert abs(q[2, 3, 0] - 65535 * g / g_int) <= 1.0
    # a corner: all three one-sided
    g = np.sqrt((a / 2) ** 2 + (b / 2) ** 2 + (c / 2) ** 2)
    assert abs(q[0, 0, 0] - 65535 * g / g_int) <= 1.0
    q2 = orc.saliency(f, 2).astype(np.int64)
    assert np.all(q2[1:-1, 1:-1, 1:-1] == 65535)
    assert abs(q2[0, 0, 0] - 65535 * (g / g_int) ** 2) <= 1.0


def test_saliency_degenerate(orc):
    f = np.full((3, 4, 5), 2.5, np.float32)
    assert np.all(orc.saliency(f, 1) == 1)  # zero gradient everywhere -> minimum weight
    rng = np.random.default_rng(1)
    f = rng.standard_normal((4, 4, 4)).astype(np.float32)
    assert np.all(orc.saliency(f, 0) == 1)
    q = orc.saliency(f, 1)
    assert q.min() >= 1 and q.max() == 65535
    with pytest.raises(orc.OracleError):
        orc.saliency(f, 5)


def _hamilton_capped(n, m, k):
    """Independent exact-fraction largest-remainder apportionment with capacity caps."""
    nb = [0] * len(m)
    capped = [False] * len(m)
    while True:
        remaining = n - sum(nb)
        if remaining == 0:
            break
        live = [i for i in range(len(m)) if not capped[i]]
        mA = sum(m[i] for i in live)
        quota = {i: Fraction(remaining * m[i], mA) for i in live}
        base = {i: int(quota[i]) for i in live}
        left = remaining - sum(base.values())
        order = sorted(live, key=lambda i: (-(quota[i] - base[i]), i))
        for i in live:
            nb[i] += base[i]
        for i in order[:left]:
            nb[i] += 1
        over = [i for i in live if nb[i] > k[i]]
        for i in over:
            nb[i] = k[i]
            capped[i] = True
        if not over:
            break
    return nb


def _strata(comp, sb):
    nz, ny, nx = comp.shape
    nbx, nby = -(-nx // sb), -(-ny // sb)
    z, y, x = np.indices(comp.shape)
    blk = (x // sb) + nbx * ((y // sb) + nby * (z // sb))
    return blk


@pytest.mark.parametrize("weighted", [False, True])
def test_seed_counts_and_apportionment(orc, weighted):
    rng = np.random.default_rng(11 if weighted else 12)
    shape = (20, 18, 22)
    f = np.cumsum(rng.standard_normal(shape), axis=2).astype(np.float32)
    band = orc.classify(f, np.array([-2.0, 0.0, 2.0], np.float32))
    comp, cb, cs, cf = orc.label_components(band)
    q = rng.integers(1, 5000, size=shape).astype(np.uint16) if weighted else None
    P, sb = 37, 8
    sp, sc, off, nc = orc.seed(comp, q, len(cb), P, sb, rng_seed=99)
    w = (q.astype(np.int64) if weighted else np.ones(shape, np.int64))
    valid = comp >= 0
    nV, mV = int(valid.sum()), int(w[valid].sum())
    blk = _strata(comp, sb)
    for c in range(len(cb)):
        sel = comp == c
        mC = int(w[sel].sum())
        want = max(-(-(nV * mC) // (P * mV)), 1)  # Eq. (nc), reading alpha = 1/P
        want = min(want, int(sel.sum()))
        assert nc[c] == want
        # apportionment over strata (blocks in increasing index)
        blocks = np.unique(blk[sel])
        m_b = [int(w[sel & (blk == b)].sum()) for b in blocks]
        k_b = [int((sel & (blk == b)).sum()) for b in blocks]
        ref = _hamilton_capped(want, m_b, k_b)
        ids = np.arange(off[c], off[c + 1])
        got_blocks = blk.ravel()[sp[ids]]
        got = [int((got_blocks == b).sum()) for b in blocks]
        assert got == ref
        assert sum(got) == want >= 1
    # site ids ordered by (component, block); sites distinct and inside their stratum
    keys = list(zip(sc.tolist(), blk.ravel()[sp].tolist()))
    assert keys == sorted(keys)
    assert len(np.unique(sp)) == len(sp)
    assert np.array_equal(comp.ravel()[sp], sc)
    assert off[-1] == len(sp)


def test_seed_uniform_closed_form_and_single_site(orc):
    comp = np.zeros((10, 10, 10), np.int32)
    sp, sc, off, nc = orc.seed(comp, None, 1, 64, 16, rng_seed=5)
    assert nc[0] == -(-1000 // 64) == len(sp)
    sp, sc, off, nc = orc.seed(comp, None, 1, 10 ** 9, 16, rng_seed=5)
    assert len(sp) == 1  # at least one site per component
    sp, sc, off, nc = orc.seed(comp, None, 1, 1, 4, rng_seed=5)
    assert len(sp) == 1000 and len(np.unique(sp)) == 1000  # every voxel a site


def test_seed_placement_ranges(orc):
    comp = np.zeros((1, 1, 40), np.int32)  # one stratum of 40 voxels (block 64)
    sp, sc, off, nc = orc.seed(comp, None, 1, 7, 64, rng_seed=3)
    n = len(sp)
    assert n == 6
    for j, p in enumerate(sp):  # rank j lies in [floor(j k/n), floor((j+1) k/n))
        assert (j * 40) // n <= p < ((j + 1) * 40) // n
    sp2, *_ = orc.seed(comp, None, 1, 7, 64, rng_seed=4)
    sp3, *_ = orc.seed(comp, None, 1, 7, 64, rng_seed=3)
    assert np.array_equal(sp, sp3) and not np.array_equal(sp, sp2)
