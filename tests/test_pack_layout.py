"""Packed batches on the host: the layout keeps the blocks inside the packed volume and at least
`gap` voxels apart (so no restricted path, traversal or site walk can join two blocks), and the
C ABI rejects overlapping or out-of-volume blocks synchronously (no GPU needed)."""
import ctypes as C

import numpy as np
import pytest

from paper_2208_06970_b300 import runtime


def _check_layout(dims, origins, ext, gap):
    assert len(origins) == len(dims)
    for (nx, ny, nz), (x0, y0, z0) in zip(dims, origins):
        assert min(x0, y0, z0) >= 0
        assert x0 + nx <= ext[0] and y0 + ny <= ext[1] and z0 + nz <= ext[2]
    boxes = [np.array([[o[a], o[a] + d[a]] for a in range(3)]) for d, o in zip(dims, origins)]
    for i in range(len(boxes)):
        for j in range(i):
            a, b = boxes[i], boxes[j]
            # separated along some axis by at least `gap` free voxels
            sep = [b[k][0] - a[k][1] >= gap or a[k][0] - b[k][1] >= gap for k in range(3)]
            assert any(sep), (i, j, boxes[i], boxes[j])


@pytest.mark.parametrize("gap", [1, 3])
def test_layout_separates_blocks(gap):
    rng = np.random.default_rng(11 + gap)
    dims = [tuple(int(v) for v in rng.integers(5, 90, size=3)) for _ in range(40)]
    origins, ext = runtime.pack_layout(dims, gap=gap)
    _check_layout(dims, origins, ext, gap)
    assert max(ext) <= 2048


def test_layout_of_the_batch_workload_is_dense():
    # 64 blocks with sides U{32..256} per axis: the height map keeps most of the packed volume
    # inside blocks
    rng = np.random.default_rng(3)
    dims = [tuple(int(v) for v in rng.integers(32, 257, size=3)) for _ in range(64)]
    origins, ext = runtime.pack_layout(dims, gap=1)
    _check_layout(dims, origins, ext, 1)
    fill = sum(a * b * c for a, b, c in dims) / float(ext[0] * ext[1] * ext[2])
    assert fill > 0.6, fill


def test_layout_single_block_and_fixed_footprint():
    origins, ext = runtime.pack_layout([(17, 9, 5)], gap=1)
    assert origins == [(0, 0, 0)] and ext == (17, 9, 5)
    dims = [(30, 30, 10)] * 4
    origins, ext = runtime.pack_layout(dims, gap=2, footprint=(64, 64))
    _check_layout(dims, origins, ext, 2)
    with pytest.raises(ValueError):
        runtime.pack_layout([(100, 10, 10)], gap=1, footprint=(64, 64))
    with pytest.raises(ValueError):
        runtime.pack_layout([(10, 10, 10)], gap=0)


def test_pack_abi_rejects_bad_tables():
    import paper_2208_06970_b300 as pkg
    from paper_2208_06970_b300 import build
    build.build()
    L = pkg.lib()
    fake = C.c_void_p(256)  # never dereferenced: validation fails first

    def table(origins, dims):
        tab = (pkg.Block * len(dims))()
        for i, ((x0, y0, z0), (nx, ny, nz)) in enumerate(zip(origins, dims)):
            tab[i] = pkg.Block(pkg.Dims(nx, ny, nz), x0, y0, z0, fake, None, fake, fake, fake, None)
        return tab

    P = pkg.Dims(40, 20, 20)
    args = lambda tab, n: (C.cast(tab, C.c_void_p), n, P, fake, None, fake, 100, fake, fake, fake, None)
    # two blocks touching (no free voxel between them): rejected
    touching = table([(0, 0, 0), (10, 0, 0)], [(10, 10, 10), (10, 10, 10)])
    assert L.lsrvt_pack_blocks(*args(touching, 2)) == 1
    # a block reaching outside the packed volume: rejected
    outside = table([(35, 0, 0)], [(10, 10, 10)])
    assert L.lsrvt_pack_blocks(*args(outside, 1)) == 1
    # no blocks, or more than the table holds: rejected
    assert L.lsrvt_pack_blocks(*args(touching, 0)) == 1
    assert L.lsrvt_pack_blocks(*args(touching, pkg.MAX_PACK_BLOCKS + 1)) == 1
    # weights asked for but a block has none: rejected
    apart = table([(0, 0, 0), (11, 0, 0)], [(10, 10, 10), (10, 10, 10)])
    assert L.lsrvt_pack_blocks(C.cast(apart, C.c_void_p), 2, P, fake, fake, fake, 100, fake, fake, fake,
                               None) == 1
    # unpacking checks the same table
    assert L.lsrvt_unpack_blocks(C.cast(touching, C.c_void_p), 2, P, fake, None, fake, fake, None) == 1


def test_block_descriptor_matches_the_header():
    # the ctypes mirror has the C layout the library asserts at compile time (72 bytes; x0 at 12,
    # band at 24, n_sites at 48, dist at 64), and the table size agrees with the header
    import os
    import re
    import paper_2208_06970_b300 as pkg
    B = pkg.Block
    assert C.sizeof(B) == 72
    assert (B.x0.offset, B.band.offset, B.n_sites.offset, B.dist.offset) == (12, 24, 48, 64)
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lsrvt.h")).read()
    assert int(re.search(r"#define LSRVT_MAX_PACK_BLOCKS (\d+)", hdr).group(1)) == pkg.MAX_PACK_BLOCKS


def test_layout_stays_below_the_volume_limit():
    # eight 1024^3 blocks cannot share a volume of fewer than 2^31 voxels
    with pytest.raises(ValueError):
        runtime.pack_layout([(1024, 1024, 1024)] * 8, gap=1)
    with pytest.raises(ValueError):
        runtime.pack_layout([(1024, 1024, 1024)] * 2, gap=1, footprint=(2048, 1024))
