"""The C ABI library loads without a GPU and exports every entry point include/lsrvt.h declares;
argument validation and workspace queries work on the host (no compute without a GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lsrvt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lsrvt_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_2208_06970_b300 import build as b
    b.build()
    import paper_2208_06970_b300 as pkg
    return pkg.lib()


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 11
    for n in names:
        assert hasattr(L, n), n
    import paper_2208_06970_b300 as pkg
    assert sorted(pkg.exported_symbols()) == names


def test_status_strings_and_version(L):
    assert L.lsrvt_status_string(0) == b"ok"
    assert b"capacity" in L.lsrvt_status_string(3)
    assert L.lsrvt_version() >= 10000


def test_workspace_queries(L):
    import paper_2208_06970_b300 as pkg
    assert pkg.workspace_bytes("classify", (64, 64, 64)) == 0
    w = pkg.workspace_bytes("cvt", (64, 64, 64), max_sites=1000)
    assert w >= 64 ** 3 * 8  # one 64-bit key per voxel at least
    assert pkg.workspace_bytes("label", (0, 4, 4)) == 0  # invalid dims
    assert pkg.workspace_bytes("seed", (512, 512, 512), max_comp=1 << 20) > 0
    # any-angle: two key + two source buffers, edge masks and clearance at least; one flag per round
    a1 = pkg.workspace_bytes("cvt_anyangle", (64, 64, 64), max_sites=1000, n_aux=64)
    a2 = pkg.workspace_bytes("cvt_anyangle", (64, 64, 64), max_sites=1000, n_aux=64 + 4096)
    assert a1 >= 64 ** 3 * (2 * 8 + 2 * 4 + 4 + 1)
    assert 4 * 4096 <= a2 - a1 <= 4 * 4096 + 256


def test_argument_errors_return_synchronously(L):
    import paper_2208_06970_b300 as pkg
    d = pkg.Dims(4, 4, 4)
    iso = (C.c_float * 2)(0.5, 0.25)
    fake = C.c_void_p(256)  # never dereferenced: validation fails first
    assert L.lsrvt_classify(fake, d, iso, 2, fake, None) == 2  # NOT_SORTED
    assert L.lsrvt_classify(None, d, iso, 1, fake, None) == 1  # NULL field
    assert L.lsrvt_classify(fake, pkg.Dims(0, 1, 1), iso, 1, fake, None) == 1
    assert L.lsrvt_classify(fake, d, iso, 255, fake, None) == 1
    # workspace too small
    assert L.lsrvt_label_components(fake, d, fake, fake, fake, fake, 8, fake, None, 0, None, None) == 8
    assert L.lsrvt_saliency_grad(fake, d, 7, fake, fake, 1 << 20, None) == 1
    sp = pkg.SeedParams(512, 17, 0, 0)  # strat_block above 16
    assert L.lsrvt_seed(fake, None, d, fake, 8, sp, fake, fake, fake, 8, fake, fake, 1 << 30, None, None) == 1
    aa = L.lsrvt_cvt_iterate_anyangle
    assert aa(fake, None, d, fake, fake, 8, 1, 0, fake, None, None, None, None, fake, 1 << 30, None, None) == 1
    assert aa(fake, None, d, None, fake, 8, 1, 16, fake, None, None, None, None, fake, 1 << 30, None, None) == 1
    assert aa(fake, None, d, fake, fake, 8, 1, 16, fake, None, None, None, None, fake, 64, None, None) == 8


def test_decompose_rejects_unknown_metric():
    import pytest
    import torch
    import paper_2208_06970_b300 as pkg
    with pytest.raises(ValueError):
        pkg.decompose(torch.zeros(2, 2, 2), [0.5], 8, 1, metric="euclid")


def test_static_labelling_scratch_covers_its_limit():
    """The allocation-free labelling accepts every volume of up to 2^18 voxels, so the
    workspace such a volume needs must fit its built-in scratch (1,310,720 bytes).  The
    workspace grows with the brick and chunk counts, so long thin shapes are the largest."""
    import paper_2208_06970_b300 as pkg
    limit = 1310720
    worst = 0
    for dims in ((64, 64, 64), (262144, 1, 1), (1, 1, 262144), (1, 4, 65536), (65536, 4, 1), (1, 262144, 1),
                 (3, 3, 29127), (2, 2, 65536), (512, 512, 1), (8, 8, 4096), (17, 15, 1028)):
        n = dims[0] * dims[1] * dims[2]
        assert n <= 1 << 18
        worst = max(worst, pkg.workspace_bytes("label", dims))
    assert 0 < worst <= limit
