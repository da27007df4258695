"""GPU parity of the joint central moments (orders 2..4: covariance, coskewness and cokurtosis
sums) over the cell, component and band ranges of a structured layout, and of their merge up
the hierarchy (Pebay 2008), against the FP64 oracle.

Bar (FP32 products summed over at most 32 voxels, FP64 beyond): counts exact; means within
1e-6 (sigma + |mean|) ... relative to the natural scale; every co-moment entry within
2e-5 * n * prod(sigma over its indices) of the oracle, sigma_i = sqrt(M2_ii / n)."""
from itertools import combinations_with_replacement as cwr

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module")
def pk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2208_06970_b300 as pkg
    from paper_2208_06970_b300 import build
    build.build()
    return pkg


def cpu(t):
    return t.detach().cpu().numpy()


def _case(dims, seed, m, P=64, iso=(0.3, 0.6), offset=0.0):
    f = workloads.blob_field(dims, seed, "cpu", n_blobs=8).numpy()
    band = oracle.classify(f, np.array(iso, np.float32))
    comp, cb, cs, cf = oracle.label_components(band)
    sp, sc, off, nc = oracle.seed(comp, None, len(cb), P, 16, seed)
    cell, dist = oracle.assign(band, sp)
    aux = workloads.correlated_aux(dims, m, seed, "cpu")[0].numpy()
    aux = (aux + np.float32(offset)).astype(np.float32)
    return cell, sc, off, cb, aux


def _check(got, ref, rows):
    m = ref["mean"].shape[1]
    cnt = ref["count"][:rows]
    assert np.array_equal(cpu(got["count"])[:rows], cnt)
    sig = np.sqrt(np.maximum(ref["m2"][:rows][:, [t for t, (i, j) in enumerate(cwr(range(m), 2)) if i == j]], 0)
                  / np.maximum(cnt, 1)[:, None])
    gm = cpu(got["mean"])[:rows]
    assert np.all(np.abs(gm - ref["mean"][:rows]) <= 1e-6 * (sig + np.abs(ref["mean"][:rows])) + 1e-12)
    for q, key in ((2, "m2"), (3, "m3"), (4, "m4")):
        tups = list(cwr(range(m), q))
        scale = cnt[:, None] * np.stack([np.prod(sig[:, list(t)], axis=1) for t in tups], 1)
        err = np.abs(cpu(got[key])[:rows] - ref[key][:rows])
        bad = err > TOL * scale + 1e-9
        assert not bad.any(), (key, np.argwhere(bad)[:5], err[bad][:5], scale[bad][:5])


def _gpu_layout(pk, cell, off, cb, aux):
    ns, nc = int(off[-1]), len(cb)
    st = pk.new_status()
    lay = pk.structured_layout(torch.from_numpy(cell).cuda(), torch.tensor([ns], dtype=torch.int32, device="cuda"),
                               ns, torch.from_numpy(off).cuda(), torch.from_numpy(cb).cuda(),
                               torch.tensor([nc], dtype=torch.int32, device="cuda"), nc,
                               aux=[torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in aux], status=st)
    pk.check_status(st, "layout")
    return lay, ns, nc


@pytest.mark.parametrize("m", [1, 3, 4, 5, 6, 7, 8])
def test_joint_cells_parity(pk, m):
    dims = (44, 30, 21)
    cell, sc, off, cb, aux = _case(dims, 3 + m, m, offset=50.0 if m == 4 else 0.0)
    lay, ns, nc = _gpu_layout(pk, cell, off, cb, aux)
    ref_lay = oracle.layout(cell, sc, cb, aux)
    ref = oracle.joint_moments(aux, ref_lay["order"], ref_lay["cell_off"])
    vals = [lay["values"][j] for j in range(m)]
    got = pk.joint_moments(vals, lay["cell_off"], torch.tensor([ns], dtype=torch.int32, device="cuda"), ns)
    torch.cuda.synchronize()
    _check(got, ref, ns)


def test_joint_long_ranges_components_and_bands(pk):
    # components and bands hold far more than one 8192-position work item
    dims = (64, 64, 48)
    m = 4
    cell, sc, off, cb, aux = _case(dims, 21, m, P=512, iso=(0.25,), offset=-7.0)
    lay, ns, nc = _gpu_layout(pk, cell, off, cb, aux)
    ref_lay = oracle.layout(cell, sc, cb, aux)
    assert np.diff(ref_lay["comp_off"]).max() > 3 * 8192
    vals = [lay["values"][j] for j in range(m)]
    for key, rows in (("comp_off", nc), ("band_off", 2)):
        ref = oracle.joint_moments(aux, ref_lay["order"], ref_lay[key][:rows + 1])
        got = pk.joint_moments(vals, lay[key][:rows + 1].contiguous(), None, rows)
        torch.cuda.synchronize()
        _check(got, ref, rows)


def test_joint_merge_hierarchy(pk):
    dims = (48, 40, 36)
    m = 3
    cell, sc, off, cb, aux = _case(dims, 31, m, P=40, iso=(0.2, 0.4, 0.6))
    lay, ns, nc = _gpu_layout(pk, cell, off, cb, aux)
    ref_lay = oracle.layout(cell, sc, cb, aux)
    ref_cells = oracle.joint_moments(aux, ref_lay["order"], ref_lay["cell_off"])
    ref_comps = oracle.joint_merge(ref_cells, off.astype(np.int64))
    n_bands = 4
    ref_bands = oracle.joint_merge(ref_comps, np.searchsorted(cb, np.arange(n_bands + 1)).astype(np.int64))
    ref_vol = oracle.joint_merge(ref_bands, np.array([0, n_bands], np.int64))
    vals = [lay["values"][j] for j in range(m)]
    ns_t = torch.tensor([ns], dtype=torch.int32, device="cuda")
    cells = pk.joint_moments(vals, lay["cell_off"], ns_t, ns)
    comps, bands, vol = pk.merge_joint_hierarchy(cells, ns_t, torch.from_numpy(off).cuda(),
                                                 torch.from_numpy(cb).cuda(),
                                                 torch.tensor([nc], dtype=torch.int32, device="cuda"), nc, n_bands)
    torch.cuda.synchronize()
    _check(cells, ref_cells, ns)
    _check(comps, ref_comps, nc)
    _check(bands, ref_bands, n_bands)
    _check(vol, ref_vol, 1)
    # the merged volume record equals the moments of all kept voxels computed directly
    direct = oracle.joint_moments(aux, ref_lay["order"], np.array([0, ref_lay["n_kept"]]))
    _check(vol, direct, 1)
