"""GPU parity of the structured hierarchical layout (Sec. 3.2 "Data Reduction and Structured
Data Layout") against the oracle, bit for bit: the order of the kept voxels, the extracted
values, and the cell / component / band offsets, on ragged volumes spanning many compaction
tiles, for several band subsets, variable counts and capacities."""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


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


def _case(dims, seed, P=200, n_iters=1, iso=(0.3, 0.6), nan_every=0):
    f = workloads.blob_field(dims, seed, "cpu", n_blobs=8).numpy()
    if nan_every:
        f.ravel()[::nan_every] = np.nan
    band = oracle.classify(f, np.array(iso, np.float32))
    comp, cb, cs, cf = oracle.label_components(band)
    sp, sc, off, nc = oracle.seed(comp, None, len(cb), P, 16, seed)
    sp2, cell, dist, tr = oracle.cvt_iterate(band, None, sp, n_iters)
    return cell, sc, off, cb


def _sites(cell, ns):
    # one voxel of each cell (its first in linear order): a valid shift voxel for the statistics
    flat = cell.ravel()
    first = np.full(ns, 0, np.int32)
    idx = np.nonzero(flat >= 0)[0]
    c = flat[idx]
    seen = np.zeros(ns, bool)
    for v, s in zip(idx, c):
        if not seen[s]:
            seen[s] = True
            first[s] = v
    return first


def _gpu_layout(pk, cell, off, cb, aux, bands, slack=0, status=None):
    ns, nc = int(off[-1]), len(cb)
    st = pk.new_status() if status is None else status
    cbt = torch.from_numpy(cb if nc else np.zeros(1, np.uint8)).cuda()  # never an empty (NULL) tensor
    out = pk.structured_layout(torch.from_numpy(cell).cuda(), torch.tensor([ns], dtype=torch.int32, device="cuda"),
                               ns + slack, torch.from_numpy(off).cuda(), cbt,
                               torch.tensor([nc], dtype=torch.int32, device="cuda"), nc + slack,
                               aux=[torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in aux], bands=bands,
                               status=st)
    return out, st


def _compare(pk, cell, sc, off, cb, aux, bands, slack=0):
    ref = oracle.layout(cell, sc, cb, aux, bands=bands)
    got, st = _gpu_layout(pk, cell, off, cb, aux, bands, slack)
    pk.check_status(st, "layout")
    r = int(got["n_kept"].item())
    ns, nc = int(off[-1]), len(cb)
    assert r == ref["n_kept"]
    assert np.array_equal(cpu(got["order"])[:r], ref["order"])
    if len(aux):
        assert np.array_equal(cpu(got["values"])[:len(aux), :r].view(np.uint32), ref["values"].view(np.uint32))
    assert np.array_equal(cpu(got["cell_off"])[:ns + 1], ref["cell_off"])
    assert np.array_equal(cpu(got["comp_off"])[:nc + 1], ref["comp_off"])
    assert np.array_equal(cpu(got["band_off"]), ref["band_off"])
    return r


@pytest.mark.parametrize("dims,m,seed", [((44, 30, 21), 3, 1), ((37, 29, 23), 5, 2), ((64, 64, 64), 0, 3),
                                         ((96, 40, 9), 9, 4), ((17, 1, 1), 1, 5), ((1, 1, 300), 2, 6)])
def test_layout_parity_shapes(pk, dims, m, seed):
    cell, sc, off, cb = _case(dims, seed, nan_every=53)
    aux = workloads.correlated_aux(dims, max(m, 1), seed, "cpu")[0].numpy()[:m]
    for bands in (None, [1], [0, 2], []):
        r = _compare(pk, cell, sc, off, cb, aux, bands)
        if bands == []:
            assert r == 0


def test_layout_capacity_slack_and_reuse(pk):
    # capacities above the live counts, repeated calls on one workspace, many cells (P = 8)
    dims = (48, 40, 36)
    cell, sc, off, cb = _case(dims, 11, P=8, iso=(0.2, 0.4, 0.6, 0.8))
    aux = workloads.correlated_aux(dims, 4, 11, "cpu")[0].numpy()
    assert len(sc) > 256 * 10  # several radix digits
    for bands in (None, [2, 3]):
        _compare(pk, cell, sc, off, cb, aux, bands, slack=1000)


def test_layout_degenerate(pk):
    # no graph nodes at all; a single voxel; one component with one site
    for f in (np.full((6, 7, 8), np.nan, np.float32), np.full((1, 1, 1), 0.5, np.float32),
              np.full((9, 10, 11), 0.5, np.float32)):
        band = oracle.classify(f, np.array([0.2, 0.8], np.float32))
        comp, cb, cs, cf = oracle.label_components(band)
        sp, sc, off, nc = oracle.seed(comp, None, len(cb), 1 << 20, 16, 1)
        cell, dist = oracle.assign(band, sp) if len(sp) else (np.full(f.shape, -1, np.int32), None)
        aux = np.stack([np.nan_to_num(f), np.ones_like(f)])
        if len(sp) == 0:
            # the entry point needs max_sites >= 1: one unused row
            off = np.zeros(1, np.int32)
            got, st = _gpu_layout(pk, cell, off, cb, aux, None, slack=1)
            pk.check_status(st, "layout")
            assert int(got["n_kept"].item()) == 0
            assert not cpu(got["band_off"]).any()
            continue
        _compare(pk, cell, sc, off, cb, aux, None)


def test_layout_reports_non_hierarchical_numbering(pk):
    # components whose bands are not in ascending order: a data-dependent argument error in
    # the status word (no fault, nothing written out of range)
    cell, sc, off, cb = _case((32, 24, 20), 7)
    assert len(cb) > 1
    bad = cb.copy()
    bad[0] = 200  # above the band of component 1
    got, st = _gpu_layout(pk, cell, off, bad, np.zeros((0,) + cell.shape, np.float32), None)
    torch.cuda.synchronize()
    assert int(st.item()) == 1  # INVALID_ARG
    # a cell id without a site
    cell2 = cell.copy()
    cell2.ravel()[5] = int(off[-1]) + 3
    got, st = _gpu_layout(pk, cell2, off, cb, np.zeros((0,) + cell.shape, np.float32), None, slack=10)
    torch.cuda.synchronize()
    assert int(st.item()) == 1


def test_layout_store_roundtrip(pk, tmp_path):
    # the GPU layout written to disk and read back one component at a time equals the oracle's
    from paper_2208_06970_b300 import store
    dims = (40, 33, 27)
    cell, sc, off, cb = _case(dims, 13)
    aux = workloads.correlated_aux(dims, 3, 13, "cpu")[0].numpy()
    got, st = _gpu_layout(pk, cell, off, cb, aux, [1, 2], slack=7)
    pk.check_status(st, "layout")
    ref = oracle.layout(cell, sc, cb, aux, bands=[1, 2])
    path = str(tmp_path / "g.lsrvt")
    store.save(path, got, int(off[-1]), len(cb))
    s = store.open_store(path)
    assert s.meta["n_kept"] == ref["n_kept"]
    for c in range(len(cb)):
        coords, vals = s.component(c)
        lo, hi = ref["comp_off"][c], ref["comp_off"][c + 1]
        assert np.array_equal(coords, ref["order"][lo:hi])
        assert np.array_equal(vals, ref["values"][:, lo:hi])


def test_statistics_on_layout_order(pk):
    # the statistics steps run on the layout (cells as contiguous runs of a 32 x 4 x N/128
    # pseudo-volume, per-position cells from the layout) give the volume form's results: counts,
    # min, max and histograms bit for bit, moments within the moment bar, co-moments within theirs
    dims = (64, 32, 24)  # N = 49152, a multiple of 128
    cell, sc, off, cb = _case(dims, 17, P=120)
    m = 6
    aux = workloads.correlated_aux(dims, m, 17, "cpu")[0].numpy()
    ns, nc = int(off[-1]), len(cb)
    st = pk.new_status()
    gcell = torch.from_numpy(cell).cuda()
    gaux = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in aux]
    lay = pk.structured_layout(gcell, torch.tensor([ns], dtype=torch.int32, device="cuda"), ns,
                               torch.from_numpy(off).cuda(), torch.from_numpy(cb).cuda(),
                               torch.tensor([nc], dtype=torch.int32, device="cuda"), nc, aux=gaux, status=st,
                               want_cells=True)
    pk.check_status(st, "layout")
    N = cell.size
    r = int(lay["n_kept"].item())
    cpos = cpu(lay["cell_pos"])
    assert np.array_equal(cpos[:r], cell.ravel()[cpu(lay["order"])[:r]]) and np.all(cpos[r:] == -1)
    shape = (N // 128, 4, 32)
    lcell = lay["cell_pos"].view(shape)
    lvals = [lay["values"][j].view(shape) for j in range(m)]
    # shift voxel of each cell: its first layout position
    lsite = torch.clamp(lay["cell_off"][:ns], max=max(r - 1, 0)).to(torch.int32).contiguous()
    ns_t = torch.tensor([ns], dtype=torch.int32, device="cuda")
    lo, scale = pk.aux_range(gcell, gaux, 16, st)
    vol = pk.aggregate(gcell, gaux, torch.from_numpy(_sites(cell, ns)).cuda(), ns_t, lo, scale, 16, cov=True,
                       status=st)
    got = pk.aggregate(lcell, lvals, lsite, ns_t, lo, scale, 16, cov=True, status=st)
    pk.check_status(st, "statistics")
    for k in ("count", "min", "max", "hist"):
        assert torch.equal(got[k][:ns], vol[k][:ns]), k
    ref = oracle.aggregate(cell, aux, ns, cpu(lo), cpu(scale), 16, cov=True)
    gm, gm2 = cpu(got["mean"])[:ns], cpu(got["m2"])[:ns]
    cnt = ref["count"][:, None]
    ex2 = ref["m2"] / np.maximum(cnt, 1) + ref["mean"] ** 2
    assert np.all(np.abs(gm - ref["mean"]) <= 1e-6 * np.maximum(np.abs(ref["mean"]), 1e-6 * ex2) + 1e-12)
    assert np.all(np.abs(gm2 / np.maximum(cnt, 1) - ref["m2"] / np.maximum(cnt, 1))
                  <= 1e-6 * np.maximum(ref["m2"] / np.maximum(cnt, 1), 1e-6 * ex2) + 1e-12)
    from itertools import combinations_with_replacement as cwr
    di = [t for t, (i, j) in enumerate(cwr(range(m), 2)) if i == j]
    R = ref["comom"]
    C = cpu(got["comom"])[:ns]
    for t, (i, j) in enumerate(cwr(range(m), 2)):
        bound = 1e-4 * np.sqrt(np.maximum(R[:, di[i]] * R[:, di[j]], 0)) + 1e-9
        assert np.all(np.abs(C[:, t] - R[:, t]) <= bound), (i, j)
