"""GPU parity of the any-angle tessellation (Sec. 3.2 region growing with src(w) shortcuts in
synchronous rounds) and of the Lloyd loop built on it (Eq. 2 with phi following src chains)
against the oracle: cells, lengths and sources bit for bit (integer arithmetic), the round
count of every tessellation, site positions and move traces of every iteration."""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

TIMEOUT, INVALID_ARG = 5, 1


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


def _case(dims, seed, P, iso=(0.3, 0.6), weights=False):
    f = workloads.blob_field(dims, seed, "cpu", n_blobs=8).numpy()
    f.ravel()[::61] = np.nan
    band = oracle.classify(f, np.array(iso, np.float32))
    comp, cb, cs, cf = oracle.label_components(band)
    sp, sc, off, nc = oracle.seed(comp, None, len(cb), P, 16, seed)
    q = np.random.default_rng(seed).integers(1, 200, band.shape).astype(np.uint16) if weights else None
    return band, q, sp


def _gpu(pk, band, q, sp, n_iters, slack=0, max_rounds=1 << 16, status=None):
    spt = torch.zeros(len(sp) + slack, dtype=torch.int32, device="cuda")
    spt[:len(sp)] = torch.from_numpy(sp.astype(np.int32)).cuda()
    if slack:
        spt[len(sp):] = -7  # capacity beyond the live sites is never read
    qt = torch.from_numpy(q.view(np.int16)).cuda() if q is not None else None
    st = pk.new_status() if status is None else status
    out = pk.cvt_iterate_anyangle(torch.from_numpy(band).cuda(), qt, spt,
                                  torch.tensor([len(sp)], dtype=torch.int32, device="cuda"), n_iters,
                                  max_rounds=max_rounds, status=st)
    return out, spt, st


def _anyangle_with_rounds(pk, band, spt, n_iters, max_rounds, st, rounds):
    """lsrvt_cvt_iterate_anyangle through the C ABI with a caller-owned rounds_host array."""
    import ctypes as C
    bt = torch.from_numpy(band).cuda()
    ns = torch.tensor([spt.numel()], dtype=torch.int32, device="cuda")
    cell = torch.empty(band.shape, dtype=torch.int32, device="cuda")
    d = pk.Dims(band.shape[2], band.shape[1], band.shape[0])
    nb = pk.workspace_bytes("cvt_anyangle", d, max_sites=spt.numel(), n_aux=max_rounds)
    buf = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    rc = pk.lib().lsrvt_cvt_iterate_anyangle(
        C.c_void_p(bt.data_ptr()), None, d, C.c_void_p(spt.data_ptr()), C.c_void_p(ns.data_ptr()), spt.numel(),
        n_iters, max_rounds, C.c_void_p(cell.data_ptr()), None, None, None, rounds.ctypes.data_as(C.c_void_p),
        C.c_void_p(buf.data_ptr()), buf.numel(), C.c_void_p(st.data_ptr()),
        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    if rc != 0:
        raise pk.LsrvtError(rc, "lsrvt_cvt_iterate_anyangle")
    return cell


@pytest.mark.parametrize("dims,P,seed", [((44, 30, 21), 200, 1), ((37, 29, 23), 64, 2), ((64, 64, 64), 512, 3),
                                         ((24, 20, 16), 2, 4), ((33, 1, 40), 16, 5), ((70, 9, 3), 40, 6)])
def test_anyangle_assignment_parity(pk, dims, P, seed):
    band, q, sp = _case(dims, seed, P)
    rc, rd, rs, rr = oracle.anyangle_assign(band, sp)
    (cell, dist, src, trace, rounds), spt, st = _gpu(pk, band, None, sp, 0, slack=3)
    pk.check_status(st, "any-angle tessellation")
    assert np.array_equal(cpu(cell), rc)
    assert np.array_equal(cpu(dist).view(np.uint32), rd)
    assert np.array_equal(cpu(src), rs)
    assert rounds[0] == rr
    # shortcuts make it no longer than the chamfer geodesic of the same sites
    cc, cd = oracle.assign(band, sp)
    m = rc >= 0
    assert np.all(rd[m].astype(np.int64) <= cd[m].astype(np.int64))


@pytest.mark.parametrize("dims,P,seed,weights,iters", [((40, 36, 28), 100, 7, True, 3), ((30, 26, 22), 64, 8, False, 4),
                                                       ((48, 20, 12), 300, 9, True, 2)])
def test_anyangle_lloyd_parity(pk, dims, P, seed, weights, iters):
    band, q, sp = _case(dims, seed, P, weights=weights)
    rsp, rc, rd, rs, rt, rr = oracle.cvt_iterate_anyangle(band, q, sp, iters)
    (cell, dist, src, trace, rounds), spt, st = _gpu(pk, band, q, sp, iters)
    pk.check_status(st, "any-angle Lloyd")
    assert np.array_equal(cpu(spt), rsp)
    assert np.array_equal(cpu(trace), rt)
    assert np.array_equal(rounds, rr)
    assert np.array_equal(cpu(cell), rc)
    assert np.array_equal(cpu(dist).view(np.uint32), rd)
    assert np.array_equal(cpu(src), rs)


def test_anyangle_degenerate(pk):
    # one band, one site: straight-line lengths everywhere
    band = np.zeros((9, 10, 11), np.uint8)
    sp = np.array([5 + 11 * (4 + 10 * 3)], np.int32)
    rc, rd, rs, rr = oracle.anyangle_assign(band, sp)
    (cell, dist, src, trace, rounds), spt, st = _gpu(pk, band, None, sp, 0)
    pk.check_status(st, "single site")
    assert np.array_equal(cpu(dist).view(np.uint32), rd) and rounds[0] == rr == 6
    assert np.all(cpu(src) == sp[0])
    # duplicate sites on one voxel: the lowest id keeps it, the other cell is empty
    band2, q2, sp2 = _case((20, 18, 16), 11, 40)
    dup = np.concatenate([sp2, sp2[:3]]).astype(np.int32)
    rc, rd, rs, rr = oracle.anyangle_assign(band2, dup)
    (cell, dist, src, trace, rounds), spt, st = _gpu(pk, band2, None, dup, 0)
    pk.check_status(st, "duplicate sites")
    assert np.array_equal(cpu(cell), rc) and np.array_equal(cpu(src), rs)
    assert not np.isin(np.arange(len(sp2), len(dup)), cpu(cell)).any()
    # an all-NaN volume: nothing reached, one round
    band3 = np.full((5, 6, 7), 255, np.uint8)
    (cell, dist, src, trace, rounds), spt, st = _gpu(pk, band3, None, np.zeros(0, np.int32), 1, slack=1)
    pk.check_status(st, "empty")
    assert np.all(cpu(cell) == -1) and np.all(cpu(src) == -1) and list(rounds) == [1, 1]


def test_anyangle_round_limit_and_bad_site(pk):
    band, q, sp = _case((44, 30, 21), 1, 200)
    rr = oracle.anyangle_assign(band, sp)[3]
    st = pk.new_status()
    with pytest.raises(pk.LsrvtError) as e:
        _gpu(pk, band, None, sp, 0, max_rounds=rr - 1, status=st)
    assert e.value.code == TIMEOUT and int(st.item()) == TIMEOUT
    # a Lloyd loop stops at the first tessellation that hits the limit: no update, no
    # further tessellation, the sites unmoved
    st = pk.new_status()
    spt = torch.from_numpy(sp.astype(np.int32)).cuda()
    rounds = np.full(4, -9, np.int32)
    with pytest.raises(pk.LsrvtError) as e:
        _anyangle_with_rounds(pk, band, spt, 3, rr - 1, st, rounds)
    assert e.value.code == TIMEOUT and int(st.item()) == TIMEOUT
    assert list(rounds) == [rr - 1, -9, -9, -9]
    assert np.array_equal(cpu(spt), sp)
    (cell, dist, src, trace, rounds), spt, st = _gpu(pk, band, None, sp, 0, max_rounds=rr)
    pk.check_status(st, "exact round limit")
    nan_voxel = int(np.flatnonzero(band.ravel() == 255)[0])
    bad = sp.copy()
    bad[1] = nan_voxel
    (cell, dist, src, trace, rounds), spt, st = _gpu(pk, band, None, bad, 0)
    torch.cuda.synchronize()
    assert int(st.item()) == INVALID_ARG


def test_decompose_anyangle_chain(pk):
    # the chained path with the any-angle metric and |grad f| weights: sites, cells, lengths,
    # sources and per-cell counts equal the oracle's chain
    w = workloads.blobs_workload(side=40, seed=3)
    f, aux = w["field"], w["aux"]
    out = pk.decompose(f.cuda(), w["iso"], 256, 2, aux=[a.cuda() for a in aux], gamma=1, rng_seed=3,
                       metric="anyangle")
    torch.cuda.synchronize()
    band = oracle.classify(f.numpy(), w["iso"])
    q = oracle.saliency(f.numpy(), 1)
    comp, cb, cs, cf = oracle.label_components(band)
    sp, sc, off, nc = oracle.seed(comp, q, len(cb), 256, 16, 3)
    rsp, rc, rd, rs, rt, rr = oracle.cvt_iterate_anyangle(band, q, sp, 2)
    ns = int(out["n_sites"].item())
    assert np.array_equal(cpu(out["site_pos"])[:ns], rsp)
    assert np.array_equal(cpu(out["cell"]), rc) and np.array_equal(cpu(out["src"]), rs)
    assert np.array_equal(cpu(out["dist"]).view(np.uint32), rd) and np.array_equal(out["rounds"], rr)
    ref = oracle.aggregate(rc, aux.numpy(), len(rsp), n_bins=32)
    assert np.array_equal(cpu(out["cells"]["count"])[:ns], ref["count"])
