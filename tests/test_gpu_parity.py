"""GPU parity: every step of the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs.  Integer results must match bit for bit; moments within
|got - ref| <= 1e-6 max(|ref|, 1e-6 <x^2>_cell) (mean and population variance).
Sizes span several bricks / tiles and ragged edges."""
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


def blob_case(side, seed=1):
    w = workloads.blobs_workload(side=side, seed=seed)
    return w


RAGGED = [(37, 29, 23), (64, 64, 64), (70, 9, 33), (1, 1, 300), (17, 1, 1)]


@pytest.mark.parametrize("dims", RAGGED)
def test_classify_parity(pk, dims):
    f = workloads.blob_field(dims, 5, "cpu", n_blobs=6).numpy()
    f.ravel()[::97] = np.nan
    for iso in ([0.3], [0.2, 0.4, 0.6, 0.8], list(np.linspace(0.05, 0.95, 8)), list(np.linspace(-1, 2, 254))):
        iso = np.array(iso, np.float32)
        ref = oracle.classify(f, iso)
        got = cpu(pk.classify(torch.from_numpy(f).cuda(), iso))
        assert np.array_equal(got, ref)
    # unaligned but contiguous input: scalar path
    n = f.size
    base = torch.empty(n + 1, dtype=torch.float32, device="cuda")
    view = base[1:].view(f.shape)
    view.copy_(torch.from_numpy(f))
    iso = np.array([0.2, 0.4, 0.6, 0.8], np.float32)
    assert np.array_equal(cpu(pk.classify(view, iso)), oracle.classify(f, iso))


def test_classify_errors(pk):
    f = torch.zeros((4, 4, 4), device="cuda")
    with pytest.raises(pk.LsrvtError) as e:
        pk.classify(f, np.array([0.5, 0.5], np.float32))
    assert e.value.code == 2


def _ccl_compare(pk, band):
    comp, cb, cs, cf = oracle.label_components(band)
    g = pk.label_components(torch.from_numpy(band).cuda(), max_comp=band.size)
    nc = int(g[4].item())
    assert nc == len(cb)
    assert np.array_equal(cpu(g[0]), comp)
    assert np.array_equal(cpu(g[1])[:nc], cb)
    assert np.array_equal(cpu(g[2])[:nc], cs)
    assert np.array_equal(cpu(g[3])[:nc], cf)


@pytest.mark.parametrize("dims,nb,seed", [((37, 29, 23), 3, 0), ((70, 9, 33), 2, 1), ((64, 64, 64), 4, 2),
                                          ((1, 1, 300), 2, 3), ((100, 3, 2), 5, 4)])
def test_ccl_parity_random(pk, dims, nb, seed):
    rng = np.random.default_rng(seed)
    shape = dims[::-1]
    band = rng.integers(0, nb, size=shape).astype(np.uint8)
    band[rng.random(shape) < 0.05] = 255
    _ccl_compare(pk, band)


def test_ccl_parity_blobs_and_checkerboard(pk):
    w = blob_case(64)
    _ccl_compare(pk, oracle.classify(w["field"].numpy(), w["iso"]))
    z, y, x = np.indices((20, 21, 22))
    _ccl_compare(pk, ((x + y + z) % 2).astype(np.uint8))
    _ccl_compare(pk, np.zeros((40, 50, 70), np.uint8))  # one component spanning every brick


def test_ccl_capacity_status(pk):
    z, y, x = np.indices((8, 8, 8))
    band = torch.from_numpy(((x + y + z) % 2).astype(np.uint8)).cuda()
    st = pk.new_status()
    g = pk.label_components(band, max_comp=100, status=st)
    assert int(g[4].item()) == 512 and int(st.item()) == 3


@pytest.mark.parametrize("gamma", [1, 2])
def test_saliency_parity(pk, gamma):
    for dims, seed in (((37, 29, 23), 3), ((64, 64, 64), 4)):
        f = workloads.blob_field(dims, seed, "cpu").numpy()
        ref = oracle.saliency(f, gamma)
        got = cpu(pk.saliency_grad(torch.from_numpy(f).cuda(), gamma)).view(np.uint16)
        assert np.array_equal(got, ref)
    f, u = workloads.flame_field((48, 40, 36), 2, "cpu")
    f = f.numpy()
    assert np.array_equal(cpu(pk.saliency_grad(torch.from_numpy(f).cuda(), gamma)).view(np.uint16),
                          oracle.saliency(f, gamma))


def _seed_compare(pk, f, iso, P, sb, rs, gamma):
    band = oracle.classify(f, iso)
    comp, cb, cs, cf = oracle.label_components(band)
    q = oracle.saliency(f, gamma) if gamma else None
    sp, sc, off, nc = oracle.seed(comp, q, len(cb), P, sb, rs)
    gb = pk.classify(torch.from_numpy(f).cuda(), iso)
    gc = pk.label_components(gb, max_comp=f.size)
    gq = pk.saliency_grad(torch.from_numpy(f).cuda(), gamma) if gamma else None
    gs = pk.seed(gc[0], gq, gc[4], f.size, P, sb, rs)
    ns = int(gs[3].item())
    assert ns == len(sp)
    assert np.array_equal(cpu(gs[0])[:ns], sp)
    assert np.array_equal(cpu(gs[1])[:ns], sc)
    assert np.array_equal(cpu(gs[2])[:len(cb) + 1], off)
    return sp


@pytest.mark.parametrize("P,sb,gamma", [(512, 16, 0), (64, 8, 0), (200, 5, 1), (37, 16, 2), (1, 4, 0)])
def test_seed_parity(pk, P, sb, gamma):
    w = blob_case(48, seed=3)
    _seed_compare(pk, w["field"].numpy(), w["iso"], P, sb, 1234, gamma)


def test_seed_parity_ragged(pk):
    f = workloads.blob_field((37, 29, 23), 9, "cpu").numpy()
    _seed_compare(pk, f, np.array([0.25, 0.5], np.float32), 100, 16, 7, 1)


def _cvt_compare(pk, f, iso, P, gamma, n_iters, rs=1):
    band = oracle.classify(f, iso)
    comp, cb, cs, cf = oracle.label_components(band)
    q = oracle.saliency(f, gamma) if gamma else None
    sp, sc, off, nc = oracle.seed(comp, q, len(cb), P, 16, rs)
    sp_ref, cell_ref, dist_ref, tr_ref = oracle.cvt_iterate(band, q, sp, n_iters)
    gband = torch.from_numpy(band).cuda()
    gq = torch.from_numpy(q.view(np.int16)).cuda() if q is not None else None
    gsp = torch.from_numpy(sp).cuda()
    ns = torch.tensor([len(sp)], dtype=torch.int32, device="cuda")
    st = pk.new_status()
    cell, dist, tr = pk.cvt_iterate(gband, gq, gsp, ns, n_iters, status=st)
    pk.check_status(st)
    assert np.array_equal(cpu(gsp), sp_ref)
    assert np.array_equal(cpu(cell), cell_ref)
    assert np.array_equal(cpu(dist).view(np.uint32), dist_ref)
    assert np.array_equal(cpu(tr), tr_ref)


@pytest.mark.parametrize("n_iters", [0, 1, 3])
def test_cvt_parity_blobs(pk, n_iters):
    w = blob_case(64)
    _cvt_compare(pk, w["field"].numpy(), w["iso"], 512, 0, n_iters)


def test_cvt_parity_weighted_ragged(pk):
    f = workloads.blob_field((45, 38, 27), 11, "cpu").numpy()
    _cvt_compare(pk, f, np.array([0.2, 0.45, 0.7], np.float32), 150, 1, 2, rs=3)


def test_cvt_parity_tall_volume(pk):
    """A volume taller than 1024 voxels along z: the path-check list keeps linear voxel indices
    (its packed coordinates hold z below 1024 only)."""
    f = workloads.blob_field((12, 10, 1100), 13, "cpu", n_blobs=40).numpy()
    _cvt_compare(pk, f, np.array([0.25, 0.5, 0.75], np.float32), 120, 0, 2, rs=5)


def test_cvt_parity_flame(pk):
    f, u = workloads.flame_field((40, 36, 32), 2, "cpu")
    _cvt_compare(pk, f.numpy(), (np.arange(1, 9, dtype=np.float32) / np.float32(9)), 300, 1, 2)


def test_cvt_config1_full(pk):
    w = blob_case(64)
    _cvt_compare(pk, w["field"].numpy(), w["iso"], 512, 0, 10)


def _moment_ok(got_mean, got_m2, ref_mean, ref_m2, count):
    n = np.maximum(count, 1)[:, None].astype(np.float64)
    var_r, var_g = ref_m2 / n, got_m2 / n
    msq = var_r + ref_mean ** 2
    floor = 1e-6 * msq
    assert np.all(np.abs(got_mean - ref_mean) <= 1e-6 * np.maximum(np.abs(ref_mean), floor) + 1e-300)
    assert np.all(np.abs(var_g - var_r) <= 1e-6 * np.maximum(np.abs(var_r), floor) + 1e-300)


def test_aggregate_and_merge_parity(pk):
    w = blob_case(64)
    f = w["field"].numpy()
    band = oracle.classify(f, w["iso"])
    comp, cb, cs, cf = oracle.label_components(band)
    sp, sc, off, nc = oracle.seed(comp, None, len(cb), 512, 16, 1)
    sp2, cell, dist, tr = oracle.cvt_iterate(band, None, sp, 2)
    aux = w["aux"].numpy()
    aux[2] += np.float32(50.0)  # far from zero: exercises the per-cell shift
    lo, hi, scale = oracle.aux_range(cell, aux, 32)
    ref = oracle.aggregate(cell, aux, len(sp2), lo, scale, 32)
    gcell = torch.from_numpy(cell).cuda()
    gaux = [torch.from_numpy(a).cuda() for a in aux]
    gsp = torch.from_numpy(sp2).cuda()
    ns = torch.tensor([len(sp2)], dtype=torch.int32, device="cuda")
    st = pk.new_status()
    glo, gsc = pk.aux_range(gcell, gaux, 32, st)
    assert np.array_equal(cpu(glo), lo) and np.array_equal(cpu(gsc), scale)
    got = pk.aggregate(gcell, gaux, gsp, ns, glo, gsc, 32, status=st)
    pk.check_status(st)
    assert np.array_equal(cpu(got["count"]), ref["count"])
    assert np.array_equal(cpu(got["min"]), ref["min"])
    assert np.array_equal(cpu(got["max"]), ref["max"])
    assert np.array_equal(cpu(got["hist"]).view(np.uint32), ref["hist"])
    _moment_ok(cpu(got["mean"]), cpu(got["m2"]), ref["mean"], ref["m2"], ref["count"])
    # hierarchy
    rc, rb, rv = oracle.merge_hierarchy(ref, sc, cb, len(w["iso"]) + 1)
    gc, gb, gv = pk.merge_hierarchy(got, ns, torch.from_numpy(off).cuda(), torch.from_numpy(cb).cuda(),
                                    torch.tensor([len(cb)], dtype=torch.int32, device="cuda"), len(cb),
                                    len(w["iso"]) + 1)
    for g, r in ((gc, rc), (gb, rb), (gv, rv)):
        assert np.array_equal(cpu(g["count"]), r["count"])
        assert np.array_equal(cpu(g["min"]), r["min"]) and np.array_equal(cpu(g["max"]), r["max"])
        assert np.array_equal(cpu(g["hist"]).view(np.uint32), r["hist"])
        _moment_ok(cpu(g["mean"]), cpu(g["m2"]), r["mean"], r["m2"], r["count"])


@pytest.mark.parametrize("dims,m,n_bins", [((44, 30, 21), 20, 31), ((37, 29, 23), 5, 32), ((96, 40, 9), 16, 64)])
def test_aggregate_parity_shapes(pk, dims, m, n_bins):
    """Statistics sweep on volumes staged by TMA tile loads (row pitch a multiple of 16 bytes:
    nx = 44, 96) and by plain loads (nx = 37), with two variable tiles (m = 20), an odd bin
    count, and more bins than the lane-private histograms hold (64)."""
    f = workloads.blob_field(dims, 7, "cpu", n_blobs=8).numpy()
    band = oracle.classify(f, np.array([0.3, 0.6], np.float32))
    comp, cb, cs, cf = oracle.label_components(band)
    sp, sc, off, nc = oracle.seed(comp, None, len(cb), 200, 16, 3)
    sp2, cell, dist, tr = oracle.cvt_iterate(band, None, sp, 1)
    aux = workloads.correlated_aux(dims, m, 9, "cpu")[0].numpy()
    lo, hi, scale = oracle.aux_range(cell, aux, n_bins)
    ref = oracle.aggregate(cell, aux, len(sp2), lo, scale, n_bins)
    gcell = torch.from_numpy(cell).cuda()
    st = pk.new_status()
    # separate allocations (one tensor map per variable) and one stacked tensor (a single 4-D
    # tensor map for all variables)
    separate = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in aux]
    stacked = list(torch.from_numpy(aux).cuda().unbind(0))
    glo, gsc = pk.aux_range(gcell, separate, n_bins, st)
    assert np.array_equal(cpu(glo), lo) and np.array_equal(cpu(gsc), scale)
    for gaux in (separate, stacked, stacked):  # repeated calls reuse the accumulators
        got = pk.aggregate(gcell, gaux, torch.from_numpy(sp2).cuda(),
                           torch.tensor([len(sp2)], dtype=torch.int32, device="cuda"), glo, gsc, n_bins, status=st)
        pk.check_status(st)
        assert np.array_equal(cpu(got["count"]), ref["count"])
        assert np.array_equal(cpu(got["min"]), ref["min"]) and np.array_equal(cpu(got["max"]), ref["max"])
        assert np.array_equal(cpu(got["hist"]).view(np.uint32), ref["hist"])
        _moment_ok(cpu(got["mean"]), cpu(got["m2"]), ref["mean"], ref["m2"], ref["count"])


def test_decompose_pipeline_config1(pk):
    w = blob_case(64)
    f = w["field"]
    out = pk.decompose(f.cuda(), w["iso"], 512, 10, aux=[a.cuda() for a in w["aux"]], gamma=0, rng_seed=1)
    band = oracle.classify(f.numpy(), w["iso"])
    comp, cb, cs, cf = oracle.label_components(band)
    sp, sc, off, nc = oracle.seed(comp, None, len(cb), 512, 16, 1)
    sp2, cell, dist, tr = oracle.cvt_iterate(band, None, sp, 10)
    ns = int(out["n_sites"].item())
    assert np.array_equal(cpu(out["site_pos"])[:ns], sp2)
    assert np.array_equal(cpu(out["cell"]), cell)
    ref = oracle.aggregate(cell, w["aux"].numpy(), len(sp2), n_bins=32)
    assert np.array_equal(cpu(out["cells"]["count"])[:ns], ref["count"])
    assert np.array_equal(cpu(out["cells"]["hist"])[:ns].view(np.uint32), ref["hist"])


@pytest.mark.parametrize("m,shape", [(32, (40, 36, 33)), (7, (64, 48, 40)), (20, (37, 29, 23))])
def test_covariance_parity(pk, m, shape):
    """Co-moments on tensor cores (BF16 split, FP32 accumulate, FP64 finalise) against the FP64
    oracle: |C_ij - R_ij| <= 1e-4 sqrt(R_ii R_jj) (correlated Gaussians with non-zero means)."""
    f = workloads.blob_field(shape[::-1], 21, "cpu").numpy()
    band = oracle.classify(f, np.array([0.3, 0.6], np.float32))
    comp, cb, cs, cf = oracle.label_components(band)
    sp, sc, off, nc = oracle.seed(comp, None, len(cb), 300, 16, 2)
    sp2, cell, dist, tr = oracle.cvt_iterate(band, None, sp, 1)
    aux, cov, mu = workloads.correlated_aux(shape[::-1], m, 31, "cpu")
    aux = aux.numpy()
    ref = oracle.aggregate(cell, aux, len(sp2), n_bins=0, cov=True)
    gaux = [torch.from_numpy(a).cuda() for a in aux]
    st = pk.new_status()
    got = pk.aggregate(torch.from_numpy(cell).cuda(), gaux, torch.from_numpy(sp2).cuda(),
                       torch.tensor([len(sp2)], dtype=torch.int32, device="cuda"), n_bins=0, cov=True, status=st)
    pk.check_status(st)
    C = cpu(got["comom"])
    R = ref["comom"]
    iu = np.triu_indices(m)
    diag_pos = [k for k, (i, j) in enumerate(zip(*iu)) if i == j]
    for k, (i, j) in enumerate(zip(*iu)):
        scale = np.sqrt(np.maximum(R[:, diag_pos[i]] * R[:, diag_pos[j]], 0.0))
        assert np.all(np.abs(C[:, k] - R[:, k]) <= 1e-4 * scale + 1e-9), (i, j)
    assert np.array_equal(cpu(got["count"]), ref["count"])


def test_cvt_rerun_and_resume_bit_identical(pk):
    # Algorithm 1 split as k1 + k2 iterations (the second call resumes from the first call's
    # sites) equals one call of k1 + k2 iterations, and reruns repeat bit for bit
    w = workloads.flame_workload(side=(70, 52, 45), seed=4, n_aux=0)
    f = w["field"].cuda()
    band = pk.classify(f, w["iso"])
    mc = pk.default_max_comp(f.numel())
    comp, cb, cs, cf, nc = pk.label_components(band, mc)
    q = pk.saliency_grad(f, 1)
    sp, sc, off, ns = pk.seed(comp, q, nc, mc, 256, 16, 4)
    runs = []
    for split in ((7, 0), (3, 4), (7, 0), (0, 7)):
        s = sp.clone()
        st = pk.new_status()
        if split[0]:
            pk.cvt_iterate(band, q, s, ns, split[0], status=st)
        cell, dist, _ = pk.cvt_iterate(band, q, s, ns, split[1], status=st)
        pk.check_status(st)
        runs.append((cpu(s), cpu(cell), cpu(dist)))
    for r in runs[1:]:
        assert all(np.array_equal(a, b) for a, b in zip(r, runs[0]))
    s_ref, c_ref, d_ref, _ = oracle.cvt_iterate(cpu(band), cpu(q).view(np.uint16), cpu(sp)[:int(ns.item())], 7)
    assert np.array_equal(runs[0][0][:int(ns.item())], s_ref) and np.array_equal(runs[0][1], c_ref)


def _oracle_pipeline(f, iso, P, n_iters, aux, n_bins=32):
    band = oracle.classify(f, iso)
    comp, cb, cs, cf = oracle.label_components(band)
    sp, sc, off, nc = oracle.seed(comp, None, len(cb), P, 16, 7)
    sp2, cell, dist, tr = oracle.cvt_iterate(band, None, sp, n_iters)
    stats = oracle.aggregate(cell, aux, len(sp2), n_bins=n_bins) if len(sp2) else None
    return band, comp, cb, sp2, cell, dist, stats


@pytest.mark.parametrize("case", ["all_invalid", "single_voxel", "constant", "single_seed", "checkerboard"])
def test_degenerate_volumes_end_to_end(pk, case):
    """The whole path on degenerate inputs against the oracle pipeline: a volume with no graph
    nodes (all NaN), one voxel, a constant field (one band, one component: a plain discrete
    CVT of the box), one site for the whole component, and a checkerboard where every voxel is
    its own component and site."""
    iso = np.array([0.2, 0.4, 0.6, 0.8], np.float32)
    P, n_iters = 512, 3
    if case == "all_invalid":
        f = np.full((8, 8, 8), np.nan, np.float32)
    elif case == "single_voxel":
        f = np.full((1, 1, 1), 0.5, np.float32)
    elif case == "constant":
        f = np.full((16, 20, 24), 0.5, np.float32)
    elif case == "single_seed":
        f = np.full((16, 16, 16), 0.5, np.float32)
        P = 1 << 20
    else:
        z, y, x = np.indices((8, 9, 10))
        f = ((x + y + z) % 2).astype(np.float32) * np.float32(0.9)
        iso = np.array([0.5], np.float32)
    aux = np.stack([np.where(np.isnan(f), 0.0, f).astype(np.float32),
                    (np.arange(f.size, dtype=np.float32).reshape(f.shape) * np.float32(0.01))])
    band, comp, cb, sp, cell, dist, stats = _oracle_pipeline(f, iso, P, n_iters, aux)
    out = pk.decompose(torch.from_numpy(f).cuda(), iso, P, n_iters, aux=[torch.from_numpy(a).cuda() for a in aux],
                       rng_seed=7)
    ns = int(out["n_sites"].item())
    assert ns == len(sp)
    assert int(out["n_comp"].item()) == len(cb)
    assert np.array_equal(cpu(out["band"]), band)
    assert np.array_equal(cpu(out["comp"]), comp)
    assert np.array_equal(cpu(out["site_pos"])[:ns], sp)
    assert np.array_equal(cpu(out["cell"]), cell)
    assert np.array_equal(cpu(out["dist"]).view(np.uint32), dist.view(np.uint32))
    if case == "single_seed":
        assert ns == 1 and np.all(cell == 0)
    if case == "checkerboard":
        # every voxel is its own component, site and cell (site ids follow the (band, component) order)
        assert ns == f.size and np.array_equal(sp[cell.ravel()], np.arange(f.size))
    if stats is not None:
        got = out["cells"]
        assert np.array_equal(cpu(got["count"])[:ns], stats["count"])
        assert np.array_equal(cpu(got["min"])[:ns], stats["min"]) and np.array_equal(cpu(got["max"])[:ns], stats["max"])
        assert np.array_equal(cpu(got["hist"])[:ns].view(np.uint32), stats["hist"])
        _moment_ok(cpu(got["mean"])[:ns], cpu(got["m2"])[:ns], stats["mean"], stats["m2"], stats["count"])


def test_cvt_parity_sharp_flame_recipe(pk):
    """The sharp flame recipe (no dissipation cutoff, 4-voxel front) at 128^3 shatters the
    thin isobands into ~10^5 components, most of a few voxels: labels, seeds (at least one per
    component), two Lloyd iterations with |grad f| weights and the final cells, bit for bit."""
    w = workloads.flame_workload(side=128, seed=2, n_aux=0, recipe="sharp")
    f = w["field"].numpy()
    band = oracle.classify(f, w["iso"])
    comp, cb, cs, cf = oracle.label_components(band)
    assert len(cb) > 100000
    gband = torch.from_numpy(band).cuda()
    st = pk.new_status()
    n = band.size
    gcomp, gcb, gcs, gcf, gnc = pk.label_components(gband, max_comp=n // 4, status=st)
    pk.check_status(st, "labels")
    k = int(gnc.item())
    assert k == len(cb) and np.array_equal(cpu(gcomp), comp) and np.array_equal(cpu(gcs)[:k], cs)
    q = oracle.saliency(f, 1)
    gq = pk.saliency_grad(torch.from_numpy(f).cuda(), 1)
    assert np.array_equal(cpu(gq).view(np.uint16), q)
    sp, sc, off, nc = oracle.seed(comp, q, len(cb), 4096, 16, 2)
    gsp, gsc, goff, gns = pk.seed(gcomp, gq, gnc, n // 4, 4096, 16, 2, status=st)
    pk.check_status(st, "seeds")
    ns = int(gns.item())
    assert ns == len(sp) and np.array_equal(cpu(gsp)[:ns], sp)
    sp_ref, cell_ref, dist_ref, tr_ref = oracle.cvt_iterate(band, q, sp, 2)
    cell, dist, tr = pk.cvt_iterate(gband, gq, gsp, gns, 2, status=st)
    pk.check_status(st, "Lloyd iterations")
    assert np.array_equal(cpu(gsp)[:ns], sp_ref)
    assert np.array_equal(cpu(cell), cell_ref) and np.array_equal(cpu(dist).view(np.uint32), dist_ref)
    assert np.array_equal(cpu(tr), tr_ref)
