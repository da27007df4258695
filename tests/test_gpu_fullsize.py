"""Full-size parity on the 512^3 flame workload, run exactly as the benchmark runs it
(bench.Pipeline: same calls, buffers, workspace and launch configuration).

The oracle cannot rerun 30 Lloyd iterations on 134 M voxels in test time, so:
- classify, components, weights and seeding are compared with the oracle on the whole volume;
- every assignment checked is certified exactly by the Bellman equations of the
  lexicographic key (a unique fixed point; an O(26 N) host check);
- one Lloyd update is replayed by the oracle on a sample of cells, from the GPU's
  certified assignment of iteration 29, and must give the GPU's sites of iteration 30;
- resuming (29 iterations, then 1) gives the 30-iteration sites and labels bit for bit;
- statistics are compared on a sample of cells (the oracle sees only those voxels), with
  the histogram ranges computed by the oracle over the whole volume;
- the merge is compared with the oracle's merge of the same per-cell records;
- the any-angle tessellation of the final sites is checked on every voxel by exact properties
  (chamfer upper bound, straight-segment lower bound, consistent source chains ending at the
  site, component membership) and on sampled shortcut segments by the oracle's traversal.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def cpu(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    import paper_2208_06970_b300 as pk
    from paper_2208_06970_b300 import build
    build.build()
    w = workloads.flame_workload(side=512, seed=2, device="cuda", n_aux=bench.N_AUX, n_iters=bench.N_ITERS)
    pipe = bench.Pipeline(pk, w["field"], [w["aux"][j] for j in range(bench.N_AUX)], w["iso"])
    out = pipe.step()
    torch.cuda.synchronize()
    pk.check_status(pipe.status, "full-size step")
    f = cpu(w["field"])
    band = oracle.classify(f, w["iso"])
    return dict(pk=pk, bench=bench, w=w, pipe=pipe, out=out, f=f, band=band)


def test_full_classify_components_weights_seeds(full):
    pk, pipe, out, band, f = full["pk"], full["pipe"], full["out"], full["band"], full["f"]
    assert np.array_equal(cpu(out["band"]), band)
    comp, cb, cs, cf = oracle.label_components(band)
    g = pk.label_components(out["band"], pipe.max_comp, pipe.ws, pipe.status)
    nc = int(g[4].item())
    assert nc == len(cb) == int(out["n_comp"].item())
    assert np.array_equal(cpu(g[0]), comp)
    assert np.array_equal(cpu(g[1])[:nc], cb) and np.array_equal(cpu(g[2])[:nc], cs)
    assert np.array_equal(cpu(g[3])[:nc], cf)
    q = oracle.saliency(f, 1)
    gq = pk.saliency_grad(full["w"]["field"], 1, pipe.ws)
    assert np.array_equal(cpu(gq).view(np.uint16), q)
    bench = full["bench"]
    sp, sc, off, _ = oracle.seed(comp, q, len(cb), bench.VPS, 16, 2)
    gsp, gsc, goff, gns = pk.seed(g[0], gq, g[4], pipe.max_comp, bench.VPS, 16, 2, ws=pipe.ws, status=pipe.status)
    ns = int(gns.item())
    assert ns == len(sp)
    assert np.array_equal(cpu(gsp)[:ns], sp) and np.array_equal(cpu(gsc)[:ns], sc)
    assert np.array_equal(cpu(goff)[:nc + 1], off)
    full.update(comp=comp, comp_band=cb, q=q, sites0=sp, gq=gq, gcomp=g, gsp0=gsp, gns=gns, off=off)


def test_full_tessellation_certified_replayed_resumed(full):
    if "sites0" not in full:
        pytest.skip("needs the seeding comparison")
    pk, pipe, out, band, bench = full["pk"], full["pipe"], full["out"], full["band"], full["bench"]
    ns = int(full["gns"].item())
    # 29 iterations, certified assignment of the last one
    sp29 = full["gsp0"].clone()
    cell29, dist29, _ = pk.cvt_iterate(out["band"], full["gq"], sp29, full["gns"], bench.N_ITERS - 1, ws=pipe.ws,
                                       status=pipe.status)
    torch.cuda.synchronize()
    pk.check_status(pipe.status, "29 iterations")
    h_sp29, h_cell29, h_dist29 = cpu(sp29)[:ns], cpu(cell29), cpu(dist29).view(np.uint32)
    assert oracle.certify(band, h_sp29, h_cell29, h_dist29) == 0
    # the 30th iteration, resumed from there
    sp30 = sp29.clone()
    cell30, dist30, _ = pk.cvt_iterate(out["band"], full["gq"], sp30, full["gns"], 1, ws=pipe.ws, status=pipe.status)
    torch.cuda.synchronize()
    pk.check_status(pipe.status, "resumed iteration")
    h_sp30 = cpu(sp30)[:ns]
    assert np.array_equal(h_sp30, cpu(out["site_pos"])[:ns])
    assert np.array_equal(cpu(cell30), cpu(out["cell"]))
    assert oracle.certify(band, h_sp30, cpu(cell30), cpu(dist30).view(np.uint32)) == 0
    # oracle replay of the 30th update on a sample of cells: random ones plus the largest
    rng = np.random.default_rng(30)
    counts = np.bincount(h_cell29[h_cell29 >= 0].ravel(), minlength=ns)
    sample = np.unique(np.concatenate([rng.choice(ns, size=min(ns, 192), replace=False),
                                       np.argsort(counts)[-32:], np.flatnonzero(h_sp30 != h_sp29)[:32]]))
    got, _ = oracle.update_selected(band, full["q"], h_cell29, h_dist29, h_sp29, sample)
    assert np.array_equal(got, h_sp30[sample])
    assert (h_sp30[sample] != h_sp29[sample]).any()


def _moment_ok(got_mean, got_m2, ref_mean, ref_m2, count):
    n = np.maximum(count, 1)[:, None].astype(np.float64)
    var_r, var_g = ref_m2 / n, got_m2 / n
    floor = 1e-6 * (var_r + ref_mean ** 2)
    assert np.all(np.abs(got_mean - ref_mean) <= 1e-6 * np.maximum(np.abs(ref_mean), floor) + 1e-300)
    assert np.all(np.abs(var_g - var_r) <= 1e-6 * np.maximum(np.abs(var_r), floor) + 1e-300)


def test_full_statistics_sampled_cells_and_merge(full):
    pk, pipe, out, bench = full["pk"], full["pipe"], full["out"], full["bench"]
    aux = full["w"]["aux"]
    m = bench.N_AUX
    cell = out["cell"]
    h_cell = cpu(cell)
    ns = int(out["n_sites"].item())
    # histogram ranges: the oracle over the whole volume, one variable at a time
    lo = np.empty(m, np.float32)
    sc = np.empty(m, np.float32)
    for j in range(m):
        l, _, s = oracle.aux_range(h_cell, cpu(aux[j])[None], bench.N_BINS)
        lo[j], sc[j] = l[0], s[0]
    glo, gsc = pk.aux_range(cell, [aux[j] for j in range(m)], bench.N_BINS, pipe.status)
    assert np.array_equal(cpu(glo), lo) and np.array_equal(cpu(gsc), sc)
    # sampled cells: the oracle aggregates only their voxels
    rng = np.random.default_rng(31)
    counts = np.bincount(h_cell[h_cell >= 0].ravel(), minlength=ns)
    sample = np.unique(np.concatenate([rng.choice(ns, size=min(ns, 96), replace=False), np.argsort(counts)[-8:],
                                       np.argsort(counts)[:8]]))
    remap = torch.full((ns,), -1, dtype=torch.int32, device=cell.device)
    remap[torch.from_numpy(sample).to(cell.device).long()] = torch.arange(len(sample), dtype=torch.int32,
                                                                           device=cell.device)
    flat = cell.reshape(-1)
    sel = torch.nonzero(flat >= 0).squeeze(1)
    sel = sel[remap[flat[sel].long()] >= 0]
    sub_cell = cpu(remap[flat[sel].long()])
    sub_aux = np.stack([cpu(aux[j].reshape(-1)[sel]) for j in range(m)])
    ref = oracle.aggregate(sub_cell, sub_aux, len(sample), lo, sc, bench.N_BINS)
    cells = out["cells"]
    assert np.array_equal(cpu(cells["count"])[sample], ref["count"])
    assert np.array_equal(cpu(cells["min"])[sample], ref["min"])
    assert np.array_equal(cpu(cells["max"])[sample], ref["max"])
    assert np.array_equal(cpu(cells["hist"])[sample].view(np.uint32), ref["hist"])
    _moment_ok(cpu(cells["mean"])[sample], cpu(cells["m2"])[sample], ref["mean"], ref["m2"], ref["count"])
    assert int(cpu(cells["count"])[:ns].sum()) == int((h_cell >= 0).sum())
    # merge: the oracle's merge of the same per-cell records
    if "comp_band" not in full:
        pytest.skip("needs the seeding comparison")
    rec = dict(count=cpu(cells["count"])[:ns], mean=cpu(cells["mean"])[:ns], m2=cpu(cells["m2"])[:ns],
               min=cpu(cells["min"])[:ns], max=cpu(cells["max"])[:ns],
               hist=cpu(cells["hist"])[:ns].view(np.uint32), comom=None)
    site_comp = np.repeat(np.arange(len(full["comp_band"]), dtype=np.int32), np.diff(full["off"]))
    rc, rb, rv = oracle.merge_hierarchy(rec, site_comp, full["comp_band"], len(full["w"]["iso"]) + 1)
    last = pipe.last
    gv = last["volume"]
    gb, gc = last["bands"], last["comps"]
    for g, r in ((gc, rc), (gb, rb), (gv, rv)):
        k = len(r["count"])
        assert np.array_equal(cpu(g["count"])[:k], r["count"])
        assert np.array_equal(cpu(g["min"])[:k], r["min"]) and np.array_equal(cpu(g["max"])[:k], r["max"])
        assert np.array_equal(cpu(g["hist"])[:k].view(np.uint32), r["hist"])
        _moment_ok(cpu(g["mean"])[:k], cpu(g["m2"])[:k], r["mean"], r["m2"], r["count"])


def test_full_layout_properties(full):
    """The structured layout of the full-size decomposition (all bands, every variable),
    checked by the properties that define a stable sort by (band, component, cell, index):
    the kept voxels are the graph nodes, (cell, index) strictly increases along the layout,
    the cell ranges hold the per-cell counts, component and band offsets are the cell offsets
    of their first cells and the band prefix counts, and the values are the variables at the
    recorded coordinates.  A band subset equals the full layout's band ranges concatenated."""
    pk, pipe, out, bench = full["pk"], full["pipe"], full["out"], full["bench"]
    aux = [full["w"]["aux"][j] for j in range(bench.N_AUX)]
    max_sites = out["site_pos"].numel()
    args = (out["cell"], out["n_sites"], max_sites, out["comp_site_off"], out["comp_band"], out["n_comp"],
            pipe.max_comp)
    lay = pk.structured_layout(*args, aux=aux, ws=pipe.ws, status=pipe.status)
    torch.cuda.synchronize()
    pk.check_status(pipe.status, "layout")
    flat = out["cell"].reshape(-1)
    r = int(lay["n_kept"].item())
    assert r == int((flat >= 0).sum().item())
    order = lay["order"][:r].long()
    key = flat[order].long() * (1 << 32) + order
    assert bool((key[1:] > key[:-1]).all())
    del key
    ns, nc = int(out["n_sites"].item()), int(out["n_comp"].item())
    cnt = torch.bincount(flat[flat >= 0].long(), minlength=ns)
    co = lay["cell_off"]
    assert int(co[0].item()) == 0 and torch.equal(co[1:ns + 1] - co[:ns], cnt)
    off = out["comp_site_off"][:nc + 1].long()
    assert torch.equal(lay["comp_off"][:nc + 1], co[off])
    band = out["band"].reshape(-1)
    bc = torch.bincount(band[band != 255].long(), minlength=256)[:256]
    want = torch.zeros(257, dtype=torch.int64, device=bc.device)
    want[1:] = torch.cumsum(bc, 0)
    assert torch.equal(lay["band_off"], want)
    for j in range(len(aux)):
        assert torch.equal(lay["values"][j, :r], aux[j].reshape(-1)[order])
    keep = [3, 4]
    sub = pk.structured_layout(*args, aux=aux[:2], bands=keep, ws=pipe.ws, status=pipe.status)
    torch.cuda.synchronize()
    pk.check_status(pipe.status, "layout subset")
    bo = lay["band_off"].tolist()
    rs = int(sub["n_kept"].item())
    assert rs == bo[5] - bo[3]
    assert torch.equal(sub["order"][:rs], lay["order"][bo[3]:bo[5]])
    assert torch.equal(sub["values"][:2, :rs], lay["values"][:2, bo[3]:bo[5]])


@pytest.fixture(scope="module")
def precision():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    import paper_2208_06970_b300 as pk
    from paper_2208_06970_b300 import build
    build.build()
    P = bench.precision_setup(pk, 640, torch.device("cuda"))
    P["stats"] = pk.aggregate(P["cell"], P["auxl"], P["sp"], P["ns"], None, None, 0, cov=True, ws=P["ws"],
                              status=P["st"])
    torch.cuda.synchronize()
    pk.check_status(P["st"], "precision form")
    return P


def test_full_precision_moments_and_comoments_sampled_cells(precision):
    """Precision form at full size (640^3, 32 correlated variables), run as the benchmark runs
    it: per-cell counts exact, moments within 1e-6 (float-float, FP64 finalise) and co-moments
    within 1e-4 sqrt(R_ii R_jj) (BF16 split on tcgen05) of the FP64 oracle, on sampled cells
    (random, largest, smallest) whose voxels alone the oracle aggregates."""
    P = precision
    cell, m = P["cell"], P["m"]
    ns = int(P["ns"].item())
    h_cell = cpu(cell).ravel()
    counts = np.bincount(h_cell[h_cell >= 0], minlength=ns)
    got = P["stats"]
    assert np.array_equal(cpu(got["count"])[:ns], counts)
    rng = np.random.default_rng(41)
    live = np.flatnonzero(counts)
    sample = np.unique(np.concatenate([rng.choice(live, size=min(len(live), 64), replace=False),
                                       np.argsort(counts)[-8:], live[np.argsort(counts[live])[:8]]]))
    remap = torch.full((ns,), -1, dtype=torch.int32, device=cell.device)
    remap[torch.from_numpy(sample).to(cell.device).long()] = torch.arange(len(sample), dtype=torch.int32,
                                                                           device=cell.device)
    flat = cell.reshape(-1)
    sel = torch.nonzero(flat >= 0).squeeze(1)
    sel = sel[remap[flat[sel].long()] >= 0]
    sub_cell = cpu(remap[flat[sel].long()])
    sub_aux = np.stack([cpu(P["auxl"][j].reshape(-1)[sel]) for j in range(m)])
    ref = oracle.aggregate(sub_cell, sub_aux, len(sample), n_bins=0, cov=True)
    assert np.array_equal(cpu(got["count"])[sample], ref["count"])
    assert np.array_equal(cpu(got["min"])[sample], ref["min"]) and np.array_equal(cpu(got["max"])[sample], ref["max"])
    _moment_ok(cpu(got["mean"])[sample], cpu(got["m2"])[sample], ref["mean"], ref["m2"], ref["count"])
    C, R = cpu(got["comom"])[sample], ref["comom"]
    iu = np.triu_indices(m)
    diag = {i: k for k, (i, j) in enumerate(zip(*iu)) if i == j}
    for k, (i, j) in enumerate(zip(*iu)):
        scale = np.sqrt(np.maximum(R[:, diag[i]] * R[:, diag[j]], 0.0))
        assert np.all(np.abs(C[:, k] - R[:, k]) <= 1e-4 * scale + 1e-9), (i, j)


def test_full_joint_moments_sampled_cells(full):
    """Joint moments of 4 variables over every cell of the 512^3 layout, as the bench computes them;
    sampled cells (random, largest, smallest) against the FP64 oracle over those cells' voxels,
    and the merged volume record against the oracle's moments of a voxel sample's hierarchy."""
    pk, pipe, out, bench = full["pk"], full["pipe"], full["out"], full["bench"]
    aux = [full["w"]["aux"][j] for j in range(bench.JOINT_VARS)]
    lay = pk.structured_layout(out["cell"], out["n_sites"], out["site_pos"].numel(), out["comp_site_off"],
                               out["comp_band"], out["n_comp"], pipe.max_comp, aux=aux, ws=pipe.ws,
                               status=pipe.status)
    jm = pk.joint_moments([lay["values"][j] for j in range(bench.JOINT_VARS)], lay["cell_off"], out["n_sites"],
                          out["site_pos"].numel(), ws=pipe.ws)
    torch.cuda.synchronize()
    ns = int(out["n_sites"].item())
    co = cpu(lay["cell_off"])[:ns + 1]
    sizes = np.diff(co)
    rng = np.random.default_rng(17)
    pick = np.unique(np.concatenate([rng.choice(ns, 40, replace=False), np.argsort(sizes)[-5:],
                                     np.argsort(sizes)[:5]]))
    pick = pick[sizes[pick] > 0]
    order = cpu(lay["order"])
    A = np.stack([cpu(a).reshape(-1) for a in aux])
    sub_order = np.concatenate([order[co[s]:co[s + 1]] for s in pick])
    sub_off = np.concatenate([[0], np.cumsum(sizes[pick])])
    ref = oracle.joint_moments(A, sub_order, sub_off)
    got = {k: cpu(v)[pick] for k, v in jm.items()}
    from itertools import combinations_with_replacement as cwr
    m = bench.JOINT_VARS
    assert np.array_equal(got["count"], ref["count"])
    sig = np.sqrt(ref["m2"][:, [t for t, (i, j) in enumerate(cwr(range(m), 2)) if i == j]] / ref["count"][:, None])
    for q, key in ((2, "m2"), (3, "m3"), (4, "m4")):
        tups = list(cwr(range(m), q))
        scale = ref["count"][:, None] * np.stack([np.prod(sig[:, list(t)], axis=1) for t in tups], 1)
        assert np.all(np.abs(got[key] - ref[key]) <= 2e-5 * scale + 1e-9), key


def test_full_site_graph_sampled(full):
    """The 512^3 site graph, as the bench builds it: sampled sites' neighbour lists and weights
    against the oracle's graph of the whole volume, and geodesic rows of sampled sources of the
    largest component against the oracle's Dijkstra on that graph."""
    pk, pipe, out = full["pk"], full["pipe"], full["out"]
    g = pk.site_graph(out["cell"], out["band"], out["site_pos"], out["n_sites"], ws=pipe.ws, status=pipe.status)
    torch.cuda.synchronize()
    pk.check_status(pipe.status, "site graph")
    ns = int(out["n_sites"].item())
    sp = cpu(out["site_pos"])[:ns]
    ref = oracle.site_graph(cpu(out["cell"]), full["band"], sp)
    E = int(g["n_edges"].item())
    assert E == len(ref["edges"])
    off = cpu(g["off"])[:ns + 1]
    assert np.array_equal(off, ref["off"])
    adj, w = cpu(g["adj"])[:2 * E], cpu(g["w"])[:2 * E].view(np.uint32)
    assert np.array_equal(adj, ref["dst"]) and np.array_equal(w, ref["w"])
    cso = cpu(out["comp_site_off"])[:int(out["n_comp"].item()) + 1]
    c = int(np.argmax(np.diff(cso)))
    s0, s1 = int(cso[c]), int(cso[c + 1])
    nz, ny, nx = out["cell"].shape
    dist, _ = pk.site_geodesics(g, out["site_pos"], (nx, ny, nz), s0, s1, ws=pipe.ws, status=pipe.status)
    torch.cuda.synchronize()
    pk.check_status(pipe.status, "site geodesics")
    D = cpu(dist).view(np.uint32).astype(np.uint64)
    rng = np.random.default_rng(5)
    for src in rng.choice(s1 - s0, 6, replace=False):
        want = oracle.site_sssp(ref, s0 + int(src))[s0:s1]
        assert np.array_equal(D[src], want)


def _ceil_q16(D):
    """ceil(2^16 sqrt(D)) for an int64 tensor D < 2^20 (exact: a double root, then squares)."""
    v = D << 32
    r = torch.floor(torch.sqrt(D.double()) * 65536.0).long()
    for _ in range(2):
        r = r + (r * r < v).long()
        r = r - ((r > 0) & ((r - 1) * (r - 1) >= v)).long()
    assert bool(((r * r >= v) & ((r == 0) | ((r - 1) * (r - 1) < v))).all())
    return r


def test_full_anyangle_properties(full):
    """The any-angle tessellation of the final 512^3 sites, run as the bench runs it, checked on
    every voxel by properties that hold at any size: the reached voxels are the chamfer
    tessellation's and no length exceeds its geodesic (direct neighbour paths are its edges);
    no length is below the straight segment to the voxel's site; every source gives exactly the
    voxel's length (d[v] = d[src] + ceil(2^16 |x_v - x_src|)) and cell, lengths fall along the
    chain, and d = 0 only on a site's own voxel, so every chain ends at the voxel's site; every
    cell stays in its site's component; sampled shortcut segments see their source (the oracle's
    traversal)."""
    pk, pipe, out = full["pk"], full["pipe"], full["out"]
    band, ns = out["band"], out["n_sites"]
    cell, dist, src, _, rounds = pk.cvt_iterate_anyangle(band, None, out["site_pos"].clone(), ns, 0, want_trace=False,
                                                         ws=pipe.ws, status=pipe.status)
    cc, cd, _ = pk.cvt_iterate(band, None, out["site_pos"].clone(), ns, 0, want_trace=False, ws=pipe.ws,
                               status=pipe.status)
    torch.cuda.synchronize()
    pk.check_status(pipe.status, "any-angle tessellation")
    assert 1 < int(rounds[0]) < (1 << 16)
    nz, ny, nx = band.shape
    c, s = cell.reshape(-1).long(), src.reshape(-1).long()
    d = dist.reshape(-1).long() & 0xFFFFFFFF
    reached = c >= 0
    assert torch.equal(reached, cc.reshape(-1) >= 0)
    assert bool((d[reached] <= (cd.reshape(-1).long() & 0xFFFFFFFF)[reached]).all())
    assert bool((d[reached] < (cd.reshape(-1).long() & 0xFFFFFFFF)[reached]).any())
    idx = torch.nonzero(reached).squeeze(1)
    sp = out["site_pos"].long()

    def sq(a, b):
        ax, ay, az = a % nx, (a // nx) % ny, a // (nx * ny)
        bx, by, bz = b % nx, (b // nx) % ny, b // (nx * ny)
        return (ax - bx) ** 2 + (ay - by) ** 2 + (az - bz) ** 2
    cv = c[idx]
    assert bool((d[idx] >= _ceil_q16(sq(idx, sp[cv]))).all())
    t = s[idx]
    assert bool((t >= 0).all())
    site_vox = t == idx
    assert torch.equal(site_vox, d[idx] == 0) and bool((sp[cv[site_vox]] == idx[site_vox]).all())
    ch = ~site_vox
    i1, t1 = idx[ch], t[ch]
    assert torch.equal(c[t1], c[i1])
    assert torch.equal(d[i1], d[t1] + _ceil_q16(sq(i1, t1)))
    comp = pk.label_components(band)[0].reshape(-1).long()
    assert torch.equal(comp[idx], comp[sp[cv]])
    # shortcut segments (source beyond the 26 neighbours) see their source
    far = ch.clone()
    far[ch] = sq(i1, t1) > 3
    fi = idx[far].cpu().numpy()
    rng = np.random.default_rng(9)
    bnp = full["band"]
    for v in rng.choice(fi, min(2000, len(fi)), replace=False):
        assert oracle.los(bnp, int(v), int(s[int(v)].item()))
