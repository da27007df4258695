"""GPU parity of the Voronoi site graph (region adjacency with integer Euclidean weights) and of
the geodesic site distances and their ratio ||x_i - x_j|| / gd (the "Voronoi Cell Views"
section) against the oracle: the CSR bit for bit, distances bit for bit (integer sums), the
ratio within float rounding."""
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


def _case(dims, seed, P, iso=(0.3, 0.6)):
    f = workloads.blob_field(dims, seed, "cpu", n_blobs=8).numpy()
    f.ravel()[::61] = np.nan
    band = oracle.classify(f, np.array(iso, np.float32))
    comp, cb, cs, cf = oracle.label_components(band)
    sp, sc, off, nc = oracle.seed(comp, None, len(cb), P, 16, seed)
    cell, dist = oracle.assign(band, sp)
    return band, cell, sp, sc, off


def _gpu_graph(pk, band, cell, sp, slack=0):
    st = pk.new_status()
    spt = torch.zeros(len(sp) + slack, dtype=torch.int32, device="cuda")
    spt[:len(sp)] = torch.from_numpy(sp.astype(np.int32)).cuda()
    g = pk.site_graph(torch.from_numpy(cell).cuda(), torch.from_numpy(band).cuda(), spt,
                      torch.tensor([len(sp)], dtype=torch.int32, device="cuda"), status=st)
    pk.check_status(st, "site graph")
    return g, spt


@pytest.mark.parametrize("dims,P,seed", [((44, 30, 21), 200, 1), ((37, 29, 23), 64, 2), ((64, 64, 64), 512, 3),
                                         ((24, 20, 16), 2, 4)])
def test_site_graph_parity(pk, dims, P, seed):
    band, cell, sp, sc, off = _case(dims, seed, P)
    ref = oracle.site_graph(cell, band, sp)
    g, spt = _gpu_graph(pk, band, cell, sp, slack=5)
    E = int(g["n_edges"].item())
    S = len(sp)
    assert E == len(ref["edges"])
    assert np.array_equal(cpu(g["off"])[:S + 1], ref["off"])
    assert np.all(cpu(g["off"])[S + 1:] == 2 * E)  # capacity rows beyond the live sites are empty
    assert np.array_equal(cpu(g["adj"])[:2 * E], ref["dst"])
    assert np.array_equal(cpu(g["w"])[:2 * E].view(np.uint32), ref["w"])


@pytest.mark.parametrize("dims,P,seed", [((44, 30, 21), 150, 5), ((40, 36, 28), 60, 6)])
def test_site_geodesics_parity(pk, dims, P, seed):
    band, cell, sp, sc, off = _case(dims, seed, P)
    ref = oracle.site_graph(cell, band, sp)
    g, spt = _gpu_graph(pk, band, cell, sp)
    INF64 = np.iinfo(np.uint64).max
    nz, ny, nx = cell.shape
    pos = np.stack([sp % nx, (sp // nx) % ny, sp // (nx * ny)], 1).astype(np.float64)
    # every component on its own, then one range over all sites (unreachable across components)
    ranges = [(int(off[c]), int(off[c + 1])) for c in range(len(off) - 1)] + [(0, len(sp))]
    for s0, s1 in ranges:
        st = pk.new_status()
        dist, ratio = pk.site_geodesics(g, spt, (nx, ny, nz), s0, s1, c_far=3.0, status=st)
        pk.check_status(st, "geodesics")
        D = cpu(dist).view(np.uint32).astype(np.uint64)
        R = cpu(ratio).astype(np.float64)
        k = s1 - s0
        for i in range(k):
            want = oracle.site_sssp(ref, s0 + i)[s0:s1]
            fin = want != INF64
            assert np.array_equal(D[i][fin], want[fin])
            assert np.all(D[i][~fin] == 0xFFFFFFFF)
            eu = np.linalg.norm(pos[s0:s1] - pos[s0 + i], axis=1) * 65536.0
            wr = np.where(fin, eu / np.maximum(want.astype(np.float64), 1), 3.0)
            wr[i] = 1.0
            assert np.allclose(R[i], wr, rtol=2e-6, atol=0)
        if (s0, s1) != (0, len(sp)):
            assert np.all(D != 0xFFFFFFFF)  # a component is connected through its cells


def test_site_geodesics_reject_open_range(pk):
    # a range that cuts a component: arcs leave it, reported in the status word
    band, cell, sp, sc, off = _case((44, 30, 21), 7, 100)
    sizes = np.diff(off)
    c = int(np.argmax(sizes))
    assert sizes[c] > 2
    g, spt = _gpu_graph(pk, band, cell, sp)
    st = pk.new_status()
    nz, ny, nx = cell.shape
    pk.site_geodesics(g, spt, (nx, ny, nz), int(off[c]), int(off[c]) + 2, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 1
