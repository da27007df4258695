"""CPU oracle of the LSRVT hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, single-threaded implementation (``lsrvt_oracle.c``) of what the GPU path
computes, written from Neuroth et al., "Level Set Restricted Voronoi Tessellation for
Large scale Spatial Statistical Analysis" (arXiv 2208.06970).  Only the test suite, the
package smoke check and the benchmark's CPU-baseline leg may import this package.  It
shares no code with the CUDA library and never calls it.

Arrays follow the volume convention of the library: a field is a C-ordered numpy array
of shape (nz, ny, nx) (x fastest), linear index i = x + nx*(y + ny*z).

Parity status of each function (what pins it; see tests/test_oracle_*.py):
  classify            closed form (brute-force count, hand cases)
  label_components    brute-force union-find + adjacency/connectivity invariants
  saliency            hand-computed gradients, closed forms on linear/quadratic fields
  seed                exact-fraction Hamilton apportionment recount, invariants,
                      SplitMix64 published vectors
  assign              per-seed Dijkstra + lexicographic min; chamfer closed form;
                      L-infinity BFS bounds
  update/cvt_iterate  independent closed-form Lloyd on a box; LOS hand cases;
                      invariants (sites stay in their component)
  anyangle_assign     single site in a convex region: ceil(2^16 |x_v - x_s|) closed form;
                      1-D line: nearest-site distances; bounds ceil-Euclidean <= d <= chamfer
                      geodesic (assign) and d >= brute-force visibility-graph shortest path;
                      src chains consistent and ending at the voxel's own site
  aggregate           numpy per-cell statistics (np.var/np.cov definitions)
  merge               direct per-component / per-band statistics
  joint_moments       numpy einsum per region; shift invariance; symmetric data (odd
                      orders vanish); merged records equal direct records of the union
  site_graph          brute-force face adjacency of the cells; weights against exact
                      integer square roots; SSSP against Floyd-Warshall; Euclidean lower bound
  layout              brute-force contiguity and membership of every band, component and
                      cell range; per-cell counts and means against aggregate
"""
import ctypes as C
import numpy as np

from . import build as _build

_lib = None

ERRORS = {0: "ok", -1: "invalid argument", -2: "isovalues not strictly increasing", -3: "capacity",
          -4: "out of memory", -5: "distance overflow", -6: "non-finite value", -7: "round limit reached"}


class OracleError(RuntimeError):
    def __init__(self, rc, what):
        super().__init__("%s: %s (%d)" % (what, ERRORS.get(rc, "?"), rc))
        self.rc = rc


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        i32, i64, u64 = C.c_int32, C.c_int64, C.c_uint64
        L.orc_classify.argtypes = [P, i64, P, i32, P]
        L.orc_label_components.argtypes = [P, i32, i32, i32, P, P, P, P, i32, P]
        L.orc_saliency.argtypes = [P, i32, i32, i32, i32, P]
        L.orc_splitmix64.argtypes = [u64]
        L.orc_splitmix64.restype = u64
        L.orc_seed.argtypes = [P, P, i32, i32, i32, i32, i64, i32, u64, P, P, P, i32, P, P]
        L.orc_assign.argtypes = [P, i32, i32, i32, P, i32, P, P]
        L.orc_los.argtypes = [P, i32, i32, i32, i32, i32]
        L.orc_update.argtypes = [P, P, i32, i32, i32, P, P, P, i32, P, P, P, P, P, P]
        L.orc_update_src.argtypes = [P, P, i32, i32, i32, P, P, P, P, i32, P, P, P, P, P, P]
        L.orc_update_selected.argtypes = [P, P, i32, i32, i32, P, P, P, i32, P, P, P]
        L.orc_cvt_iterate.argtypes = [P, P, i32, i32, i32, P, i32, i32, P, P, P]
        L.orc_anyangle_assign.argtypes = [P, i32, i32, i32, P, i32, i32, P, P, P, P]
        L.orc_cvt_iterate_anyangle.argtypes = [P, P, i32, i32, i32, P, i32, i32, i32, P, P, P, P, P]
        L.orc_aux_range.argtypes = [P, P, i32, i64, i32, P, P, P]
        L.orc_aggregate.argtypes = [P, P, i32, i64, i32, P, P, i32, i32, P, P, P, P, P, P, P]
        L.orc_merge.argtypes = [i32, P, i32, i32, i32, i32] + [P] * 7 + [P] * 7
        L.orc_certify.argtypes = [P, i32, i32, i32, P, i32, P, P]
        L.orc_certify.restype = i64
        L.orc_sssp.argtypes = [P, i32, i32, i32, i32, P]
        L.orc_layout.argtypes = [P, i64, P, i32, P, i32, P, P, i32, P, P, P, P, P, P]
        L.orc_joint_ranges.argtypes = [P, i32, i64, P, P, i32, P, P, P, P, P]
        L.orc_joint_merge.argtypes = [i32, i32, P, P, P, P, P, P, P, P, P, P, P]
        L.orc_site_weight.argtypes = [i32, i32, i32]
        L.orc_site_weight.restype = C.c_uint32
        L.orc_site_edges.argtypes = [P, P, i32, i32, i32, i64, P, P]
        L.orc_site_edges.restype = i64
        L.orc_site_sssp.argtypes = [i32, P, P, P, i32, P]
        L.orc_energy.argtypes = [P, P, P, i64, P]
        L.orc_energy.restype = None
        L.orc_lattice_lloyd.argtypes = [i32, i32, i32, P, i32, i32, P]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise OracleError(rc, what)


def _dims(vol):
    nz, ny, nx = vol.shape
    return int(nx), int(ny), int(nz)


# --------------------------------------------------------------------------- steps
def classify(field, iso):
    """Isoband index per voxel, Sec. 3.1: band = #{i : iso[i] < f}; NaN -> 255."""
    field = np.ascontiguousarray(field, dtype=np.float32)
    iso = np.ascontiguousarray(iso, dtype=np.float32)
    band = np.empty(field.shape, np.uint8)
    _check(lib().orc_classify(_p(field), field.size, _p(iso), len(iso), _p(band)), "classify")
    return band


def label_components(band, max_comp=None):
    """6-connected components of each isoband (Sec. 3.1), ids ordered by (band, min index).

    Returns (comp, comp_band, comp_size, comp_first)."""
    band = np.ascontiguousarray(band, dtype=np.uint8)
    nx, ny, nz = _dims(band)
    n = band.size
    max_comp = n if max_comp is None else max_comp
    comp = np.empty(band.shape, np.int32)
    cb = np.empty(max(max_comp, 1), np.uint8)
    cs = np.empty(max(max_comp, 1), np.int64)
    cf = np.empty(max(max_comp, 1), np.int32)
    nc = np.zeros(1, np.int32)
    _check(lib().orc_label_components(_p(band), nx, ny, nz, _p(comp), _p(cb), _p(cs), _p(cf), max_comp, _p(nc)),
           "label_components")
    k = int(nc[0])
    return comp, cb[:k].copy(), cs[:k].copy(), cf[:k].copy()


def saliency(field, gamma=1):
    """16-bit weights q = max(1, rint(|grad f|^gamma * 65535 / max)) (reading of Sec. 3.3)."""
    field = np.ascontiguousarray(field, dtype=np.float32)
    nx, ny, nz = _dims(field)
    q = np.empty(field.shape, np.uint16)
    _check(lib().orc_saliency(_p(field), nx, ny, nz, int(gamma), _p(q)), "saliency")
    return q


def splitmix64(x):
    return int(lib().orc_splitmix64(C.c_uint64(int(x) & 0xFFFFFFFFFFFFFFFF)))


def seed(comp, q, n_comp, voxels_per_site, strat_block=16, rng_seed=0, max_sites=None):
    """Stratified initial sites (Sec. 3.2, Eq. nc).  Returns (site_pos, site_comp, comp_site_off, n_c)."""
    comp = np.ascontiguousarray(comp, dtype=np.int32)
    nx, ny, nz = _dims(comp)
    if q is not None:
        q = np.ascontiguousarray(q, dtype=np.uint16)
    max_sites = comp.size if max_sites is None else max_sites
    sp = np.empty(max(max_sites, 1), np.int32)
    sc = np.empty(max(max_sites, 1), np.int32)
    off = np.empty(n_comp + 1, np.int32)
    ncomp_sites = np.empty(max(n_comp, 1), np.int64)
    ns = np.zeros(1, np.int32)
    _check(lib().orc_seed(_p(comp), _p(q), nx, ny, nz, int(n_comp), int(voxels_per_site), int(strat_block),
                          C.c_uint64(int(rng_seed) & 0xFFFFFFFFFFFFFFFF), _p(sp), _p(sc), _p(off), int(max_sites),
                          _p(ns), _p(ncomp_sites)), "seed")
    k = int(ns[0])
    return sp[:k].copy(), sc[:k].copy(), off, ncomp_sites[:n_comp].copy()


def assign(band, site_pos):
    """Restricted geodesic Voronoi assignment (Eq. 1), multi-source Dijkstra.  Returns (cell, dist)."""
    band = np.ascontiguousarray(band, dtype=np.uint8)
    site_pos = np.ascontiguousarray(site_pos, dtype=np.int32)
    nx, ny, nz = _dims(band)
    cell = np.empty(band.shape, np.int32)
    dist = np.empty(band.shape, np.uint32)
    _check(lib().orc_assign(_p(band), nx, ny, nz, _p(site_pos), len(site_pos), _p(cell), _p(dist)), "assign")
    return cell, dist


def los(band, v, s):
    band = np.ascontiguousarray(band, dtype=np.uint8)
    nx, ny, nz = _dims(band)
    return bool(lib().orc_los(_p(band), nx, ny, nz, int(v), int(s)))


def update(band, q, cell, dist, site_pos, diagnostics=False, src=None):
    """Geodesically weighted site update (Eq. 2).  Returns (new_pos, (moved, sumsq, sum_ds_q16)[, diag])
    with sum_ds_q16 the sum over moved sites of ceil(2^16 |displacement|).

    With `src` (the source map of the any-angle tessellation) phi follows src chains instead
    of the chamfer parents."""
    band = np.ascontiguousarray(band, dtype=np.uint8)
    nx, ny, nz = _dims(band)
    if q is not None:
        q = np.ascontiguousarray(q, dtype=np.uint16)
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    dist = np.ascontiguousarray(dist, dtype=np.uint32)
    site_pos = np.ascontiguousarray(site_pos, dtype=np.int32)
    S = len(site_pos)
    new_pos = np.empty(max(S, 1), np.int32)
    stats = np.zeros(3, np.int64)
    if diagnostics:
        parent = np.empty(band.shape, np.int32)
        losv = np.empty(band.shape, np.uint8)
        phi = np.empty(band.shape, np.int32)
        sums = np.empty((max(S, 1), 4), np.int64)
    else:
        parent = losv = phi = sums = None
    if src is None:
        _check(lib().orc_update(_p(band), _p(q), nx, ny, nz, _p(cell), _p(dist), _p(site_pos), S, _p(new_pos),
                                _p(stats), _p(parent), _p(losv), _p(phi), _p(sums)), "update")
    else:
        src = np.ascontiguousarray(src, dtype=np.int32)
        _check(lib().orc_update_src(_p(band), _p(q), nx, ny, nz, _p(cell), _p(dist), _p(src), _p(site_pos), S,
                                    _p(new_pos), _p(stats), _p(parent), _p(losv), _p(phi), _p(sums)), "update_src")
    out = (new_pos[:S].copy(), (int(stats[0]), int(stats[1]), int(stats[2])))
    if diagnostics:
        return out + (dict(parent=parent, los=losv.astype(bool), phi=phi, sums=sums[:S]),)
    return out


def update_selected(band, q, cell, dist, site_pos, sites):
    """Eq. 2 update restricted to the cells of `sites` (exact for those sites: parents,
    line of sight and phi stay inside a cell).  Returns (new positions of `sites`, their
    integer sums (len(sites), 4))."""
    band = np.ascontiguousarray(band, dtype=np.uint8)
    nx, ny, nz = _dims(band)
    if q is not None:
        q = np.ascontiguousarray(q, dtype=np.uint16)
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    dist = np.ascontiguousarray(dist, dtype=np.uint32)
    site_pos = np.ascontiguousarray(site_pos, dtype=np.int32)
    S = len(site_pos)
    sites = np.asarray(sites, dtype=np.int64)
    sel = np.zeros(max(S, 1), np.uint8)
    sel[sites] = 1
    new_pos = np.empty(max(S, 1), np.int32)
    sums = np.zeros((max(S, 1), 4), np.int64)
    _check(lib().orc_update_selected(_p(band), _p(q), nx, ny, nz, _p(cell), _p(dist), _p(site_pos), S, _p(sel),
                                     _p(new_pos), _p(sums)), "update_selected")
    return new_pos[sites].copy(), sums[sites].copy()


def cvt_iterate(band, q, site_pos, n_iters):
    """Algorithm 1 after seeding: n_iters x (assign, update) then a final assign.

    Returns (site_pos, cell, dist, trace[n_iters, TRACE]); a trace row is (sites moved,
    sum |d|^2, sum ceil(2^16 |d|), energy low 64 bits, energy high 64 bits) -- see
    trace_columns()."""
    band = np.ascontiguousarray(band, dtype=np.uint8)
    nx, ny, nz = _dims(band)
    if q is not None:
        q = np.ascontiguousarray(q, dtype=np.uint16)
    sp = np.array(site_pos, dtype=np.int32, copy=True)
    cell = np.empty(band.shape, np.int32)
    dist = np.empty(band.shape, np.uint32)
    trace = np.zeros((max(n_iters, 1), TRACE), np.int64)
    _check(lib().orc_cvt_iterate(_p(band), _p(q), nx, ny, nz, _p(sp), len(sp), int(n_iters), _p(cell), _p(dist),
                                 _p(trace)), "cvt_iterate")
    return sp, cell, dist, trace[:n_iters]


TRACE = 5  # columns of a Lloyd-iteration trace row


def trace_columns(trace):
    """Named columns of a trace [n_iters, TRACE]: moved, sumsq, sum_ds_q16 (int64 arrays),
    energy (exact Python ints, sum of m_v D(v)^2 in (1/2^16 voxel)^2 units) and mean_ds
    (float: mean displacement over n sites needs n, so it is left to the caller)."""
    t = np.asarray(trace, dtype=np.int64)
    lo = t[:, 3].astype(np.uint64)
    hi = t[:, 4].astype(np.uint64)
    energy = [int(h) << 64 | int(l) for l, h in zip(lo, hi)]
    return dict(moved=t[:, 0], sumsq=t[:, 1], sum_ds_q16=t[:, 2], energy=energy)


def energy(q, cell, dist):
    """CVT energy sum over assigned voxels of m_v D(v)^2 (16.16 distances), an exact int."""
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    dist = np.ascontiguousarray(dist, dtype=np.uint32)
    if q is not None:
        q = np.ascontiguousarray(q, dtype=np.uint16)
    out = np.zeros(2, np.uint64)
    lib().orc_energy(_p(q), _p(cell), _p(dist), cell.size, _p(out))
    return int(out[1]) << 64 | int(out[0])


def lattice_lloyd(shape, site_pos, n_iters):
    """Textbook Euclidean Lloyd on the lattice of a box (nearest site, centroid rounded half
    up).  shape = (nz, ny, nx).  Returns (site_pos, energy[n_iters + 1])."""
    nz, ny, nx = shape
    sp = np.array(site_pos, dtype=np.int32, copy=True)
    e = np.zeros(n_iters + 1, np.int64)
    _check(lib().orc_lattice_lloyd(nx, ny, nz, _p(sp), len(sp), int(n_iters), _p(e)), "lattice_lloyd")
    return sp, e


def anyangle_assign(band, site_pos, max_rounds=1 << 16):
    """Any-angle restricted geodesic Voronoi tessellation (Sec. 3.2 region growing with
    src(w) shortcuts, synchronous rounds).  Returns (cell, dist, src, rounds)."""
    band = np.ascontiguousarray(band, dtype=np.uint8)
    site_pos = np.ascontiguousarray(site_pos, dtype=np.int32)
    nx, ny, nz = _dims(band)
    cell = np.empty(band.shape, np.int32)
    dist = np.empty(band.shape, np.uint32)
    src = np.empty(band.shape, np.int32)
    rounds = np.zeros(1, np.int32)
    _check(lib().orc_anyangle_assign(_p(band), nx, ny, nz, _p(site_pos), len(site_pos), int(max_rounds), _p(cell),
                                     _p(dist), _p(src), _p(rounds)), "anyangle_assign")
    return cell, dist, src, int(rounds[0])


def cvt_iterate_anyangle(band, q, site_pos, n_iters, max_rounds=1 << 16):
    """Algorithm 1 with the any-angle tessellation; the Eq. 2 update follows src chains.

    Returns (site_pos, cell, dist, src, trace[n_iters, TRACE], rounds[n_iters + 1])."""
    band = np.ascontiguousarray(band, dtype=np.uint8)
    nx, ny, nz = _dims(band)
    if q is not None:
        q = np.ascontiguousarray(q, dtype=np.uint16)
    sp = np.array(site_pos, dtype=np.int32, copy=True)
    cell = np.empty(band.shape, np.int32)
    dist = np.empty(band.shape, np.uint32)
    src = np.empty(band.shape, np.int32)
    trace = np.zeros((max(n_iters, 1), TRACE), np.int64)
    rounds = np.zeros(n_iters + 1, np.int32)
    _check(lib().orc_cvt_iterate_anyangle(_p(band), _p(q), nx, ny, nz, _p(sp), len(sp), int(n_iters),
                                          int(max_rounds), _p(cell), _p(dist), _p(src), _p(trace), _p(rounds)),
           "cvt_iterate_anyangle")
    return sp, cell, dist, src, trace[:n_iters], rounds


def aux_range(cell, aux, n_bins):
    """Per-variable (lo, hi, scale) over valid voxels; scale = float32(n_bins) / (hi - lo)."""
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    aux = np.ascontiguousarray(aux, dtype=np.float32)
    m = aux.shape[0]
    lo = np.empty(max(m, 1), np.float32); hi = np.empty(max(m, 1), np.float32); sc = np.empty(max(m, 1), np.float32)
    _check(lib().orc_aux_range(_p(cell), _p(aux), m, cell.size, int(n_bins), _p(lo), _p(hi), _p(sc)), "aux_range")
    return lo[:m], hi[:m], sc[:m]


def aggregate(cell, aux, n_cells, lo=None, scale=None, n_bins=32, cov=False):
    """Per-cell statistics (FP64 two-pass definitions).  aux has shape (m, nz, ny, nx) or (m, N)."""
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    aux = np.ascontiguousarray(aux, dtype=np.float32).reshape(-1, cell.size) if np.asarray(aux).size else \
        np.zeros((0, cell.size), np.float32)
    m = aux.shape[0]
    if lo is None or scale is None:
        lo, _, scale = aux_range(cell, aux, n_bins)
    lo = np.ascontiguousarray(lo, dtype=np.float32)
    scale = np.ascontiguousarray(scale, dtype=np.float32)
    S = int(n_cells)
    T = m * (m + 1) // 2
    out = dict(count=np.empty(S, np.int64), mean=np.empty((S, m)), m2=np.empty((S, m)),
               min=np.empty((S, m), np.float32), max=np.empty((S, m), np.float32),
               hist=np.empty((S, m, n_bins), np.uint32), comom=np.empty((S, T)) if cov else None)
    _check(lib().orc_aggregate(_p(cell), _p(aux), m, cell.size, S, _p(lo), _p(scale), int(n_bins), int(bool(cov)),
                               _p(out["count"]), _p(out["mean"]), _p(out["m2"]), _p(out["min"]), _p(out["max"]),
                               _p(out["hist"]), _p(out["comom"])), "aggregate")
    return out


def merge(stats, parent, n_parent):
    """Chan pairwise merge of child records into parent records (children in id order)."""
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    S, m = stats["mean"].shape
    n_bins = stats["hist"].shape[2]
    cov = stats.get("comom") is not None
    T = m * (m + 1) // 2
    P = int(n_parent)
    out = dict(count=np.empty(P, np.int64), mean=np.empty((P, m)), m2=np.empty((P, m)),
               min=np.empty((P, m), np.float32), max=np.empty((P, m), np.float32),
               hist=np.empty((P, m, n_bins), np.uint32), comom=np.empty((P, T)) if cov else None)
    cs = {k: (None if v is None else np.ascontiguousarray(v)) for k, v in stats.items()}
    _check(lib().orc_merge(S, _p(parent), P, m, n_bins, int(cov), _p(cs["count"]), _p(cs["mean"]), _p(cs["m2"]),
                           _p(cs["min"]), _p(cs["max"]), _p(cs["hist"]), _p(cs.get("comom")),
                           _p(out["count"]), _p(out["mean"]), _p(out["m2"]), _p(out["min"]), _p(out["max"]),
                           _p(out["hist"]), _p(out["comom"])), "merge")
    return out


def merge_hierarchy(cell_stats, site_comp, comp_band, n_bands):
    """cell -> component -> band -> volume.  Returns (comp_stats, band_stats, volume_stats)."""
    comps = merge(cell_stats, site_comp, len(comp_band))
    bands = merge(comps, np.asarray(comp_band, dtype=np.int32), n_bands)
    vol = merge(bands, np.zeros(n_bands, np.int32), 1)
    return comps, bands, vol


def layout(cell, site_comp, comp_band, aux=None, bands=None):
    """Structured data layout (Sec. 3.2 "Data Reduction and Structured Data Layout"): kept
    voxels ordered by (band, component, cell, linear index).  bands: iterable of kept band
    ids (None = all).  Returns dict(order, values (m, r), cell_off, comp_off, band_off, n_kept)."""
    cell = np.ascontiguousarray(cell, dtype=np.int32).ravel()
    site_comp = np.ascontiguousarray(site_comp, dtype=np.int32)
    comp_band = np.ascontiguousarray(comp_band, dtype=np.uint8)
    n = cell.size
    aux = np.zeros((0, n), np.float32) if aux is None or np.asarray(aux).size == 0 else \
        np.ascontiguousarray(aux, dtype=np.float32).reshape(-1, n)
    m = aux.shape[0]
    mask = np.zeros(8, np.uint32)
    for b in (range(256) if bands is None else bands):
        mask[int(b) >> 5] |= np.uint32(1 << (int(b) & 31))
    S, K = site_comp.size, comp_band.size
    order = np.empty(max(n, 1), np.int32)
    values = np.empty((max(m, 1), n), np.float32)
    cell_off = np.empty(S + 1, np.int64)
    comp_off = np.empty(K + 1, np.int64)
    band_off = np.empty(257, np.int64)
    nk = np.zeros(1, np.int64)
    _check(lib().orc_layout(_p(cell), n, _p(site_comp), S, _p(comp_band), K, _p(mask), _p(aux), m, _p(order),
                            _p(values), _p(cell_off), _p(comp_off), _p(band_off), _p(nk)), "layout")
    r = int(nk[0])
    return dict(order=order[:r], values=values[:m, :r], cell_off=cell_off, comp_off=comp_off, band_off=band_off,
                n_kept=r)


def _tcounts(m):
    from math import comb
    return comb(m + 1, 2), comb(m + 2, 3), comb(m + 3, 4)


def joint_moments(aux, order, off):
    """Joint central moments of orders 2..4 (m <= 8 variables) over the ranges
    [off[r], off[r+1]) of the voxel list `order` (e.g. a structured layout).  aux: (m, N).
    Returns dict(count, mean (R, m), m2 (R, T2), m3 (R, T3), m4 (R, T4)); tuples i<=j<=k<=l
    in lexicographic order."""
    aux = np.ascontiguousarray(aux, dtype=np.float32)
    aux = aux.reshape(aux.shape[0], -1)
    m, n = aux.shape
    order = np.ascontiguousarray(order, dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int64)
    R = off.size - 1
    T2, T3, T4 = _tcounts(m)
    out = dict(count=np.empty(R, np.int64), mean=np.empty((R, m)), m2=np.empty((R, T2)), m3=np.empty((R, T3)),
               m4=np.empty((R, T4)))
    _check(lib().orc_joint_ranges(_p(aux), m, n, _p(order), _p(off), R, _p(out["count"]), _p(out["mean"]),
                                  _p(out["m2"]), _p(out["m3"]), _p(out["m4"])), "joint_moments")
    return out


def joint_merge(rec, child_off):
    """Pairwise (Pebay 2008) merge of joint-moment records: parent p combines the children
    [child_off[p], child_off[p+1]) in id order."""
    child_off = np.ascontiguousarray(child_off, dtype=np.int64)
    P = child_off.size - 1
    m = rec["mean"].shape[1]
    T2, T3, T4 = _tcounts(m)
    out = dict(count=np.empty(P, np.int64), mean=np.empty((P, m)), m2=np.empty((P, T2)), m3=np.empty((P, T3)),
               m4=np.empty((P, T4)))
    c = {k: np.ascontiguousarray(v) for k, v in rec.items()}
    _check(lib().orc_joint_merge(m, P, _p(child_off), _p(c["count"]), _p(c["mean"]), _p(c["m2"]), _p(c["m3"]),
                                 _p(c["m4"]), _p(out["count"]), _p(out["mean"]), _p(out["m2"]), _p(out["m3"]),
                                 _p(out["m4"])), "joint_merge")
    return out


def site_weight(dx, dy, dz):
    """Edge weight between two sites: ceil(2^16 * ||(dx, dy, dz)||_2) (an integer)."""
    return int(lib().orc_site_weight(int(dx), int(dy), int(dz)))


def site_graph(cell, band, site_pos):
    """Voronoi site graph ("Voronoi Cell Views": connectivity from region adjacency): cells are
    adjacent when two of their voxels are face neighbours.  Returns dict(edges (E, 2) a < b in
    (a, b) order, weight (E,) uint32, off (S+1,) int64, dst (2E,) int32, w (2E,) uint32) with the
    CSR holding both directions, neighbours in increasing order."""
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    band = np.ascontiguousarray(band, dtype=np.uint8)
    nx, ny, nz = _dims(cell)
    site_pos = np.asarray(site_pos, dtype=np.int64)
    S = site_pos.size
    cap = max(16, 13 * cell.size)
    ea = np.empty(cap, np.int32)
    eb = np.empty(cap, np.int32)
    E = lib().orc_site_edges(_p(cell), _p(band), nx, ny, nz, cap, _p(ea), _p(eb))
    if E < 0:
        raise OracleError(int(E), "site_edges")
    ea, eb = ea[:E], eb[:E]
    px, py, pz = site_pos % nx, (site_pos // nx) % ny, site_pos // (nx * ny)
    w = np.array([site_weight(px[b] - px[a], py[b] - py[a], pz[b] - pz[a]) for a, b in zip(ea, eb)], np.uint32)
    src = np.concatenate([ea, eb])
    dst = np.concatenate([eb, ea]).astype(np.int32)
    ww = np.concatenate([w, w])
    order = np.lexsort((dst, src))
    src, dst, ww = src[order], dst[order], ww[order]
    off = np.zeros(S + 1, np.int64)
    np.add.at(off, src + 1, 1)
    off = np.cumsum(off)
    return dict(edges=np.stack([ea, eb], 1), weight=w, off=off, dst=dst, w=ww)


def site_sssp(graph, src):
    """Shortest path lengths (weight units) from site `src` to every site (Dijkstra);
    2^64 - 1 where unreachable."""
    off = np.ascontiguousarray(graph["off"], dtype=np.int64)
    S = off.size - 1
    d = np.empty(S, np.uint64)
    _check(lib().orc_site_sssp(S, _p(off), _p(np.ascontiguousarray(graph["dst"], np.int32)),
                               _p(np.ascontiguousarray(graph["w"], np.uint32)), int(src), _p(d)), "site_sssp")
    return d


# --------------------------------------------------------------------------- checkers
def certify(band, site_pos, cell, dist):
    """Number of voxels violating the Bellman equations of the lexicographic key (0 = exact)."""
    band = np.ascontiguousarray(band, dtype=np.uint8)
    nx, ny, nz = _dims(band)
    site_pos = np.ascontiguousarray(site_pos, dtype=np.int32)
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    dist = np.ascontiguousarray(dist, dtype=np.uint32)
    r = lib().orc_certify(_p(band), nx, ny, nz, _p(site_pos), len(site_pos), _p(cell), _p(dist))
    if r < 0:
        raise OracleError(-1, "certify")
    return int(r)


def sssp(band, src):
    band = np.ascontiguousarray(band, dtype=np.uint8)
    nx, ny, nz = _dims(band)
    d = np.empty(band.shape, np.uint64)
    _check(lib().orc_sssp(_p(band), nx, ny, nz, int(src), _p(d)), "sssp")
    return d
