"""B300-native Level Set Restricted Voronoi Tessellation (LSRVT) hot path.

Thin Python binding of the C ABI in ``include/lsrvt.h`` (``liblsrvt.so``, hand-written
CUDA for sm_103a).  Every step runs in the library's kernels; this module only
allocates device tensors with PyTorch, passes their pointers and the current CUDA stream,
and reads the device status word.  There is no CPU fallback: without the built library
or without a CUDA device the calls raise.

Method: Neuroth et al., "Level Set Restricted Voronoi Tessellation for Large scale
Spatial Statistical Analysis" (arXiv 2208.06970).

The functions keep the C names without the ``lsrvt_`` prefix:
    classify, label_components, saliency_grad, seed, cvt_iterate, aux_range,
    aggregate, merge_hierarchy
and ``decompose`` chains them (Algorithm 1 plus statistics) on one stream.
"""
import ctypes as C
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblsrvt.so")

STATUS = {0: "ok", 1: "invalid argument", 2: "isovalues not strictly increasing", 3: "capacity exceeded",
          4: "non-finite input value", 5: "device loop limit reached", 6: "geodesic distance overflow",
          7: "CUDA launch failure", 8: "workspace missing, misaligned or too small"}
STEP = dict(classify=0, label=1, saliency=2, seed=3, cvt=4, aggregate=5, merge=6, layout=7, joint=8, graph=9,
            cvt_anyangle=10)
STATS_HIST = 1
STATS_COV = 2
TRACE = 5  # columns of a Lloyd-iteration trace record (LSRVT_TRACE)


class LsrvtError(RuntimeError):
    def __init__(self, code, where):
        super().__init__("%s: %s (%d)" % (where, STATUS.get(code, "?"), code))
        self.code = code


class Dims(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32)]


class SeedParams(C.Structure):
    _fields_ = [("voxels_per_site", C.c_int64), ("strat_block", C.c_int32), ("max_strata", C.c_int32),
                ("rng_seed", C.c_uint64)]


class Stats(C.Structure):
    _fields_ = [("count", C.c_void_p), ("mean", C.c_void_p), ("m2", C.c_void_p), ("vmin", C.c_void_p),
                ("vmax", C.c_void_p), ("hist", C.c_void_p), ("comom", C.c_void_p)]


class Block(C.Structure):
    _fields_ = [("d", Dims), ("x0", C.c_int32), ("y0", C.c_int32), ("z0", C.c_int32), ("band", C.c_void_p),
                ("q", C.c_void_p), ("site_pos", C.c_void_p), ("n_sites", C.c_void_p), ("cell", C.c_void_p),
                ("dist", C.c_void_p)]


MAX_PACK_BLOCKS = 128

_lib = None


class Joint(C.Structure):
    _fields_ = [("count", C.c_void_p), ("mean", C.c_void_p), ("m2", C.c_void_p), ("m3", C.c_void_p),
                ("m4", C.c_void_p)]


def lib():
    """Load liblsrvt.so (built in-tree by build.py); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("liblsrvt.so is not built; run paper_2208_06970_b300/build.py")
        L = C.CDLL(LIB_PATH)
        P, i32, i64, u32, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_size_t
        L.lsrvt_status_string.argtypes = [C.c_int]
        L.lsrvt_status_string.restype = C.c_char_p
        L.lsrvt_version.restype = i32
        L.lsrvt_workspace_bytes.argtypes = [C.c_int, Dims, i32, i32, i32]
        L.lsrvt_workspace_bytes.restype = sz
        L.lsrvt_classify.argtypes = [P, Dims, P, i32, P, P]
        L.lsrvt_label_components.argtypes = [P, Dims, P, P, P, P, i32, P, P, sz, P, P]
        L.lsrvt_label_components_static.argtypes = [P, Dims, P, P, P, P, i32, P, P, P]
        L.lsrvt_saliency_grad.argtypes = [P, Dims, i32, P, P, sz, P]
        L.lsrvt_seed.argtypes = [P, P, Dims, P, i32, SeedParams, P, P, P, i32, P, P, sz, P, P]
        L.lsrvt_cvt_iterate.argtypes = [P, P, Dims, P, P, i32, i32, P, P, P, P, sz, P, P]
        L.lsrvt_cvt_iterate_anyangle.argtypes = [P, P, Dims, P, P, i32, i32, i32, P, P, P, P, P, P, sz, P, P]
        L.lsrvt_aux_range.argtypes = [P, P, i32, Dims, i32, P, P, P, P]
        L.lsrvt_aggregate.argtypes = [P, P, i32, Dims, P, P, i32, u32, P, P, i32, Stats, P, sz, P, P]
        L.lsrvt_merge_hierarchy.argtypes = [Stats, P, i32, i32, i32, u32, P, P, P, i32, i32, Stats, Stats, Stats, P,
                                            sz, P]
        L.lsrvt_set_stream_share.argtypes = [P, i32]
        L.lsrvt_structured_layout.argtypes = [P, Dims, P, i32, P, P, P, i32, P, P, i32, P, P, P, P, P, P, P, P, sz, P,
                                              P]
        L.lsrvt_joint_moments.argtypes = [P, i32, i64, P, P, i32, Joint, P, sz, P]
        L.lsrvt_merge_joint_hierarchy.argtypes = [Joint, P, i32, i32, P, P, P, i32, i32, Joint, Joint, Joint, P, sz, P]
        L.lsrvt_site_graph.argtypes = [P, P, Dims, P, P, i32, P, P, P, i64, P, P, sz, P, P]
        L.lsrvt_site_geodesics.argtypes = [P, P, P, P, Dims, i32, i32, P, P, C.c_float, P, sz, P, P]
        L.lsrvt_pack_blocks.argtypes = [P, i32, Dims, P, P, P, i32, P, P, P, P]
        L.lsrvt_unpack_blocks.argtypes = [P, i32, Dims, P, P, P, P, P]
        for name in ("lsrvt_classify", "lsrvt_label_components", "lsrvt_label_components_static",
                     "lsrvt_saliency_grad", "lsrvt_seed",
                     "lsrvt_cvt_iterate", "lsrvt_cvt_iterate_anyangle", "lsrvt_aux_range", "lsrvt_aggregate",
                     "lsrvt_merge_hierarchy", "lsrvt_set_stream_share", "lsrvt_structured_layout", "lsrvt_joint_moments",
                     "lsrvt_merge_joint_hierarchy", "lsrvt_site_graph", "lsrvt_site_geodesics",
                     "lsrvt_pack_blocks", "lsrvt_unpack_blocks"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def exported_symbols():
    return ["lsrvt_status_string", "lsrvt_version", "lsrvt_workspace_bytes", "lsrvt_classify",
            "lsrvt_label_components", "lsrvt_label_components_static", "lsrvt_saliency_grad", "lsrvt_seed", "lsrvt_cvt_iterate", "lsrvt_cvt_iterate_anyangle", "lsrvt_aux_range",
            "lsrvt_aggregate", "lsrvt_merge_hierarchy", "lsrvt_set_stream_share", "lsrvt_structured_layout",
            "lsrvt_joint_moments", "lsrvt_merge_joint_hierarchy", "lsrvt_site_graph", "lsrvt_site_geodesics",
            "lsrvt_pack_blocks", "lsrvt_unpack_blocks"]


def set_stream_share(percent, stream=None):
    """Kernels launched on `stream` (default: the current stream) size their grids to `percent`
    of the SMs (1..100), so decompositions on several streams run side by side."""
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().lsrvt_set_stream_share(C.c_void_p(s.cuda_stream), int(percent)), "lsrvt_set_stream_share")


# --------------------------------------------------------------------------- helpers
def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dims(t):
    nz, ny, nx = t.shape[-3:]
    return Dims(int(nx), int(ny), int(nz))


def _check(rc, where):
    if rc != 0:
        raise LsrvtError(rc, where)


def _require_cuda(*ts):
    for t in ts:
        if t is not None and (not t.is_cuda or not t.is_contiguous()):
            raise ValueError("device tensors must be contiguous CUDA tensors")


def default_max_comp(n):
    """Default component capacity: every voxel for small volumes, N/16 (at least 2^20) otherwise."""
    return int(min(n, max(1 << 20, n // 16)))


def workspace_bytes(step, dims, max_comp=0, max_sites=0, n_aux=0):
    d = dims if isinstance(dims, Dims) else Dims(*[int(v) for v in dims])
    return int(lib().lsrvt_workspace_bytes(STEP[step], d, int(max_comp), int(max_sites), int(n_aux)))


class Workspace:
    """A growing device scratch buffer (256-byte aligned) reused across calls on one stream."""

    def __init__(self, device="cuda"):
        self.device = device
        self.buf = None

    def get(self, nbytes):
        nbytes = max(int(nbytes), 256)
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        return self.buf


def new_status(device="cuda"):
    return torch.zeros(1, dtype=torch.int32, device=device)


def check_status(status, where="device"):
    """Synchronise and raise on a data-dependent error recorded by the kernels."""
    code = int(status.item())
    if code != 0:
        raise LsrvtError(code, where)


# --------------------------------------------------------------------------- steps
def classify(field, iso, band=None):
    """Isoband index per voxel (Sec. 3.1): band = #{i : iso[i] < f}; NaN -> 255."""
    _require_cuda(field)
    iso = np.ascontiguousarray(iso, dtype=np.float32)
    if band is None:
        band = torch.empty(field.shape, dtype=torch.uint8, device=field.device)
    _check(lib().lsrvt_classify(_ptr(field), _dims(field), iso.ctypes.data_as(C.c_void_p), len(iso), _ptr(band),
                                _stream()), "lsrvt_classify")
    return band


def label_components(band, max_comp=None, ws=None, status=None):
    """6-connected components of each isoband, ids ordered by (band, min index).

    Returns (comp, comp_band, comp_size, comp_first, n_comp_dev)."""
    _require_cuda(band)
    dev = band.device
    n = band.numel()
    max_comp = default_max_comp(n) if max_comp is None else int(max_comp)
    comp = torch.empty(band.shape, dtype=torch.int32, device=dev)
    cb = torch.empty(max(max_comp, 1), dtype=torch.uint8, device=dev)
    cs = torch.empty(max(max_comp, 1), dtype=torch.int64, device=dev)
    cf = torch.empty(max(max_comp, 1), dtype=torch.int32, device=dev)
    nc = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = ws or Workspace(dev)
    status = new_status(dev) if status is None else status
    wb = workspace_bytes("label", _dims(band))
    buf = ws.get(wb)
    _check(lib().lsrvt_label_components(_ptr(band), _dims(band), _ptr(comp), _ptr(cb), _ptr(cs), _ptr(cf), max_comp,
                                        _ptr(nc), _ptr(buf), buf.numel(), _ptr(status), _stream()),
           "lsrvt_label_components")
    return comp, cb, cs, cf, nc


def label_components_static(band, max_comp=None, status=None):
    """lsrvt_label_components_static: the same labelling with the library's built-in scratch
    (no workspace, no allocation inside the call); volumes up to 2^18 voxels."""
    _require_cuda(band)
    dev = band.device
    n = band.numel()
    max_comp = default_max_comp(n) if max_comp is None else int(max_comp)
    comp = torch.empty(band.shape, dtype=torch.int32, device=dev)
    cb = torch.empty(max(max_comp, 1), dtype=torch.uint8, device=dev)
    cs = torch.empty(max(max_comp, 1), dtype=torch.int64, device=dev)
    cf = torch.empty(max(max_comp, 1), dtype=torch.int32, device=dev)
    nc = torch.zeros(1, dtype=torch.int32, device=dev)
    status = new_status(dev) if status is None else status
    _check(lib().lsrvt_label_components_static(_ptr(band), _dims(band), _ptr(comp), _ptr(cb), _ptr(cs), _ptr(cf),
                                               max_comp, _ptr(nc), _ptr(status), _stream()),
           "lsrvt_label_components_static")
    return comp, cb, cs, cf, nc


def saliency_grad(field, gamma=1, ws=None):
    """Weights q = max(1, rint(|grad f|^gamma * 65535 / max)) (uint16)."""
    _require_cuda(field)
    q = torch.empty(field.shape, dtype=torch.int16, device=field.device)
    ws = ws or Workspace(field.device)
    buf = ws.get(workspace_bytes("saliency", _dims(field)))
    _check(lib().lsrvt_saliency_grad(_ptr(field), _dims(field), int(gamma), _ptr(q), _ptr(buf), buf.numel(),
                                     _stream()), "lsrvt_saliency_grad")
    return q


def seed(comp, q, n_comp_dev, max_comp, voxels_per_site, strat_block=16, rng_seed=0, max_sites=None,
         max_strata=0, ws=None, status=None):
    """Stratified initial sites (Sec. 3.2, Eq. nc).  q is an int16 view of uint16 weights or None.

    Returns (site_pos, site_comp, comp_site_off, n_sites_dev)."""
    _require_cuda(comp, q)
    dev = comp.device
    n = comp.numel()
    if max_sites is None:
        max_sites = int(min(n, n // max(int(voxels_per_site), 1) + int(max_comp) + 1024))
    sp = torch.empty(max(max_sites, 1), dtype=torch.int32, device=dev)
    sc = torch.empty(max(max_sites, 1), dtype=torch.int32, device=dev)
    off = torch.empty(int(max_comp) + 1, dtype=torch.int32, device=dev)
    ns = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = ws or Workspace(dev)
    status = new_status(dev) if status is None else status
    params = SeedParams(int(voxels_per_site), int(strat_block), int(max_strata), int(rng_seed) & (2 ** 64 - 1))
    buf = ws.get(workspace_bytes("seed", _dims(comp), max_comp=max_comp) if not max_strata else
                 max(workspace_bytes("seed", _dims(comp), max_comp=max_comp), 64 * int(max_strata) + (1 << 24)))
    _check(lib().lsrvt_seed(_ptr(comp), _ptr(q), _dims(comp), _ptr(n_comp_dev), int(max_comp), params, _ptr(sp),
                            _ptr(sc), _ptr(off), int(max_sites), _ptr(ns), _ptr(buf), buf.numel(), _ptr(status),
                            _stream()), "lsrvt_seed")
    return sp, sc, off, ns


def cvt_iterate(band, q, site_pos, n_sites_dev, n_iters, want_dist=True, want_trace=True, ws=None, status=None,
                cell=None, dist=None):
    """Algorithm 1 after seeding: n_iters x (Eq. 1 assignment, Eq. 2 update) + final assignment.

    site_pos is updated in place.  Returns (cell, dist or None, trace[n_iters, TRACE] or None);
    trace_summary() reads a trace."""
    _require_cuda(band, q, site_pos)
    dev = band.device
    max_sites = site_pos.numel()
    if cell is None:
        cell = torch.empty(band.shape, dtype=torch.int32, device=dev)
    if want_dist and dist is None:
        dist = torch.empty(band.shape, dtype=torch.int32, device=dev)
    trace = torch.zeros((max(n_iters, 1), TRACE), dtype=torch.int64, device=dev) if want_trace else None
    ws = ws or Workspace(dev)
    status = new_status(dev) if status is None else status
    buf = ws.get(workspace_bytes("cvt", _dims(band), max_sites=max_sites))
    _check(lib().lsrvt_cvt_iterate(_ptr(band), _ptr(q), _dims(band), _ptr(site_pos), _ptr(n_sites_dev), max_sites,
                                   int(n_iters), _ptr(cell), _ptr(dist if want_dist else None),
                                   _ptr(trace), _ptr(buf), buf.numel(), _ptr(status), _stream()),
           "lsrvt_cvt_iterate")
    return cell, (dist if want_dist else None), (trace[:n_iters] if want_trace else None)


def _block_table(blocks):
    tab = (Block * len(blocks))()
    for i, b in enumerate(blocks):
        nx, ny, nz = b["dims"]
        x0, y0, z0 = b["origin"]
        tab[i] = Block(Dims(int(nx), int(ny), int(nz)), int(x0), int(y0), int(z0), _ptr(b.get("band")),
                       _ptr(b.get("q")), _ptr(b.get("site_pos")), _ptr(b.get("n_sites")), _ptr(b.get("cell")),
                       _ptr(b.get("dist")))
    return tab


def pack_blocks(blocks, packed, max_sites, want_q=False, status=None):
    """lsrvt_pack_blocks: independent blocks into one packed volume of extent packed = (nx, ny, nz).
    blocks: dicts with dims (nx, ny, nz), origin (x0, y0, z0), band, q (when want_q), site_pos and
    n_sites (device) of the block.  Returns (band, q or None, site_pos, n_sites, site_base)."""
    dev = blocks[0]["band"].device
    nx, ny, nz = (int(v) for v in packed)
    band = torch.empty((nz, ny, nx), dtype=torch.uint8, device=dev)
    q = torch.empty((nz, ny, nx), dtype=torch.int16, device=dev) if want_q else None
    sp = torch.empty(max(int(max_sites), 1), dtype=torch.int32, device=dev)
    ns = torch.empty(1, dtype=torch.int32, device=dev)
    base = torch.empty(len(blocks) + 1, dtype=torch.int32, device=dev)
    status = new_status(dev) if status is None else status
    tab = _block_table(blocks)
    _check(lib().lsrvt_pack_blocks(C.cast(tab, C.c_void_p), len(blocks), Dims(nx, ny, nz), _ptr(band), _ptr(q),
                                   _ptr(sp), int(max_sites), _ptr(ns), _ptr(base), _ptr(status), _stream()),
           "lsrvt_pack_blocks")
    return band, q, sp, ns, base


def unpack_blocks(blocks, packed, cell, dist, site_pos, site_base):
    """lsrvt_unpack_blocks: each block's cells (its own site ids), distances (when both the block's
    `dist` and the packed dist are given) and sites, from the packed results."""
    nx, ny, nz = (int(v) for v in packed)
    tab = _block_table(blocks)
    _check(lib().lsrvt_unpack_blocks(C.cast(tab, C.c_void_p), len(blocks), Dims(nx, ny, nz), _ptr(cell), _ptr(dist),
                                     _ptr(site_pos), _ptr(site_base), _stream()), "lsrvt_unpack_blocks")


def trace_summary(trace, n_sites):
    """Per-iteration figures of a Lloyd trace (host lists): sites moved, mean d_s (the paper's
    convergence measure, voxels), and the CVT energy sum q_v D(v)^2 of each iteration's
    assignment (exact ints in (2^-16 voxel)^2 units, and as floats in voxel^2), plus how many
    iterations raised the energy (recorded, not a guarantee of the method)."""
    t = trace.cpu().numpy().astype(np.int64) if hasattr(trace, "cpu") else np.asarray(trace, np.int64)
    energy = [(int(h) & (2 ** 64 - 1)) << 64 | (int(l) & (2 ** 64 - 1)) for l, h in zip(t[:, 3], t[:, 4])]
    ns = max(int(n_sites), 1)
    return dict(moved=[int(v) for v in t[:, 0]], mean_ds=[float(v) / 65536.0 / ns for v in t[:, 2]],
                energy=energy, energy_voxel2=[e / 2.0 ** 32 for e in energy],
                energy_increases=sum(1 for a, b in zip(energy[:-1], energy[1:]) if b > a))


def cvt_iterate_anyangle(band, q, site_pos, n_sites_dev, n_iters, max_rounds=1 << 16, want_dist=True,
                         want_src=True, want_trace=True, ws=None, status=None):
    """Algorithm 1 with the any-angle tessellation of Sec. 3.2 (region growing with src(w)
    shortcuts in synchronous rounds); the Eq. 2 update follows src chains.  site_pos is
    updated in place.  Returns (cell, dist or None, src or None, trace or None, rounds) with
    rounds[n_iters + 1] the rounds of each tessellation."""
    _require_cuda(band, q, site_pos)
    dev = band.device
    max_sites = site_pos.numel()
    cell = torch.empty(band.shape, dtype=torch.int32, device=dev)
    dist = torch.empty(band.shape, dtype=torch.int32, device=dev) if want_dist else None
    src = torch.empty(band.shape, dtype=torch.int32, device=dev) if want_src else None
    trace = torch.zeros((max(n_iters, 1), TRACE), dtype=torch.int64, device=dev) if want_trace else None
    rounds = np.zeros(n_iters + 1, np.int32)
    ws = ws or Workspace(dev)
    status = new_status(dev) if status is None else status
    buf = ws.get(workspace_bytes("cvt_anyangle", _dims(band), max_sites=max_sites, n_aux=max_rounds))
    _check(lib().lsrvt_cvt_iterate_anyangle(_ptr(band), _ptr(q), _dims(band), _ptr(site_pos), _ptr(n_sites_dev),
                                            max_sites, int(n_iters), int(max_rounds), _ptr(cell), _ptr(dist),
                                            _ptr(src), _ptr(trace), rounds.ctypes.data_as(C.c_void_p), _ptr(buf),
                                            buf.numel(), _ptr(status), _stream()),
           "lsrvt_cvt_iterate_anyangle")
    return cell, dist, src, (trace[:n_iters] if want_trace else None), rounds


def _aux_ptrs(aux):
    ptrs = (C.c_void_p * max(len(aux), 1))(*[t.data_ptr() for t in aux])
    return ptrs


def aux_range(cell, aux, n_bins, status=None):
    """Per-variable histogram range over valid voxels: (lo, scale) float32 device tensors."""
    aux = [a.contiguous() for a in aux]
    _require_cuda(cell, *aux)
    dev = cell.device
    m = len(aux)
    lo = torch.empty(max(m, 1), dtype=torch.float32, device=dev)
    sc = torch.empty(max(m, 1), dtype=torch.float32, device=dev)
    status = new_status(dev) if status is None else status
    ptrs = _aux_ptrs(aux)
    _check(lib().lsrvt_aux_range(_ptr(cell), C.cast(ptrs, C.c_void_p), m, _dims(cell), int(n_bins), _ptr(lo),
                                 _ptr(sc), _ptr(status), _stream()), "lsrvt_aux_range")
    return lo, sc


def alloc_stats(rows, m, n_bins, cov, device="cuda"):
    T = m * (m + 1) // 2
    return dict(count=torch.empty(max(rows, 1), dtype=torch.int64, device=device),
                mean=torch.empty((max(rows, 1), m), dtype=torch.float64, device=device),
                m2=torch.empty((max(rows, 1), m), dtype=torch.float64, device=device),
                min=torch.empty((max(rows, 1), m), dtype=torch.float32, device=device),
                max=torch.empty((max(rows, 1), m), dtype=torch.float32, device=device),
                hist=torch.empty((max(rows, 1), m, n_bins), dtype=torch.int32, device=device) if n_bins else None,
                comom=torch.empty((max(rows, 1), T), dtype=torch.float64, device=device) if cov else None)


def _stats_struct(st):
    return Stats(st["count"].data_ptr(), st["mean"].data_ptr(), st["m2"].data_ptr(), st["min"].data_ptr(),
                 st["max"].data_ptr(), st["hist"].data_ptr() if st.get("hist") is not None else None,
                 st["comom"].data_ptr() if st.get("comom") is not None else None)


def aggregate(cell, aux, site_pos, n_sites_dev, lo=None, scale=None, n_bins=32, cov=False, ws=None, status=None,
              out=None):
    """Per-cell statistics (Sec. 3.3).  Rows = site_pos.numel().  Returns a dict of device tensors."""
    aux = [a.contiguous() for a in aux]
    _require_cuda(cell, site_pos, *aux)
    dev = cell.device
    m = len(aux)
    max_sites = site_pos.numel()
    status = new_status(dev) if status is None else status
    if n_bins and m and (lo is None or scale is None):
        lo, scale = aux_range(cell, aux, n_bins, status)
    out = out or alloc_stats(max_sites, m, n_bins, cov, dev)
    ws = ws or Workspace(dev)
    buf = ws.get(workspace_bytes("aggregate", _dims(cell), max_sites=max_sites, n_aux=m))
    flags = (STATS_HIST if n_bins else 0) | (STATS_COV if cov else 0)
    ptrs = _aux_ptrs(aux)
    _check(lib().lsrvt_aggregate(_ptr(cell), C.cast(ptrs, C.c_void_p), m, _dims(cell), _ptr(lo), _ptr(scale),
                                 int(n_bins), flags, _ptr(site_pos), _ptr(n_sites_dev), max_sites,
                                 _stats_struct(out), _ptr(buf), buf.numel(), _ptr(status), _stream()),
           "lsrvt_aggregate")
    return out


def merge_hierarchy(cells, n_sites_dev, comp_site_off, comp_band, n_comp_dev, max_comp, n_bands, n_bins=32,
                    cov=False, ws=None):
    """cell -> component -> band -> volume statistics.  Returns (comps, bands, volume)."""
    dev = cells["count"].device
    m = cells["mean"].shape[1]
    max_sites = cells["count"].numel()
    comps = alloc_stats(max_comp, m, n_bins, cov, dev)
    bands = alloc_stats(n_bands, m, n_bins, cov, dev)
    vol = alloc_stats(1, m, n_bins, cov, dev)
    ws = ws or Workspace(dev)
    buf = ws.get(workspace_bytes("merge", _dims_of_nothing(), max_comp=max_comp, max_sites=max_sites, n_aux=m))
    flags = (STATS_HIST if n_bins else 0) | (STATS_COV if cov else 0)
    _check(lib().lsrvt_merge_hierarchy(_stats_struct(cells), _ptr(n_sites_dev), max_sites, m, int(n_bins), flags,
                                       _ptr(comp_site_off), _ptr(comp_band), _ptr(n_comp_dev), int(max_comp),
                                       int(n_bands), _stats_struct(comps), _stats_struct(bands), _stats_struct(vol),
                                       _ptr(buf), buf.numel(), _stream()), "lsrvt_merge_hierarchy")
    return comps, bands, vol


def structured_layout(cell, n_sites_dev, max_sites, comp_site_off, comp_band, n_comp_dev, max_comp, aux=(),
                      bands=None, ws=None, status=None, out=None, want_cells=False):
    """Structured hierarchical layout (Sec. 3.2 "Data Reduction and Structured Data Layout"):
    the voxels of the kept bands (`bands`: iterable of band ids, None = all) ordered by
    (band, component, cell, linear index), with offsets per cell / component / band and the
    variables gathered in the same order.  Returns a dict of device tensors: order [N] int32
    and values (m, N) float32 (first n_kept entries valid), cell_off [max_sites+1],
    comp_off [max_comp+1], band_off [257] int64, n_kept [1] int64; with want_cells also
    cell_pos [N] int32, the cell of each layout position (-1 past n_kept)."""
    aux = [a.contiguous() for a in aux]
    _require_cuda(cell, comp_site_off, comp_band, *aux)
    dev = cell.device
    n = cell.numel()
    m = len(aux)
    status = new_status(dev) if status is None else status
    if out is None:
        out = dict(order=torch.empty(n, dtype=torch.int32, device=dev),
                   # rows padded to a multiple of 4 floats: every row starts 16-byte aligned
                   values=torch.empty((max(m, 1), (n + 3) // 4 * 4), dtype=torch.float32, device=dev)[:, :n],
                   cell_off=torch.empty(max_sites + 1, dtype=torch.int64, device=dev),
                   comp_off=torch.empty(max_comp + 1, dtype=torch.int64, device=dev),
                   band_off=torch.empty(257, dtype=torch.int64, device=dev),
                   n_kept=torch.empty(1, dtype=torch.int64, device=dev))
    if want_cells and out.get("cell_pos") is None:
        out["cell_pos"] = torch.empty(n, dtype=torch.int32, device=dev)
    mask = None
    if bands is not None:
        words = [0] * 8
        for b in bands:
            words[int(b) >> 5] |= 1 << (int(b) & 31)
        mask = (C.c_uint32 * 8)(*words)
    ws = ws or Workspace(dev)
    buf = ws.get(workspace_bytes("layout", _dims(cell), max_sites=max_sites))
    ins = _aux_ptrs(aux)
    outs = (C.c_void_p * max(m, 1))(*[out["values"][j].data_ptr() for j in range(m)])
    _check(lib().lsrvt_structured_layout(_ptr(cell), _dims(cell), _ptr(n_sites_dev), int(max_sites),
                                         _ptr(comp_site_off), _ptr(comp_band), _ptr(n_comp_dev), int(max_comp),
                                         C.cast(mask, C.c_void_p) if mask is not None else None,
                                         C.cast(ins, C.c_void_p), m, C.cast(outs, C.c_void_p), _ptr(out["order"]),
                                         _ptr(out["cell_off"]), _ptr(out["comp_off"]), _ptr(out["band_off"]),
                                         _ptr(out["n_kept"]), _ptr(out.get("cell_pos") if want_cells else None),
                                         _ptr(buf), buf.numel(), _ptr(status), _stream()),
           "lsrvt_structured_layout")
    return out


def alloc_joint(rows, m, device="cuda"):
    from math import comb
    r = max(int(rows), 1)
    return dict(count=torch.empty(r, dtype=torch.int64, device=device),
                mean=torch.empty((r, m), dtype=torch.float64, device=device),
                m2=torch.empty((r, comb(m + 1, 2)), dtype=torch.float64, device=device),
                m3=torch.empty((r, comb(m + 2, 3)), dtype=torch.float64, device=device),
                m4=torch.empty((r, comb(m + 3, 4)), dtype=torch.float64, device=device))


def _joint_struct(j):
    return Joint(j["count"].data_ptr(), j["mean"].data_ptr(), j["m2"].data_ptr(), j["m3"].data_ptr(),
                 j["m4"].data_ptr())


def joint_moments(values, range_off, n_ranges_dev=None, max_ranges=None, ws=None, out=None):
    """Joint central moments of orders 2..4 (covariance, coskewness and cokurtosis sums) of
    m <= 8 variables over the ranges [range_off[r], range_off[r+1]) of layout-ordered values
    (e.g. structured_layout(...)["values"][:m] with its cell_off / comp_off / band_off).
    Returns a dict of device tensors: count, mean (R, m), m2, m3, m4 (R, T_q)."""
    vals = [v for v in values]
    m = len(vals)
    _require_cuda(range_off)
    dev = range_off.device
    n_pos = int(vals[0].numel()) if m else 0
    max_ranges = int(range_off.numel() - 1) if max_ranges is None else int(max_ranges)
    out = out or alloc_joint(max_ranges, m, dev)
    ws = ws or Workspace(dev)
    buf = ws.get(workspace_bytes("joint", (max(n_pos, 1), 1, 1), max_sites=max_ranges, n_aux=m))
    ptrs = (C.c_void_p * max(m, 1))(*[v.data_ptr() for v in vals])
    _check(lib().lsrvt_joint_moments(C.cast(ptrs, C.c_void_p), m, n_pos, _ptr(range_off), _ptr(n_ranges_dev),
                                     max_ranges, _joint_struct(out), _ptr(buf), buf.numel(), _stream()),
           "lsrvt_joint_moments")
    return out


def merge_joint_hierarchy(cells, n_sites_dev, comp_site_off, comp_band, n_comp_dev, max_comp, n_bands, ws=None):
    """Joint-moment records merged cell -> component -> band -> volume (Pebay 2008)."""
    dev = cells["count"].device
    m = cells["mean"].shape[1]
    comps = alloc_joint(max_comp, m, dev)
    bands = alloc_joint(n_bands, m, dev)
    vol = alloc_joint(1, m, dev)
    ws = ws or Workspace(dev)
    buf = ws.get(workspace_bytes("joint", (1, 1, 1), max_comp=max_comp, max_sites=cells["count"].numel(), n_aux=m))
    _check(lib().lsrvt_merge_joint_hierarchy(_joint_struct(cells), _ptr(n_sites_dev), cells["count"].numel(), m,
                                             _ptr(comp_site_off), _ptr(comp_band), _ptr(n_comp_dev), int(max_comp),
                                             int(n_bands), _joint_struct(comps), _joint_struct(bands),
                                             _joint_struct(vol), _ptr(buf), buf.numel(), _stream()),
           "lsrvt_merge_joint_hierarchy")
    return comps, bands, vol


def site_graph(cell, band, site_pos, n_sites_dev, ws=None, status=None, max_arcs=None):
    """Voronoi site graph (region adjacency, the "Voronoi Cell Views" section): CSR over the
    site capacity, both directions, weights ceil(2^16 * Euclidean site distance).  Returns
    dict(off [S+1] int64, adj [A] int32, w [A] int32 (uint32 bits), n_edges [1] int64)."""
    _require_cuda(cell, band, site_pos)
    dev = cell.device
    n = cell.numel()
    S = site_pos.numel()
    if max_arcs is None:
        max_arcs = 2 * min(3 * n, max(n // 8, 1 << 20))
    out = dict(off=torch.empty(S + 1, dtype=torch.int64, device=dev),
               adj=torch.empty(max(max_arcs, 1), dtype=torch.int32, device=dev),
               w=torch.empty(max(max_arcs, 1), dtype=torch.int32, device=dev),
               n_edges=torch.empty(1, dtype=torch.int64, device=dev))
    status = new_status(dev) if status is None else status
    ws = ws or Workspace(dev)
    buf = ws.get(workspace_bytes("graph", _dims(cell)))
    _check(lib().lsrvt_site_graph(_ptr(cell), _ptr(band), _dims(cell), _ptr(site_pos), _ptr(n_sites_dev), S,
                                  _ptr(out["off"]), _ptr(out["adj"]), _ptr(out["w"]), int(max_arcs),
                                  _ptr(out["n_edges"]), _ptr(buf), buf.numel(), _ptr(status), _stream()),
           "lsrvt_site_graph")
    return out


def site_geodesics(graph, site_pos, dims, s0, s1, c_far=None, ws=None, status=None):
    """Geodesic distances between the sites [s0, s1) (a union of components): (k, k) int32
    tensor of uint32 weight units (0xFFFFFFFF = no path) and, with c_far given, the paper's
    ratio ||x_i - x_j|| / gd (c_far where no path exists; 1 on the diagonal)."""
    dev = graph["off"].device
    k = int(s1) - int(s0)
    dist = torch.empty((max(k, 1), max(k, 1)), dtype=torch.int32, device=dev)
    ratio = torch.empty((max(k, 1), max(k, 1)), dtype=torch.float32, device=dev) if c_far is not None else None
    status = new_status(dev) if status is None else status
    ws = ws or Workspace(dev)
    grid = min(max(k, 1), 4 * 148)
    buf = ws.get(2 * grid * ((k + 31) // 32) * 4 + 512)
    d = dims if isinstance(dims, Dims) else Dims(*[int(v) for v in dims])
    _check(lib().lsrvt_site_geodesics(_ptr(graph["off"]), _ptr(graph["adj"]), _ptr(graph["w"]), _ptr(site_pos), d,
                                      int(s0), int(s1), _ptr(dist), _ptr(ratio),
                                      float(c_far if c_far is not None else 0.0), _ptr(buf), buf.numel(),
                                      _ptr(status), _stream()), "lsrvt_site_geodesics")
    return dist[:k, :k], (ratio[:k, :k] if ratio is not None else None)


def _dims_of_nothing():
    return Dims(1, 1, 1)


# --------------------------------------------------------------------------- pipeline
def decompose(field, iso, voxels_per_site, n_iters, aux=(), gamma=0, strat_block=16, rng_seed=0, n_bins=32,
              cov=False, max_comp=None, ws=None, check=True, metric="chamfer"):
    """The whole hot path on the current stream: classify -> CCL -> [saliency] -> seed ->
    Lloyd iterations -> per-cell statistics -> hierarchy merge.  Returns a dict of tensors.

    metric: "chamfer" (restricted 26-neighbour geodesics, lsrvt_cvt_iterate) or "anyangle"
    (Sec. 3.2 region growing with src(w) shortcuts, lsrvt_cvt_iterate_anyangle; adds the
    source map `src` and the round counts `rounds` to the result)."""
    if metric not in ("chamfer", "anyangle"):
        raise ValueError("metric must be 'chamfer' or 'anyangle', not %r" % (metric,))
    dev = field.device
    ws = ws or Workspace(dev)
    status = new_status(dev)
    band = classify(field, iso)
    n = field.numel()
    if max_comp is None:
        max_comp = default_max_comp(n)
    comp, cb, cs, cf, nc = label_components(band, max_comp, ws, status)
    q = saliency_grad(field, gamma, ws) if gamma else None
    sp, sc, off, ns = seed(comp, q, nc, max_comp, voxels_per_site, strat_block, rng_seed, ws=ws, status=status)
    extra = {}
    if metric == "anyangle":
        cell, dist, src, trace, rounds = cvt_iterate_anyangle(band, q, sp, ns, n_iters, ws=ws, status=status)
        extra = dict(src=src, rounds=rounds)
    else:
        cell, dist, trace = cvt_iterate(band, q, sp, ns, n_iters, ws=ws, status=status)
    out = dict(band=band, comp=comp, comp_band=cb, comp_size=cs, comp_first=cf, n_comp=nc, q=q, site_pos=sp,
               site_comp=sc, comp_site_off=off, n_sites=ns, cell=cell, dist=dist, trace=trace, status=status, **extra)
    if len(aux):
        cells = aggregate(cell, list(aux), sp, ns, n_bins=n_bins, cov=cov, ws=ws, status=status)
        comps, bands, vol = merge_hierarchy(cells, ns, off, cb, nc, max_comp, len(iso) + 1, n_bins, cov, ws)
        out.update(cells=cells, comps=comps, bands=bands, volume=vol)
    if check:
        check_status(status, "decompose")
    return out


def decompose_host(field, iso, voxels_per_site, n_iters, aux=None, gamma=0, strat_block=16, rng_seed=0, n_bins=32,
                   cov=False, max_comp=None, ws=None, device="cuda", buffers=None):
    """decompose() from host arrays, results back on the host.

    field: CPU float32 (nz, ny, nx); aux: CPU float32 (m, nz, ny, nx) or None (pinned memory
    makes the copies asynchronous).  The field goes up on the current stream; the auxiliary
    variables, needed only by the statistics, go up on a second stream while the
    tessellation runs, and the statistics wait for them.  Returns host tensors: the per-cell
    statistics (count, mean, m2, min, max, hist[, comom]), the sites and their count, the
    volume record, and the status word.  `buffers` (a dict) keeps the device copies between
    calls of the same shape."""
    dev = torch.device(device)
    buffers = {} if buffers is None else buffers
    main = torch.cuda.current_stream(dev)
    m = 0 if aux is None else int(aux.shape[0])
    if buffers.get("shape") != (tuple(field.shape), m):
        buffers.clear()
        buffers["shape"] = (tuple(field.shape), m)
        buffers["field"] = torch.empty(field.shape, dtype=torch.float32, device=dev)
        buffers["aux"] = torch.empty((m,) + tuple(field.shape), dtype=torch.float32, device=dev) if m else None
        buffers["copy"] = torch.cuda.Stream(device=dev)
    d_field, d_aux, copy = buffers["field"], buffers["aux"], buffers["copy"]
    d_field.copy_(field, non_blocking=True)
    aux_ready = None
    if m:
        copy.wait_stream(main)  # the previous call's statistics have read the buffer
        with torch.cuda.stream(copy):
            d_aux.copy_(aux, non_blocking=True)
            aux_ready = torch.cuda.Event()
            aux_ready.record(copy)
    ws = ws or buffers.setdefault("ws", Workspace(dev))
    status = new_status(dev)
    band = classify(d_field, iso)
    n = d_field.numel()
    if max_comp is None:
        max_comp = default_max_comp(n)
    comp, cb, cs, cf, nc = label_components(band, max_comp, ws, status)
    q = saliency_grad(d_field, gamma, ws) if gamma else None
    sp, sc, off, ns = seed(comp, q, nc, max_comp, voxels_per_site, strat_block, rng_seed, ws=ws, status=status)
    cell, dist, trace = cvt_iterate(band, q, sp, ns, n_iters, want_dist=False, ws=ws, status=status)
    out = dict(n_sites=ns, site_pos=sp, status=status)
    if m:
        main.wait_event(aux_ready)
        auxl = [d_aux[j] for j in range(m)]
        cells = aggregate(cell, auxl, sp, ns, n_bins=n_bins, cov=cov, ws=ws, status=status)
        comps, bands, vol = merge_hierarchy(cells, ns, off, cb, nc, max_comp, len(iso) + 1, n_bins, cov, ws)
        out.update(cells=cells, volume=vol)
    host = {}
    n_sites = int(ns.item())  # synchronises the main stream once
    check_status(status, "decompose_host")
    host["n_sites"] = n_sites
    host["site_pos"] = sp[:n_sites].cpu()
    if m:
        host["cells"] = {k: (v[:n_sites].cpu() if v is not None else None) for k, v in out["cells"].items()}
        host["volume"] = {k: (v.cpu() if v is not None else None) for k, v in out["volume"].items()}
    return host
