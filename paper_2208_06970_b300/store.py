"""On-disk form of the structured layout (Sec. 3.2 "Data Reduction and Structured Data Layout"):
the statistical summaries and the offsets first, then the raw data of the kept voxels ordered
by (band, component, cell), so a reader can load the light summaries, pick features, and map
only the bytes of the bands, components or cells it wants (out of core).

File format (little-endian):
  8 bytes   magic b"LSRVTLAY"
  8 bytes   header length H (uint64)
  H bytes   JSON header: {"arrays": {name: [dtype, shape, byte offset]}, "meta": {...}}
  ...       arrays at their offsets, 64-byte aligned, C order

Arrays: band_off [257], comp_off [n_comp+1], cell_off [n_sites+1] (int64 offsets into the voxel
records); order [r] (int32 linear voxel index); values [m, r] (float32, one row per variable);
and for each statistics level present ("cells", "comps", "bands", "volume") its count, mean,
m2, min, max and hist arrays under "<level>.<field>".
"""
import json
import os

import numpy as np

MAGIC = b"LSRVTLAY"
_ALIGN = 64


def _host(t):
    if t is None:
        return None
    if hasattr(t, "detach"):
        t = t.detach().cpu().numpy()
    return np.ascontiguousarray(t)


def save(path, layout, n_sites, n_comp, stats=None, meta=None):
    """Write a layout (the dict returned by structured_layout, device or host arrays) and,
    optionally, statistics levels {"cells": {...}, "comps": {...}, ...} (rows beyond the live
    counts are dropped) to `path`."""
    r = int(_host(layout["n_kept"]).reshape(-1)[0]) if np.ndim(layout["n_kept"]) else int(layout["n_kept"])
    n_sites, n_comp = int(n_sites), int(n_comp)
    arrays = {
        "band_off": _host(layout["band_off"]).astype(np.int64),
        "comp_off": _host(layout["comp_off"])[:n_comp + 1].astype(np.int64),
        "cell_off": _host(layout["cell_off"])[:n_sites + 1].astype(np.int64),
        "order": _host(layout["order"])[:r].astype(np.int32),
    }
    vals = layout.get("values")
    m = 0
    if vals is not None:
        v = _host(vals)
        m = int(v.shape[0]) if v.ndim == 2 and v.shape[1] >= r else 0
        if m:
            arrays["values"] = np.ascontiguousarray(v[:, :r].astype(np.float32))
    rows = {"cells": n_sites, "comps": n_comp}
    for level, st in (stats or {}).items():
        keep = rows.get(level)
        for field in ("count", "mean", "m2", "min", "max", "hist"):
            a = st.get(field)
            if a is None:
                continue
            a = _host(a)
            arrays["%s.%s" % (level, field)] = a[:keep] if keep is not None else a
    header = {"arrays": {}, "meta": dict(meta or {}, n_kept=r, n_sites=n_sites, n_comp=n_comp, n_vars=m)}
    # offsets: header size depends on the offsets' digits, so lay out with a generous bound
    names = list(arrays)
    off = 0
    for k in names:
        header["arrays"][k] = [arrays[k].dtype.str, list(arrays[k].shape), 0]
    hbytes = len(json.dumps(header).encode()) + 32 * len(names) + 64
    base = (16 + hbytes + _ALIGN - 1) // _ALIGN * _ALIGN
    off = base
    for k in names:
        header["arrays"][k][2] = off
        off = (off + arrays[k].nbytes + _ALIGN - 1) // _ALIGN * _ALIGN
    h = json.dumps(header).encode()
    assert 16 + len(h) <= base
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(np.uint64(len(h)).tobytes())
        f.write(h)
        for k in names:
            f.seek(header["arrays"][k][2])
            f.write(arrays[k].tobytes())
        f.truncate(off)
    return path


class Store:
    """Read side: summaries and offsets are small and loaded on demand; voxel records are
    memory-mapped, so only the ranges asked for are read from disk."""

    def __init__(self, path):
        self.path = path
        with open(path, "rb") as f:
            if f.read(8) != MAGIC:
                raise ValueError("%s: not an LSRVT layout file" % path)
            hl = int(np.frombuffer(f.read(8), np.uint64)[0])
            self.header = json.loads(f.read(hl).decode())
        self.meta = self.header["meta"]
        self._cache = {}

    def names(self):
        return list(self.header["arrays"])

    def array(self, name):
        """A read-only memory map of one stored array."""
        if name not in self._cache:
            dt, shape, off = self.header["arrays"][name]
            self._cache[name] = np.memmap(self.path, dtype=np.dtype(dt), mode="r", offset=off,
                                          shape=tuple(shape))
        return self._cache[name]

    def summary(self, level="comps"):
        """The statistics of one level as a dict of arrays (loaded into memory)."""
        pre = level + "."
        return {k[len(pre):]: np.array(self.array(k)) for k in self.names() if k.startswith(pre)}

    def _range(self, lo, hi):
        lo, hi = int(lo), int(hi)
        vals = self.array("values")[:, lo:hi] if "values" in self.header["arrays"] else None
        return np.array(self.array("order")[lo:hi]), (np.array(vals) if vals is not None else None)

    def band(self, b):
        off = self.array("band_off")
        return self._range(off[b], off[b + 1])

    def component(self, c):
        off = self.array("comp_off")
        return self._range(off[c], off[c + 1])

    def cell(self, s):
        off = self.array("cell_off")
        return self._range(off[s], off[s + 1])


def open_store(path):
    return Store(path)


def file_bytes(path):
    return os.path.getsize(path)
