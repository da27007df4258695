"""The allocation-free labelling entry point (lsrvt_label_components_static) against the
workspace entry point, called twice in a row through the C ABI.

It serves callers that cannot allocate device memory (an in-situ analysis embedded in a
simulation that owns the device memory, a plug-in without access to the host's allocator):
its scratch is a fixed array inside the library.  Consecutive calls share that array, so
the second call must not see anything of the first.  This file is collected last."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _volume(seed, shape):
    rng = np.random.default_rng(seed)
    band = rng.integers(0, 3, size=shape).astype(np.uint8)
    band[rng.random(shape) < 0.05] = 255
    return torch.from_numpy(band).cuda()


def _outputs(band, max_comp):
    comp = torch.full(band.shape, -7, dtype=torch.int32, device="cuda")
    cb = torch.zeros(max_comp, dtype=torch.uint8, device="cuda")
    cs = torch.zeros(max_comp, dtype=torch.int64, device="cuda")
    cf = torch.zeros(max_comp, dtype=torch.int32, device="cuda")
    nc = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    return comp, cb, cs, cf, nc, st


def _static_call(pk, band, max_comp, out=None):
    """One call through the C ABI into caller-allocated outputs (allocated here unless given)."""
    L = pk.lib()
    comp, cb, cs, cf, nc, st = _outputs(band, max_comp) if out is None else out
    p = lambda t: C.c_void_p(t.data_ptr())
    rc = L.lsrvt_label_components_static(p(band), pk._dims(band), p(comp), p(cb), p(cs), p(cf), max_comp, p(nc), p(st),
                                         C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return comp, cb, cs, cf, nc


def test_static_labelling_matches_workspace_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2208_06970_b300 as pk
    from paper_2208_06970_b300 import build
    build.build()
    # two different volumes, the second smaller, so stale scratch contents would show
    for seed, shape in ((11, (64, 64, 64)), (12, (23, 37, 41))):
        band = _volume(seed, shape)
        n = band.numel()
        got = _static_call(pk, band, n)
        ref = pk.label_components(band, max_comp=n)
        k = int(ref[4].item())
        assert int(got[4].item()) == k
        assert torch.equal(got[0], ref[0])
        for a, b in zip(got[1:4], ref[1:4]):
            assert torch.equal(a[:k], b[:k])


def test_static_labelling_rejects_large_volumes():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2208_06970_b300 as pk
    band = torch.zeros((65, 64, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(pk.LsrvtError) as e:
        pk.label_components_static(band)
    assert e.value.code == 8


def test_static_labelling_allocates_nothing():
    """The property the entry point exists for: with its outputs in place, a call leaves the
    caching allocator's counters and the device's free memory exactly as they were."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2208_06970_b300 as pk
    band = _volume(13, (64, 64, 64))
    n = band.numel()
    out = _outputs(band, n)
    _static_call(pk, band, n, out)  # warm: module load and the address look-up happen here
    torch.cuda.synchronize()
    keys = ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.allocated")
    before = {k: torch.cuda.memory_stats().get(k, 0) for k in keys}
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        _static_call(pk, band, n, out)
    torch.cuda.synchronize()
    after = {k: torch.cuda.memory_stats().get(k, 0) for k in keys}
    assert after == before
    assert torch.cuda.mem_get_info()[0] == free0
