"""Execution forms: blocks run concurrently (batched) and requests served with continuous
batching give the same labels (bit for bit) and statistics (within the moment tolerance) as
each run alone."""
import numpy as np
import pytest
import torch

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


def _jobs(n, lo, hi, seed):
    jobs = []
    for b in workloads.block_batch(n_blocks=n, seed=seed, lo=lo, hi=hi, device="cuda"):
        jobs.append(dict(field=b["field"], iso=b["iso"], voxels_per_site=b["voxels_per_site"], n_iters=4,
                         aux=[b["aux"][j] for j in range(b["aux"].shape[0])], gamma=0, strat_block=16,
                         rng_seed=b["rng_seed"], n_bins=32))
    return jobs


def _same(pk, a, b):
    ns = int(a["n_sites"].item())
    assert ns == int(b["n_sites"].item())
    for k in ("band", "comp", "cell", "dist"):
        assert torch.equal(a[k], b[k]), k
    assert torch.equal(a["site_pos"][:ns], b["site_pos"][:ns])
    ca, cb = a["cells"], b["cells"]
    for k in ("count", "min", "max", "hist"):
        assert torch.equal(ca[k][:ns], cb[k][:ns]), k
    ma, mb = ca["mean"][:ns].cpu().numpy(), cb["mean"][:ns].cpu().numpy()
    assert np.all(np.abs(ma - mb) <= 1e-9 * np.maximum(np.abs(mb), 1e-3))


def test_batched_blocks_equal_alone(pk):
    from paper_2208_06970_b300 import runtime
    jobs = _jobs(6, 24, 72, 3)
    alone = [pk.decompose(j["field"], j["iso"], j["voxels_per_site"], j["n_iters"], aux=j["aux"],
                          rng_seed=j["rng_seed"]) for j in jobs]
    mixed = runtime.BatchRunner(n_slots=3).run(jobs)
    for a, b in zip(alone, mixed):
        _same(pk, a, b)


def test_graph_batch_equals_alone(pk):
    # the batch captured as one CUDA graph: every replay decomposes what the input tensors hold
    # at replay time, and equals each block run alone (labels bit for bit)
    from paper_2208_06970_b300 import runtime
    jobs = _jobs(5, 24, 64, 9)
    gb = runtime.GraphBatch(jobs, n_slots=2)
    for step in range(2):
        if step == 1:  # the next "time step": new data in the same tensors
            for k, j in enumerate(jobs):
                nxt = workloads.blob_field(tuple(j["field"].shape[::-1]), 100 + k, "cuda")
                j["field"].copy_(nxt)
        got = gb.replay()
        torch.cuda.synchronize()
        gb.check()
        for j, g in zip(jobs, got):
            alone = pk.decompose(j["field"], j["iso"], j["voxels_per_site"], j["n_iters"], aux=j["aux"],
                                 rng_seed=j["rng_seed"])
            _same(pk, alone, g)


def test_autotuner_picks_a_schedule_without_changing_results(pk):
    from paper_2208_06970_b300 import runtime
    jobs = _jobs(4, 24, 56, 13)
    best, times = runtime.tune_batch(jobs, candidates=((1, 100), (2, 75), (4, 25)))
    assert best in times and len(times) == 3 and all(t > 0 for t in times.values())


@pytest.mark.parametrize("policy", ["fifo", "sjf"])
def test_served_requests_equal_alone(pk, policy):
    from paper_2208_06970_b300 import runtime
    jobs = _jobs(8, 24, 64, 5)
    reqs = [dict(arrival=0.02 * i, k=i, bytes=runtime.job_bytes(j), ws_bytes=runtime.job_bytes_split(j)[0],
                 work=j["field"].numel() * j["n_iters"]) for i, j in enumerate(jobs)]
    # a budget of about two requests forces admission to wait for memory
    budget = 2 * max(r["bytes"] for r in reqs)
    srv = runtime.Server(n_slots=3, hbm_budget=budget, policy=policy)
    recs = srv.serve(reqs, lambda r: jobs[r["k"]], keep_outputs=True)
    assert all(r is not None for r in recs)
    assert all(r["finished"] >= r["arrival"] for r in recs)
    for i, j in enumerate(jobs):
        alone = pk.decompose(j["field"], j["iso"], j["voxels_per_site"], j["n_iters"], aux=j["aux"],
                             rng_seed=j["rng_seed"])
        _same(pk, alone, recs[i]["out"])
    s = runtime.latency_summary(recs)
    assert s["p99_ms"] >= s["p50_ms"] > 0


def test_host_buffer_form_equals_device_form(pk):
    # decompose_host (host arrays in and out, auxiliary upload overlapped with the
    # tessellation on a second stream) returns what decompose returns on device arrays
    w = workloads.flame_workload(side=(72, 40, 56), seed=6, n_aux=5, n_iters=4)
    h_field = w["field"].pin_memory()
    h_aux = w["aux"].pin_memory()
    kw = dict(gamma=1, strat_block=16, rng_seed=6, n_bins=32)
    ref = pk.decompose(w["field"].cuda(), w["iso"], 256, 4, aux=[a.cuda() for a in w["aux"]], **kw)
    bufs = {}
    for _ in range(2):  # the second call reuses the device buffers
        got = pk.decompose_host(h_field, w["iso"], 256, 4, aux=h_aux, buffers=bufs, **kw)
        ns = int(ref["n_sites"].item())
        assert got["n_sites"] == ns
        assert torch.equal(got["site_pos"], ref["site_pos"][:ns].cpu())
        for k in ("count", "min", "max", "hist"):
            assert torch.equal(got["cells"][k], ref["cells"][k][:ns].cpu()), k
        assert torch.equal(got["volume"]["count"], ref["volume"]["count"].cpu())
        # FP64 atomics combine partial moments in a run-dependent order
        for k in ("mean", "m2"):
            assert torch.allclose(got["cells"][k], ref["cells"][k][:ns].cpu(), rtol=1e-12, atol=1e-12), k
            assert torch.allclose(got["volume"][k], ref["volume"][k].cpu(), rtol=1e-12, atol=1e-12), k


def test_server_stays_within_its_hbm_budget(pk):
    """Admission counts what is really held: the slots' resident workspaces (each keeps the
    largest it has needed) and each in-flight request's own inputs and outputs.  The device
    memory the serving adds never exceeds the budget (the inputs are made up front here, so
    they count before).  The per-request estimate bounds what one request allocates alone."""
    from paper_2208_06970_b300 import runtime
    jobs = _jobs(10, 24, 72, 17)
    reqs = []
    for i, j in enumerate(jobs):
        ws, rest = runtime.job_bytes_split(j)
        reqs.append(dict(arrival=0.01 * i, k=i, bytes=ws + rest, ws_bytes=ws))
    big = max(range(len(jobs)), key=lambda i: reqs[i]["bytes"])
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    base = torch.cuda.memory_allocated()
    torch.cuda.reset_peak_memory_stats()
    alone = runtime.Server(n_slots=1, hbm_budget=1 << 40).serve([dict(reqs[big], arrival=0.0)], lambda r: jobs[r["k"]])
    torch.cuda.synchronize()
    assert alone[0] is not None and torch.cuda.max_memory_allocated() - base <= reqs[big]["bytes"]
    del alone
    torch.cuda.empty_cache()
    budget = int(2.5 * reqs[big]["bytes"])
    base = torch.cuda.memory_allocated()
    torch.cuda.reset_peak_memory_stats()
    srv = runtime.Server(n_slots=3, hbm_budget=budget, policy="fifo")
    recs = srv.serve(reqs, lambda r: jobs[r["k"]])
    torch.cuda.synchronize()
    assert all(r is not None for r in recs)
    assert torch.cuda.max_memory_allocated() - base <= budget


def _energy(t):
    return ((int(t[4]) & (2 ** 64 - 1)) << 64) | (int(t[3]) & (2 ** 64 - 1))


def test_packed_batch_equals_alone(pk):
    # one Lloyd loop over blocks packed one voxel apart (ragged sides, some thinner than a brick)
    # gives each block the cells, distances, sites and statistics it gets alone; the packed
    # trace is the sum of the blocks' traces (moves, d_s and the exact 128-bit energy)
    from paper_2208_06970_b300 import runtime
    jobs = _jobs(7, 12, 70, 21)
    pb = runtime.PackedBatch(jobs, gap=1, n_slots=3, want_dist=True)
    got = pb.run()
    torch.cuda.synchronize()
    pb.check()
    tr = pb.trace.cpu().numpy()
    sums = np.zeros((tr.shape[0], 3), dtype=np.int64)
    energy = [0] * tr.shape[0]
    for j, g in zip(jobs, got):
        a = pk.decompose(j["field"], j["iso"], j["voxels_per_site"], j["n_iters"], aux=j["aux"],
                         rng_seed=j["rng_seed"])
        _same(pk, a, g)
        t = a["trace"].cpu().numpy()
        sums += t[:, :3]
        for it in range(t.shape[0]):
            energy[it] += _energy(t[it])
    assert np.array_equal(sums, tr[:, :3])
    assert energy == [_energy(tr[it]) for it in range(tr.shape[0])]


def test_packed_batch_weighted_and_wide_gap(pk):
    # saliency weights packed with the bands; a wider gap leaves the results unchanged
    from paper_2208_06970_b300 import runtime
    jobs = _jobs(4, 16, 48, 5)
    for j in jobs:
        j["gamma"] = 1
        j["aux"] = j["aux"][:1]
    for gap in (1, 5):
        got = runtime.PackedBatch(jobs, gap=gap, n_slots=2, want_dist=True).run()
        torch.cuda.synchronize()
        for j, g in zip(jobs, got):
            a = pk.decompose(j["field"], j["iso"], j["voxels_per_site"], j["n_iters"], aux=j["aux"], gamma=1,
                             rng_seed=j["rng_seed"])
            _same(pk, a, g)


def test_packed_graph_replay_equals_alone(pk):
    # the packed batch captured as one CUDA graph; new data in the input tensors between replays
    from paper_2208_06970_b300 import runtime
    jobs = _jobs(5, 20, 56, 17)
    pb = runtime.PackedBatch(jobs, n_slots=2).capture()
    for step in range(2):
        if step == 1:
            for k, j in enumerate(jobs):
                j["field"].copy_(workloads.blob_field(tuple(j["field"].shape[::-1]), 300 + k, "cuda"))
        got = pb.replay()
        torch.cuda.synchronize()
        pb.check()
        for j, g in zip(jobs, got):
            a = pk.decompose(j["field"], j["iso"], j["voxels_per_site"], j["n_iters"], aux=j["aux"],
                             rng_seed=j["rng_seed"])
            for k in ("band", "comp", "cell"):
                assert torch.equal(a[k], g[k]), k
            ns = int(a["n_sites"].item())
            assert torch.equal(a["site_pos"][:ns], g["site_pos"][:ns])


def test_packing_tuner_keeps_results(pk):
    from paper_2208_06970_b300 import runtime
    jobs = _jobs(4, 24, 56, 13)
    best, times, fills = runtime.tune_packed(jobs, candidates=((1, 2), (3, 2)))
    assert best in times and len(times) == 2 and all(0 < f <= 1 for f in fills.values())
