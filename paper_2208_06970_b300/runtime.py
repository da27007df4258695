"""Execution forms of the hot path: batched blocks and a continuous-batching server.

Both drive the C ABI (all compute in liblsrvt) from host worker threads, one CUDA stream and
one workspace per slot; ctypes releases the GIL during library calls, and each slot's stream
sizes its grids to a share of the SMs (lsrvt_set_stream_share), so the slots' kernels run side
by side on the device.  The paper's distributed form processes independent blocks with no
communication (Sec. 3.2 "Parallel Algorithm", Discussion "Block Based Distributed
Parallelism"); here independent blocks / requests share one GPU instead.

  BatchRunner(n_slots).run(jobs)     -> results in job order
  GraphBatch(jobs, n_slots).replay() -> results in job order, the batch replayed as one CUDA graph
  Server(n_slots, hbm_budget).serve(requests, make_job) -> per-request records
  tune_batch(sample_jobs) -> the fastest (slots, share) schedule, checked to leave results unchanged
  PackedBatch(jobs).run()            -> results in job order, one Lloyd loop over all blocks packed
                                        into one volume (PackedBatch.capture(): as one CUDA graph)
  tune_packed(jobs)                  -> the fastest packing schedule, checked to leave results unchanged

A job is a dict: field (CUDA float32 (nz, ny, nx)), iso, voxels_per_site, n_iters, aux (list
of CUDA tensors), gamma, strat_block, rng_seed, n_bins.
"""
import queue
import threading
import time

import numpy as np
import torch

from . import decompose, set_stream_share, Workspace


def request_bytes_split(n_voxels, n_aux, voxels_per_site, n_bins=32, dims=None):
    """Estimate of the device bytes one decomposition holds, as (workspace, the rest): the
    workspace lives in the slot and is reused by its next request; the rest (the inputs and
    every output tensor) belongs to the request."""
    from . import default_max_comp, workspace_bytes
    n = int(n_voxels)
    per_voxel = 4 + 1 + 4 + 2 + 4 + 4 + 4 * n_aux  # field, band, comp, q, cell, dist, aux
    max_comp = default_max_comp(n)
    rows = n // max(int(voxels_per_site), 1) + max_comp + 1024  # the seeding's site capacity
    per_row = 8 + 4 * 4 + n_aux * (8 + 8 + 4 + 4 + 4 * n_bins)  # counts, site tables, moments, histograms
    rest = n * per_voxel + (rows + max_comp + 64) * per_row
    if dims is None:
        side = max(int(round(n ** (1.0 / 3.0))), 1)
        dims = (side, side, side)
    ws = max(workspace_bytes(step, tuple(int(v) for v in dims), max_comp=max_comp, max_sites=rows, n_aux=n_aux)
             for step in ("label", "seed", "cvt", "aggregate", "merge"))
    return int(ws * 1.1) + (1 << 20), int(rest)


def request_bytes(n_voxels, n_aux, voxels_per_site, n_bins=32):
    """Estimate of the device bytes one decomposition holds (inputs, outputs, workspaces)."""
    ws, rest = request_bytes_split(n_voxels, n_aux, voxels_per_site, n_bins)
    return ws + rest


def job_bytes_split(job):
    nz, ny, nx = job["field"].shape
    return request_bytes_split(job["field"].numel(), len(job.get("aux", ())), job["voxels_per_site"],
                               job.get("n_bins", 32), dims=(nx, ny, nz))


def job_bytes(job):
    return sum(job_bytes_split(job))


def default_share(n_slots):
    """Share of the SMs each of n_slots concurrent slots sizes its grids to: 150 / n_slots
    percent (a mild oversubscription, so a slot running alone still gets a fair part)."""
    return max(1, min(100, 150 // max(int(n_slots), 1)))


class Slot:
    def __init__(self, device, share=100):
        self.stream = torch.cuda.Stream(device=device)
        self.ws = Workspace(device)
        set_stream_share(share, self.stream)


def _run(slot, job):
    with torch.cuda.stream(slot.stream):
        out = decompose(job["field"], job["iso"], job["voxels_per_site"], job["n_iters"], aux=job.get("aux", ()),
                        gamma=job.get("gamma", 0), strat_block=job.get("strat_block", 16),
                        rng_seed=job.get("rng_seed", 0), n_bins=job.get("n_bins", 32), ws=slot.ws, check=False)
        done = torch.cuda.Event()
        done.record(slot.stream)
    return out, done


class BatchRunner:
    """Runs many independent blocks concurrently on n_slots streams (a block per slot at a time)."""

    def __init__(self, n_slots=4, device="cuda", share=None):
        share = default_share(n_slots) if share is None else share
        self.slots = [Slot(device, share) for _ in range(n_slots)]

    def run(self, jobs):
        results = [None] * len(jobs)
        q = queue.Queue()
        for i, j in enumerate(jobs):
            q.put(i)
        errors = []

        def worker(slot):
            while True:
                try:
                    i = q.get_nowait()
                except queue.Empty:
                    return
                try:
                    out, done = _run(slot, jobs[i])
                    done.synchronize()
                    from . import check_status
                    check_status(out["status"], "block %d" % i)
                    results[i] = out
                except Exception as e:  # surfaced after all workers stop
                    errors.append(e)
                    return

        threads = [threading.Thread(target=worker, args=(s,)) for s in self.slots]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        if errors:
            raise errors[0]
        return results


class GraphBatch:
    """A batch of independent blocks captured once into one CUDA graph and replayed with one
    launch per batch: the blocks are dealt to n_slots streams (forked from and joined back into
    the capturing stream), each stream runs its blocks in order, and every step of every
    block is a library kernel recorded in the graph.  Inputs are read from the jobs' tensors at
    replay time, so new data written into the same tensors (the next time step of a volume)
    is decomposed by the next replay; outputs live in the graph's memory pool and are
    overwritten by each replay.  All data-dependent control (queues, counters, rounds) is on
    the device, so no host synchronisation breaks the capture."""

    def __init__(self, jobs, n_slots=4, device="cuda", share=None):
        share = default_share(n_slots) if share is None else share
        self.jobs = jobs
        self.slots = [Slot(device, share) for _ in range(n_slots)]
        self.device = device
        # eager warm-up: sizes every slot's workspace and loads the kernels before capture
        for k, job in enumerate(jobs):
            slot = self.slots[k % n_slots]
            out, done = _run(slot, job)
            done.synchronize()
        torch.cuda.synchronize(device)
        self.graph = torch.cuda.CUDAGraph()
        main = torch.cuda.Stream(device=device)
        main.wait_stream(torch.cuda.current_stream(device))
        self.outputs = [None] * len(jobs)
        with torch.cuda.graph(self.graph, stream=main):
            for slot in self.slots:
                slot.stream.wait_stream(main)
            for k, job in enumerate(jobs):
                slot = self.slots[k % n_slots]
                with torch.cuda.stream(slot.stream):
                    self.outputs[k] = decompose(job["field"], job["iso"], job["voxels_per_site"], job["n_iters"],
                                                aux=job.get("aux", ()), gamma=job.get("gamma", 0),
                                                strat_block=job.get("strat_block", 16),
                                                rng_seed=job.get("rng_seed", 0), n_bins=job.get("n_bins", 32),
                                                ws=slot.ws, check=False)
            for slot in self.slots:
                main.wait_stream(slot.stream)
        torch.cuda.synchronize(device)

    def replay(self):
        """One launch of the whole batch; returns the per-block outputs (graph-owned tensors)."""
        self.graph.replay()
        return self.outputs

    def check(self):
        from . import check_status
        for k, out in enumerate(self.outputs):
            check_status(out["status"], "block %d" % k)


def pick_next(pending, requests, now, used, budget, active, policy="fifo", max_work=None):
    """Admission choice of the server.  pending: indices not yet admitted, in arrival order.
    A request is eligible once it has arrived and its estimated device bytes fit in the budget
    left (any request fits when nothing runs, so the server always progresses).  'fifo' admits
    the earliest arrival and waits for it when it does not fit yet; 'sjf' admits the eligible
    request with the least work (requests[i]['work'], else its bytes), earliest arrival first on
    ties.  With max_work, only requests whose work is at most max_work are considered (the
    earliest of them for 'fifo': small requests may overtake large ones).  Returns the chosen
    index or None."""
    def fits(i):
        return used + (requests[i].get("bytes") or 0) <= budget or active == 0

    arrived = [i for i in pending if requests[i]["arrival"] <= now]
    if max_work is not None:
        arrived = [i for i in arrived if requests[i].get("work", requests[i].get("bytes") or 0) <= max_work]
    if not arrived:
        return None
    if policy == "fifo":
        return arrived[0] if fits(arrived[0]) else None
    if policy == "sjf":
        ok = [i for i in arrived if fits(i)]
        if not ok:
            return None
        return min(ok, key=lambda i: (requests[i].get("work", requests[i].get("bytes") or 0), requests[i]["arrival"]))
    raise ValueError("unknown admission policy %r" % (policy,))


class Server:
    """Continuous batching: requests are admitted whenever a slot is free and their estimated
    device bytes fit in the remaining HBM budget -- in arrival order ('fifo') or smallest work
    first among those that have arrived ('sjf'); admitted requests run concurrently on the
    slots' streams.  'fill' is size-aware: slot 0 takes every request in arrival order with all
    the SMs, the other slots take only small requests (work <= fill_work voxel-iterations, the
    earliest first) with a small SM share (fill_share percent), so they run in the gaps of the
    large ones.  Latency = completion - arrival (host clock)."""

    def __init__(self, n_slots=4, hbm_budget=64 << 30, device="cuda", share=None, policy="fifo", fill_work=None,
                 fill_share=20):
        if policy not in ("fifo", "sjf", "fill"):
            raise ValueError("unknown admission policy %r" % (policy,))
        if policy == "fill":
            shares = [100] + [fill_share] * (n_slots - 1)
            self.max_work = [None] + [fill_work] * (n_slots - 1)
        else:
            shares = [default_share(n_slots) if share is None else share] * n_slots
            self.max_work = [None] * n_slots
        self.slots = [Slot(device, sh) for sh in shares]
        self.budget = int(hbm_budget)
        self.policy = policy

    def serve(self, requests, make_job, keep_outputs=False):
        """requests: list of dicts with 'arrival' (seconds from start); make_job(req) builds the
        job (device tensors) when the request is admitted.  Returns one record per request.

        HBM accounting: the slots' workspaces are resident (each keeps the largest it has needed),
        so they are counted as they are; a request adds its own bytes (inputs, outputs: its
        'bytes' less its 'ws_bytes') plus what its slot's workspace would have to grow by; kept
        outputs stay counted after their request ends."""
        pending = sorted(range(len(requests)), key=lambda i: requests[i]["arrival"])
        records = [None] * len(requests)
        cv = threading.Condition()
        state = dict(used=0, grow=0, active=0, error=None)
        t0 = time.perf_counter()

        def ws_bytes(slot):
            return 0 if slot.ws.buf is None else slot.ws.buf.numel()

        def resident():
            return sum(ws_bytes(sl) for sl in self.slots)

        def need_on(slot, i):
            r = requests[i]
            total = r.get("bytes") or 0
            ws = min(r.get("ws_bytes") or 0, total)
            return (total - ws) + max(0, ws - ws_bytes(slot))

        def admit_loop(slot_id):
            slot = self.slots[slot_id]
            while True:
                with cv:
                    while True:
                        if state["error"] is not None or not pending:
                            return
                        now = time.perf_counter() - t0
                        # per-request needs on this slot, in the form pick_next reads
                        view = {i: dict(requests[i], bytes=need_on(slot, i)) for i in pending}
                        i = pick_next(pending, view, now, state["used"] + state["grow"] + resident(), self.budget,
                                      state["active"], "sjf" if self.policy == "sjf" else "fifo",
                                      self.max_work[slot_id])
                        if i is not None:
                            pending.remove(i)
                            grow = max(0, min(requests[i].get("ws_bytes") or 0, requests[i].get("bytes") or 0)
                                       - ws_bytes(slot))
                            need = view[i]["bytes"] - grow
                            state["used"] += need
                            # the slot's workspace growth, reserved until the request ends (then it is
                            # resident and counted by resident())
                            state["grow"] += grow
                            state["active"] += 1
                            break
                        wait = requests[pending[0]]["arrival"] - now
                        cv.wait(timeout=max(min(wait, 0.05), 0.0005) if wait > 0 else 0.01)
                try:
                    admitted = time.perf_counter() - t0
                    # the job's inputs are built on the slot's stream, ahead of its kernels
                    with torch.cuda.stream(slot.stream):
                        job = make_job(requests[i])
                    out, done = _run(slot, job)
                    done.synchronize()
                    finished = time.perf_counter() - t0
                    from . import check_status
                    check_status(out["status"], "request %d" % i)
                    records[i] = dict(arrival=requests[i]["arrival"], admitted=admitted, finished=finished,
                                      latency=finished - requests[i]["arrival"], voxels=job["field"].numel(),
                                      iters=job["n_iters"], out=out if keep_outputs else None)
                    # drop this thread's references before the bytes are released for admission
                    del out, done, job
                except Exception as e:
                    with cv:
                        state["error"] = e
                        cv.notify_all()
                    return
                finally:
                    with cv:
                        if not keep_outputs:
                            state["used"] -= need
                        state["grow"] -= grow
                        state["active"] -= 1
                        cv.notify_all()

        threads = [threading.Thread(target=admit_loop, args=(k,)) for k in range(len(self.slots))]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        if state["error"] is not None:
            raise state["error"]
        return records


def tune_batch(jobs, candidates=((1, 100), (2, 75), (4, 37), (4, 25), (8, 18)), device="cuda", reps=1):
    """Autotuner of the batching schedule: runs the sample `jobs` under each (slots, share)
    candidate, checks that every candidate reproduces the first one's labels bit for bit
    (the schedule must not change results), and returns (best candidate, {candidate: seconds})."""
    times, ref = {}, None
    for slots, share in candidates:
        runner = BatchRunner(n_slots=slots, device=device, share=share)
        runner.run(jobs[: min(len(jobs), slots)])  # warm the slots' workspaces
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        for _ in range(reps):
            outs = runner.run(jobs)
        torch.cuda.synchronize(device)
        times[(slots, share)] = (time.perf_counter() - t0) / reps
        if ref is None:
            ref = outs
        else:
            for a, b in zip(ref, outs):
                for k in ("band", "comp", "cell"):
                    if not torch.equal(a[k], b[k]):
                        raise RuntimeError("schedule (%d, %d) changed %s" % (slots, share, k))
    best = min(times, key=times.get)
    return best, times


def latency_summary(records):
    lat = sorted(r["latency"] for r in records)
    n = len(lat)

    def pct(p):
        return lat[min(n - 1, max(0, int(round(p / 100.0 * n + 0.5)) - 1))] * 1e3

    span = max(r["finished"] for r in records) - min(r["arrival"] for r in records)
    vox_it = sum(r["voxels"] * r["iters"] for r in records)
    return dict(n=n, p50_ms=pct(50), p99_ms=pct(99), mean_ms=1e3 * sum(lat) / n,
                throughput_req_s=n / span, gvoxel_iters_s=vox_it / span / 1e9, span_s=span)


# --------------------------------------------------------------------------- packed batches
def pack_layout(dims, gap=1, footprint=None, res=8, max_side=2048):
    """Origins of independent blocks in one packed volume: blocks of extents dims[i] =
    (nx, ny, nz), at least `gap` (>= 1) voxels apart, placed on a height map over a
    (width, depth) footprint kept at a resolution of `res` voxels -- the tallest block first,
    each at the lowest height its footprint (widened by the gap) allows, then the smallest y,
    then x.  footprint None: of a few candidate footprints, the one whose packed volume is the
    smallest with every side at most max_side and fewer than 2^31 voxels (the library's limit on a
    volume).  Returns (origins [(x0, y0, z0)], (NX, NY, NZ))."""
    from numpy.lib.stride_tricks import sliding_window_view as windows
    dims = [tuple(int(v) for v in d) for d in dims]
    if gap < 1:
        raise ValueError("blocks must be at least one voxel apart")
    order = sorted(range(len(dims)), key=lambda i: (-dims[i][2], -dims[i][0] * dims[i][1], i))

    def place(W, D):
        wc, dc = -(-W // res), -(-D // res)
        height = np.zeros((dc, wc), np.int64)
        org = [None] * len(dims)
        for i in order:
            nx, ny, nz = dims[i]
            fx, fy = -(-(nx + gap) // res), -(-(ny + gap) // res)
            if fx > wc or fy > dc:
                return None
            top = windows(height, fx, axis=1).max(axis=2)
            top = windows(top, fy, axis=0).max(axis=2)
            z = top.min()
            ys, xs = np.nonzero(top == z)
            k = np.lexsort((xs, ys))[0]
            y, x = int(ys[k]), int(xs[k])
            org[i] = (x * res, y * res, int(z))
            height[y:y + fy, x:x + fx] = z + nz + gap
        ext = tuple(max(org[i][a] + dims[i][a] for i in range(len(dims))) for a in range(3))
        return org, ext

    if footprint is not None:
        res_ = place(*footprint)
        if res_ is None:
            raise ValueError("a block does not fit the footprint %r" % (footprint,))
        if res_[1][0] * res_[1][1] * res_[1][2] >= 1 << 31:
            raise ValueError("the packed volume would hold 2^31 voxels or more")
        return res_
    wmin = max(d[0] for d in dims) + gap
    dmin = max(d[1] for d in dims) + gap
    best = None
    for W in range(-(-wmin // 128) * 128, max_side + 1, 128):
        for ratio in (0.75, 1.0, 1.33):
            D = max(dmin, int(round(W * ratio / res)) * res)
            if D > max_side:
                continue
            r = place(W, D)
            if r is None or max(r[1]) > max_side:
                continue
            vol = r[1][0] * r[1][1] * r[1][2]
            if vol >= 1 << 31:
                continue
            if best is None or vol < best[0]:
                best = (vol, r)
    if best is None:
        raise ValueError("the blocks do not fit a packed volume of side %d" % max_side)
    return best[1]


class PackedBatch:
    """Independent blocks (Sec. 3.2 "Parallel Algorithm", Discussion "Block Based Distributed
    Parallelism": blocks are decomposed independently, their boundaries acting as restrictions)
    decomposed with ONE Lloyd loop over all of them.  Per block, on the slots' streams:
    classification, labelling, [saliency,] seeding.  Then the blocks' bands, weights and sites
    are packed into one volume (pack_layout; the blocks at least `gap` voxels of band 0xFF
    apart), lsrvt_cvt_iterate runs once over it -- every launch of the loop a grid, or the
    relaxation's work queue, over the bricks of all blocks -- and each block gets its cells
    and sites back.  Then per block again: statistics and the hierarchy merge.

    Cells, sites and statistics equal decompose() of each block alone (tests/test_gpu_forms.py);
    the Lloyd trace is the batch's sum (`self.trace`).  All jobs share n_iters and whether they
    are weighted (gamma > 0).  capture() records the whole batch as one CUDA graph."""

    def __init__(self, jobs, gap=1, footprint=None, n_slots=4, device="cuda", share=None, want_dist=False):
        from . import MAX_PACK_BLOCKS
        if not jobs or len(jobs) > MAX_PACK_BLOCKS:
            raise ValueError("a packed batch holds 1..%d blocks" % MAX_PACK_BLOCKS)
        if len({int(j["n_iters"]) for j in jobs}) != 1 or len({bool(j.get("gamma", 0)) for j in jobs}) != 1:
            raise ValueError("the blocks of a packed batch share n_iters and weighting")
        self.jobs = jobs
        self.device = torch.device(device)
        self.dims = [(int(j["field"].shape[2]), int(j["field"].shape[1]), int(j["field"].shape[0])) for j in jobs]
        self.origins, self.packed = pack_layout(self.dims, gap, footprint)
        share = default_share(n_slots) if share is None else share
        self.slots = [Slot(self.device, share) for _ in range(n_slots)]
        # the packed loop takes the whole GPU; the share is set explicitly because a share belongs
        # to a stream handle and torch hands out recycled handles (an earlier slot's share would
        # otherwise stay with this stream)
        self.main = torch.cuda.Stream(device=self.device)
        set_stream_share(100, self.main)
        self.ws = Workspace(self.device)
        self.want_dist = want_dist
        self.graph = None
        self.trace = None

    def fill(self):
        """Voxels of the blocks over voxels of the packed volume."""
        nx, ny, nz = self.packed
        return sum(a * b * c for a, b, c in self.dims) / float(nx * ny * nz)

    def run(self):
        from . import (aggregate, classify, cvt_iterate, default_max_comp, label_components, merge_hierarchy,
                       new_status, pack_blocks, saliency_grad, seed, unpack_blocks)
        dev = self.device
        cur = torch.cuda.current_stream(dev)
        status = new_status(dev)
        for sl in self.slots:
            sl.stream.wait_stream(cur)
        outs = []
        # per block: classification, labelling, weights, seeding
        for k, job in enumerate(self.jobs):
            sl = self.slots[k % len(self.slots)]
            with torch.cuda.stream(sl.stream):
                field = job["field"]
                n = field.numel()
                max_comp = default_max_comp(n)
                band = classify(field, job["iso"])
                comp, cb, cs, cf, nc = label_components(band, max_comp, sl.ws, status)
                g = job.get("gamma", 0)
                q = saliency_grad(field, g, sl.ws) if g else None
                sp, sc, off, ns = seed(comp, q, nc, max_comp, job["voxels_per_site"], job.get("strat_block", 16),
                                       job.get("rng_seed", 0), ws=sl.ws, status=status)
                outs.append(dict(band=band, comp=comp, comp_band=cb, comp_size=cs, comp_first=cf, n_comp=nc, q=q,
                                 site_pos=sp, site_comp=sc, comp_site_off=off, n_sites=ns, max_comp=max_comp,
                                 status=status))
        for sl in self.slots:
            self.main.wait_stream(sl.stream)
        # one Lloyd loop over the packed volume
        with torch.cuda.stream(self.main):
            blocks = []
            for k, o in enumerate(outs):
                nz, ny, nx = o["band"].shape
                o["cell"] = torch.empty((nz, ny, nx), dtype=torch.int32, device=dev)
                o["dist"] = torch.empty((nz, ny, nx), dtype=torch.int32, device=dev) if self.want_dist else None
                blocks.append(dict(dims=self.dims[k], origin=self.origins[k], band=o["band"], q=o["q"],
                                   site_pos=o["site_pos"], n_sites=o["n_sites"], cell=o["cell"], dist=o["dist"]))
            # every block's site capacity, at most one site per voxel of the packed volume
            nxp, nyp, nzp = self.packed
            max_sites = min(sum(int(o["site_pos"].numel()) for o in outs), nxp * nyp * nzp)
            pband, pq, psp, pns, base = pack_blocks(blocks, self.packed, max_sites, want_q=outs[0]["q"] is not None,
                                                    status=status)
            pcell, pdist, trace = cvt_iterate(pband, pq, psp, pns, int(self.jobs[0]["n_iters"]),
                                              want_dist=self.want_dist, ws=self.ws, status=status)
            unpack_blocks(blocks, self.packed, pcell, pdist, psp, base)
            self.trace = trace
            self.n_sites_packed = pns
        for sl in self.slots:
            sl.stream.wait_stream(self.main)
        # per block: statistics and the hierarchy merge
        for k, (job, o) in enumerate(zip(self.jobs, outs)):
            sl = self.slots[k % len(self.slots)]
            aux = job.get("aux", ())
            if len(aux):
                with torch.cuda.stream(sl.stream):
                    cells = aggregate(o["cell"], list(aux), o["site_pos"], o["n_sites"], n_bins=job.get("n_bins", 32),
                                      ws=sl.ws, status=status)
                    comps, bands, vol = merge_hierarchy(cells, o["n_sites"], o["comp_site_off"], o["comp_band"],
                                                        o["n_comp"], o["max_comp"], len(job["iso"]) + 1,
                                                        job.get("n_bins", 32), False, sl.ws)
                    o.update(cells=cells, comps=comps, bands=bands, volume=vol)
        for sl in self.slots:
            cur.wait_stream(sl.stream)
        cur.wait_stream(self.main)
        self.outputs = outs
        return outs

    def capture(self):
        """Record the whole batch (per-block stages, packing, the packed Lloyd loop, unpacking,
        statistics) as one CUDA graph after an eager run that sizes every workspace; replay()
        then runs it with one launch.  Inputs are read at replay time."""
        self.run()
        torch.cuda.synchronize(self.device)
        self.graph = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(device=self.device)
        cap.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.graph(self.graph, stream=cap):
            self.run()
        torch.cuda.synchronize(self.device)
        return self

    def replay(self):
        self.graph.replay()
        return self.outputs

    def check(self):
        from . import check_status
        check_status(self.outputs[0]["status"], "packed batch")


def tune_packed(jobs, candidates=((1, 4), (1, 2), (4, 4)), device="cuda", reps=1):
    """Autotuner of the packing schedule: (gap, slots for the per-block stages) candidates,
    each run on the sample `jobs`; every candidate must reproduce the first one's cells and
    sites bit for bit (the schedule must not change results).  Returns (best candidate,
    {candidate: seconds}, {candidate: packed fill})."""
    times, fills, ref = {}, {}, None
    for gap, slots in candidates:
        pb = PackedBatch(jobs, gap=gap, n_slots=slots, device=device)
        pb.run()  # sizes the workspaces
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        for _ in range(reps):
            outs = pb.run()
        torch.cuda.synchronize(device)
        pb.check()
        times[(gap, slots)] = (time.perf_counter() - t0) / reps
        fills[(gap, slots)] = pb.fill()
        if ref is None:
            ref = [(o["cell"].clone(), o["site_pos"].clone()) for o in outs]
        else:
            for (c0, s0), o in zip(ref, outs):
                if not (torch.equal(c0, o["cell"]) and torch.equal(s0, o["site_pos"])):
                    raise RuntimeError("packing schedule %r changed the results" % ((gap, slots),))
    best = min(times, key=times.get)
    return best, times, fills
