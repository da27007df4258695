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

A job is a dict: field (CUDA float32 (nz, ny, nx)), iso, voxels_per_site, n_iters, aux (list
of CUDA tensors), gamma, strat_block, rng_seed, n_bins.
"""
import queue
import threading
import time

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
