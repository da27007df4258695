"""Benchmark of the LSRVT hot path on B300.

One step = the whole path over one synthetic 512^3 flame-like volume (8 isovalues i/9,
saliency weight |grad f| with gamma 1, one site per 4096 voxels, 30 Lloyd iterations,
16 float32 auxiliary variables, 32-bin histograms):
  classify -> connected components -> saliency -> seeding -> 30 x (restricted geodesic
  assignment + geodesically weighted update) + final assignment -> value ranges ->
  per-cell statistics -> cell/component/band/volume merge.
Metric: CVT Gvoxel-iterations per second = voxels x Lloyd iterations / step time.
Inputs are resident in HBM (field 512 MiB, aux 8 GiB: larger than L2, so no flush).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--side S]

--impl reference times the CPU oracle (the reference arm of this tier) on a bounded
sample of the same workload.  Under torchrun every rank runs its own independent volume
(replicas, weak scaling); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "CVT Gvoxel-iters/s"
UNIT = "Gvoxel-iters/s"
N_ITERS = 30
N_AUX = 16
N_BINS = 32
VPS = 4096
# algorithmic bytes of one Lloyd iteration per voxel: band in (1 B), weight in (2 B), the
# assignment materialised once (4 B label written, 4 B read back by the update)
ALG_BYTES_PER_VOXEL_ITER = 11
# DRAM bytes one Lloyd iteration moves per voxel, summed over its kernels, measured with ncu
# (dram__bytes_read.sum + dram__bytes_write.sum) on the 256^3 flame case and scaled by the
# voxel count (the traffic grows in proportion to it)
NCU_BYTES_PER_VOXEL_ITER = 71.7


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm=float(d["hbm_gbs"]), src="measured")
    return dict(hbm=6400.0, src="fallback")


# --------------------------------------------------------------------------- clocks
class Clocks:
    """Samples nvidia-smi every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            tok = [t.strip() for t in line.split(",")]
            if len(tok) < 9:
                continue
            try:
                sm.append(float(tok[1]))
                smax.append(float(tok[2]))
            except ValueError:
                continue
            for name, v in zip(names, tok[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(smax) if smax else None,
                    reasons=sorted(reasons), samples=len(sm))


# --------------------------------------------------------------------------- replicas
# The path shards into independent volumes (blocks): under torchrun each rank decomposes its own
# volume (weak scaling), no data crosses ranks; only the step time is combined.
def rank_seed(rank):
    """Workload seed of a rank: every replica gets its own volume."""
    return 2 + 1000 * rank


def max_over_ranks(ms, world, device):
    """The step time of the job: the slowest rank's (every rank gets the result)."""
    if world > 1:
        t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    return ms


def job_value(world, voxels_per_rank, iters, ms):
    """Whole-job throughput: the voxel-iterations of all ranks over the slowest rank's time."""
    return world * voxels_per_rank * iters / (ms * 1e-3) / 1e9


# --------------------------------------------------------------------------- GPU arm
class Pipeline:
    """The hot path with buffers and workspaces allocated once (all compute in liblsrvt)."""

    def __init__(self, pkg, field, aux, iso, max_comp=None):
        self.pkg = pkg
        self.field = field
        self.aux = list(aux)
        self.iso = iso
        self.dev = field.device
        self.n = field.numel()
        self.max_comp = pkg.default_max_comp(self.n) if max_comp is None else int(max_comp)
        self.ws = pkg.Workspace(self.dev)
        self.status = pkg.new_status(self.dev)
        self.n_bands = len(iso) + 1

    def step(self, marks=None):
        pk = self.pkg
        ev = (lambda name: marks.append((name, torch.cuda.Event(enable_timing=True)))) if marks is not None else None

        def mark(name):
            if ev:
                ev(name)
                marks[-1][1].record()

        mark("start")
        band = pk.classify(self.field, self.iso)
        mark("classify")
        comp, cb, cs, cf, nc = pk.label_components(band, self.max_comp, self.ws, self.status)
        mark("label")
        q = pk.saliency_grad(self.field, 1, self.ws)
        mark("saliency")
        sp, sc, off, ns = pk.seed(comp, q, nc, self.max_comp, VPS, 16, 2, ws=self.ws, status=self.status)
        mark("seed")
        cell, dist, trace = pk.cvt_iterate(band, q, sp, ns, N_ITERS, want_dist=False, ws=self.ws,
                                           status=self.status)
        mark("cvt")
        lo, scale = pk.aux_range(cell, self.aux, N_BINS, self.status)
        mark("range")
        cells = pk.aggregate(cell, self.aux, sp, ns, lo, scale, N_BINS, ws=self.ws, status=self.status)
        mark("aggregate")
        comps, bands, vol = pk.merge_hierarchy(cells, ns, off, cb, nc, self.max_comp, self.n_bands, N_BINS,
                                               ws=self.ws)
        mark("merge")
        self.last = dict(band=band, cell=cell, site_pos=sp, n_sites=ns, n_comp=nc, comp_site_off=off,
                         comp_band=cb, cells=cells, comps=comps, bands=bands, volume=vol, trace=trace)
        return self.last


def convergence_summary(trace, n_sites):
    """The Lloyd trace of the last step: sites moved, mean d_s (voxels; the paper's
    convergence measure) and the CVT energy sum q_v D(v)^2 (voxel^2) per iteration, with the
    number of iterations that raised it (recorded, not asserted: the method does not promise
    a monotone energy)."""
    import paper_2208_06970_b300 as pkg
    t = pkg.trace_summary(trace, n_sites)
    return dict(moved=t["moved"], mean_ds=[round(v, 5) for v in t["mean_ds"]],
                energy_voxel2=[float("%.6g" % v) for v in t["energy_voxel2"]],
                energy_increases=t["energy_increases"])


def count_launches(fn):
    """Kernels launched by one call of fn, from the CUDA activity trace (CUPTI via torch.profiler)."""
    from torch.profiler import ProfilerActivity, profile
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        fn()
        torch.cuda.synchronize()
    names = {}
    for e in prof.events():
        if e.device_type.name == "CUDA" and "lsrvt" in e.name:
            names[e.name] = names.get(e.name, 0) + 1
    return sum(names.values()), names


def gpu_arm(args, rank, world, local_rank):
    import paper_2208_06970_b300 as pkg
    import workloads
    from paper_2208_06970_b300 import build
    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    side = args.side
    w = workloads.flame_workload(side=side, seed=rank_seed(rank), device=dev, n_aux=N_AUX, n_iters=N_ITERS,
                                 recipe=args.flame_recipe)
    field, aux, iso = w["field"], w["aux"], w["iso"]
    n = field.numel()
    # the sharp recipe shatters the isobands into more components than the default capacity:
    # count them once and size the component (and so the site and statistics) capacity to fit
    max_comp = None
    if args.flame_recipe == "sharp":
        b0 = pkg.classify(field, iso)
        nc0 = pkg.label_components(b0, max_comp=n // 4)[4]
        max_comp = int(nc0.item()) + 1024
        del b0, nc0
        torch.cuda.empty_cache()
    pipe = Pipeline(pkg, field, [aux[j] for j in range(N_AUX)], iso, max_comp=max_comp)
    for _ in range(args.warmup):
        pipe.step()
    torch.cuda.synchronize()
    pkg.check_status(pipe.status, "warmup")
    n_sites = int(pipe.last["n_sites"].item())
    n_comp = int(pipe.last["n_comp"].item())
    trace = pipe.last["trace"].cpu().numpy()
    launches_per_step, kernel_names = count_launches(pipe.step)

    # ---- timed region: K steps, events on the launching stream
    clocks = Clocks(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    s = torch.cuda.current_stream()
    phase = {}
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(s)
    for _ in range(args.steps):
        marks = []
        pipe.step(marks)
        marks_done = marks
    t1.record(s)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1) / args.steps
    names = [m[0] for m in marks_done]
    for a, b in zip(marks_done[:-1], marks_done[1:]):
        phase[b[0]] = a[1].elapsed_time(b[1])
    pkg.check_status(pipe.status, "timed")
    ms = max_over_ranks(ms, world, dev)

    # ---- dominant kernels: one Lloyd iteration (tessellation + geodesically weighted update),
    # timed with CUDA events as cvt_iterate(k) - cvt_iterate(0) from the same sites
    sp0 = pipe.last["site_pos"].clone()
    band = pipe.last["band"]
    q = pkg.saliency_grad(field, 1, pipe.ws)
    ns = pipe.last["n_sites"]
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a2 = torch.cuda.Event(enable_timing=True)
    kk = 5
    sp_tmp = sp0.clone()
    pkg.cvt_iterate(band, q, sp_tmp, ns, 0, want_dist=False, want_trace=False, ws=pipe.ws, status=pipe.status)
    torch.cuda.synchronize()
    a0.record(s)
    sp_tmp = sp0.clone()
    pkg.cvt_iterate(band, q, sp_tmp, ns, 0, want_dist=False, want_trace=False, ws=pipe.ws, status=pipe.status)
    a1.record(s)
    sp_tmp = sp0.clone()
    pkg.cvt_iterate(band, q, sp_tmp, ns, kk, want_dist=False, want_trace=False, ws=pipe.ws, status=pipe.status)
    a2.record(s)
    torch.cuda.synchronize()
    t0_ms = a0.elapsed_time(a1)
    t_iter = (a1.elapsed_time(a2) - t0_ms) / kk  # ms per Lloyd iteration
    t_assign = t0_ms
    pk = peaks()
    iter_bytes = n * ALG_BYTES_PER_VOXEL_ITER
    achieved = iter_bytes / (t_iter * 1e-3) / 1e9
    agg_ms = phase.get("aggregate", 0.0)
    agg_bytes = n * (4 + 4 * N_AUX)
    stats_gbs = agg_bytes / (agg_ms * 1e-3) / 1e9 if agg_ms > 0 else None
    cvt_ms = phase.get("cvt", 0.0)

    # ---- end to end through the public API with host buffers: decompose_host uploads the
    # field, overlaps the auxiliary upload with the tessellation, and returns the per-cell
    # statistics and sites in host memory (the call synchronises)
    e2e = None
    h_field = field.cpu().pin_memory()
    h_aux = aux.cpu().pin_memory()
    h2d = h_field.numel() * 4 + h_aux.numel() * 4
    bufs = {}
    e_kw = dict(aux=h_aux, gamma=1, strat_block=16, rng_seed=2, n_bins=N_BINS, buffers=bufs, device=dev)
    pkg.decompose_host(h_field, iso, VPS, N_ITERS, **e_kw)  # first call allocates
    e_steps = max(1, min(args.steps, 2))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(e_steps):
        host = pkg.decompose_host(h_field, iso, VPS, N_ITERS, **e_kw)
    e1.record(s)
    torch.cuda.synchronize()
    d2h = host["site_pos"].numel() * 4 + sum(t.numel() * t.element_size() for t in host["cells"].values()
                                             if t is not None)
    e_ms = e0.elapsed_time(e1) / e_steps
    e2e = dict(value=n * N_ITERS / (e_ms * 1e-3) / 1e9, unit=UNIT, h2d_bytes_per_step=int(h2d),
               d2h_bytes_per_step=int(d2h), ms_per_step=e_ms, api="decompose_host")
    del h_aux, bufs
    layout = layout_arm(pkg, pipe, s)
    graph = graph_arm(pkg, pipe, s)
    anyangle = anyangle_arm(pkg, pipe, s)
    res = dict(ms=ms, phase=phase, clk=clk, n_sites=n_sites, n_comp=n_comp, trace=trace, t_assign=t_assign,
               t_iter=t_iter,
               achieved=achieved, peak=pk, stats_gbs=stats_gbs, cvt_ms=cvt_ms, launches=launches_per_step,
               kernels=kernel_names, e2e=e2e, n=n, field=field, aux=aux, iso=iso, layout=layout, graph=graph,
               anyangle=anyangle)
    return res


def layout_arm(pkg, pipe, s, reps=3):
    """The structured hierarchical layout of the last step's decomposition (all bands, every
    variable): compaction, stable radix sort by cell, offsets, extraction of the variables.
    Algorithmic bytes: the cell labels read once, one coordinate written and every variable
    read and written once per kept voxel."""
    L = pipe.last
    m = len(pipe.aux)
    max_sites = L["site_pos"].numel()

    def run(out=None):
        return pkg.structured_layout(L["cell"], L["n_sites"], max_sites, L["comp_site_off"], L["comp_band"],
                                     L["n_comp"], pipe.max_comp, aux=pipe.aux, ws=pipe.ws, status=pipe.status,
                                     out=out)
    out = run()
    torch.cuda.synchronize()
    pkg.check_status(pipe.status, "layout")
    r = int(out["n_kept"].item())
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        run(out)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    alg = pipe.n * 4 + r * (4 + 8 * m)
    gbs = alg / (ms * 1e-3) / 1e9
    pk = peaks()
    res = dict(ms=ms, kept_voxels=r, variables=m, algorithmic_bytes=int(alg), algorithmic_gbs=gbs,
               frac=gbs / pk["hbm"], peak_source=pk["src"],
               what="voxels of all bands ordered by (band, component, cell, index) + offsets + "
                    "extraction of every variable in layout order")
    res["joint"] = joint_arm(pkg, pipe, out, s)
    return res


JOINT_VARS = 4


def graph_arm(pkg, pipe, s, reps=3):
    """The Voronoi site graph of the last step's decomposition, then the geodesic distances
    (and the ratio ||x_i - x_j|| / gd) among all sites of its largest component.  The build
    reads the labels and bands once (5 B per voxel) plus their +x/+y/+z neighbours."""
    L = pipe.last
    band = L["band"]
    cell = L["cell"]
    sp = L["site_pos"]
    g = pkg.site_graph(cell, band, sp, L["n_sites"], ws=pipe.ws, status=pipe.status)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        g = pkg.site_graph(cell, band, sp, L["n_sites"], ws=pipe.ws, status=pipe.status)
    e1.record(s)
    torch.cuda.synchronize()
    pkg.check_status(pipe.status, "site graph")
    build_ms = e0.elapsed_time(e1) / reps
    off = L["comp_site_off"][:int(L["n_comp"].item()) + 1].cpu().numpy()
    c = int((off[1:] - off[:-1]).argmax())
    s0, s1 = int(off[c]), int(off[c + 1])
    k = s1 - s0
    nz, ny, nx = cell.shape
    dist, ratio = pkg.site_geodesics(g, sp, (nx, ny, nz), s0, s1, c_far=2.0, ws=pipe.ws, status=pipe.status)
    torch.cuda.synchronize()
    e0.record(s)
    dist, ratio = pkg.site_geodesics(g, sp, (nx, ny, nz), s0, s1, c_far=2.0, ws=pipe.ws, status=pipe.status)
    e1.record(s)
    torch.cuda.synchronize()
    pkg.check_status(pipe.status, "site geodesics")
    geo_ms = e0.elapsed_time(e1)
    n = cell.numel()
    gbs = n * 5 / (build_ms * 1e-3) / 1e9
    pk = peaks()
    arcs = int(g["off"][s1].item() - g["off"][s0].item())
    return dict(build_ms=build_ms, edges=int(g["n_edges"].item()), build_algorithmic_gbs=gbs,
                build_frac=gbs / pk["hbm"], largest_component_sites=k, largest_component_arcs=arcs,
                apsp_ms=geo_ms, apsp_pairs=k * k, apsp_arcs_scanned_lower_bound=k * arcs,
                what="site graph (face-adjacent cells, integer Euclidean weights), then geodesic distances and "
                     "||x_i - x_j|| / gd between all sites of the largest component")


def anyangle_arm(pkg, pipe, s):
    """The any-angle tessellation of Sec. 3.2 (region growing with src(w) shortcuts in
    synchronous rounds) of the last step's final sites, beside the chamfer tessellation of the
    same sites.  Algorithmic bytes per voxel and round: band 1 + edge mask 4 + key 8 + source 4
    read, key and source 12 written (neighbour states come from cache): 29 B."""
    L = pipe.last
    band, ns = L["band"], L["n_sites"]
    n = band.numel()

    def any_angle():
        sp = L["site_pos"].clone()
        return pkg.cvt_iterate_anyangle(band, None, sp, ns, 0, want_trace=False, ws=pipe.ws, status=pipe.status)

    def chamfer():
        sp = L["site_pos"].clone()
        return pkg.cvt_iterate(band, None, sp, ns, 0, want_trace=False, ws=pipe.ws, status=pipe.status)
    any_angle()
    chamfer()
    torch.cuda.synchronize()
    pkg.check_status(pipe.status, "any-angle tessellation")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    cell_a, dist_a, src_a, _, rounds = any_angle()
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    e0.record(s)
    cell_c, dist_c, _ = chamfer()
    e1.record(s)
    torch.cuda.synchronize()
    pkg.check_status(pipe.status, "any-angle tessellation")
    chamfer_ms = e0.elapsed_time(e1)
    reached = cell_c >= 0
    da = dist_a.to(torch.int64) & 0xFFFFFFFF
    dc = dist_c.to(torch.int64) & 0xFFFFFFFF
    r = int(rounds[0])
    gbs = n * 29 / (ms / r * 1e-3) / 1e9
    pk = peaks()
    return dict(ms=ms, rounds=r, ms_per_round=ms / r, algorithmic_bytes_per_voxel_round=29,
                algorithmic_gbs=gbs, frac=gbs / pk["hbm"], peak_source=pk["src"], chamfer_ms=chamfer_ms,
                same_cell_frac=float((cell_a == cell_c)[reached].float().mean().item()),
                shorter_frac=float((da < dc)[reached].float().mean().item()),
                length_ratio_mean=float((da[reached].double() / dc[reached].clamp(min=1).double()).mean().item()),
                what="any-angle tessellation (src(w) shortcuts with ray casts, synchronous rounds) of the final "
                     "sites; chamfer tessellation of the same sites for comparison")


def joint_arm(pkg, pipe, lay, s, reps=3):
    """Joint central moments of orders 2..4 of the first four variables over every cell of the
    layout, then their merge up the hierarchy.  Bound: FP32 FMA issue (each voxel contributes
    E = m + m(m+1)/2 + C(m+2,3) + C(m+3,4) products; 69 at m = 4)."""
    from math import comb
    L = pipe.last
    m = JOINT_VARS
    E = m + comb(m + 1, 2) + comb(m + 2, 3) + comb(m + 3, 4)
    ns = L["n_sites"]
    rows = L["site_pos"].numel()
    vals = [lay["values"][j] for j in range(m)]
    out = pkg.joint_moments(vals, lay["cell_off"], ns, rows, ws=pipe.ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        pkg.joint_moments(vals, lay["cell_off"], ns, rows, ws=pipe.ws, out=out)
    e1.record(s)
    for _ in range(reps):
        pkg.merge_joint_hierarchy(out, ns, L["comp_site_off"], L["comp_band"], L["n_comp"], pipe.max_comp,
                                  pipe.n_bands, ws=pipe.ws)
    e2.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    r = int(lay["n_kept"].item())
    fma = r * E
    clk = 2.032e9  # maximum SM clock
    peak = 148 * 128 * clk / 1e12  # FP32 FMA lanes x clock, T FMA/s
    ach = fma / (ms * 1e-3) / 1e12
    return dict(ms=ms, merge_ms=e1.elapsed_time(e2) / reps, variables=m, products_per_voxel=E, voxels=r,
                bound="alu", achieved=ach, peak=peak, unit="T FMA/s", frac=ach / peak,
                read_gbs=r * 4 * m / (ms * 1e-3) / 1e9,
                peak_note="148 SMs x 128 FP32 lanes x 2.032 GHz (unit counts and maximum clock)")


# --------------------------------------------------------------------------- oracle arm
def host_info():
    """Core count and CPU model of the machine the oracle runs on."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return dict(nproc=os.cpu_count(), cpu_model=model)


class PinnedCore:
    """Runs the enclosed (single-threaded) oracle call pinned to one core, then restores the
    calling thread's affinity.  The core is the highest one the process may use."""

    def __enter__(self):
        self.old = None
        self.core = None
        if hasattr(os, "sched_getaffinity"):
            self.old = os.sched_getaffinity(0)
            self.core = max(self.old)
            os.sched_setaffinity(0, {self.core})
        return self

    def __exit__(self, *exc):
        if self.old is not None:
            os.sched_setaffinity(0, self.old)
        return False


def oracle_sample(field, aux, iso, side=96, iters=2):
    """The CPU oracle on a side^3 corner of the workload (bounded sample), pinned to one core;
    returns (voxel-iterations per second, seconds, description)."""
    import oracle
    f = field[:side, :side, :side].contiguous().cpu().numpy()
    a = aux[:, :side, :side, :side].contiguous().cpu().numpy()
    with PinnedCore():
        return _oracle_path(oracle, f, a, iso, iters, side)


def _oracle_path(oracle, f, a, iso, iters, side):
    t0 = time.perf_counter()
    band = oracle.classify(f, iso)
    comp, cb, cs, cf = oracle.label_components(band)
    q = oracle.saliency(f, 1)
    sp, sc, off, nc = oracle.seed(comp, q, len(cb), VPS, 16, 2)
    sp2, cell, dist, tr = oracle.cvt_iterate(band, q, sp, iters)
    lo, hi, scale = oracle.aux_range(cell, a, N_BINS)
    st = oracle.aggregate(cell, a, len(sp2), lo, scale, N_BINS)
    oracle.merge_hierarchy(st, sc, cb, len(iso) + 1)
    dt = time.perf_counter() - t0
    vox = f.size
    return (vox * iters / dt / 1e9, dt, "%d^3 corner of the workload, %d Lloyd iterations, whole path; "
            "the metric's value is extrapolated from it (voxel-iterations of the corner / its time)" % (side, iters))


def oracle_full_size_stages(field, aux, iso):
    """The one-pass stages of the path on the whole volume, in the oracle pinned to one core:
    classification, component labelling, saliency, seeding and the statistics sweep (per-cell
    moments and histograms of every auxiliary variable; the cells for this timing are the
    oracle's own components, since a full-size oracle tessellation is out of reach).  The
    Lloyd loop itself is timed only on the corner sample.  Returns seconds per stage."""
    import oracle
    f = field.contiguous().cpu().numpy()
    out = {}
    with PinnedCore() as pc:
        t = time.perf_counter()
        band = oracle.classify(f, iso)
        out["classify"] = time.perf_counter() - t
        t = time.perf_counter()
        comp, cb, cs, cf = oracle.label_components(band)
        out["label_components"] = time.perf_counter() - t
        t = time.perf_counter()
        q = oracle.saliency(f, 1)
        out["saliency"] = time.perf_counter() - t
        t = time.perf_counter()
        oracle.seed(comp, q, len(cb), VPS, 16, 2)
        out["seed"] = time.perf_counter() - t
        del q, band
        a = aux.contiguous().cpu().numpy()
        t = time.perf_counter()
        lo, hi, scale = oracle.aux_range(comp, a, N_BINS)
        oracle.aggregate(comp, a, len(cb), lo, scale, N_BINS)
        out["aggregate"] = time.perf_counter() - t
        core = pc.core
    del a
    return dict(seconds=out, core=core, voxels=int(f.size), n_aux=int(aux.shape[0]),
                note="whole %dx%dx%d volume; statistics over the oracle's components" % tuple(f.shape[::-1]))


def reference_arm(args):
    import workloads
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    w = workloads.flame_workload(side=args.side, seed=2, device=dev, n_aux=N_AUX, n_iters=N_ITERS)
    vals = []
    times = []
    for i in range(args.warmup + args.steps):
        v, dt, desc = oracle_sample(w["field"], w["aux"], w["iso"], side=args.ref_side, iters=args.ref_iters)
        if i >= args.warmup:
            vals.append(v)
            times.append(dt)
    value = statistics.mean(vals)
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * statistics.mean(times), higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="int32/f32/f64", data="synthetic", impl="reference",
                config=dict(workload="flame %d^3 (oracle sample %d^3)" % (args.side, args.ref_side),
                            voxels_per_site=VPS, n_iters=N_ITERS, n_aux=N_AUX),
                cpu_baseline=dict(value=value, unit=UNIT, cores=1, kind="oracle", sample=desc, extrapolated=True,
                                  pinned="one core (sched_setaffinity)", host=host_info()),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def forms_arm(args, dev):
    """Batched blocks (independent blocks with sides U{32..256}, 2-12 isovalues, 20 Lloyd
    iterations, 3 aux) and a served Poisson request stream (50/s, sides U{64..hi}, 2-10
    isovalues, 0-16 aux, 10-30 iterations), each against the plain one-at-a-time form on the
    same GPU.  Throughput counts voxels x Lloyd iterations."""
    import paper_2208_06970_b300 as pkg
    import workloads
    from paper_2208_06970_b300 import runtime
    out = {}
    # ---- batching
    blocks = workloads.block_batch(n_blocks=args.blocks, seed=3, lo=32, hi=256, device=dev)
    jobs = [dict(field=b["field"], iso=b["iso"], voxels_per_site=b["voxels_per_site"], n_iters=b["n_iters"],
                 aux=[b["aux"][j] for j in range(b["aux"].shape[0])], gamma=0, strat_block=16,
                 rng_seed=b["rng_seed"], n_bins=32) for b in blocks]
    vox_it = sum(j["field"].numel() * j["n_iters"] for j in jobs)
    # the batching schedule (slots, SM share per slot) picked by the autotuner on a sample of
    # 16 blocks (untimed; every candidate is checked to reproduce the labels)
    best, tune_times = runtime.tune_batch(jobs[:16], device=dev)
    res = {}
    for name, (slots, share) in (("plain", (1, 100)), ("batched", best)):
        runner = runtime.BatchRunner(n_slots=slots, device=dev, share=share)
        runner.run(jobs[:2])  # warm the slots' workspaces
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        runner.run(jobs)
        torch.cuda.synchronize()
        res[name] = vox_it / (time.perf_counter() - t0) / 1e9
    # the same batch captured once as one CUDA graph (all blocks on the slots' streams), then
    # replayed: one launch per batch
    gb = runtime.GraphBatch(jobs, n_slots=best[0], device=dev, share=best[1])
    gb.replay()
    torch.cuda.synchronize()
    gb.check()
    reps = 2
    t0 = time.perf_counter()
    for _ in range(reps):
        gb.replay()
    torch.cuda.synchronize()
    res["graph"] = reps * vox_it / (time.perf_counter() - t0) / 1e9
    del gb
    torch.cuda.empty_cache()
    # all blocks packed into one volume and decomposed with one Lloyd loop (every launch a grid
    # over the bricks of all blocks); the packing schedule (gap, slots of the per-block stages)
    # tuned on the same 16-block sample, checked to leave cells and sites unchanged; eager, then
    # captured as one CUDA graph and replayed
    pbest, ptimes, pfills = runtime.tune_packed(jobs[:16], device=dev)
    pb = runtime.PackedBatch(jobs, gap=pbest[0], n_slots=pbest[1], device=dev)
    pb.run()
    torch.cuda.synchronize()
    pb.check()
    t0 = time.perf_counter()
    pb.run()
    torch.cuda.synchronize()
    res["packed"] = vox_it / (time.perf_counter() - t0) / 1e9
    pb.capture()
    pb.replay()
    torch.cuda.synchronize()
    pb.check()
    t0 = time.perf_counter()
    for _ in range(reps):
        pb.replay()
    torch.cuda.synchronize()
    res["packed_graph"] = reps * vox_it / (time.perf_counter() - t0) / 1e9
    packed = dict(gap=pbest[0], slots=pbest[1], extent=list(pb.packed), fill=round(pb.fill(), 4),
                  tuned={"%d/%d" % k: v for k, v in ptimes.items()}, gvoxel_iters_s=res["packed"],
                  speedup=res["packed"] / res["plain"], graph_gvoxel_iters_s=res["packed_graph"],
                  graph_speedup=res["packed_graph"] / res["plain"])
    del pb
    torch.cuda.empty_cache()
    out["batched"] = dict(blocks=len(jobs), voxels=int(sum(j["field"].numel() for j in jobs)), slots=best[0],
                          share_pct=best[1], tuned={"%d/%d" % k: v for k, v in tune_times.items()},
                          plain_gvoxel_iters_s=res["plain"], batched_gvoxel_iters_s=res["batched"],
                          speedup=res["batched"] / res["plain"], graph_gvoxel_iters_s=res["graph"],
                          graph_speedup=res["graph"] / res["plain"], packed=packed)
    del jobs, blocks
    torch.cuda.empty_cache()
    # ---- serving
    reqs = workloads.request_stream(n_requests=args.requests, rate=50.0, seed=5, lo=64, hi=args.serve_hi)
    jobs = []
    for r in reqs:
        f = workloads.blob_field(r["dims"], r["seed"], dev)
        aux = [workloads.blob_field(r["dims"], r["seed"] + 1 + j, dev, n_blobs=8, noise=0.1) for j in range(r["n_aux"])]
        jobs.append(dict(field=f, iso=r["iso"], voxels_per_site=r["voxels_per_site"], n_iters=r["n_iters"], aux=aux,
                         gamma=0, strat_block=16, rng_seed=r["seed"], n_bins=32))
        r["ws_bytes"], rest = runtime.job_bytes_split(jobs[-1])
        r["bytes"] = r["ws_bytes"] + rest
        r["work"] = int(np.prod(r["dims"])) * r["n_iters"]  # voxel-iterations: the admission estimate
    for k, r in enumerate(reqs):
        r["k"] = k
    summ = {}
    for name, slots, policy in (("plain", 1, "fifo"), ("served", args.slots, "fifo"), ("served_sjf", args.slots, "sjf")):
        srv = runtime.Server(n_slots=slots, hbm_budget=args.hbm_budget << 30, device=dev, policy=policy)
        srv.serve([dict(arrival=0.0, k=0, bytes=reqs[0]["bytes"], ws_bytes=reqs[0]["ws_bytes"])],
                  lambda r: jobs[r["k"]])  # warm-up
        torch.cuda.synchronize()
        recs = srv.serve(reqs, lambda r: jobs[r["k"]])
        summ[name] = runtime.latency_summary(recs)
    out["served"] = dict(requests=len(reqs), rate_per_s=50.0, sides="64..%d" % args.serve_hi, slots=args.slots,
                         hbm_budget_gib=args.hbm_budget, plain=summ["plain"], served=summ["served"],
                         served_sjf=summ["served_sjf"])
    return out


def serve_config5(args, dev):
    """The served form on the request stream as specified: args.requests Poisson requests at
    50/s, sides U{64..512} per axis, 2-10 isovalues, 0-16 aux variables, 10-30 Lloyd iterations,
    512 voxels per site.  Each request's field and variables are cut from resident 512^3 blob
    volumes when it is admitted (on the slot's stream, so every arm pays for it).  Arms: the
    plain form (one request at a time, FIFO), the served form (args.slots slots, FIFO) and
    shortest-work-first; each arm runs args.repeats times.  Prints one JSON line."""
    import paper_2208_06970_b300 as pkg
    import workloads
    from paper_2208_06970_b300 import runtime
    pool = workloads.CropPool(side=512, n_aux=16, seed=7, device=dev)
    reqs = workloads.request_stream(n_requests=args.requests, rate=50.0, seed=5, lo=64, hi=512)

    def make_job(r):
        f, aux = pool.request_data(r)
        return dict(field=f, iso=r["iso"], voxels_per_site=r["voxels_per_site"], n_iters=r["n_iters"], aux=aux,
                    gamma=0, strat_block=16, rng_seed=r["seed"], n_bins=32)

    for k, r in enumerate(reqs):
        r["k"] = k
        n = int(np.prod(r["dims"]))
        r["ws_bytes"], rest = runtime.request_bytes_split(n, r["n_aux"], 512, 32, dims=tuple(r["dims"]))
        r["bytes"] = r["ws_bytes"] + rest
        r["work"] = n * r["n_iters"]
    # size-aware filling: requests up to the stream's lower quartile of work may run beside the
    # large ones, on a slot with a fifth of the SMs
    fill_work = sorted(r["work"] for r in reqs)[len(reqs) // 4]
    all_arms = {"plain": (1, "fifo"), "served": (args.slots, "fifo"), "served_sjf": (args.slots, "sjf"),
                "served_fill": (args.slots, "fill")}
    arms = [(a, all_arms[a][0], all_arms[a][1]) for a in args.arms.split(",")]
    runs = {name: [] for name, _, _ in arms}
    for rep in range(args.repeats):
        for name, slots, policy in arms:
            srv = runtime.Server(n_slots=slots, hbm_budget=args.hbm_budget << 30, device=dev, policy=policy,
                                 fill_work=fill_work, fill_share=20)
            srv.serve([dict(reqs[0], arrival=0.0)], make_job)  # warm-up
            torch.cuda.synchronize()
            runs[name].append(runtime.latency_summary(srv.serve(reqs, make_job)))
            del srv
            torch.cuda.empty_cache()
    summ = {}
    for name, rs in runs.items():
        thr = [r["throughput_req_s"] for r in rs]
        summ[name] = dict(throughput_req_s=thr, mean_throughput=sum(thr) / len(thr), spread=max(thr) - min(thr),
                          p50_ms=[r["p50_ms"] for r in rs], p99_ms=[r["p99_ms"] for r in rs],
                          gvoxel_iters_s=[r["gvoxel_iters_s"] for r in rs])
    vox_it = sum(r["work"] for r in reqs)
    print(json.dumps(dict(form="served", requests=len(reqs), rate_per_s=50.0, sides="64..512", isovalues="2..10",
                          aux="0..16", iters="10..30", slots=args.slots, hbm_budget_gib=args.hbm_budget,
                          repeats=args.repeats, gvoxel_iters=vox_it / 1e9, data="synthetic: crops of 512^3 blob volumes",
                          fill_work=fill_work,
                          arms=summ)))


def precision_setup(pkg, side, dev, m=32):
    """The precision form's inputs and labels: blob field (seed 4), 32 correlated variables,
    classify -> components -> seeds (512 voxels per site) -> 10 Lloyd iterations."""
    import workloads
    f = workloads.blob_field((side,) * 3, 4, dev)
    aux = workloads.correlated_aux((side,) * 3, m, 4, dev)[0]
    ws = pkg.Workspace(dev)
    st = pkg.new_status(dev)
    n = f.numel()
    mc = pkg.default_max_comp(n)
    band = pkg.classify(f, np.array([0.2, 0.4, 0.6, 0.8], np.float32))
    comp, cb, cs, cf, nc = pkg.label_components(band, mc, ws, st)
    sp, sc, off, ns = pkg.seed(comp, None, nc, mc, 512, 16, 4, ws=ws, status=st)
    cell, _, _ = pkg.cvt_iterate(band, None, sp, ns, 10, want_dist=False, want_trace=False, ws=ws, status=st)
    del f, band, comp
    return dict(side=side, m=m, n=n, cell=cell, aux=aux, auxl=[aux[j] for j in range(m)], sp=sp, ns=ns, ws=ws, st=st,
                off=off, cb=cb, nc=nc, mc=mc)


def precision_arm(args, dev):
    """Precision form on its own workload: a 640^3 blob field (the 64^3 generator at the same
    blob density, 4 isovalues, 512 voxels per site, 10 Lloyd iterations) with 32 correlated
    Gaussian variables; per-cell moments (float-float, FP64 finalise) and co-moments (BF16
    split products on tcgen05 tensor cores, FP32 accumulation, FP64 finalise), timed with CUDA
    events on the launching stream; errors against the FP64 oracle are checked by the
    full-size tests."""
    import paper_2208_06970_b300 as pkg
    P = precision_setup(pkg, args.prec_side, dev)
    side, m, n, cell, auxl, sp, ns, ws, st = (P[k] for k in ("side", "m", "n", "cell", "auxl", "sp", "ns", "ws", "st"))
    s = torch.cuda.current_stream()

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        for _ in range(reps):
            fn()
        b.record(s)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    mom = timed(lambda: pkg.aggregate(cell, auxl, sp, ns, None, None, 0, ws=ws, status=st))
    both = timed(lambda: pkg.aggregate(cell, auxl, sp, ns, None, None, 0, cov=True, ws=ws, status=st))
    pkg.check_status(st, "precision form")
    gb = n * 4 * (1 + m) / 1e9
    # the same statistics on the structured layout: every cell a contiguous run of a 32 x 4 x N/128
    # pseudo-volume (per-position cells from the layout), so the co-moments read contiguous runs
    # instead of gathering each cell's voxels from the volume
    on_layout = None
    if n % 128 == 0:
        rows = sp.numel()
        lay = pkg.structured_layout(cell, ns, rows, P["off"], P["cb"], P["nc"], P["mc"], aux=auxl, ws=ws, status=st,
                                    want_cells=True)
        t_lay = timed(lambda: pkg.structured_layout(cell, ns, rows, P["off"], P["cb"], P["nc"], P["mc"], aux=auxl,
                                                    ws=ws, status=st, out=lay, want_cells=True))
        r = int(lay["n_kept"].item())
        shape = (n // 128, 4, 32)
        lcell = lay["cell_pos"].view(shape)
        lvals = [lay["values"][j].view(shape) for j in range(m)]
        lsite = torch.clamp(lay["cell_off"][:rows], max=max(r - 1, 0)).to(torch.int32).contiguous()
        lmom = timed(lambda: pkg.aggregate(lcell, lvals, lsite, ns, None, None, 0, ws=ws, status=st))
        lboth = timed(lambda: pkg.aggregate(lcell, lvals, lsite, ns, None, None, 0, cov=True, ws=ws, status=st))
        pkg.check_status(st, "precision form on the layout")
        on_layout = dict(layout_ms=t_lay, moments_ms=lmom, comoments_ms=lboth - lmom,
                         comoments_gbs=gb / ((lboth - lmom) * 1e-3), total_ms=t_lay + lboth,
                         volume_form_total_ms=both)
        del lay, lcell, lvals, lsite
    res = dict(workload="blobs %d^3, 4 isovalues, 1 site/512 voxels, 10 Lloyd iters, %d correlated aux vars" % (side, m),
               voxels=n, sites=int(ns.item()), moments_ms=mom, moments_gbs=gb / (mom * 1e-3),
               comoments_ms=both - mom, comoments_gbs=gb / ((both - mom) * 1e-3),
               comoments_flop_per_voxel=3 * 2 * 32 * 32, on_layout=on_layout,
               precision="moments: float-float sums per brick, FP64 finalise; co-moments: BF16 hi+lo split, "
                         "hi.hi + hi.lo + lo.hi on tcgen05 (FP32 accumulate), FP64 finalise")
    del P, auxl, cell
    torch.cuda.empty_cache()
    return res


def profile_step(args):
    """Workload generation plus two identical steps, no extra instrumentation (ncu target)."""
    import paper_2208_06970_b300 as pkg
    import workloads
    from paper_2208_06970_b300 import build
    build.build()
    dev = torch.device("cuda", 0)
    w = workloads.flame_workload(side=args.side, seed=2, device=dev, n_aux=N_AUX, n_iters=N_ITERS)
    pipe = Pipeline(pkg, w["field"], [w["aux"][j] for j in range(N_AUX)], w["iso"])
    for _ in range(2):
        pipe.step()
    torch.cuda.synchronize()
    pkg.check_status(pipe.status, "profile step")
    print("profile step ok: %d sites" % int(pipe.last["n_sites"].item()))


def profile_layout(args):
    """One step of the workload, then two structured layouts of it, each followed by the joint
    moments of its cells and their merge, then the site graph and the geodesics of the largest
    component, then the any-angle tessellation of the final sites (ncu target)."""
    import paper_2208_06970_b300 as pkg
    import workloads
    from paper_2208_06970_b300 import build
    build.build()
    dev = torch.device("cuda", 0)
    w = workloads.flame_workload(side=args.side, seed=2, device=dev, n_aux=N_AUX, n_iters=N_ITERS)
    pipe = Pipeline(pkg, w["field"], [w["aux"][j] for j in range(N_AUX)], w["iso"])
    pipe.step()
    L = pipe.last
    out = None
    for _ in range(2):
        out = pkg.structured_layout(L["cell"], L["n_sites"], L["site_pos"].numel(), L["comp_site_off"],
                                    L["comp_band"], L["n_comp"], pipe.max_comp, aux=pipe.aux, ws=pipe.ws,
                                    status=pipe.status, out=out)
        jm = pkg.joint_moments([out["values"][j] for j in range(JOINT_VARS)], out["cell_off"], L["n_sites"],
                               L["site_pos"].numel(), ws=pipe.ws)
        pkg.merge_joint_hierarchy(jm, L["n_sites"], L["comp_site_off"], L["comp_band"], L["n_comp"], pipe.max_comp,
                                  pipe.n_bands, ws=pipe.ws)
    g = pkg.site_graph(L["cell"], L["band"], L["site_pos"], L["n_sites"], ws=pipe.ws, status=pipe.status)
    off = L["comp_site_off"][:int(L["n_comp"].item()) + 1].cpu().numpy()
    c = int((off[1:] - off[:-1]).argmax())
    nz, ny, nx = L["cell"].shape
    pkg.site_geodesics(g, L["site_pos"], (nx, ny, nz), int(off[c]), int(off[c + 1]), c_far=2.0, ws=pipe.ws,
                       status=pipe.status)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    aa = pkg.cvt_iterate_anyangle(L["band"], None, L["site_pos"].clone(), L["n_sites"], 0, want_trace=False,
                                  ws=pipe.ws, status=pipe.status)
    e1.record()
    torch.cuda.synchronize()
    pkg.check_status(pipe.status, "profile layout")
    print("profile layout ok: %d voxels, %d graph edges, any-angle %d rounds in %.1f ms"
          % (int(out["n_kept"].item()), int(g["n_edges"].item()), int(aa[4][0]), e0.elapsed_time(e1)))


def profile_precision(args):
    """The precision form's inputs, then two moment + co-moment aggregations (ncu target)."""
    import paper_2208_06970_b300 as pkg
    from paper_2208_06970_b300 import build
    build.build()
    dev = torch.device("cuda", 0)
    P = precision_setup(pkg, args.prec_side, dev)
    for _ in range(2):
        pkg.aggregate(P["cell"], P["auxl"], P["sp"], P["ns"], None, None, 0, cov=True, ws=P["ws"], status=P["st"])
    torch.cuda.synchronize()
    pkg.check_status(P["st"], "profile precision")
    print("profile precision ok: %d sites" % int(P["ns"].item()))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lsrvt")
    ap.add_argument("--side", type=int, default=512)
    ap.add_argument("--flame-recipe", default="resolved", choices=("resolved", "sharp"),
                    help="flame field: resolved front (default) or the sharp one: eta = 0, 4-voxel front")
    ap.add_argument("--ref-side", type=int, default=96)
    ap.add_argument("--ref-iters", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-full", action="store_true", help="skip the full-size oracle stage timings")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched / served comparison")
    ap.add_argument("--blocks", type=int, default=64)
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--serve-hi", type=int, default=384)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--serve-config5", action="store_true",
                    help="only the served form on the specified request stream (sides 64..512), --repeats times")
    ap.add_argument("--repeats", type=int, default=3)
    ap.add_argument("--arms", default="plain,served,served_sjf,served_fill",
                    help="arms of --serve-config5 (plain, served, served_sjf, served_fill)")
    ap.add_argument("--hbm-budget", type=int, default=96, help="GiB admitted at once by the server")
    ap.add_argument("--prec-side", type=int, default=640, help="side of the precision-form workload")
    ap.add_argument("--no-precision", action="store_true", help="skip the precision form")
    ap.add_argument("--profile-precision", action="store_true",
                    help="build the precision-form inputs and run two co-moment aggregations (for ncu)")
    ap.add_argument("--profile-layout", action="store_true",
                    help="one step, then two structured layouts and joint moments of it (for ncu)")
    ap.add_argument("--profile-step", action="store_true",
                    help="generate the workload and run two plain steps (for ncu); prints nothing else")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            reference_arm(args)
        return
    if args.profile_step:
        profile_step(args)
        return
    if args.profile_precision:
        profile_precision(args)
        return
    if args.profile_layout:
        profile_layout(args)
        return
    if args.serve_config5:
        from paper_2208_06970_b300 import build
        build.build()
        serve_config5(args, torch.device("cuda", local_rank))
        return
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    r = gpu_arm(args, rank, world, local_rank)
    if rank == 0:
        n = r["n"]
        value = job_value(world, n, N_ITERS, r["ms"])
        forms = None
        if not args.no_forms and world == 1:
            forms = forms_arm(args, torch.device("cuda", local_rank))
        precision = None
        if not args.no_precision and world == 1:
            precision = precision_arm(args, torch.device("cuda", local_rank))
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            v, dt, desc = oracle_sample(r["field"], r["aux"], r["iso"], side=args.ref_side, iters=args.ref_iters)
            cpu = dict(value=v, unit=UNIT, cores=1, kind="oracle", sample=desc, seconds=dt, extrapolated=True,
                       pinned="one core (sched_setaffinity)", host=host_info())
            if not args.no_oracle_full:
                cpu["full_size_stages"] = oracle_full_size_stages(r["field"], r["aux"], r["iso"])
        pk = r["peak"]
        line = dict(
            metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
            ms_per_step=r["ms"], higher_is_better=True, scaling="weak", vs_baseline=None,
            dtype="int32/u64 labels, f32 float-float + f64 stats", data="synthetic",
            config=dict(workload="flame %d^3%s, 8 isovalues, |grad| weight, 1 site/4096 voxels, %d Lloyd iters, "
                                 "%d aux vars, %d bins" % (args.side, "" if args.flame_recipe == "resolved"
                                                           else " (sharp recipe: eta 0, front width 4)", N_ITERS,
                                                           N_AUX, N_BINS),
                        voxels=n, sites=r["n_sites"], components=r["n_comp"], parallelism="replicas" if world > 1
                        else "single", l2="inputs larger than L2 (field 512 MiB + aux 8 GiB), no flush"),
            roofline=dict(kernel="one Lloyd iteration: site bins + cell lists + cfi_kernel + check_paths_kernel + "
                                 "relax_async_kernel + update_voxels_kernel + update_nonlos_kernel + "
                                 "move_sites_kernel",
                          # the roofline axis is HBM (algorithmic bytes against the measured copy rate);
                          # the measured limiter is issue and latency (dependent loads in the path and
                          # line-of-sight walks, barriers between the filter's per-brick phases)
                          bound="issue/latency", roofline_axis="hbm", achieved=r["achieved"], peak=pk["hbm"],
                          unit="GB/s",
                          frac=r["achieved"] / pk["hbm"],
                          traffic=(NCU_BYTES_PER_VOXEL_ITER * n if NCU_BYTES_PER_VOXEL_ITER and args.side in (256, 512)
                                   else None),
                          traffic_note="ncu DRAM bytes per iteration, 256^3 capture scaled by voxels",
                          peak_source=pk["src"],
                          algorithmic_bytes_per_voxel=ALG_BYTES_PER_VOXEL_ITER, ms_per_launch=r["t_iter"],
                          ms_per_tessellation=r["t_assign"]),
            stats=dict(aggregate_ms=r["phase"].get("aggregate"), algorithmic_gbs=r["stats_gbs"],
                       frac=(r["stats_gbs"] / pk["hbm"]) if r["stats_gbs"] else None),
            phases_ms=r["phase"], cvt_gvoxel_iters_per_s=n * N_ITERS / (r["cvt_ms"] * 1e-3) / 1e9,
            convergence=convergence_summary(r["trace"], r["n_sites"]), clocks=r["clk"], e2e=r["e2e"],
            gpu_launches=int(r["launches"] * args.steps), launches_per_step=r["launches"], cpu_baseline=cpu,
            layout=r["layout"], graph=r["graph"], anyangle=r["anyangle"], forms=forms, precision=precision)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
