// aggregate.cu -- per-cell statistics of the auxiliary variables (Sec. 3.3 "Aggregation";
// introduction: statistical aggregation within the segments of the tessellation).
//
// Per cell s and variable j: count, mean, M2 (population variance M2/n), exact min and
// max, an n_bins histogram, and optionally co-moments (tensor cores, below).
//
// B300 design (statistics sweep).  The volume is cut into 32x8x4 bricks (1024 voxels).  A
// CTA of 16 consumer warps and one producer warp walks its bricks; the producer streams
// each brick's cell labels and up to 16 variables (one 4 KB tile each) into shared memory
// with TMA tile loads, double buffered on mbarriers, so HBM reads of the next brick overlap
// the arithmetic on the current one.  Per brick the consumers group the voxels by cell
// with a counting sort (shared hash of the brick's cells -> dense slots -> per-slot runs of
// local indices).  The sorted runs are cut into 32-position chunks shared out to the warps
// in order.  Inside a warp, lane (j, h) owns variable j and every second position of the
// chunk (h = 0, 1), so one cell's 16 variables are reduced in parallel and only the two
// halves of the warp have to be combined when a cell ends.  A lane accumulates x - c and
// (x - c)^2 (c = the variable at the cell's site voxel, a shift common to all bricks of the
// cell) in float-float (TwoSum / FMA error-free transforms) over at most 51 elements, then
// folds them into a normalised float-float sum by accurate double-word additions (FP64 only
// once per cell and warp, for the atomics); min / max are exact; the histogram goes to lane-private 16-bit
// counters in shared memory (no bank conflicts, no atomics).  One FP64 atomic
// per (brick, cell, variable) and moment combines the bricks; a finalize pass forms
// mean = c + S1/n and M2 = S2 - S1^2/n in FP64.  HBM traffic is the algorithmic 4 B (cell)
// + 4 m B (variables) per voxel.  Volumes whose row pitch is not a multiple of 16 bytes
// (TMA cannot describe them) take the same kernel with tiles staged by plain loads.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tcgen05.cuh"
#include "tma.cuh"

namespace lsrvt {
namespace {

constexpr int kMaxBins = 256;

struct AggParams {
    const float *aux[64];
    int32_t m;
    int32_t n_bins;
    uint32_t flags;
};

struct AggAcc {
    double *s1, *s2;          // [max_sites][m]
    unsigned *vmin, *vmax;    // ordered encodings [max_sites][m]
    unsigned long long *cnt;  // [max_sites]
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly, for |a| >= |b| (Dekker)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// (xh, xl) += (yh, yl): accurate double-word addition (Joldes, Muller & Popescu 2017,
// relative error below 3 u^2), FP32 operations only
__device__ __forceinline__ void dw_add(float &xh, float &xl, float yh, float yl) {
    float sh, sl, th, tl, vh, vl;
    two_sum(xh, yh, sh, sl);
    two_sum(xl, yl, th, tl);
    fast_two_sum(sh, __fadd_rn(sl, th), vh, vl);
    fast_two_sum(vh, __fadd_rn(tl, vl), xh, xl);
}

// ------------------------------------------------------------------ statistics sweep
constexpr int GX = 32, GY = 4, GZ = 4, GV = GX * GY * GZ;  // 512-voxel brick, rows of 128 bytes
constexpr int kG = 16;                   // variables per tile: one per lane of a half warp
constexpr int kCW = 8;                   // consumer warps per CTA (two CTAs per SM)
constexpr int kCT = kCW * 32;            // consumer threads
constexpr int kAggBlock = kCT + 32;      // + the producer warp
constexpr int kVPT = GV / kCT;           // voxels per consumer thread in the sort
constexpr int kChunk = 32;               // sorted positions per work chunk
constexpr int kHashN = 2 * GV;           // twice the brick's voxels: the table never fills
constexpr int kLaneBins = 32;            // lane-private histograms up to 32 bins
constexpr int kShiftSlots = 64;          // slots per brick whose shifts are staged in shared memory
constexpr int kStackBox = 4;             // stacked variables per 4-D tensor box (8 KB)
constexpr int kRun = 16;                 // consecutive bricks (along x) a CTA takes at a time
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s bound on every mbarrier wait

struct AggMaps {
    CUtensorMap cell;
    CUtensorMap stack;    // all variables as one 4-D tensor (when they are stacked at a constant pitch)
    CUtensorMap var[64];  // one 3-D tensor per variable otherwise
};

// how the tiles reach shared memory
enum AggLoad { kLoadPlain = 0, kLoadTma = 1, kLoadTmaStack = 2 };

struct AggSmem {
    float vars[2][kG][GV];                     // TMA tiles (128-byte rows)
    int32_t cells[2][GV];
    // per warp and lane, 16 words: word w holds bin w (low half) and bin w + 16 (high half)
    uint32_t hist[kCW][16][32];
    int32_t tab[kHashN];                       // hash of the brick's cell ids (-1 empty)
    int16_t tslot[kHashN];                     // table position -> dense slot
    int16_t vt[GV];                            // voxel -> table position, then slot (-1 none)
    uint16_t sorted[GV];                       // local voxel indices grouped by slot
    int32_t off[GV + 1];                       // counts, then run offsets per slot
    int32_t cho[GV + 1];                       // first chunk of each slot
    int32_t cur[GV];                           // scatter cursors
    int32_t cellOf[GV];                        // slot -> cell id
    float shift[kShiftSlots][kG];              // per slot and variable of the tile: x at the site voxel
    uint64_t full[2], empty[2];
    int32_t wsa[2][kCW], wsb[2][kCW];
    int32_t nslots, nchunks;
};
constexpr size_t kAggSmem = sizeof(AggSmem) + 1024;
static_assert(2 * (kAggSmem + 1024) <= 228 * 1024, "two statistics CTAs must fit one SM");

// Bricks go to CTAs in runs of kRun consecutive bricks (x-neighbours in the x-fastest order),
// runs dealt round-robin over the grid; only the last run of the volume can be short.
struct RunMap {
    int64_t nbricks, nruns;
    __device__ RunMap(int64_t nb) : nbricks(nb), nruns((nb + kRun - 1) / kRun) {}
    __device__ int64_t my_bricks() const {
        if ((int64_t)blockIdx.x >= nruns) return 0;
        const int64_t runs = (nruns - 1 - blockIdx.x) / gridDim.x + 1;
        const int64_t last = blockIdx.x + (runs - 1) * (int64_t)gridDim.x;
        return (runs - 1) * kRun + (nbricks - last * kRun < kRun ? nbricks - last * kRun : kRun);
    }
    // the bi-th brick of this CTA
    __device__ int64_t brick(int64_t bi) const { return (blockIdx.x + (bi / kRun) * (int64_t)gridDim.x) * kRun + bi % kRun; }
};

// exclusive scan of two ints over the consumer threads; totals in ta, tb.  `buf` alternates
// between calls so one barrier suffices.
__device__ __forceinline__ void consumer_scan2(AggSmem &S, int buf, int a, int b, int &ea, int &eb, int &ta,
                                               int &tb) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int ua = __shfl_up_sync(0xffffffffu, ia, o), ub = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) { ia += ua; ib += ub; }
    }
    if (lane == 31) { S.wsa[buf][w] = ia; S.wsb[buf][w] = ib; }
    named_bar_sync(1, kCT);
    int pa = 0, pb = 0;
    ta = 0; tb = 0;
#pragma unroll
    for (int q = 0; q < kCW; ++q) {
        const int va = S.wsa[buf][q], vb = S.wsb[buf][q];
        if (q < w) { pa += va; pb += vb; }
        ta += va; tb += vb;
    }
    ea = pa + ia - a;
    eb = pb + ib - b;
}

// Groups the brick's voxels by cell: slots (dense, in hash-table order), run offsets, the
// sorted local indices, chunk offsets, and the per-cell voxel counts.  On entry the hash
// table is empty (cleared by the previous brick's sort, or at kernel start).
__device__ void sort_brick(AggSmem &S, const int32_t *cells_tile, Dims d, int ox, int oy, int oz, int32_t max_sites,
                           AggAcc acc, const float *__restrict__ shift_tab, int m, int j0, int G) {
    const int tid = threadIdx.x, lane = tid & 31;
    bool val[kVPT];
#pragma unroll
    for (int r = 0; r < kVPT; ++r) {
        const int v = tid + r * kCT;
        const int gx = ox + (v & (GX - 1)), gy = oy + ((v / GX) & (GY - 1)), gz = oz + v / (GX * GY);
        const int32_t c = cells_tile[v];
        const bool valid = gx < d.nx && gy < d.ny && gz < d.nz && c >= 0 && c < max_sites;
        const unsigned mm = __match_any_sync(0xffffffffu, valid ? c : -1);
        const int leader = __ffs(mm) - 1;
        int h = 0;
        if (valid && lane == leader) {
            h = (int)(((uint32_t)c * 2654435761u) >> (32 - 10));
            for (int probe = 0; probe < kHashN; ++probe) {
                const int old = atomicCAS(&S.tab[h], -1, c);
                if (old == -1 || old == c) break;
                h = (h + 1) & (kHashN - 1);
            }
        }
        h = __shfl_sync(0xffffffffu, h, leader);
        S.vt[v] = valid ? (int16_t)h : (int16_t)-1;
        val[r] = valid;
    }
    named_bar_sync(1, kCT);
    {
        // occupied table entries -> dense slots (kHashN / kCT entries per thread); clear the
        // per-slot counts on the way
        constexpr int E = kHashN / kCT;
        int f = 0;
#pragma unroll
        for (int q = 0; q < E; ++q) f += S.tab[tid * E + q] != -1;
        for (int i = tid; i <= GV; i += kCT) S.off[i] = 0;
        int e0, e1, t0, t1;
        consumer_scan2(S, 0, f, 0, e0, e1, t0, t1);
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int h = tid * E + q;
            const int c = S.tab[h];
            if (c != -1) {
                S.tslot[h] = (int16_t)e0;
                S.cellOf[e0] = c;
                ++e0;
            }
        }
        if (tid == 0) S.nslots = t0;
    }
    named_bar_sync(1, kCT);
    // the tile's shifts (site values of its cells): loads issued now, stored after the scatter,
    // so their latency hides behind the remaining phases
    constexpr int kShPT = kShiftSlots * kG / kCT;
    float shv[kShPT];
    {
        const int nsh = S.nslots < kShiftSlots ? S.nslots : kShiftSlots;
#pragma unroll
        for (int r = 0; r < kShPT; ++r) {
            const int i = tid + r * kCT, sl2 = i / kG, jj = i % kG;
            shv[r] = (sl2 < nsh && jj < G) ? __ldg(shift_tab + (int64_t)S.cellOf[sl2] * m + j0 + jj) : 0.0f;
        }
    }
    int sl[kVPT];
#pragma unroll
    for (int r = 0; r < kVPT; ++r) {
        const int v = tid + r * kCT;
        const int s = val[r] ? (int)S.tslot[S.vt[v]] : -1;
        sl[r] = s;
        const unsigned mm = __match_any_sync(0xffffffffu, s);
        if (s >= 0 && lane == __ffs(mm) - 1) atomicAdd(&S.off[s], __popc(mm));
    }
    for (int i = tid; i < kHashN; i += kCT) S.tab[i] = -1;  // empty again for the next brick
    named_bar_sync(1, kCT);
    {
        const int ns = S.nslots;
        int a[2], c[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int i = 2 * tid + r;
            a[r] = i < ns ? S.off[i] : 0;
            c[r] = (a[r] + kChunk - 1) / kChunk;
        }
        int ea, ec, ta, tc;
        consumer_scan2(S, 1, a[0] + a[1], c[0] + c[1], ea, ec, ta, tc);
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int i = 2 * tid + r;
            if (i < ns) {
                S.off[i] = ea; S.cur[i] = ea; S.cho[i] = ec;
                atomicAdd(&acc.cnt[S.cellOf[i]], (unsigned long long)a[r]);
            }
            ea += a[r];
            ec += c[r];
        }
        if (tid == 0) {
            S.off[ns] = ta;
            S.cho[ns] = tc;
            S.nchunks = tc;
        }
    }
    named_bar_sync(1, kCT);
#pragma unroll
    for (int r = 0; r < kVPT; ++r) {
        const int v = tid + r * kCT;
        const int s = sl[r];
        const unsigned mm = __match_any_sync(0xffffffffu, s);
        const int leader = __ffs(mm) - 1;
        int base = 0;
        if (s >= 0 && lane == leader) base = atomicAdd(&S.cur[s], __popc(mm));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (s >= 0) S.sorted[base + __popc(mm & lanemask_lt())] = (uint16_t)v;
    }
#pragma unroll
    for (int r = 0; r < kShPT; ++r) (&S.shift[0][0])[tid + r * kCT] = shv[r];
    named_bar_sync(1, kCT);
}

// the shifts of a later pass over the same brick (the sort ran on its first pass)
__device__ void load_shifts(AggSmem &S, const float *__restrict__ shift_tab, int m, int j0, int G) {
    const int tid = threadIdx.x;
    const int nsh = S.nslots < kShiftSlots ? S.nslots : kShiftSlots;
    for (int i = tid; i < kShiftSlots * kG; i += kCT) {
        const int sl2 = i / kG, jj = i % kG;
        (&S.shift[0][0])[i] = (sl2 < nsh && jj < G) ? __ldg(shift_tab + (int64_t)S.cellOf[sl2] * m + j0 + jj) : 0.0f;
    }
    named_bar_sync(1, kCT);
}

// shift of every (site, variable): the variable at the site voxel
__global__ void shift_table_kernel(const __grid_constant__ AggParams p, const int32_t *__restrict__ site_pos,
                                   const int32_t *n_sites_dev, int32_t max_sites, float *shift) {
    const int32_t ns = min(*n_sites_dev, max_sites);
    const int64_t total = (int64_t)ns * p.m;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / p.m;
        const int j = (int)(i - c * p.m);
        shift[i] = __ldg(p.aux[j] + site_pos[c]);
    }
}

template <int kLoad>
__global__ void __launch_bounds__(kAggBlock, 2) aggregate_kernel(const int32_t *__restrict__ cell, Dims d,
                                                                 const __grid_constant__ AggParams p,
                                                                 const __grid_constant__ AggMaps maps,
                                                                 const float *__restrict__ lo,
                                                                 const float *__restrict__ scale,
                                                                 const float *__restrict__ shift_tab,
                                                                 int32_t max_sites, AggAcc acc, uint32_t *hist,
                                                                 int32_t *status) {
    extern __shared__ __align__(16) unsigned char agg_smem_raw[];
    // align in the shared address space (pointer arithmetic keeps the accesses shared-memory
    // instructions; a round trip through an integer would turn them into generic ones)
    const uint32_t raw_addr = smem_u32(agg_smem_raw);
    AggSmem &S = *reinterpret_cast<AggSmem *>(agg_smem_raw + (((raw_addr + 1023u) & ~1023u) - raw_addr));
    constexpr bool kTma = kLoad != kLoadPlain;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nbx = (d.nx + GX - 1) / GX, nby = (d.ny + GY - 1) / GY, nbz = (d.nz + GZ - 1) / GZ;
    const int64_t nbricks = (int64_t)nbx * nby * nbz;
    const int m = p.m, B = p.n_bins;
    const int npass = m > 0 ? (m + kG - 1) / kG : 1;
    const RunMap runs(nbricks);
    const int64_t ntiles = runs.my_bricks() * npass;
    if (tid == 0) {
        mbar_init(&S.full[0], 1);
        mbar_init(&S.full[1], 1);
        mbar_init(&S.empty[0], kCW);
        mbar_init(&S.empty[1], kCW);
        fence_mbar_init();
    }
    for (int i = tid; i < kCW * 16 * 32; i += blockDim.x) (&S.hist[0][0][0])[i] = 0u;
    for (int i = tid; i < kHashN; i += blockDim.x) S.tab[i] = -1;
    __syncthreads();

    if (warp == kCW) {
        // ---------------- producer warp.  A thread keeps about one tensor copy in flight at a
        // time, so the boxes of a tile are spread over lanes: lane 0 arms the stage's barrier with
        // the tile's bytes, then one lane per box issues it (stage 1 starts at lane 16, so the two
        // stages' copies are in flight together).  Stacked variables go four per 4-D box.
        if (kTma) {
            constexpr int kVarsPerBox = kLoad == kLoadTmaStack ? kStackBox : 1;
            int64_t t = 0;
            bool alive = true;
            for (; t < ntiles; ++t) {
                const int st = (int)(t & 1);
                const uint32_t ph = (uint32_t)(t >> 1) & 1u;
                int ok = 1;
                if (lane == 0) ok = mbar_wait(&S.empty[st], ph ^ 1u, kWaitNs) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) set_status(status, LSRVT_ERR_TIMEOUT);
                    alive = false;
                    break;
                }
                const int64_t brick = runs.brick(t / npass);
                const int pass = (int)(t % npass);
                const int j0 = pass * kG, G = m - j0 < kG ? m - j0 : kG;
                const int ox = (int)(brick % nbx) * GX, oy = (int)((brick / nbx) % nby) * GY,
                          oz = (int)(brick / ((int64_t)nbx * nby)) * GZ;
                const int nvbox = G > 0 ? (G + kVarsPerBox - 1) / kVarsPerBox : 0;
                const uint32_t bytes = (uint32_t)nvbox * kVarsPerBox * GV * 4u + (pass == 0 ? GV * 4u : 0u);
                if (lane == 0) mbar_arrive_expect_tx(&S.full[st], bytes);
                __syncwarp();
                const int li = (lane - 16 * st) & 31;  // this lane's box of the tile: 0 = cells, 1..16 = variables
                if (li == 0 && pass == 0) tma_load_3d(S.cells[st], &maps.cell, ox, oy, oz, &S.full[st]);
                if (li >= 1 && li <= nvbox) {
                    const int jj = (li - 1) * kVarsPerBox;
                    if (kLoad == kLoadTmaStack) tma_load_4d(S.vars[st][jj], &maps.stack, ox, oy, oz, j0 + jj, &S.full[st]);
                    else tma_load_3d(S.vars[st][jj], &maps.var[j0 + jj], ox, oy, oz, &S.full[st]);
                }
            }
            (void)alive;
            // never leave with copies in flight: wait (bounded) for the last tile of each stage
            if (lane == 0)
                for (int64_t u = t - 2 < 0 ? 0 : t - 2; u < t; ++u)
                    mbar_wait(&S.full[u & 1], (uint32_t)(u >> 1) & 1u, kWaitNs);
        }
        return;
    }

    // ---------------- consumers
    const int j = lane & 15, hh = lane >> 4;
    uint32_t *hw = &S.hist[warp][0][lane];  // this lane's 16 words, stride 32
    const bool lane_hist = B > 0 && B <= kLaneBins;
    const float Bm1 = (float)(B > 0 ? B - 1 : 0);
    // Accumulator state, carried from brick to brick of a run while this warp stays in the same
    // cell (one variable tile per brick): a cell that spans many bricks is flushed once per run.
    int cur_cell = -1, kacc = 0;
    bool act = false;
    int jv = 0;
    float nsh = 0.0f;
    // two independent float-float accumulator sets (even / odd steps) for instruction-level
    // parallelism
    float h1[2] = {0.0f, 0.0f}, l1[2] = {0.0f, 0.0f}, h2[2] = {0.0f, 0.0f}, l2[2] = {0.0f, 0.0f};
    // second level: normalised float-float sums (accurate double-word additions), FP64 only
    // once per flush
    float H1 = 0.0f, L1 = 0.0f, H2 = 0.0f, L2 = 0.0f;
    float mn = __int_as_float(0x7f800000), mx = -__int_as_float(0x7f800000);
    int64_t cj = 0;
    auto fold = [&]() {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            float a, b;
            two_sum(h1[u], l1[u], a, b);  // normalise the first-level pair
            dw_add(H1, L1, a, b);
            two_sum(h2[u], l2[u], a, b);
            dw_add(H2, L2, a, b);
            h1[u] = l1[u] = h2[u] = l2[u] = 0.0f;
        }
        kacc = 0;
    };
    auto flush = [&]() {
        fold();
        dw_add(H1, L1, __shfl_down_sync(0xffffffffu, H1, 16), __shfl_down_sync(0xffffffffu, L1, 16));
        dw_add(H2, L2, __shfl_down_sync(0xffffffffu, H2, 16), __shfl_down_sync(0xffffffffu, L2, 16));
        mn = fminf(mn, __shfl_down_sync(0xffffffffu, mn, 16));
        mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, 16));
        if (hh == 0 && act) {
            const double D1 = (double)H1 + (double)L1, D2 = (double)H2 + (double)L2;
            atomicAdd(&acc.s1[cj], D1);
            atomicAdd(&acc.s2[cj], D2);
            atomicMin(&acc.vmin[cj], float_to_ordered(mn));
            atomicMax(&acc.vmax[cj], float_to_ordered(mx));
            if (!isfinite(D1) || !isfinite(D2)) set_status(status, LSRVT_ERR_NONFINITE);
        }
        if (lane_hist) {
            const int words = B < 16 ? B : 16;
            for (int w2 = 0; w2 < words; ++w2) {
                const uint32_t own = hw[w2 * 32];
                const uint32_t tot = own + __shfl_down_sync(0xffffffffu, own, 16);
                hw[w2 * 32] = 0u;
                if (hh == 0 && act) {
                    const uint32_t c0 = tot & 0xFFFFu, c1 = tot >> 16;
                    if (c0) atomicAdd(&hist[cj * B + w2], c0);
                    if (c1) atomicAdd(&hist[cj * B + w2 + 16], c1);
                }
            }
        }
        H1 = L1 = H2 = L2 = 0.0f;
        mn = __int_as_float(0x7f800000);
        mx = -__int_as_float(0x7f800000);
        cur_cell = -1;
    };
    float loj = 0.0f, scj = 0.0f;
    auto acc_one = [&](const float x, int u) {
        mn = fminf(mn, x);
        mx = fmaxf(mx, x);
        float dh, dl, s_, e_;
        two_sum(x, nsh, dh, dl);  // x - c = dh + dl exactly
        two_sum(h1[u], dh, s_, e_);
        h1[u] = s_;
        l1[u] = __fadd_rn(l1[u], __fadd_rn(e_, dl));
        const float pp = __fmul_rn(dh, dh);
        const float corr = __fmaf_rn(__fadd_rn(dh, dh), dl, __fmaf_rn(dh, dh, -pp));  // (dh+dl)^2 - pp
        two_sum(h2[u], pp, s_, e_);
        h2[u] = s_;
        l2[u] = __fadd_rn(l2[u], __fadd_rn(e_, corr));
        if (B) {
            float tt = __fmul_rn(__fsub_rn(x, loj), scj);
            tt = fminf(fmaxf(tt, 0.0f), Bm1);  // NaN and t <= 0 -> bin 0, t >= B -> B - 1
            // x + 2^23 rounded toward zero is 2^23 + floor(x) for 0 <= x < 2^23: its low
            // mantissa bits are the bin
            const uint32_t bits = __float_as_uint(__fadd_rz(tt, 8388608.0f));
            // the lane's own words: a reduction with no result keeps the steps independent
            if (lane_hist) atomicAdd(hw + ((bits & 15u) << 5), 1u << (bits & 16u));
            else atomicAdd(&hist[cj * B + (bits - 0x4B000000u)], 1u);
        }
    };
    for (int64_t t = 0; t < ntiles; ++t) {
        const int st = kTma ? (int)(t & 1) : 0;
        const int64_t bi = t / npass;
        const int64_t brick = runs.brick(bi);
        const int pass = (int)(t % npass);
        const int j0 = pass * kG, G = m - j0 < kG ? m - j0 : kG;
        const int ox = (int)(brick % nbx) * GX, oy = (int)((brick / nbx) % nby) * GY,
                  oz = (int)(brick / ((int64_t)nbx * nby)) * GZ;
        act = j < G;
        jv = j0 + (act ? j : 0);
        loj = (B && act) ? lo[jv] : 0.0f;  // issued before the wait
        scj = (B && act) ? scale[jv] : 0.0f;
        bool ok = true;
        if (kTma) {
            ok = mbar_wait(&S.full[st], (uint32_t)(t >> 1) & 1u, kWaitNs);
            if (!ok && lane == 0) set_status(status, LSRVT_ERR_TIMEOUT);
        } else {
            named_bar_sync(1, kCT);  // every warp is done with the previous tile
            const int nload = (pass == 0 ? GV : 0) + G * GV;
            for (int i = tid; i < nload; i += kCT) {
                const bool is_cell = pass == 0 && i < GV;
                const int k = is_cell ? i : i - (pass == 0 ? GV : 0);
                const int v = k & (GV - 1), jj = k / GV;
                const int gx = ox + (v & (GX - 1)), gy = oy + ((v / GX) & (GY - 1)), gz = oz + v / (GX * GY);
                const bool inb = gx < d.nx && gy < d.ny && gz < d.nz;
                const int64_t g = gx + (int64_t)d.nx * (gy + (int64_t)d.ny * gz);
                if (is_cell) S.cells[0][v] = inb ? __ldcs(cell + g) : -1;
                else S.vars[0][jj][v] = inb ? __ldcs(p.aux[j0 + jj] + g) : 0.0f;
            }
        }
        // a timed-out wait anywhere ends every consumer warp at the same point; the barrier also
        // orders this tile's sort after the previous tile's reads of the sort data
        if (named_bar_or(1, kCT, !ok)) break;
        if (pass == 0) sort_brick(S, S.cells[st], d, ox, oy, oz, max_sites, acc, shift_tab, m, j0, G);
        else load_shifts(S, shift_tab, m, j0, G);
        // ---- this warp's share of the chunks, in order
        const int ns = S.nslots, T = S.nchunks;
        const int q0 = (int)((int64_t)warp * T / kCW), q1 = (int)((int64_t)(warp + 1) * T / kCW);
        const float *xt = S.vars[st][j];
        int s = 0;
        for (int q = q0; q < q1; ++q) {
            while (s + 1 < ns && S.cho[s + 1] <= q) ++s;  // slot of chunk q (chunks are in slot order)
            const int c = S.cellOf[s];
            if (c != cur_cell) {
                if (cur_cell >= 0) flush();
                cur_cell = c;
                cj = (int64_t)c * m + jv;
                nsh = !act ? 0.0f : (s < kShiftSlots ? -S.shift[s][j] : -__ldg(shift_tab + cj));
            }
            const int p0 = S.off[s] + (q - S.cho[s]) * kChunk;
            const int pe = S.off[s + 1] < p0 + kChunk ? S.off[s + 1] : p0 + kChunk;
            const int L = pe - p0, Le = L & ~1;
            if (act && Le) {
                // lane (j, h) takes the chunk positions of parity h, starting at 2j + h (mod the
                // even length), so the 32 lanes read 32 different banks; every lane makes Le / 2
                // steps, so the warp stays converged
                int o = 2 * j + hh;
                while (o >= Le) o -= Le;
                const uint16_t *sp = S.sorted + p0;
                const int n2 = Le >> 1;
                int k = 0;
                for (; k + 1 < n2; k += 2) {
                    int ob = o + 2;
                    ob = ob >= Le ? ob - Le : ob;
                    const float xa = xt[sp[o]], xb = xt[sp[ob]];
                    acc_one(xa, 0);
                    acc_one(xb, 1);
                    o = ob + 2;
                    o = o >= Le ? o - Le : o;
                }
                if (k < n2) acc_one(xt[sp[o]], 0);
            }
            if (act && (L & 1) && hh == 0) acc_one(xt[S.sorted[pe - 1]], 1);
            kacc += (Le >> 1) + 1;
            if (kacc > 34) fold();  // at most 51 float-float additions before a fold
        }
        // flush at the end of a run, and after every tile when the variables come in several
        // tiles per brick (the next tile holds other variables)
        const bool run_end = npass > 1 || bi % kRun == kRun - 1 || t + 1 == ntiles;
        if (run_end && cur_cell >= 0) flush();
        __syncwarp();
        if (kTma && lane == 0) mbar_arrive(&S.empty[st]);
    }
}

// Clears the accumulators, histograms and co-moments of the live rows only (rows < n_sites):
// the row capacity is a bound chosen by the caller and can exceed the sites by orders of
// magnitude.
__global__ void aggregate_init_kernel(AggAcc acc, const int32_t *n_sites_dev, int32_t max_sites, int32_t m,
                                      int32_t B, int32_t T, lsrvt_stats out) {
    const int32_t ns = min(*n_sites_dev, max_sites);
    const int64_t total = (int64_t)ns * m;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = i0; i < total; i += step) {
        acc.s1[i] = 0.0;
        acc.s2[i] = 0.0;
        acc.vmin[i] = float_to_ordered(__int_as_float(0x7f800000));
        acc.vmax[i] = float_to_ordered(-__int_as_float(0x7f800000));
    }
    for (int64_t i = i0; i < ns; i += step) acc.cnt[i] = 0;
    if (B > 0)
        for (int64_t i = i0; i < total * B; i += step) out.hist[i] = 0u;
    if (T > 0)
        for (int64_t i = i0; i < (int64_t)ns * T; i += step) out.comom[i] = 0.0;
}

__global__ void aggregate_finalize_kernel(AggAcc acc, const int32_t *n_sites_dev, int32_t max_sites, int32_t m,
                                          const __grid_constant__ AggParams p, const int32_t *__restrict__ site_pos,
                                          lsrvt_stats out) {
    int32_t ns = min(*n_sites_dev, max_sites);
    int64_t total = (int64_t)ns * m;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = (int32_t)(i / (m > 0 ? m : 1));
        int32_t j = (int32_t)(i - (int64_t)c * m);
        long long n = (long long)acc.cnt[c];
        double mean = 0.0, m2 = 0.0;
        if (n > 0) {
            double sh = (double)__ldg(p.aux[j] + site_pos[c]);
            double s1 = acc.s1[i], s2 = acc.s2[i];
            mean = sh + s1 / (double)n;
            m2 = s2 - s1 * (s1 / (double)n);
            if (m2 < 0.0) m2 = 0.0;
        }
        out.mean[i] = mean;
        out.m2[i] = m2;
        out.vmin[i] = ordered_to_float(acc.vmin[i]);
        out.vmax[i] = ordered_to_float(acc.vmax[i]);
    }
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ns; c += (int64_t)gridDim.x * blockDim.x)
        out.count[c] = (int64_t)acc.cnt[c];
}

// ------------------------------------------------------------------ co-moments on tcgen05 tensor cores
// C_ij = sum over the cell (x_i - mean_i)(x_j - mean_j), a grouped contraction X_c^T X_c over
// the cells.  The voxels are first ordered by cell (a counting sort with the counts of the
// moments pass), so each cell is contracted by exactly one CTA and its co-moments are written
// once, with no atomics.  A CTA takes groups of kCoGroup consecutive cells from a work counter;
// each cell's voxels are gathered in 16-voxel chunks (the last one zero-padded), centred by
// c = float(mean) of the cell, split d = hi + lo into two BF16 numbers (lo = the float remainder
// rounded to BF16), and staged in the K-major canonical layout of the tensor core: a chunk holds
// 64 rows (32 hi variables, then 32 lo) x 16 voxels as 2 K-cores x 8 row groups of 8 x 16-byte
// core matrices.  One thread issues, per chunk, tcgen05.mma kind::f16 with M = 128 (A = the
// chunk's 64 rows; rows 64..127 read the following bytes and land in accumulator rows nobody
// reads), N = 32 (B = the 32 hi rows), K = 16, FP32 accumulation in the cell's 32-column TMEM
// accumulator; cells longer than a staging round keep accumulating across rounds.  TMEM lanes
// 0..31 then hold hi.hi^T and lanes 32..63 lo.hi^T, so C' = hi.hi^T + lo.hi^T + (lo.hi^T)^T
// (the lo.lo term is below 2^-16 relative); the epilogue removes the centring offset exactly,
// C = C' - n (mean_i - c_i)(mean_j - c_j), and takes the diagonal from the float-float M2 of
// the moments pass.
constexpr int kCovVars = 32;                 // variables the contraction holds
constexpr int kCoThreads = 256;
constexpr int kCoWarps = kCoThreads / 32;
constexpr int kCoChunkBytes = 2048;          // one K-step (16 voxels) of A
constexpr int kCoChunks = 16;                // chunks staged per round
// Bytes past the last chunk the descriptors may touch: an M = 128 read covers 16 row groups and
// 2 K-cores; even with the two strides exchanged it stays below 15 * 1024 + 128 + 128 bytes.
constexpr int kCoSlack = 16384;
constexpr int kCoGroup = 4;                  // cells per group, one 32-column accumulator each
constexpr uint32_t kCoTmemCols = 128;
constexpr uint32_t kCoIdesc = umma_idesc_bf16_f32(128, 32);

struct CoSmem {
    unsigned char a[kCoChunks * kCoChunkBytes + kCoSlack];  // tensor-core operands (first)
    float mean_f[kCoGroup][kCovVars];
    float tr[2][32][33];                     // lo.hi^T blocks for the transposition
    int64_t start[kCoGroup];                 // first sorted position of each cell of the group
    int32_t count[kCoGroup];
    int32_t chunk0[kCoGroup + 1];            // first chunk of each cell of the group
    uint64_t mma_bar;
    uint32_t tmem_base;
    int32_t group;
};
constexpr size_t kCoSmem = sizeof(CoSmem) + 1024;
static_assert(3 * (kCoSmem + 1024) <= 228 * 1024, "three co-moment CTAs must fit one SM");

__device__ __forceinline__ unsigned short bf16_bits(float f) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}

// cell offsets of the voxel order: off[c] = counts of the cells before c (counts of rows
// beyond the live sites are zero)
__global__ void cell_count_kernel(const int64_t *__restrict__ count, const int32_t *n_sites_dev, int32_t max_sites,
                                  int64_t *off) {
    const int32_t ns = min(*n_sites_dev, max_sites);
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= max_sites; c += (int64_t)gridDim.x * blockDim.x)
        off[c] = c < ns ? count[c] : 0;
}

// perm[off[c] + k] = the k-th voxel of cell c (the order inside a cell follows the atomics)
__global__ void cell_scatter_kernel(const int32_t *__restrict__ cell, int64_t n, const int32_t *n_sites_dev,
                                    int32_t max_sites, const int64_t *__restrict__ off, int32_t *cur, int32_t *perm,
                                    int32_t *status) {
    const int32_t ns = min(*n_sites_dev, max_sites);
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = base + (threadIdx.x & 31);
        const int32_t c0 = v < n ? cell[v] : -1;
        const int32_t c = (c0 >= 0 && c0 < ns) ? c0 : -1;
        const unsigned mm = __match_any_sync(0xffffffffu, c);
        const int leader = __ffs(mm) - 1;
        int pos = 0;
        if (c >= 0 && (int)(threadIdx.x & 31) == leader) pos = atomicAdd(&cur[c], __popc(mm));
        pos = __shfl_sync(0xffffffffu, pos, leader);
        if (c >= 0) {
            // the counts come from the moments pass; a position past the cell's range means
            // they do not describe these labels
            const int64_t at = off[c] + pos + __popc(mm & lanemask_lt());
            if (at < off[c + 1]) perm[at] = (int32_t)v;
            else set_status(status, LSRVT_ERR_CAPACITY);
        }
    }
}

__global__ void __launch_bounds__(kCoThreads, 3) covariance_kernel(const int32_t *__restrict__ perm,
                                                                   const int64_t *__restrict__ off,
                                                                   const __grid_constant__ AggParams p,
                                                                   const int64_t *__restrict__ count,
                                                                   const double *__restrict__ mean,
                                                                   const double *__restrict__ m2,
                                                                   const int32_t *n_sites_dev, int32_t max_sites,
                                                                   int32_t *work, double *comom, int32_t *status) {
    extern __shared__ __align__(16) unsigned char co_smem_raw[];
    const uint32_t raw_addr = smem_u32(co_smem_raw);
    CoSmem &S = *reinterpret_cast<CoSmem *>(co_smem_raw + (((raw_addr + 1023u) & ~1023u) - raw_addr));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m = p.m, T = m * (m + 1) / 2;
    const int32_t ns = min(*n_sites_dev, max_sites);
    if (tid == 0) {
        mbar_init(&S.mma_bar, 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&S.tmem_base, kCoTmemCols);
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = S.tmem_base;
    const uint32_t a_base = smem_u32(S.a);
    uint32_t rounds = 0;  // MMA rounds completed (mbarrier phase)
    bool failed = false;
    while (!failed) {
        if (tid == 0) S.group = atomicAdd(work, kCoGroup);
        __syncthreads();
        const int32_t g0 = S.group;
        if (g0 >= ns) break;
        const int nk = ns - g0 < kCoGroup ? ns - g0 : kCoGroup;
        if (tid < nk) {
            const int32_t c = g0 + tid;
            S.start[tid] = off[c];
            S.count[tid] = (int32_t)count[c];
        }
        for (int i = tid; i < nk * kCovVars; i += kCoThreads) {
            const int k = i / kCovVars, j = i % kCovVars;
            S.mean_f[k][j] = j < m ? (float)mean[(int64_t)(g0 + k) * m + j] : 0.0f;
        }
        __syncthreads();
        if (tid == 0) {
            int c0 = 0;
            for (int k = 0; k < nk; ++k) {
                S.chunk0[k] = c0;
                c0 += (S.count[k] + 15) / 16;
            }
            S.chunk0[nk] = c0;
        }
        __syncthreads();
        const int total = S.chunk0[nk];
        for (int r0 = 0; r0 < total && !failed; r0 += kCoChunks) {
            const int nch = total - r0 < kCoChunks ? total - r0 : kCoChunks;
            // stage: thread per position of the round, all variables of that voxel (up to 32
            // independent loads in flight)
            for (int pp = tid; pp < nch * 16; pp += kCoThreads) {
                const int cg = r0 + (pp >> 4), k16 = pp & 15;
                int k = 0;
                while (k + 1 < nk && S.chunk0[k + 1] <= cg) ++k;
                const int q = (cg - S.chunk0[k]) * 16 + k16;
                const bool live = q < S.count[k];
                const int v = live ? __ldg(perm + S.start[k] + q) : 0;
                unsigned char *ck = S.a + (size_t)(pp >> 4) * kCoChunkBytes + (k16 >> 3) * 1024 + (k16 & 7) * 2;
                float xv[kCovVars];
#pragma unroll
                for (int j = 0; j < kCovVars; ++j) xv[j] = (live && j < m) ? __ldg(p.aux[j] + v) : 0.0f;  // all in flight
#pragma unroll
                for (int j = 0; j < kCovVars; ++j) {
                    float dd = 0.0f;
                    if (live && j < m) dd = __fsub_rn(xv[j], S.mean_f[k][j]);
                    const unsigned short h2 = bf16_bits(dd);
                    const unsigned short l2 = bf16_bits(__fsub_rn(dd, __bfloat162float(__ushort_as_bfloat16(h2))));
                    *reinterpret_cast<unsigned short *>(ck + (j >> 3) * 128 + (j & 7) * 16) = h2;
                    *reinterpret_cast<unsigned short *>(ck + ((j + 32) >> 3) * 128 + (j & 7) * 16) = l2;
                }
            }
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after_sync();
                int k = 0;
                for (int lc = 0; lc < nch; ++lc) {
                    const int cg = r0 + lc;
                    while (k + 1 < nk && S.chunk0[k + 1] <= cg) ++k;
                    const uint64_t ad = umma_sdesc(a_base + (uint32_t)lc * kCoChunkBytes, 1024, 128);
                    umma_bf16(tmem + (uint32_t)k * 32, ad, ad, kCoIdesc, cg > S.chunk0[k]);
                }
                umma_commit(&S.mma_bar);
            }
            const bool ok = mbar_wait(&S.mma_bar, rounds & 1u, kWaitNs);
            ++rounds;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    set_status(status, LSRVT_ERR_TIMEOUT);
                    mbar_wait(&S.mma_bar, (rounds - 1) & 1u, kWaitNs);  // the MMAs may still be running
                }
                failed = true;
            }
            tc_fence_after_sync();
        }
        if (failed) break;
        // epilogue: warps 0 / 4 read hi.hi^T (lanes 0..31), warps 1 / 5 lo.hi^T (lanes 32..63);
        // the two warp pairs take alternate cells; each co-moment is written once
        const int pair = warp >> 2, wq = warp & 3;
        if (wq < 2) {
            for (int k = pair; k < nk; k += 2) {
                const int64_t c = g0 + k;
                const int64_t n = S.count[k];
                float v[32];
                if (n > 0) tmem_ld32(tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)k * 32, v);
                if (wq == 1 && n > 0) {
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) S.tr[pair][lane][jj] = v[jj];
                }
                if (pair == 0) named_bar_sync(2, 64); else named_bar_sync(3, 64);
                if (wq == 0 && lane < m) {
                    const int i = lane;
                    const int64_t base = c * T + (int64_t)i * m - (int64_t)i * (i - 1) / 2 - i;
                    const double mi = mean[c * m + i], di = mi - (double)(float)mi;
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) {
                        if (jj < i || jj >= m) continue;
                        double val = 0.0;
                        if (n > 0) {
                            if (jj == i) {
                                val = m2[c * m + i];
                            } else {
                                const double mj = mean[c * m + jj], dj = mj - (double)(float)mj;
                                val = (double)(v[jj] + S.tr[pair][i][jj] + S.tr[pair][jj][i]) - (double)n * di * dj;
                            }
                        }
                        comom[base + jj] = val;
                    }
                }
                if (pair == 0) named_bar_sync(2, 64); else named_bar_sync(3, 64);
            }
        }
        tc_fence_before_sync();
        __syncthreads();
    }
    __syncthreads();
    tc_fence_after_sync();
    if (warp == 0) tmem_dealloc(tmem, kCoTmemCols);
}

// ------------------------------------------------------------------ value ranges
__global__ void range_init_kernel(unsigned *lo_bits, unsigned *hi_bits, int32_t m) {
    int j = threadIdx.x + blockIdx.x * blockDim.x;
    if (j < m) {
        lo_bits[j] = float_to_ordered(__int_as_float(0x7f800000));
        hi_bits[j] = float_to_ordered(-__int_as_float(0x7f800000));
    }
}

// Global min / max of up to 16 variables over the valid voxels (cell >= 0) in one sweep: the
// cell labels are read once, and each thread keeps 16 loads in flight per step.
constexpr int kRangeVars = 16;

__global__ void __launch_bounds__(256) range_kernel(const int32_t *__restrict__ cell, const __grid_constant__ AggParams p,
                                                    int j0, int G, int64_t n, unsigned *lo_bits, unsigned *hi_bits,
                                                    int32_t *status) {
    float mn[kRangeVars], mx[kRangeVars];
#pragma unroll
    for (int jj = 0; jj < kRangeVars; ++jj) {
        mn[jj] = __int_as_float(0x7f800000);
        mx[jj] = -__int_as_float(0x7f800000);
    }
    bool bad = false;
    bool vec = ((uintptr_t)cell & 15) == 0;
    for (int jj = 0; jj < G; ++jj) vec = vec && (((uintptr_t)p.aux[j0 + jj] & 15) == 0);
    const int64_t n4 = vec ? n / 4 : 0;
    const int4 *c4 = (const int4 *)cell;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const int4 c = __ldcs(c4 + i);
        float4 v[kRangeVars];
#pragma unroll
        for (int jj = 0; jj < kRangeVars; ++jj)
            if (jj < G) v[jj] = __ldcs(reinterpret_cast<const float4 *>(p.aux[j0 + jj]) + i);
#pragma unroll
        for (int jj = 0; jj < kRangeVars; ++jj) {
            if (jj >= G) continue;
            const float vv[4] = {v[jj].x, v[jj].y, v[jj].z, v[jj].w};
            const int cc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (cc[k] >= 0) {
                    if (!isfinite(vv[k])) bad = true;
                    else { mn[jj] = fminf(mn[jj], vv[k]); mx[jj] = fmaxf(mx[jj], vv[k]); }
                }
        }
    }
    for (int64_t i = n4 * 4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (cell[i] < 0) continue;
#pragma unroll
        for (int jj = 0; jj < kRangeVars; ++jj) {
            if (jj >= G) continue;
            const float v = p.aux[j0 + jj][i];
            if (!isfinite(v)) bad = true;
            else { mn[jj] = fminf(mn[jj], v); mx[jj] = fmaxf(mx[jj], v); }
        }
    }
#pragma unroll
    for (int jj = 0; jj < kRangeVars; ++jj) {
        if (jj >= G) continue;
        float a = mn[jj], b = mx[jj];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(lo_bits + j0 + jj, float_to_ordered(a));
            atomicMax(hi_bits + j0 + jj, float_to_ordered(b));
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) set_status(status, LSRVT_ERR_NONFINITE);
}

__global__ void range_finalize_kernel(float *lo, float *scale, int32_t m, int32_t n_bins) {
    int j = threadIdx.x + blockIdx.x * blockDim.x;
    if (j >= m) return;
    float a = ordered_to_float(__float_as_uint(lo[j]));
    float b = ordered_to_float(__float_as_uint(scale[j]));
    if (a > b) { a = 0.0f; b = 0.0f; }
    float wdt = __fsub_rn(b, a);
    lo[j] = a;
    scale[j] = wdt > 0.0f ? __fdiv_rn((float)n_bins, wdt) : 0.0f;
}

struct AggWs {
    AggAcc acc;
    float *shift;     // [max_sites][m]: the variable at each site voxel
    int32_t *perm;    // [N]: voxels ordered by cell (co-moments)
    int64_t *off;     // [max_sites + 1]: first position of each cell in perm
    int32_t *cur;     // [max_sites]: scatter cursors
    int32_t *work;    // co-moment work counter
    void *scan;       // scan temporaries
};

AggWs carve_agg(void *ws, size_t bytes, Dims d, int32_t max_sites, int32_t m, size_t *need) {
    Carver c(ws, bytes);
    AggWs w;
    int64_t sm = (int64_t)max_sites * (m > 0 ? m : 1);
    w.acc.s1 = c.take<double>(sm);
    w.acc.s2 = c.take<double>(sm);
    w.acc.vmin = c.take<unsigned>(sm);
    w.acc.vmax = c.take<unsigned>(sm);
    w.acc.cnt = c.take<unsigned long long>(max_sites > 0 ? max_sites : 1);
    w.shift = c.take<float>(sm);
    w.perm = c.take<int32_t>(d.n());
    w.off = c.take<int64_t>((int64_t)max_sites + 1);
    w.cur = c.take<int32_t>(max_sites > 0 ? max_sites : 1);
    w.work = c.take<int32_t>(1);
    w.scan = c.take<char>(scan_temp_bytes((int64_t)max_sites + 1));
    *need = c.used;
    return w;
}

}  // namespace

size_t aggregate_workspace(Dims d, int32_t max_sites, int32_t m) {
    size_t need;
    carve_agg(nullptr, 0, d, max_sites, m, &need);
    return need;
}

}  // namespace lsrvt

using namespace lsrvt;

extern "C" lsrvt_status lsrvt_aux_range(const int32_t *cell, const float *const *aux_host, int32_t n_aux,
                                        lsrvt_dims dd, int32_t n_bins, float *lo_dev, float *scale_dev,
                                        int32_t *status_dev, void *stream) {
    if (!dims_ok(dd) || !cell || n_aux < 0 || n_aux > 64 || n_bins < 0 || n_bins > kMaxBins ||
        (n_aux > 0 && (!aux_host || !lo_dev || !scale_dev)))
        return LSRVT_ERR_INVALID_ARG;
    for (int j = 0; j < n_aux; ++j)
        if (!aux_host[j]) return LSRVT_ERR_INVALID_ARG;
    if (n_aux == 0) return LSRVT_OK;
    cudaStream_t s = as_stream(stream);
    int64_t n = (int64_t)dd.nx * dd.ny * dd.nz;
    AggParams p;
    for (int j = 0; j < 64; ++j) p.aux[j] = j < n_aux ? aux_host[j] : nullptr;
    p.m = n_aux;
    p.n_bins = n_bins;
    p.flags = 0;
    range_init_kernel<<<1, 64, 0, s>>>((unsigned *)lo_dev, (unsigned *)scale_dev, n_aux);
    for (int j0 = 0; j0 < n_aux; j0 += kRangeVars)
        range_kernel<<<grid_for(n / 4 + 1, 256, kSMs * 4), 256, 0, s>>>(
            cell, p, j0, n_aux - j0 < kRangeVars ? n_aux - j0 : kRangeVars, n, (unsigned *)lo_dev,
            (unsigned *)scale_dev, status_dev);
    range_finalize_kernel<<<1, 64, 0, s>>>(lo_dev, scale_dev, n_aux, n_bins);
    return launch_status();
}

extern "C" lsrvt_status lsrvt_aggregate(const int32_t *cell, const float *const *aux_host, int32_t n_aux,
                                        lsrvt_dims dd, const float *lo_dev, const float *scale_dev, int32_t n_bins,
                                        uint32_t flags, const int32_t *site_pos, const int32_t *n_sites_dev,
                                        int32_t max_sites, lsrvt_stats out, void *ws, size_t ws_bytes,
                                        int32_t *status_dev, void *stream) {
    bool want_hist = (flags & LSRVT_STATS_HIST) && n_bins > 0;
    bool want_cov = (flags & LSRVT_STATS_COV) != 0;
    if (!dims_ok(dd) || !cell || n_aux < 0 || n_aux > 64 || n_bins < 0 || n_bins > kMaxBins || !site_pos ||
        !n_sites_dev || max_sites < 0 || !out.count || (n_aux > 0 && (!aux_host || !out.mean || !out.m2 ||
                                                                       !out.vmin || !out.vmax)) ||
        (want_hist && n_aux > 0 && (!out.hist || !lo_dev || !scale_dev)) || (want_cov && n_aux > 0 && !out.comom))
        return LSRVT_ERR_INVALID_ARG;
    if (want_cov && n_aux > kCovVars) return LSRVT_ERR_INVALID_ARG;  // tensor-core path holds up to 32 variables
    AggParams p;
    for (int j = 0; j < 64; ++j) p.aux[j] = nullptr;
    for (int j = 0; j < n_aux; ++j) {
        if (!aux_host[j]) return LSRVT_ERR_INVALID_ARG;
        p.aux[j] = aux_host[j];
    }
    p.m = n_aux;
    p.n_bins = want_hist ? n_bins : 0;
    p.flags = flags;
    size_t need;
    AggWs w = carve_agg(ws, ws_bytes, Dims{dd.nx, dd.ny, dd.nz}, max_sites, n_aux, &need);
    size_t cov_need = 0;
    if (!ws || ws_bytes < need + cov_need || ((uintptr_t)ws & 255)) return LSRVT_ERR_WORKSPACE;
    cudaStream_t s = as_stream(stream);
    Dims d{dd.nx, dd.ny, dd.nz};
    aggregate_init_kernel<<<kSMs * 8, 256, 0, s>>>(w.acc, n_sites_dev, max_sites, n_aux,
                                                   (want_hist && n_aux > 0) ? n_bins : 0,
                                                   0, out);  // co-moments are written whole, no clearing
    {
        // TMA tile loads when every array can be described by a tensor map (row pitch a
        // multiple of 16 bytes, 16-byte aligned bases); otherwise plain-load staging
        AggMaps maps;  // encoded per call on the host stack; copied into the launch parameters
        // TMA tile loads when every array can be described by a tensor map (row pitch a
        // multiple of 16 bytes, 16-byte aligned bases): one 4-D box for all variables when they
        // are stacked at a constant pitch, else one box per variable; otherwise plain loads
        int mode = encode_volume_map(&maps.cell, cell, CU_TENSOR_MAP_DATA_TYPE_INT32, 4, d.nx, d.ny, d.nz, GX, GY, GZ)
                       ? kLoadTma
                       : kLoadPlain;
        if (mode == kLoadTma && n_aux > 0) {
            const int64_t pitch = n_aux > 1 ? (const char *)aux_host[1] - (const char *)aux_host[0] : d.n() * 4;
            bool stacked = pitch >= d.n() * 4;
            for (int j = 1; j < n_aux && stacked; ++j)
                stacked = (const char *)aux_host[j] - (const char *)aux_host[0] == (int64_t)j * pitch;
            if (stacked && encode_stack_map(&maps.stack, aux_host[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, d.nx, d.ny,
                                            d.nz, n_aux, pitch, GX, GY, GZ, kStackBox)) {
                mode = kLoadTmaStack;
            } else {
                for (int j = 0; j < n_aux && mode == kLoadTma; ++j)
                    if (!encode_volume_map(&maps.var[j], aux_host[j], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, d.nx, d.ny,
                                           d.nz, GX, GY, GZ))
                        mode = kLoadPlain;
            }
        }
        const int64_t nbricks = (int64_t)((d.nx + GX - 1) / GX) * ((d.ny + GY - 1) / GY) * ((d.nz + GZ - 1) / GZ);
        const int nsm = stream_sms(s);  // this stream's share of the SMs
        if (n_aux > 0)
            shift_table_kernel<<<grid_for((int64_t)max_sites * n_aux, 256, kSMs * 4), 256, 0, s>>>(
                p, site_pos, n_sites_dev, max_sites, w.shift);
        auto launch = [&](auto kern) {
            // two CTAs per SM: one CTA's sort and barriers overlap the other's arithmetic, which
            // needs the largest shared-memory carveout
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAggSmem);
            cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            int occ = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kAggBlock, kAggSmem);
            if (occ < 1) occ = 1;
            const int64_t nruns = (nbricks + kRun - 1) / kRun;
            const int grid = (int)(nruns < (int64_t)nsm * occ ? nruns : (int64_t)nsm * occ);
            kern<<<grid, kAggBlock, kAggSmem, s>>>(cell, d, p, maps, lo_dev, scale_dev, w.shift, max_sites, w.acc,
                                                   out.hist, status_dev);
        };
        if (mode == kLoadTmaStack) launch(aggregate_kernel<kLoadTmaStack>);
        else if (mode == kLoadTma) launch(aggregate_kernel<kLoadTma>);
        else launch(aggregate_kernel<kLoadPlain>);
    }
    aggregate_finalize_kernel<<<kSMs * 8, 256, 0, s>>>(
        w.acc, n_sites_dev, max_sites, n_aux, p, site_pos, out);
    if (want_cov && n_aux > 0) {
        // voxels ordered by cell, then one CTA per group of cells
        const int64_t n = d.n();
        cell_count_kernel<<<grid_for((int64_t)max_sites + 1, 256, kSMs * 4), 256, 0, s>>>(out.count, n_sites_dev,
                                                                                           max_sites, w.off);
        exclusive_scan_i64(w.off, (int64_t)max_sites + 1, nullptr, w.scan, s);
        cudaMemsetAsync(w.cur, 0, sizeof(int32_t) * (size_t)(max_sites > 0 ? max_sites : 1), s);
        cudaMemsetAsync(w.work, 0, sizeof(int32_t), s);
        cell_scatter_kernel<<<grid_for(n, 256, kSMs * 8), 256, 0, s>>>(cell, n, n_sites_dev, max_sites, w.off, w.cur,
                                                                        w.perm, status_dev);
        cudaFuncSetAttribute(covariance_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCoSmem);
        cudaFuncSetAttribute(covariance_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        // three CTAs per SM (shared memory, registers and barriers allow it; 3 x 128 TMEM columns
        // fit an SM's 512), set directly: the occupancy query reports one for this kernel.  The
        // CTAs take cell groups from a work counter, so a CTA that does not find room simply
        // starts later.
        const int occ = 3;
        const int nsm2 = stream_sms(s);
        covariance_kernel<<<nsm2 * occ, kCoThreads, kCoSmem, s>>>(w.perm, w.off, p, out.count, out.mean, out.m2,
                                                                   n_sites_dev, max_sites, w.work, out.comom,
                                                                   status_dev);
    }
    return launch_status();
}
