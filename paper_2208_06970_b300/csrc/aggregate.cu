// aggregate.cu -- per-cell statistics of the auxiliary variables (Sec. 3.3 "Aggregation";
// introduction: statistical aggregation within the segments of the tessellation).
//
// Per cell s and variable j: count, mean, M2 (population variance M2/n), exact min and
// max, an n_bins histogram, and optionally co-moments (tensor cores, below).
//
// B300 design (statistics sweep), two kernels.  The volume is cut into 32x4x4 bricks (512
// voxels, rows of 128 bytes).  (1) A grouping pass orders each brick's valid voxels by cell (a
// counting sort: shared hash of the brick's cell ids -> dense slots -> runs), counts every
// cell's voxels, and writes the order (512 local indices, 1 KB) and a 128-byte record of the
// run starts per brick.  It keeps little shared state, so many bricks are in flight per SM and
// the sort's barriers overlap.  (2) The sweep: a producer warp streams each brick's cell
// labels, its order and record, and up to 16 variables (one 2 KB tile each) into a ring of
// shared-memory tiles with TMA (tensor tile loads and bulk copies, mbarrier completion), so HBM
// reads of the next brick overlap the arithmetic on the current one.  The consumer warps split
// the brick's valid positions evenly and walk them in chunks of at most 32 positions inside one
// run; they never wait for each other, only for the tile's mbarrier.  Inside a warp, lane (j, h)
// owns variable j and every second position of the chunk (h = 0, 1), so one cell's 16
// variables are reduced in parallel and only the two halves of the warp have to be combined
// when the warp's segment of a cell ends.  A lane accumulates x - s and (x - s)^2 (s = the
// variable at the first position of the segment) in float-float (TwoSum / FMA error-free
// transforms) over at most 51 elements, then folds them into a normalised float-float sum by
// accurate double-word additions; at the segment's end the sums move, in FP64, to the cell's
// common shift c (the variable at its site voxel) and go out with one FP64 atomic per moment.
// min / max are exact; the histogram goes to lane-private 16-bit counters in shared memory (no
// bank conflicts, no contention), and a flush visits only the words the segment touched.  A
// finalize pass forms mean = c + S1/n and M2 = S2 - S1^2/n in FP64.  HBM traffic is the
// algorithmic 4 B (cell) + 4 m B (variables) per voxel, plus 4 B (labels) and 2.25 B (order)
// per voxel for the grouping pass and 2.25 B per voxel of order read back.  Volumes whose row
// pitch is not a multiple of 16 bytes (TMA cannot describe them) take the same kernel with
// tiles staged by plain loads.
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
constexpr int kStages = 2;               // tiles in flight per CTA
constexpr int kChunk = 32;               // sorted positions per work chunk
constexpr int kLaneBins = 32;            // lane-private histograms up to 32 bins
constexpr int kStackBox = 4;             // stacked variables per 4-D tensor box (8 KB)
constexpr int kRun = 16;                 // consecutive bricks (along x) a CTA takes at a time
constexpr int kRecRuns = 8;              // runs whose shifts the brick record carries
constexpr int kRecHead = 32;             // record head: run-start mask (16 words), valid voxels, runs
constexpr int kRecWords = kRecHead + kRecRuns * kG;  // + the shifts of the first runs' cells
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s bound on every mbarrier wait

struct AggMaps {
    CUtensorMap cell;
    CUtensorMap stack;    // all variables as one 4-D tensor (when they are stacked at a constant pitch)
    CUtensorMap var[64];  // one 3-D tensor per variable otherwise
};

// how the tiles reach shared memory
enum AggLoad { kLoadPlain = 0, kLoadTma = 1, kLoadTmaStack = 2 };

// The brick grouping: for every brick, its valid voxels ordered by cell (local indices, one
// run per cell) and a record of the run starts.  Written by group_bricks_kernel, read by the
// sweep with bulk copies.
struct BrickOrder {
    uint16_t *perm;  // [nbricks][GV]
    uint32_t *rec;   // [nbricks][kRecWords]: words 0..15 run-start bits, 16 valid voxels, 17 runs, then
                     // the shift (variable at the site voxel) of run r's cell for variable j at 32 + 16 r + j
};

// ---- grouping pass: one warp per brick, no block barriers.  Lane l holds the brick's voxels
// l + 32 r (row r = y + 4 z).  The runs are found one at a time: the cell of the first voxel
// (in index order) not yet placed leads, and every voxel of that cell is placed after the
// previous runs, in index order (a ballot per row and prefix counts).  The work per brick grows
// with its number of cells (about three on average in the flame volumes, 40 % of the bricks a
// single cell), not with the size of a hash table.
constexpr int kGrpWarps = 8;
constexpr int kGrpThreads = kGrpWarps * 32;
constexpr int kRows = GV / 32;

__global__ void __launch_bounds__(kGrpThreads, 6) group_bricks_kernel(const int32_t *__restrict__ cell, Dims d,
                                                                   int32_t max_sites, unsigned long long *cnt,
                                                                   const float *__restrict__ shift_tab, int32_t m,
                                                                   BrickOrder ord) {
    __shared__ __align__(16) uint16_t sorted_s[kGrpWarps][GV];
    __shared__ __align__(16) uint32_t rec_s[kGrpWarps][kRecWords];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    uint16_t *sorted = sorted_s[wl];
    uint32_t *rec = rec_s[wl];
    const int nbx = (d.nx + GX - 1) / GX, nby = (d.ny + GY - 1) / GY, nbz = (d.nz + GZ - 1) / GZ;
    const int64_t nbricks = (int64_t)nbx * nby * nbz;
    const int64_t wstride = (int64_t)gridDim.x * kGrpWarps;
    for (int64_t brick = (int64_t)blockIdx.x * kGrpWarps + wl; brick < nbricks; brick += wstride) {
        const int ox = (int)(brick % nbx) * GX, oy = (int)((brick / nbx) % nby) * GY,
                  oz = (int)(brick / ((int64_t)nbx * nby)) * GZ;
        int32_t cv[kRows];
        uint32_t pend = 0u;  // bit r: voxel (lane, r) valid and not yet placed
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const int gx = ox + lane, gy = oy + (r & (GY - 1)), gz = oz + r / GY;
            const bool inb = gx < d.nx && gy < d.ny && gz < d.nz;
            cv[r] = inb ? __ldg(cell + gx + (int64_t)d.nx * (gy + (int64_t)d.ny * gz)) : -1;
            pend |= (uint32_t)(cv[r] >= 0 && cv[r] < max_sites) << r;
        }
        for (int i = lane; i < kRecWords; i += 32) rec[i] = 0u;
        __syncwarp();
        int base = 0, nruns = 0;
        uint32_t mword = 0u;  // lane w < 16: run-start bits of positions 32 w .. 32 w + 31
        while (true) {
            // the first pending voxel in index order: lowest row with one, then lowest lane
            const unsigned rows = __reduce_or_sync(0xffffffffu, pend);
            if (!rows) break;
            const int rs = __ffs(rows) - 1;
            const int ls = __ffs(__ballot_sync(0xffffffffu, (pend >> rs) & 1u)) - 1;
            int cr = cv[0];
#pragma unroll
            for (int r = 1; r < kRows; ++r) cr = r == rs ? cv[r] : cr;
            const int32_t cur = __shfl_sync(0xffffffffu, cr, ls);
            int pos = base;
            uint32_t hit = 0u;
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                const bool e = ((pend >> r) & 1u) && cv[r] == cur;
                const unsigned bm = __ballot_sync(0xffffffffu, e);
                if (e) sorted[pos + __popc(bm & lanemask_lt())] = (uint16_t)(lane + 32 * r);
                pos += __popc(bm);
                hit |= (uint32_t)e << r;
            }
            pend &= ~hit;
            if (lane == (base >> 5)) mword |= 1u << (base & 31);
            if (lane == 0) atomicAdd(&cnt[cur], (unsigned long long)(pos - base));
            if (nruns < kRecRuns && lane < kG && lane < m)
                rec[kRecHead + nruns * kG + lane] = __float_as_uint(__ldg(shift_tab + (int64_t)cur * m + lane));
            base = pos;
            ++nruns;
        }
        if (lane < 16) rec[lane] = mword;
        if (lane == 0) {
            rec[16] = (uint32_t)base;
            rec[17] = (uint32_t)nruns;
        }
        __syncwarp();
        // positions at and beyond the valid count are never read; the whole 1 KB line is written
        const uint4 *src = reinterpret_cast<const uint4 *>(sorted);
        uint4 *dst = reinterpret_cast<uint4 *>(ord.perm + brick * GV);
        dst[lane] = src[lane];
        dst[lane + 32] = src[lane + 32];
        for (int i = lane; i < kRecWords; i += 32) ord.rec[brick * kRecWords + i] = rec[i];
        __syncwarp();  // the staging is reused by the next brick
    }
}

// ---- the sweep
struct AggTile {
    float vars[kG][GV];          // TMA tiles (128-byte rows)
    int32_t cells[GV];
    uint16_t perm[GV];           // the brick's valid voxels grouped by cell
    uint32_t rec[kRecWords];
};
static_assert(sizeof(AggTile) % 128 == 0, "tiles stay 128-byte aligned");

struct AggSmem {
    AggTile tile[kStages];
    // per warp and lane, 16 words: word w holds bin w (low half) and bin w + 16 (high half); rows
    // padded to 33 words so a flush can read one word of 16 lanes without bank conflicts
    uint32_t hist[kCW][16][33];
    uint64_t full[kStages], empty[kStages];
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

// The sweep.  A producer warp streams each brick's cell labels, its order (from the grouping
// pass) and up to 16 variables into a ring of shared-memory tiles; the consumer warps share
// each brick's valid positions out evenly (no barrier between them: each waits for the tile's
// mbarrier and releases it when done).  A warp walks its positions in chunks of at most 32
// inside one run (one cell).  Lane (j, h) owns variable j and the chunk positions of parity h;
// it accumulates x - c and (x - c)^2, c = the variable at the first position of the warp's
// current segment of the cell, in float-float (TwoSum / FMA error-free transforms), folded
// every <= 51 steps into a normalised float-float sum by accurate double-word additions.  At
// the end of a segment the two halves of the warp are combined and the sums are moved, in FP64,
// to the cell's common shift (the variable at its site voxel) before one FP64 atomic per moment;
// only the histogram words the segment touched are flushed.
enum AggHist { kHistNone = 0, kHistLane = 1, kHistGlobal = 2 };

template <int kLoad, int kHist>
__global__ void __launch_bounds__(kAggBlock, 2) aggregate_kernel(const int32_t *__restrict__ cell, Dims d,
                                                                 const __grid_constant__ AggParams p,
                                                                 const __grid_constant__ AggMaps maps,
                                                                 BrickOrder ord,
                                                                 const float *__restrict__ lo,
                                                                 const float *__restrict__ scale,
                                                                 const float *__restrict__ shift_tab,
                                                                 AggAcc acc, uint32_t *hist, int32_t *status) {
    extern __shared__ __align__(16) unsigned char agg_smem_raw[];
    // align in the shared address space (pointer arithmetic keeps the accesses shared-memory
    // instructions; a round trip through an integer would turn them into generic ones)
    const uint32_t raw_addr = smem_u32(agg_smem_raw);
    AggSmem &S = *reinterpret_cast<AggSmem *>(agg_smem_raw + (((raw_addr + 1023u) & ~1023u) - raw_addr));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nbx = (d.nx + GX - 1) / GX, nby = (d.ny + GY - 1) / GY, nbz = (d.nz + GZ - 1) / GZ;
    const int64_t nbricks = (int64_t)nbx * nby * nbz;
    const int m = p.m, B = p.n_bins;
    const int npass = m > 0 ? (m + kG - 1) / kG : 1;
    const RunMap runs(nbricks);
    const int64_t ntiles = runs.my_bricks() * npass;
    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) {
            mbar_init(&S.full[st], 1);
            mbar_init(&S.empty[st], kCW);
        }
        fence_mbar_init();
    }
    for (int i = tid; i < kCW * 16 * 33; i += blockDim.x) (&S.hist[0][0][0])[i] = 0u;
    __syncthreads();

    if (warp == kCW) {
        // ---------------- producer warp.  A thread keeps about one tensor copy in flight at a
        // time, so the copies of a tile are spread over lanes: lane 0 arms the stage's barrier
        // with the tile's bytes, then one lane per copy issues it (odd stages start at lane 16).
        constexpr int kVarsPerBox = kLoad == kLoadTmaStack ? kStackBox : 1;
        int64_t t = 0;
        for (; t < ntiles; ++t) {
            const int st = (int)(t % kStages);
            const uint32_t ph = (uint32_t)(t / kStages) & 1u;
            int ok = 1;
            if (lane == 0) ok = mbar_wait(&S.empty[st], ph ^ 1u, kWaitNs) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) set_status(status, LSRVT_ERR_TIMEOUT);
                break;
            }
            const int64_t brick = runs.brick(t / npass);
            const int pass = (int)(t % npass);
            const int j0 = pass * kG, G = m - j0 < kG ? m - j0 : kG;
            const int ox = (int)(brick % nbx) * GX, oy = (int)((brick / nbx) % nby) * GY,
                      oz = (int)(brick / ((int64_t)nbx * nby)) * GZ;
            AggTile &T = S.tile[st];
            if (kLoad != kLoadPlain) {
                const int nvbox = G > 0 ? (G + kVarsPerBox - 1) / kVarsPerBox : 0;
                const uint32_t bytes = (uint32_t)nvbox * kVarsPerBox * GV * 4u + GV * 4u + GV * 2u + kRecWords * 4u;
                static_assert(kRecWords * 4 % 16 == 0, "bulk copies move multiples of 16 bytes");
                if (lane == 0) mbar_arrive_expect_tx(&S.full[st], bytes);
                __syncwarp();
                const int li = (lane - 16 * (st & 1)) & 31;  // 0 = cells, 1 = order, 2 = record, 3.. = variables
                if (li == 0) tma_load_3d(T.cells, &maps.cell, ox, oy, oz, &S.full[st]);
                if (li == 1) bulk_load(T.perm, ord.perm + brick * GV, GV * 2u, &S.full[st]);
                if (li == 2) bulk_load(T.rec, ord.rec + brick * kRecWords, kRecWords * 4u, &S.full[st]);
                if (li >= 3 && li < 3 + nvbox) {
                    const int jj = (li - 3) * kVarsPerBox;
                    if (kLoad == kLoadTmaStack) tma_load_4d(T.vars[jj], &maps.stack, ox, oy, oz, j0 + jj, &S.full[st]);
                    else tma_load_3d(T.vars[jj], &maps.var[j0 + jj], ox, oy, oz, &S.full[st]);
                }
            } else {
                // plain loads (arrays TMA cannot describe); the order and record with them
                for (int i = lane; i < GV * (1 + G); i += 32) {
                    const int k = i & (GV - 1), jj = i / GV - 1;
                    const int gx = ox + (k & (GX - 1)), gy = oy + ((k / GX) & (GY - 1)), gz = oz + k / (GX * GY);
                    const bool inb = gx < d.nx && gy < d.ny && gz < d.nz;
                    const int64_t g = gx + (int64_t)d.nx * (gy + (int64_t)d.ny * gz);
                    if (jj < 0) T.cells[k] = inb ? __ldcs(cell + g) : -1;
                    else T.vars[jj][k] = inb ? __ldcs(p.aux[j0 + jj] + g) : 0.0f;
                }
                for (int i = lane; i < GV / 2; i += 32)
                    reinterpret_cast<uint32_t *>(T.perm)[i] = reinterpret_cast<const uint32_t *>(ord.perm + brick * GV)[i];
                for (int i = lane; i < kRecWords; i += 32) T.rec[i] = ord.rec[brick * kRecWords + i];
                __syncwarp();
                if (lane == 0) mbar_arrive(&S.full[st]);
            }
        }
        // never leave with copies in flight: wait (bounded) for the last tile of each stage
        if (lane == 0)
            for (int64_t u = t - kStages < 0 ? 0 : t - kStages; u < t; ++u)
                mbar_wait(&S.full[u % kStages], (uint32_t)(u / kStages) & 1u, kWaitNs);
        return;
    }

    // ---------------- consumers
    const int j = lane & 15, hh = lane >> 4;
    uint32_t *hw = &S.hist[warp][0][lane];  // this lane's 16 words, stride 33
    const float Bm1 = (float)(B > 0 ? B - 1 : 0);
    // Accumulator state, carried from brick to brick of a run while this warp stays in the same
    // cell (one variable tile per brick): a cell that spans many bricks is flushed once per run.
    int cur_cell = -1, kacc = 0;
    int tj0 = 0, tG = 0;               // the current tile's first variable and variable count
    bool act = false;
    int jv = 0;
    float nsh = 0.0f;                  // minus the cell's shift
    uint32_t tmask = 0u;               // histogram words this lane touched in the segment
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
        if (kHist == kHistLane) {
            if (__reduce_or_sync(0xffffffffu, tmask)) {
                // transposed: per variable, lane q takes bin q (word q & 15, half q & 16 of the
                // variable's two lanes) and the warp adds one coalesced row of bins
                __syncwarp();
                const uint32_t *col = &S.hist[warp][lane & 15][0];
                const int shq = lane & 16;
                for (int jj = 0; jj < tG; ++jj) {
                    const uint32_t n_q = ((col[jj] >> shq) & 0xFFFFu) + ((col[jj + 16] >> shq) & 0xFFFFu);
                    if (n_q && lane < B) atomicAdd(&hist[((int64_t)cur_cell * m + tj0 + jj) * B + lane], n_q);
                }
                __syncwarp();
#pragma unroll
                for (int w2 = 0; w2 < 16; ++w2) hw[w2 * 33] = 0u;
                tmask = 0u;
            }
        }
        H1 = L1 = H2 = L2 = 0.0f;
        mn = __int_as_float(0x7f800000);
        mx = -__int_as_float(0x7f800000);
        cur_cell = -1;
    };
    float loj = 0.0f, scj = 0.0f;
    // one step of lane (j, h); inc = 0 makes it neutral (x is then the segment's shift, which adds
    // nothing to the sums and is inside the segment's min / max)
    auto acc_one = [&](const float x, int u, uint32_t inc) {
        mn = fminf(mn, x);
        mx = fmaxf(mx, x);
        float dh, dl, s_, e_;
        two_sum(x, nsh, dh, dl);  // x - s = dh + dl exactly
        two_sum(h1[u], dh, s_, e_);
        h1[u] = s_;
        l1[u] = __fadd_rn(l1[u], __fadd_rn(e_, dl));
        const float pp = __fmul_rn(dh, dh);
        const float corr = __fmaf_rn(__fadd_rn(dh, dh), dl, __fmaf_rn(dh, dh, -pp));  // (dh+dl)^2 - pp
        two_sum(h2[u], pp, s_, e_);
        h2[u] = s_;
        l2[u] = __fadd_rn(l2[u], __fadd_rn(e_, corr));
        if (kHist != kHistNone) {
            float tt = __fmul_rn(__fsub_rn(x, loj), scj);
            tt = fminf(fmaxf(tt, 0.0f), Bm1);  // NaN and t <= 0 -> bin 0, t >= B -> B - 1
            // x + 2^23 rounded toward zero is 2^23 + floor(x) for 0 <= x < 2^23: its low
            // mantissa bits are the bin
            const uint32_t bits = __float_as_uint(__fadd_rz(tt, 8388608.0f));
            if (kHist == kHistLane) {
                // the lane's own words: a reduction with no result keeps the steps independent
                atomicAdd(hw + (bits & 15u) * 33u, inc << (bits & 16u));
                tmask |= inc << (bits & 15u);
            } else if (inc) {
                atomicAdd(&hist[cj * B + (bits - 0x4B000000u)], 1u);
            }
        }
    };
    for (int64_t t = 0; t < ntiles; ++t) {
        const int st = (int)(t % kStages);
        const int64_t bi = t / npass;
        const int pass = (int)(t % npass);
        const int j0 = pass * kG, G = m - j0 < kG ? m - j0 : kG;
        act = j < G;
        jv = j0 + (act ? j : 0);
        tj0 = j0;
        tG = G;
        loj = (B && act) ? lo[jv] : 0.0f;  // issued before the wait
        scj = (B && act) ? scale[jv] : 0.0f;
        if (!mbar_wait(&S.full[st], (uint32_t)(t / kStages) & 1u, kWaitNs)) {
            if (lane == 0) set_status(status, LSRVT_ERR_TIMEOUT);
            break;
        }
        const AggTile &T = S.tile[st];
        const float *xt = T.vars[j];
        const int nv = (int)T.rec[16];
        const uint32_t mw = lane < 16 ? T.rec[lane] : 0u;  // run-start bits, word per lane
        // this warp's share of the brick's valid positions
        const int pe = (int)(((warp + 1) * nv) / kCW);
        int pos = (int)((warp * nv) / kCW);
        while (pos < pe) {
            // end of the run that holds pos: the next run start after it
            int re = nv;
            {
                const int q = pos + 1;
                const int qw = q >> 5;
                const uint32_t mine = lane < qw ? 0u : (lane == qw ? (mw & (0xffffffffu << (q & 31))) : mw);
                const unsigned nz = __ballot_sync(0xffffffffu, mine != 0u);
                if (nz) {
                    const int wl = __ffs(nz) - 1;
                    const uint32_t word = __shfl_sync(0xffffffffu, mine, wl);
                    re = min(nv, wl * 32 + __ffs(word) - 1);
                }
            }
            const int ce = min(min(pe, re), pos + kChunk);
            const int c = T.cells[T.perm[pos]];
            if (c != cur_cell) {
                if (cur_cell >= 0) flush();
                cur_cell = c;
                cj = (int64_t)c * m + jv;
                // the cell's shift: from the brick record for its first runs (the run index is the
                // number of run starts at or before pos, less one), else from the table
                const int pw = pos >> 5;
                const uint32_t upto = lane < pw ? mw : lane == pw ? (mw & ((2u << (pos & 31)) - 1u)) : 0u;
                const int r = __reduce_add_sync(0xffffffffu, (unsigned)__popc(upto)) - 1;
                nsh = !act ? 0.0f
                           : -(r < kRecRuns && pass == 0 ? __uint_as_float(T.rec[kRecHead + r * kG + j])
                                                         : __ldg(shift_tab + cj));
            }
            const int L = ce - pos;
            if (act) {
                // lane (j, h) takes the positions of parity h, starting at index (j * n_h) / 16 of
                // its n_h positions and wrapping, so the 32 lanes read 32 different banks; every
                // lane makes ceil(L / 2) steps, the odd lanes' last one neutral when L is odd
                const int n0 = (L + 1) >> 1, nh = hh ? (L >> 1) : n0;
                const uint16_t *sp = T.perm + pos + hh;
                const float sx = -nsh;
                int i = (j * nh) >> 4;
                int k = 0;
                for (; k + 1 < n0; k += 2) {
                    int ib = i + 1;
                    ib = ib == nh ? 0 : ib;
                    const bool vb = k + 1 < nh;
                    const float xa = xt[sp[2 * i]];
                    const float xb = xt[sp[2 * (vb ? ib : i)]];
                    acc_one(xa, 0, 1u);
                    acc_one(vb ? xb : sx, 1, vb ? 1u : 0u);
                    i = ib + 1;
                    i = i >= nh ? i - nh : i;
                }
                if (k < n0) {
                    const bool va = k < nh;
                    const float xa = xt[va ? sp[2 * i] : T.perm[pos]];
                    acc_one(va ? xa : sx, 0, va ? 1u : 0u);
                }
            }
            kacc += (L + 1) >> 1;
            if (kacc > 34) fold();  // at most 51 float-float additions before a fold
            pos = ce;
        }
        // flush at the end of a run, and after every tile when the variables come in several
        // tiles per brick (the next tile holds other variables)
        const bool run_end = npass > 1 || bi % kRun == kRun - 1 || t + 1 == ntiles;
        if (run_end && cur_cell >= 0) flush();
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[st]);
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
// once, with no atomics.  A CTA takes groups of kCoGroup cells from a work counter, the cells in
// the raster order of their site voxels, so cells that share cache lines (neighbours along x) are
// gathered at about the same time and the lines are read from DRAM once;
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
    float dmean[kCoGroup][kCovVars];         // mean - float(mean): the centring offset, exactly
    float tr[2][32][33];                     // one cell's hi.hi^T and lo.hi^T, read from TMEM
    uint16_t tri[kCovVars * (kCovVars + 1) / 2];  // (row << 8 | column) of each upper-triangle entry
    int64_t start[kCoGroup];                 // first sorted position of each cell of the group
    int32_t cellid[kCoGroup];                // the group's cells
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

// (site voxel, cell) pairs of the live cells, to be sorted into the co-moments' cell order
__global__ void cell_order_keys_kernel(const int32_t *__restrict__ site_pos, const int32_t *n_sites_dev,
                                       int32_t max_sites, uint32_t *key, uint32_t *val) {
    const int32_t ns = min(*n_sites_dev, max_sites);
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ns; c += (int64_t)gridDim.x * blockDim.x) {
        key[c] = (uint32_t)site_pos[c];
        val[c] = (uint32_t)c;
    }
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
                                                                   const uint32_t *__restrict__ order, int32_t *work,
                                                                   double *comom, int32_t *status) {
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
    // the upper triangle in its stored (row-major) order
    for (int i = tid; i < m; i += kCoThreads) {
        const int row0 = i * m - i * (i - 1) / 2;
        for (int jj = i; jj < m; ++jj) S.tri[row0 + jj - i] = (uint16_t)(i << 8 | jj);
    }
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
            const int32_t c = (int32_t)order[g0 + tid];
            S.cellid[tid] = c;
            S.start[tid] = off[c];
            S.count[tid] = (int32_t)count[c];
        }
        for (int i = tid; i < nk * kCovVars; i += kCoThreads) {
            const int k = i / kCovVars, j = i % kCovVars;
            const double mu = j < m ? mean[(int64_t)order[g0 + k] * m + j] : 0.0;
            S.mean_f[k][j] = (float)mu;
            S.dmean[k][j] = (float)(mu - (double)(float)mu);
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
        // epilogue, one cell at a time: warp 0 reads hi.hi^T (TMEM lanes 0..31) and warp 1 lo.hi^T
        // (lanes 32..63) into shared memory; then every thread writes entries of the upper
        // triangle in their stored order (coalesced), C_ij = hi.hi^T + lo.hi^T + (lo.hi^T)^T
        // - n d_i d_j in FP32 (d = the centring offset), the diagonal from the moments' M2
        for (int k = 0; k < nk; ++k) {
            const int64_t c = S.cellid[k];
            const int32_t n = S.count[k];
            if (warp < 2 && n > 0) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)k * 32, v);
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) S.tr[warp][lane][jj] = v[jj];
            }
            __syncthreads();
            for (int t = tid; t < T; t += kCoThreads) {
                const int i = S.tri[t] >> 8, jj = S.tri[t] & 255;
                double val = 0.0;
                if (n > 0)
                    val = i == jj ? m2[c * m + i]
                                  : (double)(S.tr[0][i][jj] + S.tr[1][i][jj] + S.tr[1][jj][i] -
                                             (float)n * S.dmean[k][i] * S.dmean[k][jj]);
                comom[c * T + t] = val;
            }
            __syncthreads();
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
    BrickOrder ord;   // the sweep's per-brick order (same memory as perm)
    int64_t *off;     // [max_sites + 1]: first position of each cell in perm
    int32_t *cur;     // [max_sites]: scatter cursors
    int32_t *work;    // co-moment work counter
    uint32_t *okey, *oval;  // cells by the raster position of their site voxel (co-moment order)
    void *rtemp;      // radix sort temporaries
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
    // the brick order of the sweep and the co-moments' voxel order are never live together
    const int64_t nbricks = (int64_t)((d.nx + GX - 1) / GX) * ((d.ny + GY - 1) / GY) * ((d.nz + GZ - 1) / GZ);
    const int64_t order_bytes = nbricks * (GV * 2 + kRecWords * 4);
    w.perm = (int32_t *)c.take<char>(d.n() * 4 > order_bytes ? d.n() * 4 : order_bytes);
    w.ord.perm = (uint16_t *)w.perm;
    w.ord.rec = (uint32_t *)((char *)w.perm + nbricks * GV * 2);
    w.off = c.take<int64_t>((int64_t)max_sites + 1);
    w.cur = c.take<int32_t>(max_sites > 0 ? max_sites : 1);
    w.work = c.take<int32_t>(1);
    w.okey = c.take<uint32_t>(max_sites > 0 ? max_sites : 1);
    w.oval = c.take<uint32_t>(max_sites > 0 ? max_sites : 1);
    w.rtemp = c.take<char>(radix_temp_bytes(max_sites > 0 ? max_sites : 1));
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
        // every brick's voxels grouped by cell (and the cells' voxel counts), a warp per brick
        const int64_t gblocks = (nbricks + kGrpWarps - 1) / kGrpWarps;  // six CTAs per SM are resident
        group_bricks_kernel<<<(int)(gblocks < (int64_t)nsm * 6 ? gblocks : (int64_t)nsm * 6), kGrpThreads, 0, s>>>(
            cell, d, max_sites, w.acc.cnt, w.shift, n_aux, w.ord);
        auto launch = [&](auto kern) {
            // two CTAs per SM, which needs the largest shared-memory carveout
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAggSmem);
            cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            int occ = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kAggBlock, kAggSmem);
            if (occ < 1) occ = 1;
            const int64_t nruns = (nbricks + kRun - 1) / kRun;
            const int grid = (int)(nruns < (int64_t)nsm * occ ? nruns : (int64_t)nsm * occ);
            kern<<<grid, kAggBlock, kAggSmem, s>>>(cell, d, p, maps, w.ord, lo_dev, scale_dev, w.shift, w.acc,
                                                   out.hist, status_dev);
        };
        const int hm = p.n_bins == 0 ? kHistNone : p.n_bins <= kLaneBins ? kHistLane : kHistGlobal;
        auto launch_h = [&](auto k0, auto k1, auto k2) {
            if (hm == kHistNone) launch(k0);
            else if (hm == kHistLane) launch(k1);
            else launch(k2);
        };
        if (mode == kLoadTmaStack)
            launch_h(aggregate_kernel<kLoadTmaStack, kHistNone>, aggregate_kernel<kLoadTmaStack, kHistLane>,
                     aggregate_kernel<kLoadTmaStack, kHistGlobal>);
        else if (mode == kLoadTma)
            launch_h(aggregate_kernel<kLoadTma, kHistNone>, aggregate_kernel<kLoadTma, kHistLane>,
                     aggregate_kernel<kLoadTma, kHistGlobal>);
        else
            launch_h(aggregate_kernel<kLoadPlain, kHistNone>, aggregate_kernel<kLoadPlain, kHistLane>,
                     aggregate_kernel<kLoadPlain, kHistGlobal>);
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
        cell_order_keys_kernel<<<grid_for(max_sites, 256, kSMs * 4), 256, 0, s>>>(site_pos, n_sites_dev, max_sites,
                                                                                   w.okey, w.oval);
        int bits = 1;
        while (bits < 32 && (int64_t(1) << bits) < n) ++bits;
        radix_sort_pairs(w.okey, w.oval, max_sites, n_sites_dev, bits, w.rtemp, s);
        covariance_kernel<<<nsm2 * occ, kCoThreads, kCoSmem, s>>>(w.perm, w.off, p, out.count, out.mean, out.m2,
                                                                   n_sites_dev, max_sites, w.oval, w.work, out.comom,
                                                                   status_dev);
    }
    return launch_status();
}
