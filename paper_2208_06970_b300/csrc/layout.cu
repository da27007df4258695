// layout.cu -- structured hierarchical data layout of a decomposition (Sec. 3.2 "Data Reduction
// and Structured Data Layout", Fig. hierarchy): the voxels of the kept isobands ordered by
// (band, component, cell) and, inside a cell, by linear index, so that every band, component
// and cell is one contiguous, directly indexable range; the raw variables are extracted in the
// same order next to one coordinate (the linear voxel index) per voxel.
//
// Site ids are grouped by component in ascending order and components by band (the numbering
// of lsrvt_label_components and lsrvt_seed), so ordering by cell id alone is ordering by
// (band, component, cell): a stable sort of the kept voxels by cell.
//
// Design: cells are spatially compact, so a tile of 2048 consecutive voxels holds few distinct
// cells, each as a few runs ("segments") of equal labels.  Instead of sorting voxels, each tile
// sorts its segments by (cell, position) in shared memory; only the (cell, tile) pairs are
// sorted globally (stable radix sort; millions of pairs instead of a hundred million voxels),
// and an exclusive scan of the pair counts in that order gives every pair's start in the
// layout.  Three passes over the tiles share the same in-tile procedure:
//   group   -- the tile's pairs (cell, count) in cell order, written to the tile's own slot
//              range (2048 per tile) with their number; a scan of the numbers and a compaction
//              of the slots give the global pair list;
//   scatter -- each voxel's layout position = its pair's start + the lengths of the earlier
//              segments of its cell in the tile + its offset in its segment; writes the
//              coordinate and every variable (variables read in linear order, written in runs).
// Two passes over the voxels, both deterministic; no voxel-level sort.
#include "common.cuh"

namespace lsrvt {
namespace {

constexpr int kTile = 2048;
constexpr int kTileThreads = 256;
constexpr int kTilePer = kTile / kTileThreads;  // 8 consecutive voxels per thread
constexpr int kSegBits = 11;                     // segment ids < 2048
constexpr int kLayMaxVars = 64;
constexpr uint16_t kNoSeg = 0xFFFF;

enum TileMode { kGroup = 0, kScatter = 1 };

struct KeepMask {
    uint32_t w[8];  // bit b of word b / 32: band b is kept
};
struct VarIn {
    const float *p[kLayMaxVars];
};
struct VarOut {
    float *p[kLayMaxVars];
};

// per cell: 1 if the band of its component is kept.  Also checks the numbering the layout
// relies on (component offsets non-decreasing from 0 to the site count, component bands
// non-decreasing).
__global__ void cell_keep_kernel(const int32_t *__restrict__ comp_site_off, const uint8_t *__restrict__ comp_band,
                                 const int32_t *n_comp_dev, int32_t max_comp, const int32_t *n_sites_dev,
                                 int32_t max_sites, KeepMask km, uint8_t *keep, int32_t *status) {
    const int32_t nc = min(*n_comp_dev, max_comp), ns = min(*n_sites_dev, max_sites);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t c = t0; c <= nc; c += stride) {
        const bool bad = (c == 0 && comp_site_off[0] != 0) || (c > 0 && comp_site_off[c] < comp_site_off[c - 1]) ||
                         (c > 0 && c < nc && comp_band[c] < comp_band[c - 1]) ||
                         (c == nc && comp_site_off[nc] != ns);
        if (bad) set_status(status, LSRVT_ERR_INVALID_ARG);
    }
    for (int64_t s = t0; s < ns; s += stride) {
        int32_t lo = 0, hi = nc;  // first c in [0, nc] with comp_site_off[c] > s
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (comp_site_off[mid] <= s) lo = mid + 1;
            else hi = mid;
        }
        const int32_t c = lo - 1;
        uint8_t k = 0;
        if (c >= 0 && c < nc) {
            const unsigned b = comp_band[c];
            k = (uint8_t)((km.w[b >> 5] >> (b & 31)) & 1u);
        }
        keep[s] = k;
    }
}

// the cell of voxel v if it is kept, else -1 (a cell id without a site is an argument error)
__device__ __forceinline__ int32_t kept_cell(int32_t s, int32_t ns, const uint8_t *__restrict__ keep,
                                             int32_t *status) {
    if (s >= ns) {
        set_status(status, LSRVT_ERR_INVALID_ARG);
        return -1;
    }
    return (s >= 0 && keep[s]) ? s : -1;
}

// exclusive block scan of one int per thread; returns the block total in `total`
__device__ __forceinline__ int block_scan_excl(int v, int &total) {
    __shared__ int wsum[kTileThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    int before = 0;
    total = 0;
#pragma unroll
    for (int k = 0; k < kTileThreads / 32; ++k) {
        const int t = wsum[k];
        before += k < w ? t : 0;
        total += t;
    }
    __syncthreads();  // wsum is reused by the next call
    return before + x - v;
}

struct TileSmem {
    unsigned long long skey[kTile];  // (cell << 11) | segment id; sorted by cell, then position
    int32_t seg_start[kTile];        // tile position of each segment's first voxel (position order)
    int32_t seg_len[kTile];
    int32_t seg_base[kTile];         // scatter: layout position of each segment's first voxel
    uint16_t segid[kTile];           // scatter: segment of each tile position (kNoSeg: not kept)
};

struct TileArgs {
    const int32_t *cell;
    int64_t n;
    const int32_t *n_sites_dev;
    int32_t max_sites;
    const uint8_t *keep;
    int64_t *tile_np;          // group: pairs per tile; scatter: scanned offsets
    uint32_t *slot_key;        // group: pair cells in the tile's slots [t * kTile, t * kTile + npairs)
    int32_t *slot_cnt;         // group: pair voxel counts, same slots
    const int32_t *pstart;     // scatter: layout start of each pair (by pair index)
    int32_t *order;            // scatter
    int32_t *cell_out;         // scatter (nullable): the cell of each layout position
    VarIn in;                  // scatter
    VarOut out;                // scatter
    int m;
    int32_t *status;
};

template <int kMode>
__global__ void __launch_bounds__(kTileThreads) layout_tile_kernel(TileArgs a) {
    __shared__ TileSmem sm;
    const int32_t ns = min(*a.n_sites_dev, a.max_sites);
    const int64_t ntiles = (a.n + kTile - 1) / kTile;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t base = t * kTile;
        const int64_t v0 = base + (int64_t)tid * kTilePer;
        int32_t c[kTilePer];
        if (v0 + kTilePer <= a.n) {
            const int4 x = __ldg(reinterpret_cast<const int4 *>(a.cell + v0));
            const int4 y = __ldg(reinterpret_cast<const int4 *>(a.cell + v0) + 1);
            c[0] = x.x; c[1] = x.y; c[2] = x.z; c[3] = x.w;
            c[4] = y.x; c[5] = y.y; c[6] = y.z; c[7] = y.w;
        } else {
#pragma unroll
            for (int k = 0; k < kTilePer; ++k) c[k] = v0 + k < a.n ? __ldg(a.cell + v0 + k) : -1;
        }
#pragma unroll
        for (int k = 0; k < kTilePer; ++k) c[k] = kept_cell(c[k], ns, a.keep, kMode == kGroup ? a.status : nullptr);
        // the previous voxel's kept cell (segments never cross a tile boundary)
        int32_t prev = __shfl_up_sync(0xffffffffu, c[kTilePer - 1], 1);
        if (lane == 0) prev = (tid == 0 || v0 > a.n) ? -1 : kept_cell(__ldg(a.cell + v0 - 1), ns, a.keep, nullptr);
        unsigned starts = 0;
#pragma unroll
        for (int k = 0; k < kTilePer; ++k)
            starts |= (unsigned)(c[k] >= 0 && c[k] != (k ? c[k - 1] : prev)) << k;
        // segments in position order: start, sort key, voxel count (a thread's leading run may
        // belong to a segment an earlier thread started, hence the counters are cleared before
        // the scan's barrier and filled with atomics after it)
        for (int i = tid; i < kTile; i += kTileThreads) sm.seg_len[i] = 0;
        int nseg;
        const int sid0 = block_scan_excl(__popc(starts), nseg);
        {
            int cur = sid0 - 1, run = 0;
#pragma unroll
            for (int k = 0; k < kTilePer; ++k) {
                if ((starts >> k) & 1u) {
                    if (run) atomicAdd(&sm.seg_len[cur], run);
                    ++cur;
                    run = 0;
                    sm.seg_start[cur] = tid * kTilePer + k;
                    sm.skey[cur] = ((unsigned long long)(uint32_t)c[k] << kSegBits) | (unsigned)cur;
                }
                if (c[k] >= 0) ++run;
                if (kMode == kScatter) sm.segid[tid * kTilePer + k] = c[k] >= 0 ? (uint16_t)cur : kNoSeg;
            }
            if (run) atomicAdd(&sm.seg_len[cur], run);
        }
        int npow2 = 1;
        while (npow2 < nseg) npow2 <<= 1;
        for (int i = nseg + tid; i < npow2; i += kTileThreads) sm.skey[i] = ~0ULL;
        if (npow2 > 1) block_bitonic_sort(sm.skey, npow2);
        else __syncthreads();
        // cell groups in sorted order: a head starts each distinct cell
        unsigned heads = 0;
#pragma unroll
        for (int k = 0; k < kTilePer; ++k) {
            const int j = tid * kTilePer + k;
            if (j < nseg && (j == 0 || (sm.skey[j] >> kSegBits) != (sm.skey[j - 1] >> kSegBits))) heads |= 1u << k;
        }
        int npairs;
        int q = block_scan_excl(__popc(heads), npairs);
        if (kMode == kGroup && tid == 0) a.tile_np[t] = npairs;
        {
            const int64_t poff = kMode == kScatter ? a.tile_np[t] : 0;
#pragma unroll
            for (int k = 0; k < kTilePer; ++k) {
                if (!((heads >> k) & 1u)) continue;
                const int j = tid * kTilePer + k;
                const uint32_t cellid = (uint32_t)(sm.skey[j] >> kSegBits);
                const int64_t run = kMode == kScatter ? a.pstart[poff + q] : 0;
                int cnt = 0;
                for (int jj = j; jj < nseg && (uint32_t)(sm.skey[jj] >> kSegBits) == cellid; ++jj) {
                    const int sid = (int)(sm.skey[jj] & ((1u << kSegBits) - 1));
                    if (kMode == kScatter) sm.seg_base[sid] = (int32_t)(run + cnt);
                    cnt += sm.seg_len[sid];
                }
                if (kMode == kGroup) {
                    a.slot_key[t * kTile + q] = cellid;
                    a.slot_cnt[t * kTile + q] = cnt;
                }
                ++q;
            }
        }
        if (kMode == kScatter) {
            __syncthreads();
            // voxel i = r * 256 + tid: a warp covers 32 consecutive voxels, so reads of the
            // variables are coalesced and writes go out in runs along each segment
            int32_t pos[kTilePer];
#pragma unroll
            for (int r = 0; r < kTilePer; ++r) {
                const int i = r * kTileThreads + tid;
                const uint16_t sid = sm.segid[i];
                pos[r] = (base + i < a.n && sid != kNoSeg) ? sm.seg_base[sid] + (i - sm.seg_start[sid]) : -1;
                if (pos[r] >= 0) {
                    a.order[pos[r]] = (int32_t)(base + i);
                    if (a.cell_out) a.cell_out[pos[r]] = __ldg(a.cell + base + i);
                }
            }
            // four variables at a time: 32 independent loads in flight per thread
            for (int j0 = 0; j0 < a.m; j0 += 4) {
                const int nj = a.m - j0 < 4 ? a.m - j0 : 4;
                float x[4][kTilePer];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    if (jj >= nj) break;
                    const float *src = a.in.p[j0 + jj] + base;
#pragma unroll
                    for (int r = 0; r < kTilePer; ++r)
                        x[jj][r] = pos[r] >= 0 ? __ldcs(src + r * kTileThreads + tid) : 0.f;
                }
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    if (jj >= nj) break;
                    float *dst = a.out.p[j0 + jj];
#pragma unroll
                    for (int r = 0; r < kTilePer; ++r)
                        if (pos[r] >= 0) dst[pos[r]] = x[jj][r];
                }
            }
        }
        __syncthreads();  // shared memory is reused by the next tile
    }
}

// the tiles' pair slots, compacted in tile order: pair index = scanned tile offset + slot
__global__ void layout_compact_pairs_kernel(const uint32_t *__restrict__ slot_key,
                                            const int32_t *__restrict__ slot_cnt,
                                            const int64_t *__restrict__ tile_off, int64_t ntiles, uint32_t *pkey,
                                            uint32_t *pval, int32_t *pcnt) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp; t < ntiles; t += nwarps) {
        const int64_t off = tile_off[t], np = tile_off[t + 1] - off;
        for (int64_t q = lane; q < np; q += 32) {
            pkey[off + q] = slot_key[t * kTile + q];
            pval[off + q] = (uint32_t)(off + q);
            pcnt[off + q] = slot_cnt[t * kTile + q];
        }
    }
}

// the number of pairs: the exclusive scan's entry at ntiles
// positions past the kept voxels: no cell (so the per-position cells form a complete label array)
__global__ void layout_cell_tail_kernel(const int64_t *n_kept, int64_t n, int32_t *cell_out) {
    for (int64_t p = *n_kept + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        cell_out[p] = -1;
}

__global__ void layout_pairs_total_kernel(const int64_t *tile_off, int64_t ntiles, int64_t *np64, int32_t *np32) {
    *np64 = tile_off[ntiles];
    *np32 = (int32_t)tile_off[ntiles];
}

// counts of the pairs in sorted order (the scan of these gives each pair's layout start)
__global__ void layout_permute_kernel(const uint32_t *__restrict__ pval, const int32_t *__restrict__ pcnt,
                                      const int64_t *np, int64_t *cs) {
    const int64_t P = *np;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < P; j += (int64_t)gridDim.x * blockDim.x)
        cs[j] = pcnt[pval[j]];
}

__global__ void layout_starts_kernel(const uint32_t *__restrict__ pval, const int64_t *__restrict__ cs,
                                     const int64_t *np, int32_t *pstart) {
    const int64_t P = *np;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < P; j += (int64_t)gridDim.x * blockDim.x)
        pstart[pval[j]] = (int32_t)cs[j];
}

__device__ __forceinline__ int64_t lower_bound_u32(const uint32_t *__restrict__ a, int64_t n, uint32_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// layout start of the first pair whose cell is >= s (n_kept if none)
__device__ __forceinline__ int64_t start_of_cell(const uint32_t *__restrict__ pkey, const int64_t *__restrict__ cs,
                                                 int64_t P, int64_t r, uint32_t s) {
    const int64_t j = lower_bound_u32(pkey, P, s);
    return j < P ? cs[j] : r;
}

// Offsets from the sorted pairs: cell_off[s] (s <= ns), comp_off[c] (c <= nc), band_off[b]
// (b <= 256)
__global__ void layout_offsets_kernel(const uint32_t *__restrict__ pkey, const int64_t *__restrict__ cs,
                                      const int64_t *np, const int64_t *n_kept, const int32_t *n_sites_dev,
                                      int32_t max_sites, const int32_t *__restrict__ comp_site_off,
                                      const uint8_t *__restrict__ comp_band, const int32_t *n_comp_dev,
                                      int32_t max_comp, int64_t *cell_off, int64_t *comp_off, int64_t *band_off) {
    const int64_t P = *np, r = *n_kept;
    const int32_t ns = min(*n_sites_dev, max_sites), nc = min(*n_comp_dev, max_comp);
    const int64_t total = (int64_t)(ns + 1) + (nc + 1) + 257;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i <= ns) {
            cell_off[i] = start_of_cell(pkey, cs, P, r, (uint32_t)i);
        } else if (i <= (int64_t)ns + 1 + nc) {
            const int32_t c = (int32_t)(i - ns - 1);
            comp_off[c] = start_of_cell(pkey, cs, P, r, (uint32_t)comp_site_off[c]);
        } else {
            const int32_t b = (int32_t)(i - ns - 2 - nc);
            int32_t lo = 0, hi = nc;  // first component of band >= b
            while (lo < hi) {
                const int32_t mid = (lo + hi) >> 1;
                if ((int32_t)comp_band[mid] < b) lo = mid + 1;
                else hi = mid;
            }
            band_off[b] = lo < nc ? start_of_cell(pkey, cs, P, r, (uint32_t)comp_site_off[lo]) : r;
        }
    }
}

struct LayoutWs {
    uint8_t *keep;
    int64_t *tile_np;
    void *scan_tiles;
    int64_t *np64;
    int32_t *np32;
    uint32_t *pkey, *pval;
    uint32_t *slot_key;
    int32_t *slot_cnt;
    int32_t *pcnt;
    int64_t *cs;
    int32_t *pstart;
    void *scan_pairs;
    void *radix_tmp;
};

// pairs: at most one per kept voxel
LayoutWs carve_layout(void *ws, size_t bytes, Dims d, int32_t max_sites, size_t *need) {
    Carver c(ws, bytes);
    LayoutWs w;
    const int64_t n = d.n();
    const int64_t ntiles = (n + kTile - 1) / kTile;
    w.keep = c.take<uint8_t>((size_t)max_sites + 1);
    w.tile_np = c.take<int64_t>(ntiles + 1);
    w.scan_tiles = c.take<char>(scan_temp_bytes(ntiles + 1));
    w.np64 = c.take<int64_t>(1);
    w.np32 = c.take<int32_t>(1);
    w.pkey = c.take<uint32_t>(n);
    w.pval = c.take<uint32_t>(n);
    w.slot_key = c.take<uint32_t>(ntiles * kTile);
    w.slot_cnt = c.take<int32_t>(ntiles * kTile);
    w.pcnt = c.take<int32_t>(n);
    w.cs = c.take<int64_t>(n);
    w.pstart = c.take<int32_t>(n);
    w.scan_pairs = c.take<char>(scan_temp_bytes(n));
    w.radix_tmp = c.take<char>(radix_temp_bytes(n));
    *need = c.used;
    return w;
}

}  // namespace

size_t layout_workspace(Dims d, int32_t max_sites) {
    size_t need;
    carve_layout(nullptr, 0, d, max_sites, &need);
    return need;
}

}  // namespace lsrvt

using namespace lsrvt;

extern "C" lsrvt_status lsrvt_structured_layout(const int32_t *cell, lsrvt_dims dd, const int32_t *n_sites_dev,
                                                int32_t max_sites, const int32_t *comp_site_off,
                                                const uint8_t *comp_band, const int32_t *n_comp_dev, int32_t max_comp,
                                                const uint32_t *band_mask_host, const float *const *aux_host,
                                                int32_t n_aux, float *const *values_host, int32_t *order,
                                                int64_t *cell_off, int64_t *comp_off, int64_t *band_off,
                                                int64_t *n_kept_dev, int32_t *cell_out, void *ws, size_t ws_bytes,
                                                int32_t *status_dev, void *stream) {
    if (!dims_ok(dd) || !cell || !n_sites_dev || max_sites < 1 || !comp_site_off || !comp_band || !n_comp_dev ||
        max_comp < 0 || n_aux < 0 || n_aux > kLayMaxVars || (n_aux > 0 && (!aux_host || !values_host)) || !order ||
        !cell_off || !comp_off || !band_off || !n_kept_dev)
        return LSRVT_ERR_INVALID_ARG;
    TileArgs a{};
    for (int j = 0; j < n_aux; ++j) {
        a.in.p[j] = aux_host[j];
        a.out.p[j] = values_host[j];
        if (!a.in.p[j] || !a.out.p[j]) return LSRVT_ERR_INVALID_ARG;
    }
    if ((uintptr_t)cell & 15) return LSRVT_ERR_INVALID_ARG;  // 16-byte loads of the labels
    const Dims d{dd.nx, dd.ny, dd.nz};
    size_t need;
    LayoutWs w = carve_layout(ws, ws_bytes, d, max_sites, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) return LSRVT_ERR_WORKSPACE;
    KeepMask km;
    for (int k = 0; k < 8; ++k) km.w[k] = band_mask_host ? band_mask_host[k] : ~0u;
    cudaStream_t s = as_stream(stream);
    const int sms = stream_sms(s);
    const int64_t n = d.n();
    const int64_t ntiles = (n + kTile - 1) / kTile;
    cell_keep_kernel<<<grid_for(max_sites + 1, 256, sms * 4), 256, 0, s>>>(comp_site_off, comp_band, n_comp_dev,
                                                                            max_comp, n_sites_dev, max_sites, km,
                                                                            w.keep, status_dev);
    a.cell = cell;
    a.n = n;
    a.n_sites_dev = n_sites_dev;
    a.max_sites = max_sites;
    a.keep = w.keep;
    a.tile_np = w.tile_np;
    a.slot_key = w.slot_key;
    a.slot_cnt = w.slot_cnt;
    a.pstart = w.pstart;
    a.order = order;
    a.cell_out = cell_out;
    a.m = n_aux;
    a.status = status_dev;
    const int tgrid = (int)(ntiles < sms * 5 ? ntiles : sms * 5);
    layout_tile_kernel<kGroup><<<tgrid, kTileThreads, 0, s>>>(a);
    exclusive_scan_i64(w.tile_np, ntiles + 1, nullptr, w.scan_tiles, s);  // entry ntiles: the total
    layout_pairs_total_kernel<<<1, 1, 0, s>>>(w.tile_np, ntiles, w.np64, w.np32);
    layout_compact_pairs_kernel<<<sms * 8, 256, 0, s>>>(w.slot_key, w.slot_cnt, w.tile_np, ntiles, w.pkey, w.pval,
                                                        w.pcnt);
    int bits = 0;
    while (bits < 31 && ((int64_t)1 << bits) < max_sites) ++bits;
    radix_sort_pairs(w.pkey, w.pval, n, w.np32, bits, w.radix_tmp, s);
    const int pgrid = sms * 8;
    layout_permute_kernel<<<pgrid, 256, 0, s>>>(w.pval, w.pcnt, w.np64, w.cs);
    exclusive_scan_i64_dev(w.cs, n, w.np64, n_kept_dev, w.scan_pairs, s);
    layout_starts_kernel<<<pgrid, 256, 0, s>>>(w.pval, w.cs, w.np64, w.pstart);
    layout_offsets_kernel<<<grid_for((int64_t)max_sites + max_comp + 259, 256, sms * 4), 256, 0, s>>>(
        w.pkey, w.cs, w.np64, n_kept_dev, n_sites_dev, max_sites, comp_site_off, comp_band, n_comp_dev, max_comp,
        cell_off, comp_off, band_off);
    layout_tile_kernel<kScatter><<<tgrid, kTileThreads, 0, s>>>(a);
    if (cell_out) layout_cell_tail_kernel<<<sms * 4, 256, 0, s>>>(n_kept_dev, n, cell_out);
    return launch_status();
}
