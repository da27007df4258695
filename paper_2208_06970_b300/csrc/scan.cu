// scan.cu -- device-wide exclusive scan (int64) and stable LSD radix sort of uint32
// (key, value) pairs.  Building blocks for dense relabelling (components), stratum
// grouping and site numbering.  Both are deterministic.
#include "common.cuh"

namespace lsrvt {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ int64_t block_exclusive_scan(int64_t v, int64_t *out_excl) {
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t block_total;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        int64_t t = lane < nw ? warp_tot[lane] : 0;
        int64_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t u = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += u;
        }
        if (lane < nw) warp_tot[lane] = ti - t;  // exclusive warp offsets
        if (lane == nw - 1) block_total = ti;
    }
    __syncthreads();
    *out_excl = warp_tot[w] + inc - v;
    int64_t total = block_total;
    __syncthreads();
    return total;
}

// n_dev (nullable): a device-side count <= n; entries at and beyond it are left alone
__device__ __forceinline__ int64_t scan_n(int64_t n, const int64_t *n_dev) {
    if (!n_dev) return n;
    const int64_t m = *n_dev;
    return m < n ? (m < 0 ? 0 : m) : n;
}

__global__ void scan_reduce_kernel(const int64_t *data, int64_t n, const int64_t *n_dev, int64_t *tile_sums) {
    n = scan_n(n, n_dev);
    if ((int64_t)blockIdx.x * kScanTile >= n) {  // a tile past the live entries sums to 0
        if (threadIdx.x == 0) tile_sums[blockIdx.x] = 0;
        return;
    }
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += data[base + i];
    int64_t excl;
    int64_t tot = block_exclusive_scan(s, &excl);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// Single-block scan of the tile sums (any count), carrying across chunks.
__global__ void scan_tiles_kernel(int64_t *tile_sums, int64_t ntiles, int64_t *total) {
    int64_t carry = 0;
    for (int64_t base = 0; base < ntiles; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < ntiles ? tile_sums[i] : 0;
        int64_t excl;
        int64_t tot = block_exclusive_scan(v, &excl);
        if (i < ntiles) tile_sums[i] = carry + excl;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void scan_apply_kernel(int64_t *data, int64_t n, const int64_t *n_dev, const int64_t *tile_offs) {
    n = scan_n(n, n_dev);
    if ((int64_t)blockIdx.x * kScanTile >= n) return;
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? data[base + i] : 0;
        s += v[i];
    }
    int64_t excl;
    block_exclusive_scan(s, &excl);
    int64_t run = tile_offs[blockIdx.x] + excl;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) data[base + i] = run;
        run += v[i];
    }
}

// ------------------------------------------------------------------ radix sort
constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixPerWarp = 256;  // items per warp sub-tile (8 rounds of 32)
constexpr int kRadixTile = kRadixWarps * kRadixPerWarp;  // 2048

__device__ __forceinline__ int64_t radix_n(int64_t n, const int32_t *n_dev) {
    if (n_dev) {
        int64_t m = *n_dev;
        return m < n ? (m < 0 ? 0 : m) : n;
    }
    return n;
}

// Tiles of the live items (device count): ceil(n / kRadixTile).  The histogram is digit-major
// over the live tiles, hist[d * ntiles + tile], so its exclusive scan (over 256 * ntiles entries)
// gives every (digit, tile) its output offset.  Kernels loop over the live tiles with a fixed
// grid, so a large capacity costs no idle blocks.
__device__ __forceinline__ int64_t radix_tiles(int64_t n) { return (n + kRadixTile - 1) / kRadixTile; }

__global__ void radix_count_kernel(int64_t n_max, const int32_t *n_dev, int64_t *hist_n) {
    *hist_n = radix_tiles(radix_n(n_max, n_dev)) * 256;
}

__global__ void radix_hist_kernel(const uint32_t *keys, int64_t n_max, const int32_t *n_dev, int shift,
                                  int64_t *hist) {
    __shared__ unsigned cnt[256];
    const int64_t n = radix_n(n_max, n_dev);
    const int64_t ntiles = radix_tiles(n);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) cnt[i] = 0;
        __syncthreads();
        const int64_t base = tile * kRadixTile;
        for (int i = threadIdx.x; i < kRadixTile; i += blockDim.x) {
            const int64_t j = base + i;
            if (j < n) atomicAdd(&cnt[(keys[j] >> shift) & 255u], 1u);
        }
        __syncthreads();
        for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(int64_t)d * ntiles + tile] = cnt[d];
        __syncthreads();
    }
}

__global__ void radix_scatter_kernel(const uint32_t *keys, const uint32_t *vals, uint32_t *okeys, uint32_t *ovals,
                                     int64_t n_max, const int32_t *n_dev, int shift, const int64_t *offs) {
    __shared__ unsigned wcnt[kRadixWarps][256];
    const int64_t n = radix_n(n_max, n_dev);
    const int64_t ntiles = radix_tiles(n);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        for (int i = threadIdx.x; i < kRadixWarps * 256; i += blockDim.x) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        const int64_t wbase = tile * kRadixTile + (int64_t)w * kRadixPerWarp;
        // pass 1: per-warp digit counts
        for (int r = 0; r < kRadixPerWarp; r += 32) {
            const int64_t j = wbase + r + lane;
            const bool ok = j < n;
            const unsigned d = ok ? ((keys[j] >> shift) & 255u) : 256u;
            const unsigned m = __match_any_sync(0xffffffffu, d);
            if (ok && (m & lanemask_lt()) == 0) wcnt[w][d] += __popc(m);
            __syncwarp();
        }
        __syncthreads();
        // exclusive prefix over warps per digit
        for (int d = threadIdx.x; d < 256; d += blockDim.x) {
            unsigned run = 0;
            for (int k = 0; k < kRadixWarps; ++k) {
                const unsigned c = wcnt[k][d];
                wcnt[k][d] = run;
                run += c;
            }
        }
        __syncthreads();
        // pass 2: stable placement
        for (int r = 0; r < kRadixPerWarp; r += 32) {
            const int64_t j = wbase + r + lane;
            const bool ok = j < n;
            const uint32_t key = ok ? keys[j] : 0u;
            const unsigned d = ok ? ((key >> shift) & 255u) : 256u;
            const unsigned m = __match_any_sync(0xffffffffu, d);
            if (ok) {
                const unsigned rank = __popc(m & lanemask_lt());
                const int64_t pos = offs[(int64_t)d * ntiles + tile] + wcnt[w][d] + rank;
                okeys[pos] = key;
                ovals[pos] = vals[j];
            }
            __syncwarp();
            if (ok && (m & lanemask_lt()) == 0) wcnt[w][d] += __popc(m);
            __syncwarp();
        }
        __syncthreads();
    }
}

}  // namespace

size_t scan_temp_bytes(int64_t n) {
    int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    return (size_t)(ntiles > 0 ? ntiles : 1) * sizeof(int64_t) + 256;
}

void exclusive_scan_i64_dev(int64_t *data, int64_t n, const int64_t *n_dev, int64_t *total, void *temp,
                           cudaStream_t s) {
    int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    int64_t *tile = (int64_t *)temp;
    if (ntiles == 0) {
        if (total) cudaMemsetAsync(total, 0, sizeof(int64_t), s);
        return;
    }
    scan_reduce_kernel<<<(unsigned)ntiles, kScanThreads, 0, s>>>(data, n, n_dev, tile);
    scan_tiles_kernel<<<1, 1024, 0, s>>>(tile, ntiles, total);
    scan_apply_kernel<<<(unsigned)ntiles, kScanThreads, 0, s>>>(data, n, n_dev, tile);
}

void exclusive_scan_i64(int64_t *data, int64_t n, int64_t *total, void *temp, cudaStream_t s) {
    exclusive_scan_i64_dev(data, n, nullptr, total, temp, s);
}

size_t radix_temp_bytes(int64_t n) {
    int64_t ntiles = (n + kRadixTile - 1) / kRadixTile;
    if (ntiles < 1) ntiles = 1;
    size_t b = 0;
    b += ((size_t)n * 4 + 256) * 2;                  // ping-pong keys + values
    b += (size_t)ntiles * 256 * sizeof(int64_t) + 256;  // histograms
    b += scan_temp_bytes(ntiles * 256) + 256;
    b += 256;                                        // live histogram length
    return b;
}

void radix_sort_pairs(uint32_t *keys, uint32_t *vals, int64_t n, const int32_t *n_dev, int bits, void *temp,
                      cudaStream_t s) {
    if (n <= 0) return;
    int64_t ntiles = (n + kRadixTile - 1) / kRadixTile;
    Carver c(temp, ~size_t(0));
    uint32_t *k2 = c.take<uint32_t>(n);
    uint32_t *v2 = c.take<uint32_t>(n);
    int64_t *hist = c.take<int64_t>(ntiles * 256);
    void *stemp = c.take<char>(scan_temp_bytes(ntiles * 256));
    int64_t *hist_n = c.take<int64_t>(1);
    uint32_t *ka = keys, *va = vals, *kb = k2, *vb = v2;
    int passes = (bits + 7) / 8;
    if (passes < 1) passes = 1;
    if (passes & 1) passes += 1;  // even number of passes: the result lands back in keys/vals
    const int sms = stream_sms(s);
    const int grid = (int)(ntiles < sms * 8 ? ntiles : sms * 8);
    radix_count_kernel<<<1, 1, 0, s>>>(n, n_dev, hist_n);
    for (int p = 0; p < passes; ++p) {
        int shift = p * 8;
        if (shift >= 32) shift = 24;  // padding pass on an already-sorted top digit is stable
        radix_hist_kernel<<<grid, kRadixThreads, 0, s>>>(ka, n, n_dev, shift, hist);
        exclusive_scan_i64_dev(hist, ntiles * 256, hist_n, nullptr, stemp, s);
        radix_scatter_kernel<<<grid, kRadixThreads, 0, s>>>(ka, va, kb, vb, n, n_dev, shift, hist);
        uint32_t *t = ka; ka = kb; kb = t;
        t = va; va = vb; vb = t;
    }
}

}  // namespace lsrvt
