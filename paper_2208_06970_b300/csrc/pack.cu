// pack.cu -- packed batches of independent blocks (Discussion "Block Based Distributed
// Parallelism": the blocks of a volume are decomposed independently, their boundaries acting
// as restrictions; Sec. 3.2 "Parallel Algorithm").
//
// Many blocks are placed in one packed volume, apart from each other by voxels of band 0xFF,
// which are no graph nodes, so that one Lloyd loop over the packed volume runs each of its
// launches over the bricks of every block.  Packing copies each block's bands (and weights)
// to its origin and renumbers its sites after the sites of the blocks before it; unpacking
// hands each block its cells (site ids less that offset), distances and sites.  The block
// table travels as a kernel parameter, so a packed batch captures into a CUDA graph without
// host memory behind it, and the sites' offsets are prefix sums taken on the device from the
// blocks' device counts.
#include <cstddef>

#include "common.cuh"

// the descriptor layout the Python binding mirrors (LP64): dims and origin, then six pointers
static_assert(sizeof(lsrvt_block) == 72, "lsrvt_block layout");
static_assert(offsetof(lsrvt_block, x0) == 12 && offsetof(lsrvt_block, band) == 24 &&
                  offsetof(lsrvt_block, n_sites) == 48 && offsetof(lsrvt_block, dist) == 64,
              "lsrvt_block layout");

namespace lsrvt {
namespace {

struct Blk {
    int32_t nx, ny, nz, x0, y0, z0;
    const uint8_t *band;
    const uint16_t *q;
    int32_t *site_pos;
    const int32_t *n_sites;
    int32_t *cell;
    uint32_t *dist;
};

struct BlockTable {
    int32_t n;
    Blk b[LSRVT_MAX_PACK_BLOCKS];
};

// site_base[b] = sum of the counts of the blocks before b; site_base[n] = the total
__global__ void pack_base_kernel(const __grid_constant__ BlockTable t, int32_t *site_base, int32_t *n_sites_dev,
                                 int32_t max_sites, int32_t *status) {
    __shared__ int32_t cnt[LSRVT_MAX_PACK_BLOCKS];
    const int b = threadIdx.x;
    cnt[b] = b < t.n ? max(*t.b[b].n_sites, 0) : 0;
    __syncthreads();
    if (b == 0) {
        int64_t acc = 0;
        for (int i = 0; i < t.n; ++i) {
            site_base[i] = (int32_t)min(acc, (int64_t)max_sites);
            acc += cnt[i];
        }
        const bool fits = acc <= max_sites;
        site_base[t.n] = fits ? (int32_t)acc : max_sites;
        *n_sites_dev = fits ? (int32_t)acc : 0;
        if (!fits) set_status(status, LSRVT_ERR_CAPACITY);
    }
}

// one row (fixed y, z) of a block per CTA turn, its voxels along x by the threads
__global__ void __launch_bounds__(256) pack_voxels_kernel(const __grid_constant__ BlockTable t, Dims P,
                                                          uint8_t *__restrict__ band, uint16_t *__restrict__ q) {
    const Blk &B = t.b[blockIdx.y];
    const int64_t rows = (int64_t)B.ny * B.nz;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const int y = (int)(r % B.ny), z = (int)(r / B.ny);
        const int64_t src = (int64_t)B.nx * r;
        const int64_t dst = B.x0 + (int64_t)P.nx * ((int64_t)(B.y0 + y) + (int64_t)P.ny * (B.z0 + z));
        for (int x = threadIdx.x; x < B.nx; x += blockDim.x) {
            band[dst + x] = B.band[src + x];
            if (q) q[dst + x] = B.q[src + x];
        }
    }
}

__global__ void __launch_bounds__(256) pack_sites_kernel(const __grid_constant__ BlockTable t, Dims P,
                                                         const int32_t *__restrict__ site_base,
                                                         int32_t *__restrict__ site_pos) {
    const Blk &B = t.b[blockIdx.y];
    const int32_t base = site_base[blockIdx.y], cnt = site_base[blockIdx.y + 1] - base;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        const int32_t p = B.site_pos[i];
        const int x = p % B.nx, y = (p / B.nx) % B.ny, z = p / (B.nx * B.ny);
        site_pos[base + i] =
            (int32_t)((B.x0 + x) + (int64_t)P.nx * ((int64_t)(B.y0 + y) + (int64_t)P.ny * (B.z0 + z)));
    }
}

__global__ void __launch_bounds__(256) unpack_voxels_kernel(const __grid_constant__ BlockTable t, Dims P,
                                                            const int32_t *__restrict__ cell,
                                                            const uint32_t *__restrict__ dist,
                                                            const int32_t *__restrict__ site_base) {
    const Blk &B = t.b[blockIdx.y];
    if (!B.cell && !(dist && B.dist)) return;
    const int32_t base = site_base[blockIdx.y];
    const int64_t rows = (int64_t)B.ny * B.nz;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const int y = (int)(r % B.ny), z = (int)(r / B.ny);
        const int64_t src = (int64_t)B.nx * r;
        const int64_t dst = B.x0 + (int64_t)P.nx * ((int64_t)(B.y0 + y) + (int64_t)P.ny * (B.z0 + z));
        for (int x = threadIdx.x; x < B.nx; x += blockDim.x) {
            if (B.cell) {
                const int32_t c = cell[dst + x];
                B.cell[src + x] = c >= 0 ? c - base : -1;
            }
            if (dist && B.dist) B.dist[src + x] = dist[dst + x];
        }
    }
}

__global__ void __launch_bounds__(256) unpack_sites_kernel(const __grid_constant__ BlockTable t, Dims P,
                                                           const int32_t *__restrict__ site_base,
                                                           const int32_t *__restrict__ site_pos) {
    const Blk &B = t.b[blockIdx.y];
    const int32_t base = site_base[blockIdx.y], cnt = site_base[blockIdx.y + 1] - base;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        const int32_t p = site_pos[base + i];
        const int X = p % P.nx, Y = (p / P.nx) % P.ny, Z = p / (P.nx * P.ny);
        B.site_pos[i] = (X - B.x0) + B.nx * ((Y - B.y0) + B.ny * (Z - B.z0));
    }
}

// Host: the descriptors as a kernel parameter; INVALID_ARG for a block outside the packed
// volume, NULL arrays the call needs, or two blocks whose boxes, each widened by one voxel on
// its upper side, overlap on every axis (their voxels would be 26-neighbours or shared).
lsrvt_status make_table(const lsrvt_block *blocks, int32_t n_blocks, lsrvt_dims packed, bool packing, bool need_q,
                        BlockTable &t) {
    if (!blocks || n_blocks < 1 || n_blocks > LSRVT_MAX_PACK_BLOCKS || !dims_ok(packed)) return LSRVT_ERR_INVALID_ARG;
    memset(&t, 0, sizeof(t));
    t.n = n_blocks;
    for (int i = 0; i < n_blocks; ++i) {
        const lsrvt_block &b = blocks[i];
        if (!dims_ok(b.d) || b.x0 < 0 || b.y0 < 0 || b.z0 < 0 || (int64_t)b.x0 + b.d.nx > packed.nx ||
            (int64_t)b.y0 + b.d.ny > packed.ny || (int64_t)b.z0 + b.d.nz > packed.nz || !b.site_pos)
            return LSRVT_ERR_INVALID_ARG;
        if (packing && (!b.band || !b.n_sites || (need_q && !b.q))) return LSRVT_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j) {
            const lsrvt_block &a = blocks[j];
            const bool ox = a.x0 < (int64_t)b.x0 + b.d.nx + 1 && b.x0 < (int64_t)a.x0 + a.d.nx + 1;
            const bool oy = a.y0 < (int64_t)b.y0 + b.d.ny + 1 && b.y0 < (int64_t)a.y0 + a.d.ny + 1;
            const bool oz = a.z0 < (int64_t)b.z0 + b.d.nz + 1 && b.z0 < (int64_t)a.z0 + a.d.nz + 1;
            if (ox && oy && oz) return LSRVT_ERR_INVALID_ARG;
        }
        t.b[i] = Blk{b.d.nx, b.d.ny, b.d.nz, b.x0, b.y0, b.z0, b.band, b.q, b.site_pos, b.n_sites, b.cell, b.dist};
    }
    return LSRVT_OK;
}

int voxel_grid(const BlockTable &t, int sms) {
    // about eight CTAs per SM over all blocks' rows
    const int per_block = (8 * sms + t.n - 1) / t.n;
    return per_block < 1 ? 1 : per_block;
}

}  // namespace
}  // namespace lsrvt

using namespace lsrvt;

extern "C" lsrvt_status lsrvt_pack_blocks(const lsrvt_block *blocks_host, int32_t n_blocks, lsrvt_dims packed,
                                          uint8_t *band, uint16_t *q, int32_t *site_pos, int32_t max_sites,
                                          int32_t *n_sites_dev, int32_t *site_base, int32_t *status_dev,
                                          void *stream) {
    BlockTable tab;  // the kernel parameter (copied at each launch)
    lsrvt_status st = make_table(blocks_host, n_blocks, packed, true, q != nullptr, tab);
    if (st != LSRVT_OK) return st;
    if (!band || !site_pos || max_sites < 1 || !n_sites_dev || !site_base) return LSRVT_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    const Dims P{packed.nx, packed.ny, packed.nz};
    const int64_t n = P.n();
    if (cudaMemsetAsync(band, 0xFF, (size_t)n, s) != cudaSuccess) return LSRVT_ERR_CUDA;
    if (q && cudaMemsetAsync(q, 0, (size_t)n * sizeof(uint16_t), s) != cudaSuccess) return LSRVT_ERR_CUDA;
    pack_base_kernel<<<1, LSRVT_MAX_PACK_BLOCKS, 0, s>>>(tab, site_base, n_sites_dev, max_sites, status_dev);
    const int sms = stream_sms(s);
    pack_voxels_kernel<<<dim3(voxel_grid(tab, sms), n_blocks), 256, 0, s>>>(tab, P, band, q);
    pack_sites_kernel<<<dim3(voxel_grid(tab, sms), n_blocks), 256, 0, s>>>(tab, P, site_base, site_pos);
    return launch_status();
}

extern "C" lsrvt_status lsrvt_unpack_blocks(const lsrvt_block *blocks_host, int32_t n_blocks, lsrvt_dims packed,
                                            const int32_t *cell, const uint32_t *dist, const int32_t *site_pos,
                                            const int32_t *site_base, void *stream) {
    BlockTable tab;
    lsrvt_status st = make_table(blocks_host, n_blocks, packed, false, false, tab);
    if (st != LSRVT_OK) return st;
    if (!cell || !site_pos || !site_base) return LSRVT_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    const Dims P{packed.nx, packed.ny, packed.nz};
    const int sms = stream_sms(s);
    unpack_voxels_kernel<<<dim3(voxel_grid(tab, sms), n_blocks), 256, 0, s>>>(tab, P, cell, dist, site_base);
    unpack_sites_kernel<<<dim3(voxel_grid(tab, sms), n_blocks), 256, 0, s>>>(tab, P, site_base, site_pos);
    return launch_status();
}
