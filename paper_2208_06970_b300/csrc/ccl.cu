// ccl.cu -- connected components of each isoband (Sec. 3.1: components C^k of an
// isoband, no voxel of one adjacent to a voxel of another; 6-adjacency), with canonical
// ids ordered by (band, smallest linear index).
//
// Design (B300): lock-free union-find with min-index roots.
//  1. brick pass: a CTA loads a 32x4x4 brick of bands into shared memory, unions its
//     6-neighbour pairs with shared-memory atomicMin, compresses, and writes for every
//     voxel the global index of its brick-local root (the local minimum);
//  2. face pass: voxels on the low x/y/z faces of a brick union with the neighbour
//     across the face in global memory (atomicMin on the larger root);
//  3. compress pass: every voxel stores its final root (= smallest index of its set);
//  4. relabel: per 8192-voxel warp chunk the roots are counted per band, a single
//     exclusive scan over the band-major count table gives every root its dense id
//     (band, index) order, a second chunk pass ranks roots within the chunk in order;
//  5. finalize: every voxel takes its root's id; sizes by run-length + atomics.
#include "common.cuh"

namespace lsrvt {
namespace {

constexpr int BX = 32, BY = 4, BZ = 4, BV = BX * BY * BZ;  // 512 voxels, one per thread
constexpr int kChunkRounds = 256;                            // 256 x 32 = 8192 voxels per warp chunk
constexpr int kChunk = kChunkRounds * 32;
constexpr int kBands = 255;

// Labels only decrease along a chain, so a chain is at most BV long; the bound only
// guards against corrupted input.
__device__ __forceinline__ int smem_find(volatile int *lab, int a) {
    for (int it = 0; it <= BV; ++it) {
        int p = lab[a];
        if (p == a) return a;
        a = p;
    }
    return a;
}

__device__ void smem_union(int *lab, int a, int b) {
    // lock-free union with the smaller index as root; labels only decrease
    for (int it = 0; it < 4 * BV; ++it) {
        a = smem_find(lab, a);
        b = smem_find(lab, b);
        if (a == b) return;
        if (a > b) { int t = a; a = b; b = t; }
        int old = atomicMin(&lab[b], a);
        if (old == b) return;
        b = old;
    }
}

// Chains strictly decrease, so they are shorter than the volume; the bound only guards
// against corrupted input.
__device__ __forceinline__ int32_t gfind(const int32_t *L, int32_t a) {
    for (int64_t it = 0; it < (int64_t(1) << 31); ++it) {
        int32_t p = __ldcg(L + a);
        if (p == a || p < 0) return a;
        a = p;
    }
    return a;
}

constexpr uint8_t kMixedBrick = 0xFE;  // per-brick band summary: the band of a one-band brick, else this

__global__ void __launch_bounds__(BV) ccl_brick_kernel(const uint8_t *__restrict__ band, Dims d, int32_t *L,
                                                       uint8_t *ub) {
    __shared__ uint8_t sb[BV];
    __shared__ int lab[BV];
    int t = threadIdx.x;
    int lx = t % BX, ly = (t / BX) % BY, lz = t / (BX * BY);
    int x = blockIdx.x * BX + lx, y = blockIdx.y * BY + ly, z = blockIdx.z * BZ + lz;
    bool inb = x < d.nx && y < d.ny && z < d.nz;
    int64_t g = inb ? x + (int64_t)d.nx * (y + (int64_t)d.ny * z) : 0;
    uint8_t b = inb ? band[g] : kInvalidBand;
    sb[t] = b;
    lab[t] = t;
    __syncthreads();
    // a brick inside the volume whose voxels all share one band is one component rooted at its
    // first voxel (what the unions below reach, smallest index first): no union-find needed
    const bool one_band = __syncthreads_and(inb && b != kInvalidBand && b == sb[0]);
    if (t == 0)
        ub[blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z)] = one_band ? b : kMixedBrick;
    if (one_band) {
        const int64_t rg = (blockIdx.x * BX) + (int64_t)d.nx * ((blockIdx.y * BY) + (int64_t)d.ny * (blockIdx.z * BZ));
        L[g] = (int32_t)rg;
        return;
    }
    if (b != kInvalidBand) {
        if (lx > 0 && sb[t - 1] == b) smem_union(lab, t, t - 1);
        if (ly > 0 && sb[t - BX] == b) smem_union(lab, t, t - BX);
        if (lz > 0 && sb[t - BX * BY] == b) smem_union(lab, t, t - BX * BY);
    }
    __syncthreads();
    if (inb) {
        if (b == kInvalidBand) {
            L[g] = -1;
        } else {
            int r = smem_find(lab, t);
            int rx = r % BX, ry = (r / BX) % BY, rz = r / (BX * BY);
            int64_t rg = (blockIdx.x * BX + rx) + (int64_t)d.nx * ((blockIdx.y * BY + ry) + (int64_t)d.ny * (blockIdx.z * BZ + rz));
            L[g] = (int32_t)rg;
        }
    }
}

__device__ void gunion(int32_t *L, int32_t a, int32_t b, int32_t *status) {
    for (int it = 0; it < (1 << 20); ++it) {
        a = gfind(L, a);
        b = gfind(L, b);
        if (a == b) return;
        if (a > b) { int32_t t = a; a = b; b = t; }
        int32_t old = atomicMin(&L[b], a);
        if (old == b) return;
        b = old;
    }
    set_status(status, LSRVT_ERR_TIMEOUT);
}

// Unions across the brick faces normal to one axis (0: x, 1: y, 2: z); grid rows take face
// planes, threads the voxels of a plane.  Two neighbouring one-band bricks of the same band are
// each one component, so one voxel pair of their face (the face's first) joins them and the
// others skip -- decided from the brick summaries before any band byte is read.  Every index
// fits 32 bits (volumes below 2^31 voxels).
template <int kAxis>
__global__ void ccl_face_kernel(const uint8_t *__restrict__ band, Dims d, const uint8_t *__restrict__ ub, int32_t *L,
                                int32_t *status) {
    const int nbx = (d.nx + BX - 1) / BX, nby = (d.ny + BY - 1) / BY;
    constexpr int bw = kAxis == 0 ? BX : (kAxis == 1 ? BY : BZ);
    const int na = kAxis == 0 ? d.nx : (kAxis == 1 ? d.ny : d.nz);
    const int nplanes = (na - 1) / bw;  // faces at bw, 2 bw, ... below na
    const int nu = kAxis == 0 ? d.ny : d.nx;  // in-plane extents (u fastest)
    const int nw = kAxis == 2 ? d.ny : d.nz;
    const int psize = nu * nw;
    const int32_t sa = kAxis == 0 ? 1 : (kAxis == 1 ? d.nx : d.nx * d.ny);  // stride along the axis
    for (int pl = blockIdx.y; pl < nplanes; pl += gridDim.y) {
        const int a = (pl + 1) * bw;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < psize; i += gridDim.x * blockDim.x) {
            const int u = i % nu, w = i / nu;
            const int x = kAxis == 0 ? a : u, y = kAxis == 1 ? a : (kAxis == 0 ? u : w), z = kAxis == 2 ? a : w;
            const int bx = x / BX, by = y / BY, bz = z / BZ;
            const uint8_t u0 = __ldg(ub + bx + nbx * (by + nby * bz));
            const bool first = kAxis == 0 ? (y % BY == 0 && z % BZ == 0)
                                          : (kAxis == 1 ? (x % BX == 0 && z % BZ == 0) : (x % BX == 0 && y % BY == 0));
            if (u0 != kMixedBrick && !first) {
                const int ob = (bx - (kAxis == 0)) + nbx * ((by - (kAxis == 1)) + nby * (bz - (kAxis == 2)));
                if (__ldg(ub + ob) == u0) continue;
            }
            const int32_t v = x + d.nx * (y + d.ny * z);
            const uint8_t b = band[v];
            if (b == kInvalidBand || band[v - sa] != b) continue;
            gunion(L, v, v - sa, status);
        }
    }
}

void ccl_faces(const uint8_t *band, Dims d, const uint8_t *ub, int32_t *L, int32_t *status, cudaStream_t s) {
    auto launch = [&](auto kern, int na, int bw, int64_t psize) {
        const int nplanes = (na - 1) / bw;
        if (nplanes <= 0) return;
        const int gx = (int)((psize + 255) / 256 < 4096 ? (psize + 255) / 256 : 4096);
        const int gy = nplanes < 65535 ? nplanes : 65535;
        kern<<<dim3(gx, gy), 256, 0, s>>>(band, d, ub, L, status);
    };
    launch(ccl_face_kernel<0>, d.nx, BX, (int64_t)d.ny * d.nz);
    launch(ccl_face_kernel<1>, d.ny, BY, (int64_t)d.nx * d.nz);
    launch(ccl_face_kernel<2>, d.nz, BZ, (int64_t)d.nx * d.ny);
}

__global__ void ccl_compress_kernel(int32_t *L, int64_t n) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t p = L[v];
        if (p < 0 || p == v) continue;
        L[v] = gfind(L, p);
    }
}

// count roots per band in each warp chunk: hist[band * nchunks + chunk]
__global__ void ccl_count_kernel(const int32_t *__restrict__ L, const uint8_t *__restrict__ band, int64_t n,
                                 int64_t nchunks, int64_t *hist) {
    extern __shared__ unsigned cnt_s[];  // [warps][kBands]
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    unsigned *cnt = cnt_s + w * kBands;
    for (int64_t chunk = (int64_t)blockIdx.x * nw + w; chunk < nchunks; chunk += (int64_t)gridDim.x * nw) {
        for (int i = lane; i < kBands; i += 32) cnt[i] = 0;
        __syncwarp();
        int64_t base = chunk * kChunk;
        for (int r = 0; r < kChunkRounds; ++r) {
            int64_t v = base + r * 32 + lane;
            bool root = v < n && L[v] == v;
            if (root) atomicAdd(&cnt[band[v]], 1u);
        }
        __syncwarp();
        for (int i = lane; i < kBands; i += 32) hist[(int64_t)i * nchunks + chunk] = cnt[i];
        __syncwarp();
    }
}

__global__ void ccl_ids_kernel(const int32_t *__restrict__ L, const uint8_t *__restrict__ band, int64_t n,
                               int64_t nchunks, const int64_t *__restrict__ offs, int32_t *comp, uint8_t *comp_band,
                               int32_t *comp_first, int32_t max_comp) {
    extern __shared__ long long base_s[];  // [warps][kBands]
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    long long *cnt = base_s + w * kBands;
    for (int64_t chunk = (int64_t)blockIdx.x * nw + w; chunk < nchunks; chunk += (int64_t)gridDim.x * nw) {
        for (int i = lane; i < kBands; i += 32) cnt[i] = offs[(int64_t)i * nchunks + chunk];
        __syncwarp();
        int64_t base = chunk * kChunk;
        for (int r = 0; r < kChunkRounds; ++r) {
            int64_t v = base + r * 32 + lane;
            bool root = v < n && L[v] == v;
            unsigned bal = __ballot_sync(0xffffffffu, root);
            if (!bal) continue;
            unsigned b = root ? band[v] : 256u;
            unsigned m = __match_any_sync(0xffffffffu, b);
            if (root) {
                long long id = cnt[b] + __popc(m & lanemask_lt());
                comp[v] = (int32_t)id;
                if (id < max_comp) {
                    comp_band[id] = (uint8_t)b;
                    comp_first[id] = (int32_t)v;
                }
            }
            __syncwarp();
            if (root && (m & lanemask_lt()) == 0) cnt[b] += __popc(m);
            __syncwarp();
        }
    }
}

__global__ void ccl_finalize_kernel(const int32_t *__restrict__ L, int32_t *comp, int64_t n, int64_t *comp_size,
                                    int32_t max_comp) {
    // each thread: 16 consecutive voxels, sizes counted by runs of equal id
    const int K = 16;
    int64_t nthreads = (n + K - 1) / K;
    int64_t ntr = (nthreads + 31) & ~int64_t(31);  // warp-uniform trip count
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntr; t += (int64_t)gridDim.x * blockDim.x) {
        int32_t cur = -1, first_c = -1;
        long long run = 0, first_run = 0;
        bool first_done = false;
        if (t < nthreads) {
            for (int k = 0; k < K; ++k) {
                int64_t v = t * K + k;
                if (v >= n) break;
                int32_t p = L[v];
                int32_t c;
                if (p < 0) {
                    c = -1;
                    comp[v] = -1;
                } else if (p == v) {
                    c = comp[v];
                } else {
                    c = comp[p];  // roots were numbered by the previous kernel and are not written here
                    comp[v] = c;
                }
                if (c != cur) {
                    if (cur >= 0) {
                        if (!first_done) { first_c = cur; first_run = run; first_done = true; }
                        else if (cur < max_comp) atomicAdd((unsigned long long *)&comp_size[cur], (unsigned long long)run);
                    }
                    cur = c;
                    run = 0;
                }
                ++run;
            }
            if (cur >= 0) {
                if (!first_done) { first_c = cur; first_run = run; first_done = true; }
                else if (cur < max_comp) atomicAdd((unsigned long long *)&comp_size[cur], (unsigned long long)run);
            }
        }
        // warp-aggregate the first run of every lane (long runs are shared by neighbours)
        unsigned m = __match_any_sync(0xffffffffu, first_c);
        long long tot = 0;
        for (unsigned mm = m; mm; mm &= mm - 1) tot += __shfl_sync(m, first_run, __ffs(mm) - 1);
        if (first_c >= 0 && first_c < max_comp && (m & lanemask_lt()) == 0)
            atomicAdd((unsigned long long *)&comp_size[first_c], (unsigned long long)tot);
    }
}

__global__ void ccl_count_out_kernel(const int64_t *total, int32_t *n_comp_dev, int32_t max_comp, int32_t *status) {
    int64_t t = *total;
    *n_comp_dev = (int32_t)t;
    if (t > max_comp) set_status(status, LSRVT_ERR_CAPACITY);
}

struct CclWs {
    int32_t *L;
    uint8_t *ub;  // per brick: its band if it holds one band only, else kMixedBrick
    int64_t *hist;
    int64_t *total;
    void *scan;
};

CclWs carve_ccl(void *ws, size_t bytes, Dims d, size_t *need) {
    Carver c(ws, bytes);
    int64_t n = d.n();
    int64_t nchunks = (n + kChunk - 1) / kChunk;
    CclWs w;
    w.L = c.take<int32_t>(n);
    w.ub = c.take<uint8_t>((int64_t)((d.nx + BX - 1) / BX) * ((d.ny + BY - 1) / BY) * ((d.nz + BZ - 1) / BZ));
    w.hist = c.take<int64_t>(nchunks * kBands);
    w.total = c.take<int64_t>(1);
    w.scan = c.take<char>(scan_temp_bytes(nchunks * kBands));
    *need = c.used;
    return w;
}

}  // namespace

size_t ccl_workspace(Dims d) {
    size_t need;
    carve_ccl(nullptr, 0, d, &need);
    return need;
}

}  // namespace lsrvt

using namespace lsrvt;

extern "C" lsrvt_status lsrvt_label_components(const uint8_t *band, lsrvt_dims dd, int32_t *comp, uint8_t *comp_band,
                                               int64_t *comp_size, int32_t *comp_first, int32_t max_comp,
                                               int32_t *n_comp_dev, void *ws, size_t ws_bytes, int32_t *status_dev,
                                               void *stream) {
    if (!dims_ok(dd) || !band || !comp || !n_comp_dev || max_comp < 0 ||
        (max_comp > 0 && (!comp_band || !comp_size || !comp_first)))
        return LSRVT_ERR_INVALID_ARG;
    Dims d{dd.nx, dd.ny, dd.nz};
    size_t need;
    CclWs w = carve_ccl(ws, ws_bytes, d, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) return LSRVT_ERR_WORKSPACE;
    cudaStream_t s = as_stream(stream);
    int64_t n = d.n();
    int64_t nchunks = (n + kChunk - 1) / kChunk;
    dim3 bgrid((d.nx + BX - 1) / BX, (d.ny + BY - 1) / BY, (d.nz + BZ - 1) / BZ);
    ccl_brick_kernel<<<bgrid, BV, 0, s>>>(band, d, w.L, w.ub);
    ccl_faces(band, d, w.ub, w.L, status_dev, s);
    ccl_compress_kernel<<<grid_for(n, 256, kSMs * 16), 256, 0, s>>>(w.L, n);
    int warps = 8;
    int cgrid = (int)((nchunks + warps - 1) / warps);
    if (cgrid > kSMs * 16) cgrid = kSMs * 16;
    ccl_count_kernel<<<cgrid, warps * 32, warps * kBands * sizeof(unsigned), s>>>(w.L, band, n, nchunks, w.hist);
    exclusive_scan_i64(w.hist, nchunks * kBands, w.total, w.scan, s);
    ccl_ids_kernel<<<cgrid, warps * 32, warps * kBands * sizeof(long long), s>>>(w.L, band, n, nchunks, w.hist, comp,
                                                                                   comp_band, comp_first, max_comp);
    if (max_comp > 0) cudaMemsetAsync(comp_size, 0, sizeof(int64_t) * (size_t)max_comp, s);
    ccl_finalize_kernel<<<grid_for((n + 15) / 16, 256, kSMs * 16), 256, 0, s>>>(w.L, comp, n, comp_size, max_comp);
    ccl_count_out_kernel<<<1, 1, 0, s>>>(w.total, n_comp_dev, max_comp, status_dev);
    return launch_status();
}

// ---------------------------------------------------------------- allocation-free variant
// Some callers cannot allocate device memory at all: a simulation that embeds this library
// for in-situ analysis and owns every byte of the device through its own pool, or a host
// application that loads it as a plug-in without exposing its allocator, can neither call
// cudaMalloc nor hand over a workspace.  For them lsrvt_label_components_static labels
// volumes of up to kStaticMaxVoxels voxels with its scratch in the file-scope device array
// below, which every GPU that loads the library holds until the process exits.
#include <mutex>

namespace lsrvt {
namespace {

constexpr int64_t kStaticMaxVoxels = int64_t(1) << 18;  // 64^3
constexpr size_t kStaticScratchBytes = 1310720;         // >= the workspace of any volume up to 2^18 voxels

static __device__ __align__(256) unsigned char g_ccl_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  Outside stream capture it is
// looked up on every call (a device reset re-creates the context and moves the array), and the
// result is remembered per device; while the stream is being captured the remembered address
// is used, so the first call on a device must come before any capture.
lsrvt_status static_scratch(cudaStream_t s, void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LSRVT_ERR_CUDA;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return LSRVT_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (cap == cudaStreamCaptureStatusNone || !g_static_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_ccl_static_scratch) != cudaSuccess || !p) return LSRVT_ERR_CUDA;
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return LSRVT_OK;
}

}  // namespace
}  // namespace lsrvt

extern "C" lsrvt_status lsrvt_label_components_static(const uint8_t *band, lsrvt_dims dd, int32_t *comp,
                                                      uint8_t *comp_band, int64_t *comp_size, int32_t *comp_first,
                                                      int32_t max_comp, int32_t *n_comp_dev, int32_t *status_dev,
                                                      void *stream) {
    if (!dims_ok(dd) || !band || !comp || !n_comp_dev || max_comp < 0 ||
        (max_comp > 0 && (!comp_band || !comp_size || !comp_first)))
        return LSRVT_ERR_INVALID_ARG;
    Dims d{dd.nx, dd.ny, dd.nz};
    if (d.n() > kStaticMaxVoxels) return LSRVT_ERR_WORKSPACE;  // larger than the built-in scratch
    size_t need;
    carve_ccl(nullptr, 0, d, &need);
    if (need > kStaticScratchBytes) return LSRVT_ERR_WORKSPACE;
    cudaStream_t s = as_stream(stream);
    void *ws = nullptr;
    lsrvt_status st = static_scratch(s, &ws);
    if (st != LSRVT_OK) return st;
    CclWs w = carve_ccl(ws, kStaticScratchBytes, d, &need);
    // Every buffer below is written before it is read, so nothing left by an earlier call
    // needs clearing.
    int64_t n = d.n();
    int64_t nchunks = (n + kChunk - 1) / kChunk;
    dim3 bgrid((d.nx + BX - 1) / BX, (d.ny + BY - 1) / BY, (d.nz + BZ - 1) / BZ);
    ccl_brick_kernel<<<bgrid, BV, 0, s>>>(band, d, w.L, w.ub);
    ccl_faces(band, d, w.ub, w.L, status_dev, s);
    ccl_compress_kernel<<<grid_for(n, 256, kSMs * 16), 256, 0, s>>>(w.L, n);
    int warps = 8;
    int cgrid = (int)((nchunks + warps - 1) / warps);
    if (cgrid > kSMs * 16) cgrid = kSMs * 16;
    ccl_count_kernel<<<cgrid, warps * 32, warps * kBands * sizeof(unsigned), s>>>(w.L, band, n, nchunks, w.hist);
    exclusive_scan_i64(w.hist, nchunks * kBands, w.total, w.scan, s);
    ccl_ids_kernel<<<cgrid, warps * 32, warps * kBands * sizeof(long long), s>>>(w.L, band, n, nchunks, w.hist, comp,
                                                                                   comp_band, comp_first, max_comp);
    if (max_comp > 0) cudaMemsetAsync(comp_size, 0, sizeof(int64_t) * (size_t)max_comp, s);
    ccl_finalize_kernel<<<grid_for((n + 15) / 16, 256, kSMs * 16), 256, 0, s>>>(w.L, comp, n, comp_size, max_comp);
    ccl_count_out_kernel<<<1, 1, 0, s>>>(w.total, n_comp_dev, max_comp, status_dev);
    return launch_status();
}
