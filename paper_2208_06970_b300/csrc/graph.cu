// graph.cu -- Voronoi site graph and geodesic site distances ("Voronoi Cell Views" section of the
// paper: the connectivity of the sites from region adjacency, shortest paths between adjacent
// sites restricted to the component, and the distance ||x_i - x_j|| / gd(s_i, s_j), or c where
// no path exists).
//
// Two cells are adjacent when a voxel of one and a voxel of the other are face neighbours of one
// band (6-adjacency; such voxels lie in one component).  The edge weight between sites a and b
// is ceil(2^16 ||x_a - x_b||_2), an integer, so path lengths are exact sums and the result does
// not depend on the relaxation order.
//
// Graph build: one CTA per 16x8x8 brick collects the (a, b) pairs of its voxels' +x/+y/+z
// faces in a shared-memory hash set (duplicates inside the brick folded), appends them to a
// global candidate list; two stable radix sorts (by b, then a) order them, adjacent duplicates
// are dropped, weights computed, and the arcs of both directions sorted by (source, target)
// into a CSR.  Geodesics: one CTA per source site runs Bellman-Ford over frontier bitmaps
// (bounded rounds) inside a site range closed under adjacency (a union of components).
#include <math.h>

#include "common.cuh"

namespace lsrvt {
namespace {

constexpr int kGX = 16, kGY = 8, kGZ = 8, kGV = kGX * kGY * kGZ;  // brick
constexpr int kGThreads = 256;
constexpr int kGHash = 2048;  // pair slots per brick (3 * 1024 faces at most)
constexpr unsigned long long kGEmpty = ~0ULL;

__device__ __forceinline__ uint32_t site_weight(int dx, int dy, int dz) {
    // ceil(2^16 sqrt(D)) = smallest w with w^2 >= 2^32 D; the double root is within one of it
    const unsigned long long D = (unsigned long long)((long long)dx * dx + (long long)dy * dy + (long long)dz * dz);
    const unsigned long long v = D << 32;
    unsigned long long r = (unsigned long long)sqrt((double)v);
    while (r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return (uint32_t)(r * r == v ? r : r + 1);
}

__global__ void __launch_bounds__(kGThreads) graph_candidates_kernel(const int32_t *__restrict__ cell,
                                                                      const uint8_t *__restrict__ band, Dims d,
                                                                      int32_t ns, uint32_t *ca, uint32_t *cb,
                                                                      int64_t cap, unsigned long long *n_cand,
                                                                      int32_t *status) {
    __shared__ unsigned long long set[kGHash];
    __shared__ int cnt_s;
    __shared__ unsigned long long base_s;
    const int nbx = (d.nx + kGX - 1) / kGX, nby = (d.ny + kGY - 1) / kGY, nbz = (d.nz + kGZ - 1) / kGZ;
    const int64_t nbricks = (int64_t)nbx * nby * nbz;
    const int64_t sxy = (int64_t)d.nx * d.ny;
    for (int64_t brick = blockIdx.x; brick < nbricks; brick += gridDim.x) {
        const int bx = (int)(brick % nbx), by = (int)((brick / nbx) % nby), bz = (int)(brick / ((int64_t)nbx * nby));
        for (int i = threadIdx.x; i < kGHash; i += kGThreads) set[i] = kGEmpty;
        if (threadIdx.x == 0) cnt_s = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < kGV; i += kGThreads) {
            const int x = bx * kGX + (i % kGX), y = by * kGY + (i / kGX) % kGY, z = bz * kGZ + i / (kGX * kGY);
            if (x >= d.nx || y >= d.ny || z >= d.nz) continue;
            const int64_t v = x + (int64_t)d.nx * y + sxy * z;
            const int32_t s = __ldg(cell + v);
            if (s < 0) continue;
            if (s >= ns) {
                set_status(status, LSRVT_ERR_INVALID_ARG);
                continue;
            }
            const uint8_t b = __ldg(band + v);
            const int64_t nb[3] = {x + 1 < d.nx ? v + 1 : -1, y + 1 < d.ny ? v + d.nx : -1, z + 1 < d.nz ? v + sxy : -1};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (nb[k] < 0) continue;
                const int32_t t = __ldg(cell + nb[k]);
                if (t < 0 || t == s || t >= ns || __ldg(band + nb[k]) != b) continue;
                const unsigned long long key = ((unsigned long long)(uint32_t)min(s, t) << 32) | (uint32_t)max(s, t);
                // open addressing; a full probe sequence appends the pair directly (duplicates
                // across bricks are dropped after the global sort anyway)
                unsigned h = (unsigned)((key * 0x9E3779B97F4A7C15ULL) >> 53) & (kGHash - 1);
                bool placed = false;
                for (int probe = 0; probe < 32; ++probe) {
                    const unsigned long long old = atomicCAS(&set[h], kGEmpty, key);
                    if (old == kGEmpty || old == key) {
                        placed = true;
                        break;
                    }
                    h = (h + 1) & (kGHash - 1);
                }
                if (!placed) {
                    const unsigned long long at = atomicAdd(n_cand, 1ULL);
                    if ((int64_t)at < cap) {
                        ca[at] = (uint32_t)(key >> 32);
                        cb[at] = (uint32_t)key;
                    } else {
                        set_status(status, LSRVT_ERR_CAPACITY);
                    }
                }
            }
        }
        __syncthreads();
        // compact the set and append it with one global atomic
        for (int i = threadIdx.x; i < kGHash; i += kGThreads)
            if (set[i] != kGEmpty) atomicAdd(&cnt_s, 1);
        __syncthreads();
        if (threadIdx.x == 0) base_s = cnt_s ? atomicAdd(n_cand, (unsigned long long)cnt_s) : 0ULL;
        if (threadIdx.x == 0) cnt_s = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < kGHash; i += kGThreads) {
            const unsigned long long key = set[i];
            if (key == kGEmpty) continue;
            const unsigned long long at = base_s + (unsigned long long)atomicAdd(&cnt_s, 1);
            if ((int64_t)at < cap) {
                ca[at] = (uint32_t)(key >> 32);
                cb[at] = (uint32_t)key;
            } else {
                set_status(status, LSRVT_ERR_CAPACITY);
            }
        }
        __syncthreads();
    }
}

__global__ void graph_count_kernel(const unsigned long long *n_cand, int64_t cap, int32_t *n32, int64_t *n64) {
    const int64_t n = (int64_t)min((unsigned long long)cap, *n_cand);
    *n32 = (int32_t)n;
    *n64 = n;
}

// 1 where (a, b) differs from its predecessor in the sorted list
__global__ void graph_unique_flags_kernel(const uint32_t *a, const uint32_t *b, const int64_t *n_dev, int64_t *flag) {
    const int64_t n = *n_dev;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || a[i] != a[i - 1] || b[i] != b[i - 1]) ? 1 : 0;
}

// unique edges -> both arcs: arc 2k = (a, b), arc 2k+1 = (b, a)
__global__ void graph_arcs_kernel(const uint32_t *a, const uint32_t *b, const int64_t *n_dev,
                                  const int64_t *__restrict__ pos, uint32_t *src, uint32_t *dst) {
    const int64_t n = *n_dev;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!(i == 0 || a[i] != a[i - 1] || b[i] != b[i - 1])) continue;
        const int64_t k = pos[i];
        src[2 * k] = a[i];
        dst[2 * k] = b[i];
        src[2 * k + 1] = b[i];
        dst[2 * k + 1] = a[i];
    }
}

__global__ void graph_edges_total_kernel(const int64_t *n_edges, int64_t *n_arcs, int32_t *n_arcs32) {
    *n_arcs = 2 * *n_edges;
    *n_arcs32 = (int32_t)(2 * *n_edges);
}

// CSR offsets (first arc with source >= s) and arc weights
__global__ void graph_csr_kernel(const uint32_t *__restrict__ src, const uint32_t *__restrict__ dst,
                                 const int64_t *n_arcs_dev, const int32_t *__restrict__ site_pos, Dims d,
                                 const int32_t *n_sites_dev, int32_t max_sites, int64_t max_arcs, int64_t *off,
                                 int32_t *adj, uint32_t *w, int32_t *status) {
    const int32_t ns = min(max(*n_sites_dev, 0), max_sites);  // rows past the live sites are empty
    const int64_t n_all = *n_arcs_dev;
    if (n_all > max_arcs && blockIdx.x == 0 && threadIdx.x == 0) set_status(status, LSRVT_ERR_CAPACITY);
    const int64_t n = n_all < max_arcs ? n_all : max_arcs;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t s = t0; s <= max_sites; s += stride) {
        if (s > ns) {
            off[s] = n;
            continue;
        }
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (src[mid] < (uint32_t)s) lo = mid + 1;
            else hi = mid;
        }
        off[s] = lo;
    }
    for (int64_t i = t0; i < n; i += stride) {
        const int32_t a = (int32_t)src[i], b = (int32_t)dst[i];
        const int32_t pa = site_pos[a], pb = site_pos[b];
        const int ax = pa % d.nx, ay = (pa / d.nx) % d.ny, az = pa / (d.nx * d.ny);
        const int bx = pb % d.nx, by = (pb / d.nx) % d.ny, bz = pb / (d.nx * d.ny);
        adj[i] = b;
        w[i] = site_weight(bx - ax, by - ay, bz - az);
    }
}

struct GraphWs {
    uint32_t *ca, *cb, *src, *dst;  // candidates (cap), arcs (2 cap: two per unique edge)
    unsigned long long *n_cand;
    int32_t *n32, *n_arcs32;
    int64_t *n64, *flag, *n_edges, *n_arcs;
    void *scan, *radix;
};

GraphWs carve_graph(void *ws, size_t bytes, int64_t cap, size_t *need) {
    Carver c(ws, bytes);
    GraphWs w;
    w.ca = c.take<uint32_t>(cap);
    w.cb = c.take<uint32_t>(cap);
    w.src = c.take<uint32_t>(2 * cap);
    w.dst = c.take<uint32_t>(2 * cap);
    w.n_cand = c.take<unsigned long long>(1);
    w.n32 = c.take<int32_t>(1);
    w.n_arcs32 = c.take<int32_t>(1);
    w.n64 = c.take<int64_t>(1);
    w.n_edges = c.take<int64_t>(1);
    w.n_arcs = c.take<int64_t>(1);
    w.flag = c.take<int64_t>(cap);
    w.scan = c.take<char>(scan_temp_bytes(cap));
    w.radix = c.take<char>(radix_temp_bytes(2 * cap));
    *need = c.used;
    return w;
}

// ---------------------------------------------------------------- geodesics
constexpr int kSThreads = 256;
constexpr unsigned kSInf = 0xFFFFFFFFu;

// One CTA per source: Bellman-Ford over frontier bitmaps within [s0, s1).  Arcs that leave
// the range are reported (the range must be closed under adjacency).  At most k rounds.  With
// kShared the distance row and both bitmaps live in shared memory (ranges up to kSharedMax
// sites) and the row is copied out at the end; otherwise they live in global memory.
constexpr int kSharedMax = 12000;  // distance row + frontier list + bitmaps: 8 k + k / 4 bytes

template <bool kShared>
__global__ void __launch_bounds__(kSThreads) graph_sssp_kernel(const int64_t *__restrict__ off,
                                                                const int32_t *__restrict__ adj,
                                                                const uint32_t *__restrict__ w, int32_t s0,
                                                                int32_t s1, uint32_t *dist, uint32_t *fa,
                                                                uint32_t *fb, const int32_t *__restrict__ site_pos,
                                                                Dims d, float c_far, float *ratio, int32_t *status) {
    extern __shared__ uint32_t dyn[];
    __shared__ int any_s, nlist_s;
    const int k = s1 - s0;
    const int nw = (k + 31) / 32;
    uint32_t *cur = kShared ? dyn + k : fa + (int64_t)blockIdx.x * nw;
    uint32_t *nxt = kShared ? dyn + k + nw : fb + (int64_t)blockIdx.x * nw;
    for (int src = blockIdx.x; src < k; src += gridDim.x) {
        uint32_t *row = dist + (int64_t)src * k;
        uint32_t *D = kShared ? dyn : row;
        for (int i = threadIdx.x; i < k; i += kSThreads) D[i] = i == src ? 0u : kSInf;
        for (int i = threadIdx.x; i < nw; i += kSThreads) {
            cur[i] = i == (src >> 5) ? (1u << (src & 31)) : 0u;
            nxt[i] = 0u;
        }
        __syncthreads();
        for (int round = 0; round <= k; ++round) {
            if (threadIdx.x == 0) any_s = 0;
            __syncthreads();
            // relax the arcs of frontier node u (the latest distance of u is read atomically)
            auto relax = [&](int u) {
                const uint32_t du = atomicAdd(&D[u], 0u);
                const int64_t e0 = off[s0 + u], e1 = off[s0 + u + 1];
                for (int64_t e = e0; e < e1; ++e) {
                    const int t = adj[e] - s0;
                    if (t < 0 || t >= k) {
                        set_status(status, LSRVT_ERR_INVALID_ARG);
                        continue;
                    }
                    const unsigned long long nd = (unsigned long long)du + w[e];
                    if (nd >= kSInf) {
                        set_status(status, LSRVT_ERR_OVERFLOW);
                        continue;
                    }
                    if ((uint32_t)nd < atomicMin(&D[t], (uint32_t)nd)) {
                        atomicOr(&nxt[t >> 5], 1u << (t & 31));
                        any_s = 1;
                    }
                }
            };
            if (kShared) {
                // the frontier as a list, so every thread takes whole nodes (frontier bits cluster
                // in a few words: site ids are ordered in space)
                int *list = reinterpret_cast<int *>(dyn + k + 2 * nw);
                if (threadIdx.x == 0) nlist_s = 0;
                __syncthreads();
                for (int wi = threadIdx.x; wi < nw; wi += kSThreads) {
                    uint32_t bits = cur[wi];
                    if (!bits) continue;
                    int at = atomicAdd(&nlist_s, __popc(bits));
                    while (bits) {
                        list[at++] = wi * 32 + __ffs(bits) - 1;
                        bits &= bits - 1;
                    }
                }
                __syncthreads();
                const int nl = nlist_s;
                for (int li = threadIdx.x; li < nl; li += kSThreads) relax(list[li]);
            } else {
                for (int wi = threadIdx.x; wi < nw; wi += kSThreads) {
                    uint32_t bits = cur[wi];
                    while (bits) {
                        const int u = wi * 32 + __ffs(bits) - 1;
                        bits &= bits - 1;
                        relax(u);
                    }
                }
            }
            __syncthreads();
            const bool more = any_s != 0;
            uint32_t *tmp = cur;
            cur = nxt;
            nxt = tmp;
            for (int i = threadIdx.x; i < nw; i += kSThreads) nxt[i] = 0u;
            __syncthreads();
            if (!more) break;
            if (round == k && threadIdx.x == 0) set_status(status, LSRVT_ERR_TIMEOUT);
        }
        if (kShared)
            for (int i = threadIdx.x; i < k; i += kSThreads) row[i] = D[i];
        if (ratio) {
            const int32_t ps = site_pos[s0 + src];
            const int sx = ps % d.nx, sy = (ps / d.nx) % d.ny, sz = ps / (d.nx * d.ny);
            for (int i = threadIdx.x; i < k; i += kSThreads) {
                const uint32_t g = D[i];
                float r;
                if (i == src) {
                    r = 1.f;
                } else if (g == kSInf) {
                    r = c_far;
                } else {
                    const int32_t pt = site_pos[s0 + i];
                    const float dx = (float)(pt % d.nx - sx), dy = (float)((pt / d.nx) % d.ny - sy),
                                dz = (float)(pt / (d.nx * d.ny) - sz);
                    r = sqrtf(dx * dx + dy * dy + dz * dz) * 65536.f / (float)g;
                }
                ratio[(int64_t)src * k + i] = r;
            }
        }
        __syncthreads();
    }
}

}  // namespace

int64_t graph_candidate_cap(Dims d) {
    const int64_t n = d.n();
    const int64_t a = n / 8 > (1 << 20) ? n / 8 : (1 << 20);
    return a < 3 * n ? a : 3 * n;
}

size_t graph_workspace(Dims d) {
    size_t need;
    carve_graph(nullptr, 0, graph_candidate_cap(d), &need);
    return need;
}

size_t geodesic_workspace(int32_t k, int grid) {
    const int64_t nw = (k + 31) / 32;
    return (size_t)(2 * grid * nw) * sizeof(uint32_t) + 512;
}

}  // namespace lsrvt

using namespace lsrvt;

extern "C" lsrvt_status lsrvt_site_graph(const int32_t *cell, const uint8_t *band, lsrvt_dims dd,
                                         const int32_t *site_pos, const int32_t *n_sites_dev, int32_t max_sites,
                                         int64_t *adj_off, int32_t *adj, uint32_t *adj_w, int64_t max_arcs,
                                         int64_t *n_edges_dev, void *ws, size_t ws_bytes, int32_t *status_dev,
                                         void *stream) {
    if (!dims_ok(dd) || !cell || !band || !site_pos || !n_sites_dev || max_sites < 0 || !adj_off || !adj || !adj_w ||
        max_arcs < 0 || !n_edges_dev)
        return LSRVT_ERR_INVALID_ARG;
    const Dims d{dd.nx, dd.ny, dd.nz};
    const int64_t cap = graph_candidate_cap(d);
    size_t need;
    GraphWs w = carve_graph(ws, ws_bytes, cap, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) return LSRVT_ERR_WORKSPACE;
    cudaStream_t s = as_stream(stream);
    const int sms = stream_sms(s);
    // cell ids are checked against the site capacity (an id beyond it is an argument error)
    cudaMemsetAsync(w.n_cand, 0, sizeof(unsigned long long), s);
    graph_candidates_kernel<<<sms * 4, kGThreads, 0, s>>>(cell, band, d, max_sites, w.ca, w.cb, cap, w.n_cand,
                                                          status_dev);
    graph_count_kernel<<<1, 1, 0, s>>>(w.n_cand, cap, w.n32, w.n64);
    int bits = 0;
    while (bits < 31 && ((int64_t)1 << bits) < max_sites) ++bits;
    radix_sort_pairs(w.cb, w.ca, cap, w.n32, bits, w.radix, s);  // by b
    radix_sort_pairs(w.ca, w.cb, cap, w.n32, bits, w.radix, s);  // then by a, stable: (a, b) order
    graph_unique_flags_kernel<<<sms * 8, 256, 0, s>>>(w.ca, w.cb, w.n64, w.flag);
    exclusive_scan_i64_dev(w.flag, cap, w.n64, n_edges_dev, w.scan, s);
    graph_arcs_kernel<<<sms * 8, 256, 0, s>>>(w.ca, w.cb, w.n64, w.flag, w.src, w.dst);
    graph_edges_total_kernel<<<1, 1, 0, s>>>(n_edges_dev, w.n_arcs, w.n_arcs32);
    // arcs by (source, target): sort by target, then by source (stable)
    radix_sort_pairs(w.dst, w.src, 2 * cap, w.n_arcs32, bits, w.radix, s);
    radix_sort_pairs(w.src, w.dst, 2 * cap, w.n_arcs32, bits, w.radix, s);
    // the CSR itself: offsets over max_sites + 1 rows, arcs up to max_arcs
    graph_csr_kernel<<<sms * 8, 256, 0, s>>>(w.src, w.dst, w.n_arcs, site_pos, d, n_sites_dev, max_sites, max_arcs,
                                             adj_off, adj, adj_w, status_dev);
    return launch_status();
}

extern "C" lsrvt_status lsrvt_site_geodesics(const int64_t *adj_off, const int32_t *adj, const uint32_t *adj_w,
                                             const int32_t *site_pos, lsrvt_dims dd, int32_t s0, int32_t s1,
                                             uint32_t *dist, float *ratio, float c_far, void *ws, size_t ws_bytes,
                                             int32_t *status_dev, void *stream) {
    if (!adj_off || !adj || !adj_w || s0 < 0 || s1 < s0 || !dist || (ratio && (!site_pos || !dims_ok(dd))))
        return LSRVT_ERR_INVALID_ARG;
    const int k = s1 - s0;
    if (k == 0) return LSRVT_OK;
    cudaStream_t s = as_stream(stream);
    const int sms = stream_sms(s);
    const int grid = k < sms * 4 ? k : sms * 4;
    const size_t need = geodesic_workspace(k, grid);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) return LSRVT_ERR_WORKSPACE;
    const int64_t nw = (k + 31) / 32;
    uint32_t *fa = reinterpret_cast<uint32_t *>(ws), *fb = fa + (int64_t)grid * nw;
    const Dims d{dd.nx > 0 ? dd.nx : 1, dd.ny > 0 ? dd.ny : 1, dd.nz > 0 ? dd.nz : 1};
    if (k <= kSharedMax) {
        const size_t smem = (size_t)(2 * k + 2 * nw) * sizeof(uint32_t);
        cudaFuncSetAttribute(graph_sssp_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        graph_sssp_kernel<true><<<grid, kSThreads, smem, s>>>(adj_off, adj, adj_w, s0, s1, dist, fa, fb, site_pos, d,
                                                              c_far, ratio, status_dev);
    } else {
        graph_sssp_kernel<false><<<grid, kSThreads, 0, s>>>(adj_off, adj, adj_w, s0, s1, dist, fa, fb, site_pos, d,
                                                               c_far, ratio, status_dev);
    }
    return launch_status();
}
