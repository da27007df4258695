// merge.cu -- statistics merged up the hierarchy cell -> component -> band -> volume
// (introduction: aggregations may be merged over Voronoi cells, connected components and
// isobands; Sec. 3.2 "Data Reduction and Structured Data Layout": the hierarchy).
//
// Children of a parent are contiguous (site ids are ordered by component, component ids
// by band), so each level is a segmented reduction over offsets.  Exact parts (count,
// min, max, histogram) use integer / ordered-float atomics, one thread per child.  The
// moments use the closed form of the pairwise update of Chan, Golub & LeVeque (1979):
//   mean = sum n_i mean_i / n,  M2 = sum (M2_i + n_i (mean_i - mean)^2),
//   C_ab = sum (C_i,ab + n_i (mean_i,a - mean_a)(mean_i,b - mean_b)),
// evaluated in FP64 with fixed reduction trees (deterministic): a warp per parent with few
// children, a CTA per parent with many.
#include "common.cuh"

namespace lsrvt {
namespace {


struct Level {
    const int64_t *count;
    const double *mean, *m2, *comom;
    const float *vmin, *vmax;
    const uint32_t *hist;
};

__global__ void parent_of_kernel(const int32_t *off32, const int64_t *off64, const int32_t *n_parent_dev,
                                 int32_t n_parent_max, int32_t *parent) {
    int32_t np = n_parent_dev ? min(*n_parent_dev, n_parent_max) : n_parent_max;
    for (int32_t p = blockIdx.x; p < np; p += gridDim.x) {
        int64_t a = off32 ? off32[p] : off64[p];
        int64_t b = off32 ? off32[p + 1] : off64[p + 1];
        for (int64_t c = a + threadIdx.x; c < b; c += blockDim.x) parent[c] = p;
    }
}

// clears the live parent rows only (rows < the device-side count)
__global__ void merge_init_kernel(lsrvt_stats out, const int32_t *n_parent_dev, int32_t n_parent_max, int32_t m,
                                  int32_t B, unsigned *omin, unsigned *omax) {
    const int32_t rows = n_parent_dev ? min(*n_parent_dev, n_parent_max) : n_parent_max;
    int64_t rm = (int64_t)rows * m;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rm; i += (int64_t)gridDim.x * blockDim.x) {
        omin[i] = float_to_ordered(__int_as_float(0x7f800000));
        omax[i] = float_to_ordered(-__int_as_float(0x7f800000));
    }
    if (B > 0 && out.hist)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rm * B; i += (int64_t)gridDim.x * blockDim.x)
            out.hist[i] = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x)
        out.count[i] = 0;
}

// Exact parts (count, min, max, histogram).  Children of a parent are contiguous, so a CTA
// takes 256 consecutive children (a thread each) and aggregates before touching memory: a warp
// combines the lanes of one parent (match on the parent id, warp reductions) and one lane
// issues the atomics; when the whole chunk has one parent (the upper levels, where few parents
// own very many children) the warps combine in shared memory first, so a parent receives one
// atomic per chunk and bin instead of one per child and bin.
constexpr int kMX = 256;

__global__ void __launch_bounds__(kMX) merge_exact_kernel(Level in, const int32_t *n_child_dev, int32_t n_child_max,
                                                          const int32_t *parent, int32_t m, int32_t B,
                                                          lsrvt_stats out, unsigned *omin, unsigned *omax,
                                                          bool shared_ok) {
    extern __shared__ unsigned msh[];  // [m * B] histogram, [m] min, [m] max, [2] count (when shared_ok)
    unsigned *sh_hist = msh, *sh_min = msh + (size_t)m * B, *sh_max = sh_min + m;
    unsigned long long *sh_cnt = reinterpret_cast<unsigned long long *>(sh_max + m + ((m * B + 2 * m) & 1));
    const int32_t nc = n_child_dev ? min(*n_child_dev, n_child_max) : n_child_max;
    const int tid = threadIdx.x;
    for (int32_t c0 = blockIdx.x * kMX; c0 < nc; c0 += gridDim.x * kMX) {
        const int32_t c = c0 + tid;
        const int64_t n = c < nc ? in.count[c] : 0;
        const int32_t p = n > 0 ? parent[c] : -1;
        const bool one = shared_ok && parent[c0] == parent[min(c0 + kMX, nc) - 1];  // parents are sorted
        if (one) {
            for (int i = tid; i < m * B; i += kMX) sh_hist[i] = 0u;
            for (int i = tid; i < m; i += kMX) {
                sh_min[i] = float_to_ordered(__int_as_float(0x7f800000));
                sh_max[i] = float_to_ordered(-__int_as_float(0x7f800000));
            }
            if (tid == 0) *sh_cnt = 0ull;
            __syncthreads();
        }
        const unsigned mk = __match_any_sync(0xffffffffu, p);
        const bool lead = p >= 0 && (mk & lanemask_lt()) == 0;
        {
            const unsigned s = __reduce_add_sync(mk, (unsigned)n);  // N < 2^31: a warp's sum fits
            if (lead) {
                if (one) atomicAdd(sh_cnt, (unsigned long long)s);
                else atomicAdd((unsigned long long *)&out.count[p], (unsigned long long)s);
            }
        }
        for (int j = 0; j < m; ++j) {
            const int64_t cj = (int64_t)c * m + j, pj = (int64_t)p * m + j;
            const unsigned lo = __reduce_min_sync(mk, n > 0 ? float_to_ordered(in.vmin[cj]) : 0xFFFFFFFFu);
            const unsigned hi = __reduce_max_sync(mk, n > 0 ? float_to_ordered(in.vmax[cj]) : 0u);
            if (lead) {
                if (one) {
                    atomicMin(&sh_min[j], lo);
                    atomicMax(&sh_max[j], hi);
                } else {
                    atomicMin(&omin[pj], lo);
                    atomicMax(&omax[pj], hi);
                }
            }
            if (B > 0 && in.hist)
                for (int b = 0; b < B; ++b) {
                    const unsigned h = __reduce_add_sync(mk, n > 0 ? in.hist[cj * B + b] : 0u);
                    if (lead && h) {
                        if (one) atomicAdd(&sh_hist[j * B + b], h);
                        else atomicAdd(&out.hist[pj * B + b], h);
                    }
                }
        }
        if (one) {
            __syncthreads();
            const int32_t pp = parent[c0];
            for (int i = tid; i < m * B; i += kMX)
                if (sh_hist[i]) atomicAdd(&out.hist[(int64_t)pp * m * B + i], sh_hist[i]);
            for (int i = tid; i < m; i += kMX) {
                atomicMin(&omin[(int64_t)pp * m + i], sh_min[i]);
                atomicMax(&omax[(int64_t)pp * m + i], sh_max[i]);
            }
            if (tid == 0 && *sh_cnt) atomicAdd((unsigned long long *)&out.count[pp], *sh_cnt);
            __syncthreads();
        }
    }
}

// Moments (Chan et al.): the parent's mean first, then M2 (and co-moments) around it, in FP64
// with fixed reduction trees (deterministic).  Variables (and co-moment entries) go in groups of
// kMG so the per-thread partial sums stay in registers.  Parents with at most kSmallKids children
// (the cell -> component level: a component holds few cells) take a warp each, with no barriers;
// larger parents (components -> bands, bands -> volume: few parents, very many children) take a
// CTA each, every thread streaming whole child rows.
constexpr int kMG = 8;
constexpr int kSmallKids = 128;

__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ long long warp_allsum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum over the CTA of the kMG values of every thread (fixed order: warp trees, then warps in
// order); every thread receives the totals
__device__ __forceinline__ void block_allsum(double *v, double (*red)[kMG], int nw) {
#pragma unroll
    for (int k = 0; k < kMG; ++k) v[k] = warp_allsum(v[k]);
    __syncthreads();
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < kMG; ++k) red[threadIdx.x >> 5][k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kMG; ++k) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += red[w][k];
        v[k] = s;
    }
}

// The moments of one parent with children [a, b).  Lanes of a group of G threads (a warp, or a
// whole CTA) step over the children; reduce(v) sums the kMG values over the group.
template <typename R>
__device__ __forceinline__ void parent_moments(const Level &in, int64_t a, int64_t b, long long n, int32_t m, bool cov,
                                               int32_t p, lsrvt_stats &out, const unsigned *omin,
                                               const unsigned *omax, double *mu, int gl, int G, R reduce) {
    const int32_t T = m * (m + 1) / 2;
    for (int j0 = 0; j0 < m; j0 += kMG) {
        const int g = m - j0 < kMG ? m - j0 : kMG;
        double v[kMG];
#pragma unroll
        for (int k = 0; k < kMG; ++k) v[k] = 0.0;
        for (int64_t c = a + gl; c < b; c += G) {
            const double nc = (double)in.count[c];
#pragma unroll
            for (int k = 0; k < kMG; ++k)
                if (k < g) v[k] += nc * in.mean[c * m + j0 + k];
        }
        reduce(v);
#pragma unroll
        for (int k = 0; k < kMG; ++k) v[k] = n > 0 ? v[k] / (double)n : 0.0;
        if (gl == 0)
#pragma unroll
            for (int k = 0; k < kMG; ++k)
                if (k < g) mu[j0 + k] = v[k];
        double mj[kMG];
#pragma unroll
        for (int k = 0; k < kMG; ++k) { mj[k] = v[k]; v[k] = 0.0; }
        for (int64_t c = a + gl; c < b; c += G) {
            const int64_t nc = in.count[c];
            if (nc == 0) continue;
#pragma unroll
            for (int k = 0; k < kMG; ++k)
                if (k < g) {
                    const double dd = in.mean[c * m + j0 + k] - mj[k];
                    v[k] += in.m2[c * m + j0 + k] + (double)nc * dd * dd;
                }
        }
        reduce(v);
        if (gl == 0)
#pragma unroll
            for (int k = 0; k < kMG; ++k) {
                if (k >= g) continue;
                const int64_t pj = (int64_t)p * m + j0 + k;
                out.mean[pj] = mj[k];
                out.m2[pj] = v[k];
                out.vmin[pj] = ordered_to_float(omin[pj]);
                out.vmax[pj] = ordered_to_float(omax[pj]);
            }
    }
    if (!cov || !in.comom || !out.comom) return;
    for (int t0 = 0; t0 < T; t0 += kMG) {
        const int g = T - t0 < kMG ? T - t0 : kMG;
        // the (i, j) of entry t0 + k (upper triangle, rows in order)
        int ii[kMG], jj[kMG];
        {
            int t = 0, i = 0, j = 0;
            while (t < t0) { ++t; if (++j == m) { ++i; j = i; } }
#pragma unroll
            for (int k = 0; k < kMG; ++k) {
                ii[k] = i; jj[k] = j;
                if (k < g - 1 && ++j == m) { ++i; j = i; }
            }
        }
        double v[kMG];
#pragma unroll
        for (int k = 0; k < kMG; ++k) v[k] = 0.0;
        for (int64_t c = a + gl; c < b; c += G) {
            const int64_t nc = in.count[c];
            if (nc == 0) continue;
#pragma unroll
            for (int k = 0; k < kMG; ++k)
                if (k < g)
                    v[k] += in.comom[c * T + t0 + k] +
                            (double)nc * (in.mean[c * m + ii[k]] - mu[ii[k]]) * (in.mean[c * m + jj[k]] - mu[jj[k]]);
        }
        reduce(v);
        if (gl == 0)
#pragma unroll
            for (int k = 0; k < kMG; ++k)
                if (k < g) out.comom[(int64_t)p * T + t0 + k] = v[k];
    }
}

__global__ void __launch_bounds__(256) merge_small_kernel(Level in, const int32_t *off32, const int64_t *off64,
                                                           const int32_t *n_parent_dev, int32_t n_parent_max,
                                                           int32_t m, bool cov, lsrvt_stats out,
                                                           const unsigned *omin, const unsigned *omax) {
    __shared__ double mu_s[256 / 32][64];
    const int32_t np = n_parent_dev ? min(*n_parent_dev, n_parent_max) : n_parent_max;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double *mu = mu_s[w];
    for (int32_t p = blockIdx.x * (blockDim.x >> 5) + w; p < np; p += gridDim.x * (blockDim.x >> 5)) {
        const int64_t a = off32 ? off32[p] : off64[p], b = off32 ? off32[p + 1] : off64[p + 1];
        if (b - a > kSmallKids) continue;  // warp-uniform
        long long nl = 0;
        for (int64_t c = a + lane; c < b; c += 32) nl += in.count[c];
        const long long n = warp_allsum_ll(nl);
        parent_moments(in, a, b, n, m, cov, p, out, omin, omax, mu, lane, 32, [&](double *v) {
#pragma unroll
            for (int k = 0; k < kMG; ++k) v[k] = warp_allsum(v[k]);
            __syncwarp();
        });
        __syncwarp();
    }
}

__global__ void __launch_bounds__(256) merge_large_kernel(Level in, const int32_t *off32, const int64_t *off64,
                                                           const int32_t *n_parent_dev, int32_t n_parent_max,
                                                           int32_t m, bool cov, lsrvt_stats out,
                                                           const unsigned *omin, const unsigned *omax) {
    __shared__ double red[256 / 32][kMG];
    __shared__ double mu[64];
    __shared__ long long redl[256 / 32];
    const int32_t np = n_parent_dev ? min(*n_parent_dev, n_parent_max) : n_parent_max;
    const int nw = blockDim.x >> 5;
    for (int32_t p = blockIdx.x; p < np; p += gridDim.x) {
        const int64_t a = off32 ? off32[p] : off64[p], b = off32 ? off32[p + 1] : off64[p + 1];
        if (b - a <= kSmallKids) continue;  // CTA-uniform
        long long nl = 0;
        for (int64_t c = a + threadIdx.x; c < b; c += blockDim.x) nl += in.count[c];
        nl = warp_allsum_ll(nl);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) redl[threadIdx.x >> 5] = nl;
        __syncthreads();
        long long n = 0;
        for (int k = 0; k < nw; ++k) n += redl[k];
        parent_moments(in, a, b, n, m, cov, p, out, omin, omax, mu, threadIdx.x, blockDim.x,
                       [&](double *v) { block_allsum(v, red, nw); });
        __syncthreads();
    }
}

__global__ void band_offsets_kernel(const uint8_t *comp_band, const int32_t *n_comp_dev, int32_t max_comp,
                                    int32_t n_bands, int64_t *band_off) {
    // band_off[b] = first component id of band b (components are ordered by band)
    int32_t nc = min(*n_comp_dev, max_comp);
    for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b <= n_bands; b += gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = nc;  // first c with comp_band[c] >= b
        while (lo < hi) {
            int32_t mid = (lo + hi) / 2;
            if ((int32_t)comp_band[mid] < b) lo = mid + 1;
            else hi = mid;
        }
        band_off[b] = lo;
    }
}

__global__ void volume_offsets_kernel(int64_t *off, int32_t n) {
    off[0] = 0;
    off[1] = n;
}

Level as_level(lsrvt_stats s) { return Level{s.count, s.mean, s.m2, s.comom, s.vmin, s.vmax, s.hist}; }

struct MergeWs {
    int32_t *parent;
    unsigned *omin, *omax;
    int64_t *band_off;
    int64_t *vol_off;
};

MergeWs carve_merge(void *ws, size_t bytes, int32_t max_sites, int32_t max_comp, int32_t n_bands, int32_t m,
                    size_t *need) {
    Carver c(ws, bytes);
    MergeWs w;
    int64_t rows = max_sites > max_comp ? max_sites : max_comp;
    if (rows < n_bands) rows = n_bands;
    w.parent = c.take<int32_t>(rows + 1);
    int64_t pm = (int64_t)(max_comp > n_bands ? max_comp : n_bands) * (m > 0 ? m : 1) + 64;
    w.omin = c.take<unsigned>(pm);
    w.omax = c.take<unsigned>(pm);
    w.band_off = c.take<int64_t>(n_bands + 1);
    w.vol_off = c.take<int64_t>(2);
    *need = c.used;
    return w;
}

void merge_level(lsrvt_stats child, const int32_t *n_child_dev, int32_t n_child_max, const int32_t *off32,
                 const int64_t *off64, const int32_t *n_parent_dev, int32_t n_parent_max, int32_t m, int32_t B,
                 bool cov, lsrvt_stats parent_out, MergeWs &w, cudaStream_t s) {
    parent_of_kernel<<<kSMs * 4, 128, 0, s>>>(off32, off64, n_parent_dev, n_parent_max, w.parent);
    merge_init_kernel<<<kSMs * 8, 256, 0, s>>>(parent_out, n_parent_dev, n_parent_max, m, B, w.omin, w.omax);
    const size_t xsm = sizeof(unsigned) * ((size_t)m * B + 2 * m + 4);
    const bool shared_ok = xsm <= 48 * 1024;
    merge_exact_kernel<<<grid_for(n_child_max, kMX, kSMs * 8), kMX, shared_ok ? xsm : 0, s>>>(
        as_level(child), n_child_dev, n_child_max, w.parent, m, B, parent_out, w.omin, w.omax, shared_ok);
    merge_small_kernel<<<grid_for((int64_t)n_parent_max * 32, 256, kSMs * 8), 256, 0, s>>>(
        as_level(child), off32, off64, n_parent_dev, n_parent_max, m, cov, parent_out, w.omin, w.omax);
    merge_large_kernel<<<kSMs * 2, 256, 0, s>>>(as_level(child), off32, off64, n_parent_dev, n_parent_max, m, cov,
                                                parent_out, w.omin, w.omax);
}

}  // namespace

size_t merge_workspace(int32_t max_sites, int32_t max_comp, int32_t n_bands, int32_t m) {
    size_t need;
    carve_merge(nullptr, 0, max_sites, max_comp, n_bands, m, &need);
    return need;
}

}  // namespace lsrvt

using namespace lsrvt;

extern "C" lsrvt_status lsrvt_merge_hierarchy(lsrvt_stats cells, const int32_t *n_sites_dev, int32_t max_sites,
                                              int32_t n_aux, int32_t n_bins, uint32_t flags,
                                              const int32_t *comp_site_off, const uint8_t *comp_band,
                                              const int32_t *n_comp_dev, int32_t max_comp, int32_t n_bands,
                                              lsrvt_stats comps, lsrvt_stats bands, lsrvt_stats volume, void *ws,
                                              size_t ws_bytes, void *stream) {
    bool hist = (flags & LSRVT_STATS_HIST) && n_bins > 0;
    bool cov = (flags & LSRVT_STATS_COV) != 0;
    if (n_aux < 0 || n_aux > 64 || n_bins < 0 || !n_sites_dev || max_sites < 0 || !comp_site_off || !comp_band ||
        !n_comp_dev || max_comp < 0 || n_bands < 1 || n_bands > 255 || !cells.count || !comps.count ||
        !bands.count || !volume.count)
        return LSRVT_ERR_INVALID_ARG;
    if (n_aux > 0) {
        lsrvt_stats *all[4] = {&cells, &comps, &bands, &volume};
        for (auto *st : all) {
            if (!st->mean || !st->m2 || !st->vmin || !st->vmax) return LSRVT_ERR_INVALID_ARG;
            if (hist && !st->hist) return LSRVT_ERR_INVALID_ARG;
            if (cov && !st->comom) return LSRVT_ERR_INVALID_ARG;
        }
    }
    size_t need;
    MergeWs w = carve_merge(ws, ws_bytes, max_sites, max_comp, n_bands, n_aux, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) return LSRVT_ERR_WORKSPACE;
    cudaStream_t s = as_stream(stream);
    int32_t B = hist ? n_bins : 0;
    merge_level(cells, n_sites_dev, max_sites, comp_site_off, nullptr, n_comp_dev, max_comp, n_aux, B, cov, comps, w, s);
    band_offsets_kernel<<<1, 256, 0, s>>>(comp_band, n_comp_dev, max_comp, n_bands, w.band_off);
    merge_level(comps, n_comp_dev, max_comp, nullptr, w.band_off, nullptr, n_bands, n_aux, B, cov, bands, w, s);
    volume_offsets_kernel<<<1, 1, 0, s>>>(w.vol_off, n_bands);
    merge_level(bands, nullptr, n_bands, nullptr, w.vol_off, nullptr, 1, n_aux, B, cov, volume, w, s);
    return launch_status();
}
