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
// evaluated in FP64 by one CTA per parent with a fixed reduction tree (deterministic).
#include "common.cuh"

namespace lsrvt {
namespace {

constexpr int kMergeThreads = 128;

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

__global__ void merge_exact_kernel(Level in, const int32_t *n_child_dev, int32_t n_child_max, const int32_t *parent,
                                   int32_t m, int32_t B, lsrvt_stats out, unsigned *omin, unsigned *omax) {
    int32_t nc = n_child_dev ? min(*n_child_dev, n_child_max) : n_child_max;
    int64_t per = (int64_t)(m > 0 ? m : 1);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)nc * per;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = (int32_t)(i / per);
        int32_t j = (int32_t)(i - (int64_t)c * per);
        int64_t n = in.count[c];
        if (n == 0) continue;
        int32_t p = parent[c];
        if (j == 0) atomicAdd((unsigned long long *)&out.count[p], (unsigned long long)n);
        if (m == 0) continue;
        int64_t cj = (int64_t)c * m + j, pj = (int64_t)p * m + j;
        atomicMin(&omin[pj], float_to_ordered(in.vmin[cj]));
        atomicMax(&omax[pj], float_to_ordered(in.vmax[cj]));
        if (B > 0 && in.hist)
            for (int b = 0; b < B; ++b) {
                uint32_t h = in.hist[cj * B + b];
                if (h) atomicAdd(&out.hist[pj * B + b], h);
            }
    }
}

__device__ double block_sum_d(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    return s;
}

__device__ long long block_sum_ll(long long v, long long *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    long long s = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    return s;
}

__global__ void __launch_bounds__(kMergeThreads) merge_moments_kernel(Level in, const int32_t *off32,
                                                                       const int64_t *off64, const int32_t *n_parent_dev,
                                                                       int32_t n_parent_max, int32_t m, bool cov,
                                                                       lsrvt_stats out, const unsigned *omin,
                                                                       const unsigned *omax) {
    __shared__ double red[kMergeThreads / 32];
    __shared__ long long redl[kMergeThreads / 32];
    __shared__ double mu[64];
    int32_t np = n_parent_dev ? min(*n_parent_dev, n_parent_max) : n_parent_max;
    int32_t T = m * (m + 1) / 2;
    for (int32_t p = blockIdx.x; p < np; p += gridDim.x) {
        int64_t a = off32 ? off32[p] : off64[p];
        int64_t b = off32 ? off32[p + 1] : off64[p + 1];
        long long nloc = 0;
        for (int64_t c = a + threadIdx.x; c < b; c += blockDim.x) nloc += in.count[c];
        long long n = block_sum_ll(nloc, redl);
        for (int j = 0; j < m; ++j) {
            double s = 0.0;
            for (int64_t c = a + threadIdx.x; c < b; c += blockDim.x) s += (double)in.count[c] * in.mean[c * m + j];
            s = block_sum_d(s, red);
            double meanj = n > 0 ? s / (double)n : 0.0;
            if (threadIdx.x == 0) mu[j] = meanj;
            double q = 0.0;
            for (int64_t c = a + threadIdx.x; c < b; c += blockDim.x) {
                int64_t nc = in.count[c];
                if (nc == 0) continue;
                double dd = in.mean[c * m + j] - meanj;
                q += in.m2[c * m + j] + (double)nc * dd * dd;
            }
            q = block_sum_d(q, red);
            if (threadIdx.x == 0) {
                out.mean[(int64_t)p * m + j] = meanj;
                out.m2[(int64_t)p * m + j] = q;
                out.vmin[(int64_t)p * m + j] = ordered_to_float(omin[(int64_t)p * m + j]);
                out.vmax[(int64_t)p * m + j] = ordered_to_float(omax[(int64_t)p * m + j]);
            }
        }
        __syncthreads();
        if (cov && in.comom && out.comom) {
            int t = 0;
            for (int i = 0; i < m; ++i)
                for (int j = i; j < m; ++j, ++t) {
                    double q = 0.0;
                    for (int64_t c = a + threadIdx.x; c < b; c += blockDim.x) {
                        int64_t nc = in.count[c];
                        if (nc == 0) continue;
                        q += in.comom[c * T + t] + (double)nc * (in.mean[c * m + i] - mu[i]) * (in.mean[c * m + j] - mu[j]);
                    }
                    q = block_sum_d(q, red);
                    if (threadIdx.x == 0) out.comom[(int64_t)p * T + t] = q;
                }
        }
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
    merge_exact_kernel<<<grid_for((int64_t)n_child_max * (m > 0 ? m : 1), 256, kSMs * 8), 256, 0, s>>>(
        as_level(child), n_child_dev, n_child_max, w.parent, m, B, parent_out, w.omin, w.omax);
    merge_moments_kernel<<<kSMs * 4, kMergeThreads, 0, s>>>(as_level(child), off32, off64, n_parent_dev, n_parent_max,
                                                            m, cov, parent_out, w.omin, w.omax);
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
