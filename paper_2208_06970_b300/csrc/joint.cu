// joint.cu -- joint central moments of orders 2..4 (covariance, coskewness and cokurtosis sums)
// of up to 8 variables per region, and their merge up the hierarchy.  The joint-plot section of
// the paper evaluates summaries by how well they keep the mean, covariance, coskewness and
// cokurtosis of the raw data; Sec. 3.3 merges summaries over cells, components and bands.
//
// Regions are contiguous ranges of a structured layout (lsrvt_structured_layout): the variables
// of a cell, component or band are one coalesced stream.  Work items are ranges, or chunks of
// 1024 positions of long ones; d = x - c with c the mean of the range's first 32 voxels (a shift
// close to the range's mean, the same for all its chunks, which keeps the shift corrections
// below small).  The raw sums
//   S1_i = sum d_i, S2_ij = sum d_i d_j, S3_ijk = sum d_i (d_j d_k), S4_ijkl = sum (d_i d_j)(d_k d_l)
// are accumulated in one of two ways:
//   m <= 4 -- a lane per voxel with all sums (at most 69) in registers, FP32 over the lane's
//             <= 32 voxels of the item, then a butterfly reduction across the warp;
//   m <= 8 -- 32 voxels' vectors z = (1, d_i, d_i d_j) staged in shared memory and the sums, as
//             products of two z entries, dealt out to the lanes; FP32 partials go to FP64 every
//             32 voxels.
// The central moments follow exactly (in FP64) from the shift formulas:
//   e = S1 / n, M2 = S2 - n e e, M3 = S3 - sum_3 e S2 + 2 n e e e,
//   M4 = S4 - sum_4 e S3 + sum_6 e e S2 - 3 n e e e e.
// Merges combine records pairwise (Pebay 2008), children in id order, in FP64.
#include "common.cuh"

namespace lsrvt {
namespace {

constexpr int kJMax = 8;                 // variables
constexpr int kJZ = 1 + kJMax + 36;      // z entries: 1, d_i, d_i d_j (i <= j)
constexpr int kJE = kJMax + 36 + 120 + 330;  // accumulated sums at m = 8
constexpr int kJT = 36 + 120 + 330;      // output co-moments at m = 8
constexpr int kJWarps = 8;
constexpr int kJChunk = 1024;            // positions per work item (longer ranges are split)

__host__ __device__ constexpr int binom2(int a) { return a * (a - 1) / 2; }
__host__ __device__ constexpr int binom3(int a) { return a * (a - 1) * (a - 2) / 6; }

struct JointTables {
    int m, Z, E, T2, T3, T4;
    uint8_t za[kJE], zb[kJE];   // accumulated sum e = product z[za[e]] * z[zb[e]]
    uint8_t tup[kJT][4];        // output entry -> sorted index tuple (orders 2, 3, 4 in turn)
    uint8_t pairz[kJMax][kJMax];  // z index of d_i d_j (i <= j)
};

// position of a non-decreasing tuple among the tuples of its length, lexicographic order
__host__ __device__ inline int tuple_pos(const int *t, int q, int m) {
    int idx = 0, prev = 0;
    for (int pos = 0; pos < q; ++pos) {
        const int L = q - pos - 1;
        for (int v = prev; v < t[pos]; ++v) {
            // number of non-decreasing tuples of length L over [v, m): C(m - v + L - 1, L)
            const int a = m - v + L - 1;
            idx += L == 0 ? 1 : (L == 1 ? a : (L == 2 ? binom2(a) : binom3(a)));
        }
        prev = t[pos];
    }
    return idx;
}

JointTables make_tables(int m) {
    JointTables T{};
    if (m < 1 || m > kJMax) return T;  // callers validate m first
    T.m = m;
    T.T2 = m * (m + 1) / 2;
    T.T3 = m * (m + 1) * (m + 2) / 6;
    T.T4 = m * (m + 1) * (m + 2) * (m + 3) / 24;
    T.Z = 1 + m + T.T2;
    int zp = 1 + m;
    for (int i = 0; i < m; ++i)
        for (int j = i; j < m; ++j) T.pairz[i][j] = T.pairz[j][i] = (uint8_t)zp++;
    int e = 0;
    for (int i = 0; i < m; ++i) { T.za[e] = 0; T.zb[e] = (uint8_t)(1 + i); ++e; }
    for (int i = 0; i < m; ++i)
        for (int j = i; j < m; ++j) { T.za[e] = 0; T.zb[e] = T.pairz[i][j]; ++e; }
    for (int i = 0; i < m; ++i)
        for (int j = i; j < m; ++j)
            for (int k = j; k < m; ++k) { T.za[e] = (uint8_t)(1 + i); T.zb[e] = T.pairz[j][k]; ++e; }
    for (int i = 0; i < m; ++i)
        for (int j = i; j < m; ++j)
            for (int k = j; k < m; ++k)
                for (int l = k; l < m; ++l) { T.za[e] = T.pairz[i][j]; T.zb[e] = T.pairz[k][l]; ++e; }
    T.E = e;
    int t = 0;
    for (int i = 0; i < m; ++i)
        for (int j = i; j < m; ++j) { T.tup[t][0] = (uint8_t)i; T.tup[t][1] = (uint8_t)j; ++t; }
    for (int i = 0; i < m; ++i)
        for (int j = i; j < m; ++j)
            for (int k = j; k < m; ++k) {
                T.tup[t][0] = (uint8_t)i; T.tup[t][1] = (uint8_t)j; T.tup[t][2] = (uint8_t)k; ++t;
            }
    for (int i = 0; i < m; ++i)
        for (int j = i; j < m; ++j)
            for (int k = j; k < m; ++k)
                for (int l = k; l < m; ++l) {
                    T.tup[t][0] = (uint8_t)i; T.tup[t][1] = (uint8_t)j; T.tup[t][2] = (uint8_t)k;
                    T.tup[t][3] = (uint8_t)l; ++t;
                }
    return T;
}

struct JVars {
    const float *p[kJMax];
};

__device__ __forceinline__ int64_t n_live(const int32_t *n_dev, int32_t cap) {
    if (!n_dev) return cap;
    const int32_t v = *n_dev;
    return v < 0 ? 0 : (v < cap ? v : cap);
}

// work items: one per range, or one per kJChunk positions of a long range; long ranges get an
// accumulator slot
__global__ void joint_items_kernel(const int64_t *__restrict__ off, const int32_t *n_dev, int32_t cap,
                                   int64_t *items, int64_t *slots, int64_t *n_scan) {
    const int64_t R = n_live(n_dev, cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_scan = R + 1;  // the scans cover the live ranges only
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= R; r += (int64_t)gridDim.x * blockDim.x) {
        int64_t nch = 0, lng = 0;
        if (r < R) {
            const int64_t L = off[r + 1] - off[r];
            nch = L <= kJChunk ? 1 : (L + kJChunk - 1) / kJChunk;
            lng = nch > 1;
        }
        items[r] = nch;
        slots[r] = lng;
    }
}

// item -> range, one entry per work item, so the moment kernels read their range with one load
// (the searches run here, all independent)
__global__ void joint_item_range_kernel(const int64_t *__restrict__ item_off, const int32_t *n_dev, int32_t cap,
                                        int32_t *item_range) {
    const int64_t R = n_live(n_dev, cap);
    const int64_t nitems = R > 0 ? item_off[R] : 0;
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < nitems;
         it += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = R;  // last r with item_off[r] <= it
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (item_off[mid] <= it) lo = mid;
            else hi = mid;
        }
        item_range[it] = (int32_t)lo;
    }
}

// central moments of one range from its raw sums around c (S: [E] in the table's order)
__device__ void joint_finalize(const JointTables &T, int lane, int64_t n, const float *c, const double *S,
                               int64_t r, lsrvt_joint out) {
    const int m = T.m;
    const double dn = (double)n;
    double e[kJMax];
#pragma unroll
    for (int i = 0; i < kJMax; ++i) e[i] = (i < m && n > 0) ? S[i] / dn : 0.0;
    const double *S2 = S + m, *S3 = S2 + T.T2, *S4 = S3 + T.T3;
    if (lane == 0) out.count[r] = n;
    for (int i = lane; i < m; i += 32) out.mean[r * m + i] = n > 0 ? (double)c[i] + e[i] : 0.0;
    const int total = T.T2 + T.T3 + T.T4;
    for (int t = lane; t < total; t += 32) {
        const int i = T.tup[t][0], j = T.tup[t][1], k = T.tup[t][2], l = T.tup[t][3];
        double v = 0.0;
        if (n > 0) {
            if (t < T.T2) {
                v = S2[t] - dn * e[i] * e[j];
            } else if (t < T.T2 + T.T3) {
                const int a[2] = {j, k}, b[2] = {i, k}, cc[2] = {i, j};
                v = S3[t - T.T2] - (e[i] * S2[tuple_pos(a, 2, m)] + e[j] * S2[tuple_pos(b, 2, m)] +
                                    e[k] * S2[tuple_pos(cc, 2, m)]) +
                    2.0 * dn * e[i] * e[j] * e[k];
            } else {
                const int q[4] = {i, j, k, l};
                double s3 = 0.0, s2 = 0.0;
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    int rest[3], w = 0;
#pragma unroll
                    for (int y = 0; y < 4; ++y)
                        if (y != x) rest[w++] = q[y];
                    s3 += e[q[x]] * S3[tuple_pos(rest, 3, m)];
                }
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = x + 1; y < 4; ++y) {
                        int rest[2], w = 0;
#pragma unroll
                        for (int z = 0; z < 4; ++z)
                            if (z != x && z != y) rest[w++] = q[z];
                        s2 += e[q[x]] * e[q[y]] * S2[tuple_pos(rest, 2, m)];
                    }
                v = S4[t - T.T2 - T.T3] - s3 + s2 - 3.0 * dn * e[i] * e[j] * e[k] * e[l];
            }
        }
        double *dst = t < T.T2 ? out.m2 + r * T.T2 + t
                               : (t < T.T2 + T.T3 ? out.m3 + r * T.T3 + (t - T.T2)
                                                  : out.m4 + r * T.T4 + (t - T.T2 - T.T3));
        *dst = v;
    }
}

struct JointWarpSmem {
    float z[32][kJZ];  // odd row length: lane-per-row writes hit 32 different banks
};

// the shift of a range: the mean of its first min(32, length) voxels, summed in a fixed order
// (every chunk of the range computes the same value)
__device__ __forceinline__ void range_shift(const JVars &V, int m, int64_t beg, int64_t end, int lane, float *c) {
    const int k = (int)min((int64_t)32, end - beg);
#pragma unroll
    for (int i = 0; i < kJMax; ++i) {
        float x = (i < m && lane < k) ? __ldg(V.p[i] + beg + lane) : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        c[i] = k > 0 ? x / (float)k : 0.f;
    }
}

// QN = sums per lane: ceil(E / 32) for the variable count
template <int QN>
__global__ void __launch_bounds__(32 * kJWarps) joint_ranges_kernel(JVars V, const int64_t *__restrict__ off,
                                                                    const int32_t *n_dev, int32_t cap,
                                                                    const int64_t *__restrict__ item_off,
                                                                    const int32_t *__restrict__ item_range,
                                                                    const int64_t *__restrict__ slot_off,
                                                                    double *acc, JointTables T, lsrvt_joint out) {
    __shared__ JointWarpSmem sm[kJWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t R = n_live(n_dev, cap);
    const int64_t nitems = R > 0 ? item_off[R] : 0;
    const int m = T.m, E = T.E;
    int za[QN], zb[QN];
#pragma unroll
    for (int q = 0; q < QN; ++q) {
        const int e = lane + 32 * q;
        za[q] = e < E ? T.za[e] : 0;
        zb[q] = e < E ? T.zb[e] : 0;
    }
    float(*z)[kJZ] = sm[w].z;
    for (int64_t it = (int64_t)blockIdx.x * kJWarps + w; it < nitems; it += (int64_t)gridDim.x * kJWarps) {
        // the range of this item: last r with item_off[r] <= it
        const int64_t r = item_range[it], chunk = it - item_off[r];
        const int64_t beg = off[r], end = off[r + 1];
        const int64_t pb = beg + chunk * kJChunk, pe = min(end, pb + kJChunk);
        const bool single = end - beg <= kJChunk;
        float c[kJMax];
        range_shift(V, m, beg, end, lane, c);
        float af[QN];
        double ad[QN];
#pragma unroll
        for (int q = 0; q < QN; ++q) { af[q] = 0.f; ad[q] = 0.0; }
        // the next batch's values are loaded while the current one is accumulated
        float xn[kJMax];
#pragma unroll
        for (int i = 0; i < kJMax; ++i) xn[i] = (i < m && pb + lane < pe) ? __ldcs(V.p[i] + pb + lane) : 0.f;
        for (int64_t b = pb; b < pe; b += 32) {
            const int64_t p = b + lane;
            float d[kJMax];
#pragma unroll
            for (int i = 0; i < kJMax; ++i) d[i] = (i < m && p < pe) ? xn[i] - c[i] : 0.f;
#pragma unroll
            for (int i = 0; i < kJMax; ++i) xn[i] = (i < m && p + 32 < pe) ? __ldcs(V.p[i] + p + 32) : 0.f;
            z[lane][0] = 1.f;
#pragma unroll
            for (int i = 0; i < kJMax; ++i)
                if (i < m) z[lane][1 + i] = d[i];
            {
                int zp = 1 + m;
#pragma unroll
                for (int i = 0; i < kJMax; ++i)
#pragma unroll
                    for (int j = i; j < kJMax; ++j)
                        if (j < m) z[lane][zp++] = d[i] * d[j];
            }
            __syncwarp();
            const int nv = (int)min((int64_t)32, pe - b);
            for (int v = 0; v < nv; ++v) {
#pragma unroll
                for (int q = 0; q < QN; ++q) af[q] = fmaf(z[v][za[q]], z[v][zb[q]], af[q]);
            }
#pragma unroll
            for (int q = 0; q < QN; ++q) { ad[q] += (double)af[q]; af[q] = 0.f; }
            __syncwarp();
        }
        if (single) {
            // the whole range in this warp: stage the sums, finalize, write
            double *S = reinterpret_cast<double *>(&z[0][0]);  // kJE doubles fit in the staging rows
#pragma unroll
            for (int q = 0; q < QN; ++q)
                if (lane + 32 * q < E) S[lane + 32 * q] = ad[q];
            __syncwarp();
            joint_finalize(T, lane, end - beg, c, S, r, out);
            __syncwarp();
        } else {
            double *A = acc + slot_off[r] * (int64_t)E;
#pragma unroll
            for (int q = 0; q < QN; ++q)
                if (lane + 32 * q < E) atomicAdd(A + lane + 32 * q, ad[q]);
        }
    }
}

// m <= 4: a lane per voxel with every sum in registers (E <= 69), no shared staging; each lane
// sums its <= 32 voxels of the item in FP32, a butterfly reduction gives the warp's sums, FP64
// from there.  The sums come in the table's order (orders 1, 2, 3, 4; lexicographic tuples).
template <int M>
struct JSmall {
    static constexpr int T2 = M * (M + 1) / 2;
    static constexpr int T3 = M * (M + 1) * (M + 2) / 6;
    static constexpr int T4 = M * (M + 1) * (M + 2) * (M + 3) / 24;
    static constexpr int E = M + T2 + T3 + T4;
};

template <int M>
__device__ __forceinline__ void joint_accumulate(const float (&d)[M], float (&acc)[JSmall<M>::E]) {
    float P[JSmall<M>::T2];
    int e = 0, t = 0;
#pragma unroll
    for (int i = 0; i < M; ++i) acc[e++] += d[i];
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
        for (int j = i; j < M; ++j) {
            P[t] = d[i] * d[j];
            acc[e++] += P[t++];
        }
    // P index of (j, k), j <= k: position in the lexicographic pair list
#define LSRVT_PIDX(a, b) ((a) * M - ((a) * ((a) - 1)) / 2 + ((b) - (a)))
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
        for (int j = i; j < M; ++j)
#pragma unroll
            for (int k = j; k < M; ++k) {
                acc[e] = fmaf(d[i], P[LSRVT_PIDX(j, k)], acc[e]);
                ++e;
            }
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
        for (int j = i; j < M; ++j)
#pragma unroll
            for (int k = j; k < M; ++k)
#pragma unroll
                for (int l = k; l < M; ++l) {
                    acc[e] = fmaf(P[LSRVT_PIDX(i, j)], P[LSRVT_PIDX(k, l)], acc[e]);
                    ++e;
                }
#undef LSRVT_PIDX
}

constexpr int kJRegWarps = 4;  // 128-thread CTAs: the sums take up to ~140 registers at m = 4

template <int M>
__global__ void __launch_bounds__(32 * kJRegWarps) joint_ranges_reg_kernel(JVars V, const int64_t *__restrict__ off,
                                                                        const int32_t *n_dev, int32_t cap,
                                                                        const int64_t *__restrict__ item_off,
                                                                        const int32_t *__restrict__ item_range,
                                                                        const int64_t *__restrict__ slot_off,
                                                                        double *acc_g, JointTables T, lsrvt_joint out) {
    constexpr int E = JSmall<M>::E;
    __shared__ double S[kJRegWarps][JSmall<M>::E];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t R = n_live(n_dev, cap);
    const int64_t nitems = R > 0 ? item_off[R] : 0;
    for (int64_t it = (int64_t)blockIdx.x * kJRegWarps + w; it < nitems; it += (int64_t)gridDim.x * kJRegWarps) {
        const int64_t r = item_range[it], chunk = it - item_off[r];
        const int64_t beg = off[r], end = off[r + 1];
        const int64_t pb = beg + chunk * kJChunk, pe = min(end, pb + kJChunk);
        float c[kJMax];
        range_shift(V, M, beg, end, lane, c);
        float acc[E];
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = 0.f;
        // U voxels per lane and step, the next step's values loaded while these are accumulated
        constexpr int U = M <= 2 ? 4 : 2;
        float xn[U][M];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int i = 0; i < M; ++i) {
                const int64_t q = pb + lane + 32 * u;
                xn[u][i] = q < pe ? __ldcs(V.p[i] + q) : 0.f;
            }
        for (int64_t p = pb + lane; p < pe; p += 32 * U) {
            float x[U][M];
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int i = 0; i < M; ++i) {
                    x[u][i] = xn[u][i];
                    const int64_t q = p + 32 * (U + u);
                    xn[u][i] = q < pe ? __ldcs(V.p[i] + q) : 0.f;
                }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (p + 32 * u >= pe) break;
                float d[M];
#pragma unroll
                for (int i = 0; i < M; ++i) d[i] = x[u][i] - c[i];
                joint_accumulate<M>(d, acc);
            }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = warp_sum(acc[e]);
        if (end - beg <= kJChunk) {
#pragma unroll
            for (int e = 0; e < E; ++e)
                if ((e & 31) == lane) S[w][e] = (double)acc[e];
            __syncwarp();
            joint_finalize(T, lane, end - beg, c, S[w], r, out);
            __syncwarp();
        } else {
            double *A = acc_g + slot_off[r] * (int64_t)E;
#pragma unroll
            for (int e = 0; e < E; ++e)
                if ((e & 31) == lane) atomicAdd(A + e, (double)acc[e]);
        }
    }
}

__global__ void joint_zero_kernel(double *acc, const int64_t *slot_off, const int32_t *n_dev, int32_t cap, int E) {
    const int64_t R = n_live(n_dev, cap);
    const int64_t n = (R > 0 ? slot_off[R] : 0) * (int64_t)E;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc[i] = 0.0;
}

// finalize the long ranges from their accumulators (one warp per range)
__global__ void joint_long_finalize_kernel(JVars V, const int64_t *__restrict__ off, const int32_t *n_dev,
                                           int32_t cap, const int64_t *__restrict__ slot_off, const double *acc,
                                           JointTables T, lsrvt_joint out) {
    __shared__ double S[kJWarps][kJE];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t R = n_live(n_dev, cap);
    for (int64_t r = (int64_t)blockIdx.x * kJWarps + w; r < R; r += (int64_t)gridDim.x * kJWarps) {
        if (slot_off[r + 1] == slot_off[r]) continue;  // a single-item range, written already
        const double *A = acc + slot_off[r] * (int64_t)T.E;
        for (int e = lane; e < T.E; e += 32) S[w][e] = A[e];
        float c[kJMax];
        range_shift(V, T.m, off[r], off[r + 1], lane, c);
        __syncwarp();
        joint_finalize(T, lane, off[r + 1] - off[r], c, S[w], r, out);
        __syncwarp();
    }
}

// ---------------------------------------------------------------- merge (Pebay 2008)
// Parent p combines its children [cbeg, cend) in id order; one warp per parent, the running
// record in shared memory, updated in place order-by-order (M4 reads the old M3 and M2, M3 the
// old M2), lanes owning entries.
struct JointRec {
    double mean[kJMax];
    double m2[36], m3[120], m4[330];
};

__device__ void joint_merge_step(const JointTables &T, int lane, JointRec &A, double &nA_, int64_t nB_,
                                 const double *muB, const double *B2, const double *B3, const double *B4) {
    const int m = T.m;
    if (nB_ == 0) return;
    if (nA_ == 0.0) {
        for (int i = lane; i < m; i += 32) A.mean[i] = muB[i];
        for (int t = lane; t < T.T2; t += 32) A.m2[t] = B2[t];
        for (int t = lane; t < T.T3; t += 32) A.m3[t] = B3[t];
        for (int t = lane; t < T.T4; t += 32) A.m4[t] = B4[t];
        __syncwarp();
        nA_ = (double)nB_;
        return;
    }
    const double nA = nA_, nB = (double)nB_, n = nA + nB;
    double d[kJMax];
#pragma unroll
    for (int i = 0; i < kJMax; ++i) d[i] = i < m ? muB[i] - A.mean[i] : 0.0;
    // order 4 (reads the old M3, M2)
    for (int t = lane; t < T.T4; t += 32) {
        const uint8_t *q = T.tup[T.T2 + T.T3 + t];
        const int ix[4] = {q[0], q[1], q[2], q[3]};
        double s6 = 0.0, s4 = 0.0;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = a + 1; b < 4; ++b) {
                int rest[2], w = 0;
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (c != a && c != b) rest[w++] = ix[c];
                const int pr = tuple_pos(rest, 2, m);
                s6 += d[ix[a]] * d[ix[b]] * (nA * nA * B2[pr] + nB * nB * A.m2[pr]);
            }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            int rest[3], w = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (c != a) rest[w++] = ix[c];
            const int pr = tuple_pos(rest, 3, m);
            s4 += d[ix[a]] * (nA * B3[pr] - nB * A.m3[pr]);
        }
        A.m4[t] = A.m4[t] + B4[t] + d[ix[0]] * d[ix[1]] * d[ix[2]] * d[ix[3]] * nA * nB * (nA * nA - nA * nB + nB * nB) /
                                        (n * n * n) +
                  s6 / (n * n) + s4 / n;
    }
    __syncwarp();
    // order 3 (reads the old M2)
    for (int t = lane; t < T.T3; t += 32) {
        const uint8_t *q = T.tup[T.T2 + t];
        const int i = q[0], j = q[1], k = q[2];
        const int jk[2] = {j, k}, ik[2] = {i, k}, ij[2] = {i, j};
        const int p1 = tuple_pos(jk, 2, m), p2 = tuple_pos(ik, 2, m), p3 = tuple_pos(ij, 2, m);
        const double s3 = d[i] * (nA * B2[p1] - nB * A.m2[p1]) + d[j] * (nA * B2[p2] - nB * A.m2[p2]) +
                          d[k] * (nA * B2[p3] - nB * A.m2[p3]);
        A.m3[t] = A.m3[t] + B3[t] + d[i] * d[j] * d[k] * nA * nB * (nA - nB) / (n * n) + s3 / n;
    }
    __syncwarp();
    for (int t = lane; t < T.T2; t += 32) {
        const uint8_t *q = T.tup[t];
        A.m2[t] = A.m2[t] + B2[t] + d[q[0]] * d[q[1]] * nA * nB / n;
    }
    __syncwarp();
    for (int i = lane; i < m; i += 32) A.mean[i] += d[i] * nB / n;
    __syncwarp();
    nA_ = n;
}

// Two levels: blocks of kJMergeBlock consecutive children of one parent are merged by one warp
// each (in id order) into partial records, then each parent merges its partials in order.
constexpr int kJMergeBlock = 64;

__device__ __forceinline__ int64_t child_begin(const int32_t *off32, const int64_t *off64, int64_t p) {
    return off32 ? (int64_t)off32[p] : off64[p];
}

// blocks per parent (at least one, so every parent gets a record) and, for parents with more
// than one block, partial-record rows
__global__ void joint_merge_blocks_kernel(const int32_t *off32, const int64_t *off64, const int32_t *n_parent_dev,
                                          int32_t n_parent_max, int64_t *nblk, int64_t *npart, int64_t *n_scan) {
    const int64_t P = n_live(n_parent_dev, n_parent_max);
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_scan = P + 1;  // the scans cover the live parents only
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= P; p += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = 0;
        if (p < P) {
            const int64_t nc = child_begin(off32, off64, p + 1) - child_begin(off32, off64, p);
            k = nc <= kJMergeBlock ? 1 : (nc + kJMergeBlock - 1) / kJMergeBlock;
        }
        nblk[p] = k;
        npart[p] = k > 1 ? k : 0;
    }
}

__device__ void write_record(const JointTables &T, int lane, const JointRec &A, double n, int64_t p,
                             lsrvt_joint out) {
    const int m = T.m;
    const bool any = n > 0.0;
    if (lane == 0) out.count[p] = (int64_t)n;
    for (int i = lane; i < m; i += 32) out.mean[p * m + i] = any ? A.mean[i] : 0.0;
    for (int t = lane; t < T.T2; t += 32) out.m2[p * T.T2 + t] = any ? A.m2[t] : 0.0;
    for (int t = lane; t < T.T3; t += 32) out.m3[p * T.T3 + t] = any ? A.m3[t] : 0.0;
    for (int t = lane; t < T.T4; t += 32) out.m4[p * T.T4 + t] = any ? A.m4[t] : 0.0;
    __syncwarp();
}

// stage 1: one warp per block of children; a parent of one block is written directly, the
// blocks of a larger parent become partial records
__global__ void joint_merge_stage1_kernel(lsrvt_joint child, const int32_t *off32, const int64_t *off64,
                                          const int32_t *n_parent_dev, int32_t n_parent_max,
                                          const int64_t *__restrict__ blk_off, const int64_t *__restrict__ part_off,
                                          JointTables T, lsrvt_joint part, lsrvt_joint parent) {
    __shared__ JointRec rec[kJWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t P = n_live(n_parent_dev, n_parent_max);
    const int64_t NB = P > 0 ? blk_off[P] : 0;
    const int m = T.m;
    for (int64_t k = (int64_t)blockIdx.x * kJWarps + w; k < NB; k += (int64_t)gridDim.x * kJWarps) {
        int64_t lo = 0, hi = P;  // parent of block k: last p with blk_off[p] <= k
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (blk_off[mid] <= k) lo = mid;
            else hi = mid;
        }
        const int64_t p = lo, kb = k - blk_off[p];
        const int64_t c0 = child_begin(off32, off64, p) + kb * kJMergeBlock;
        const int64_t c1 = min(child_begin(off32, off64, p + 1), c0 + kJMergeBlock);
        double n = 0.0;
        JointRec &A = rec[w];
        for (int64_t c = c0; c < c1; ++c)
            joint_merge_step(T, lane, A, n, child.count[c], child.mean + c * m, child.m2 + c * T.T2,
                             child.m3 + c * T.T3, child.m4 + c * T.T4);
        if (blk_off[p + 1] - blk_off[p] == 1) write_record(T, lane, A, n, p, parent);
        else write_record(T, lane, A, n, part_off[p] + kb, part);
    }
}

// stage 2: one warp per parent of several blocks merges its partials in order
__global__ void joint_merge_stage2_kernel(lsrvt_joint part, const int64_t *__restrict__ part_off,
                                          const int32_t *n_parent_dev, int32_t n_parent_max, JointTables T,
                                          lsrvt_joint parent) {
    __shared__ JointRec rec[kJWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t P = n_live(n_parent_dev, n_parent_max);
    const int m = T.m;
    for (int64_t p = (int64_t)blockIdx.x * kJWarps + w; p < P; p += (int64_t)gridDim.x * kJWarps) {
        if (part_off[p + 1] == part_off[p]) continue;  // one block: written by stage 1
        double n = 0.0;
        JointRec &A = rec[w];
        for (int64_t k = part_off[p]; k < part_off[p + 1]; ++k)
            joint_merge_step(T, lane, A, n, part.count[k], part.mean + k * m, part.m2 + k * T.T2,
                             part.m3 + k * T.T3, part.m4 + k * T.T4);
        write_record(T, lane, A, n, p, parent);
    }
}

__global__ void joint_band_offsets_kernel(const uint8_t *comp_band, const int32_t *n_comp_dev, int32_t max_comp,
                                          int32_t n_bands, int64_t *band_off) {
    const int32_t nc = min(*n_comp_dev, max_comp);
    for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b <= n_bands; b += gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = nc;  // first component of band >= b
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if ((int32_t)comp_band[mid] < b) lo = mid + 1;
            else hi = mid;
        }
        band_off[b] = lo;
    }
}

__global__ void joint_volume_offsets_kernel(int64_t *off, int32_t n) {
    off[0] = 0;
    off[1] = n;
}

struct JointWs {
    int64_t *items, *slots, *n_scan;
    int32_t *item_range;
    void *scan_items, *scan_slots;
    double *acc;
};

JointWs carve_joint(void *ws, size_t bytes, int32_t max_ranges, int64_t n_positions, int E, size_t *need) {
    Carver c(ws, bytes);
    JointWs w;
    const int64_t R = (int64_t)max_ranges + 1;
    w.items = c.take<int64_t>(R);
    w.slots = c.take<int64_t>(R);
    w.n_scan = c.take<int64_t>(1);
    w.scan_items = c.take<char>(scan_temp_bytes(R));
    w.scan_slots = c.take<char>(scan_temp_bytes(R));
    // items: one per range plus one per extra 1024-position chunk of a long range
    w.item_range = c.take<int32_t>(R + n_positions / kJChunk + 1);
    // long ranges hold more than kJChunk positions each: at most n_positions / kJChunk of them
    w.acc = c.take<double>((n_positions / kJChunk + 1) * (int64_t)E);
    *need = c.used;
    return w;
}

bool joint_ok(lsrvt_joint j) { return j.count && j.mean && j.m2 && j.m3 && j.m4; }

// merge scratch: per-parent block and partial counts (scanned to offsets) and the partial records
// of one level; a parent with more than one block has more than kJMergeBlock children, so the
// partial rows are fewer than 2 * children / kJMergeBlock + 1 (the levels run one after another
// and reuse the scratch)
struct JointMergeWs {
    int64_t *nblk, *npart, *n_scan;
    void *scan;
    lsrvt_joint part;
    int64_t *band_off, *vol_off;
};

JointMergeWs carve_joint_merge(void *ws, size_t bytes, int32_t max_children, int32_t max_parents, int32_t m,
                               size_t *need) {
    Carver c(ws, bytes);
    JointMergeWs w;
    const int64_t P = (int64_t)max_parents + 1;
    const int64_t NB = 2 * ((int64_t)max_children / kJMergeBlock) + 1;
    const int mm = m < 1 ? 1 : (m > kJMax ? kJMax : m);
    w.nblk = c.take<int64_t>(P);
    w.npart = c.take<int64_t>(P);
    w.n_scan = c.take<int64_t>(1);
    w.scan = c.take<char>(scan_temp_bytes(P));
    w.part.count = c.take<int64_t>(NB);
    w.part.mean = c.take<double>(NB * mm);
    w.part.m2 = c.take<double>(NB * (mm * (mm + 1) / 2));
    w.part.m3 = c.take<double>(NB * (mm * (mm + 1) * (mm + 2) / 6));
    w.part.m4 = c.take<double>(NB * (mm * (mm + 1) * (mm + 2) * (mm + 3) / 24));
    w.band_off = c.take<int64_t>(257);
    w.vol_off = c.take<int64_t>(2);
    *need = c.used;
    return w;
}

void joint_merge_level(lsrvt_joint child, const int32_t *off32, const int64_t *off64, const int32_t *n_parent_dev,
                       int32_t n_parent_max, const JointTables &T, lsrvt_joint parent, JointMergeWs &w, int sms,
                       cudaStream_t s) {
    joint_merge_blocks_kernel<<<grid_for((int64_t)n_parent_max + 1, 256, sms * 4), 256, 0, s>>>(
        off32, off64, n_parent_dev, n_parent_max, w.nblk, w.npart, w.n_scan);
    exclusive_scan_i64_dev(w.nblk, (int64_t)n_parent_max + 1, w.n_scan, nullptr, w.scan, s);
    exclusive_scan_i64_dev(w.npart, (int64_t)n_parent_max + 1, w.n_scan, nullptr, w.scan, s);
    joint_merge_stage1_kernel<<<sms * 4, 32 * kJWarps, 0, s>>>(child, off32, off64, n_parent_dev, n_parent_max,
                                                               w.nblk, w.npart, T, w.part, parent);
    joint_merge_stage2_kernel<<<grid_for(n_parent_max, kJWarps, sms * 4), 32 * kJWarps, 0, s>>>(
        w.part, w.npart, n_parent_dev, n_parent_max, T, parent);
}

}  // namespace

int joint_sums(int m) { return m + m * (m + 1) / 2 + m * (m + 1) * (m + 2) / 6 + m * (m + 1) * (m + 2) * (m + 3) / 24; }

size_t joint_workspace(int32_t max_ranges, int64_t n_positions, int32_t m) {
    size_t need;
    carve_joint(nullptr, 0, max_ranges, n_positions, joint_sums(m < 1 ? 1 : (m > kJMax ? kJMax : m)), &need);
    return need;
}

size_t joint_merge_workspace(int32_t max_sites, int32_t max_comp, int32_t m) {
    size_t a, b, c;
    carve_joint_merge(nullptr, 0, max_sites, max_comp, m, &a);
    carve_joint_merge(nullptr, 0, max_comp, 255, m, &b);
    carve_joint_merge(nullptr, 0, 255, 1, m, &c);
    return a > b ? (a > c ? a : c) : (b > c ? b : c);
}

}  // namespace lsrvt

using namespace lsrvt;

extern "C" lsrvt_status lsrvt_joint_moments(const float *const *values_host, int32_t m, int64_t n_positions,
                                            const int64_t *range_off, const int32_t *n_ranges_dev,
                                            int32_t max_ranges, lsrvt_joint out, void *ws, size_t ws_bytes,
                                            void *stream) {
    if (m < 1 || m > kJMax || !values_host || !range_off || max_ranges < 0 || n_positions < 0 || !joint_ok(out))
        return LSRVT_ERR_INVALID_ARG;
    JVars V{};
    for (int i = 0; i < m; ++i) {
        V.p[i] = values_host[i];
        if (!V.p[i]) return LSRVT_ERR_INVALID_ARG;
    }
    size_t need;
    JointWs w = carve_joint(ws, ws_bytes, max_ranges, n_positions, joint_sums(m), &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) return LSRVT_ERR_WORKSPACE;
    if (max_ranges == 0) return LSRVT_OK;
    const JointTables T = make_tables(m);
    cudaStream_t s = as_stream(stream);
    const int sms = stream_sms(s);
    joint_items_kernel<<<grid_for(max_ranges, 256, sms * 4), 256, 0, s>>>(range_off, n_ranges_dev, max_ranges,
                                                                           w.items, w.slots, w.n_scan);
    exclusive_scan_i64_dev(w.items, (int64_t)max_ranges + 1, w.n_scan, nullptr, w.scan_items, s);
    exclusive_scan_i64_dev(w.slots, (int64_t)max_ranges + 1, w.n_scan, nullptr, w.scan_slots, s);
    joint_zero_kernel<<<sms * 4, 256, 0, s>>>(w.acc, w.slots, n_ranges_dev, max_ranges, T.E);
    joint_item_range_kernel<<<sms * 8, 256, 0, s>>>(w.items, n_ranges_dev, max_ranges, w.item_range);
    if (m <= 4) {
#define LSRVT_JOINT_REG(M_)                                                                                      \
    joint_ranges_reg_kernel<M_><<<sms * 8, 32 * kJRegWarps, 0, s>>>(V, range_off, n_ranges_dev, max_ranges,    \
                                                                    w.items, w.item_range, w.slots, w.acc, T, out)
        if (m == 1) LSRVT_JOINT_REG(1);
        else if (m == 2) LSRVT_JOINT_REG(2);
        else if (m == 3) LSRVT_JOINT_REG(3);
        else LSRVT_JOINT_REG(4);
#undef LSRVT_JOINT_REG
        joint_long_finalize_kernel<<<sms * 4, 32 * kJWarps, 0, s>>>(V, range_off, n_ranges_dev, max_ranges, w.slots,
                                                                    w.acc, T, out);
        return launch_status();
    }
    const int qn = (T.E + 31) / 32;
#define LSRVT_JOINT_LAUNCH(Q)                                                                                \
    joint_ranges_kernel<Q><<<sms * 4, 32 * kJWarps, 0, s>>>(V, range_off, n_ranges_dev, max_ranges, w.items, \
                                                            w.item_range, w.slots, w.acc, T, out)
    if (qn <= 1) LSRVT_JOINT_LAUNCH(1);
    else if (qn <= 2) LSRVT_JOINT_LAUNCH(2);
    else if (qn <= 3) LSRVT_JOINT_LAUNCH(3);
    else if (qn <= 4) LSRVT_JOINT_LAUNCH(4);
    else if (qn <= 7) LSRVT_JOINT_LAUNCH(7);
    else if (qn <= 11) LSRVT_JOINT_LAUNCH(11);
    else LSRVT_JOINT_LAUNCH(16);
#undef LSRVT_JOINT_LAUNCH
    joint_long_finalize_kernel<<<sms * 4, 32 * kJWarps, 0, s>>>(V, range_off, n_ranges_dev, max_ranges, w.slots,
                                                                w.acc, T, out);
    return launch_status();
}

extern "C" lsrvt_status lsrvt_merge_joint_hierarchy(lsrvt_joint cells, const int32_t *n_sites_dev,
                                                    int32_t max_sites, int32_t m, const int32_t *comp_site_off,
                                                    const uint8_t *comp_band, const int32_t *n_comp_dev,
                                                    int32_t max_comp, int32_t n_bands, lsrvt_joint comps,
                                                    lsrvt_joint bands, lsrvt_joint volume, void *ws,
                                                    size_t ws_bytes, void *stream) {
    if (m < 1 || m > kJMax || !n_sites_dev || max_sites < 0 || !comp_site_off || !comp_band || !n_comp_dev ||
        max_comp < 0 || n_bands < 1 || n_bands > 255 || !joint_ok(cells) || !joint_ok(comps) || !joint_ok(bands) ||
        !joint_ok(volume))
        return LSRVT_ERR_INVALID_ARG;
    size_t need1, need2, need3;
    carve_joint_merge(nullptr, 0, max_sites, max_comp, m, &need1);
    carve_joint_merge(nullptr, 0, max_comp, n_bands, m, &need2);
    carve_joint_merge(nullptr, 0, n_bands, 1, m, &need3);
    const size_t need = need1 > need2 ? (need1 > need3 ? need1 : need3) : (need2 > need3 ? need2 : need3);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) return LSRVT_ERR_WORKSPACE;
    const JointTables T = make_tables(m);
    cudaStream_t s = as_stream(stream);
    const int sms = stream_sms(s);
    // each level carves the same scratch (levels run in stream order)
    JointMergeWs w1 = carve_joint_merge(ws, ws_bytes, max_sites, max_comp, m, &need1);
    joint_merge_level(cells, comp_site_off, nullptr, n_comp_dev, max_comp, T, comps, w1, sms, s);
    JointMergeWs w2 = carve_joint_merge(ws, ws_bytes, max_comp, n_bands, m, &need2);
    joint_band_offsets_kernel<<<1, 256, 0, s>>>(comp_band, n_comp_dev, max_comp, n_bands, w2.band_off);
    joint_merge_level(comps, nullptr, w2.band_off, nullptr, n_bands, T, bands, w2, sms, s);
    JointMergeWs w3 = carve_joint_merge(ws, ws_bytes, n_bands, 1, m, &need2);
    joint_volume_offsets_kernel<<<1, 1, 0, s>>>(w3.vol_off, n_bands);
    joint_merge_level(bands, nullptr, w3.vol_off, nullptr, 1, T, volume, w3, sms, s);
    return launch_status();
}
