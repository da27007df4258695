// aggregate.cu -- per-cell statistics of the auxiliary variables (Sec. 3.3 "Aggregation";
// introduction: statistical aggregation within the segments of the tessellation).
//
// Per cell s and variable j: count, mean, M2 (population variance M2/n), exact min and
// max, an n_bins histogram, and optionally co-moments (tensor cores, covariance.cu).
//
// B300 design: a CTA takes a 32x8x8 brick (rows of 32 floats = 128-byte coalesced
// loads), sorts the brick's (cell, local index) keys in shared memory so every cell is a
// contiguous run, then streams the variables eight at a time through shared memory.  The
// warps share the (variable, run) items, so bricks with one or two cells keep every warp
// busy.  For an item a warp's lanes accumulate x - c (c = the variable at the cell's site voxel, a
// per-cell shift common to all bricks) and (x - c)^2 in float-float (TwoSum / FMA
// error-free transforms, ~44 significant bits), min / max, and a per-warp shared
// histogram.  One FP64 atomic per (brick, cell, variable) and moment combines the bricks;
// a finalize pass forms mean = c + S1/n and M2 = S2 - S1^2/n in FP64.  HBM traffic is the
// algorithmic 4 B (cell) + 4 m B (variables) per voxel.
#include <cuda_bf16.h>

#include "common.cuh"

namespace lsrvt {
namespace {

constexpr int AX = 32, AY = 8, AZ = 8, AV = AX * AY * AZ;  // 2048 voxels
constexpr int kAggThreads = 256;
constexpr int kAggWarps = kAggThreads / 32;
constexpr int kMaxBins = 256;
constexpr size_t kAggDyn = sizeof(float) * kAggWarps * AV;  // staged variables (64 KB)

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

// float-float accumulator
struct FF {
    float hi, lo;
    __device__ void add(float a) {
        float s, e;
        two_sum(hi, a, s, e);
        hi = s;
        lo = __fadd_rn(lo, e);
    }
};

__global__ void __launch_bounds__(kAggThreads) aggregate_kernel(const int32_t *__restrict__ cell, Dims d,
                                                                 const __grid_constant__ AggParams p,
                                                                 const float *__restrict__ lo,
                                                                 const float *__restrict__ scale,
                                                                 const int32_t *__restrict__ site_pos,
                                                                 int32_t max_sites, AggAcc acc, uint32_t *hist,
                                                                 int32_t *status) {
    __shared__ unsigned long long keys[AV];
    extern __shared__ float xs[];  // kAggWarps variables of the brick, [kAggWarps][AV]
    __shared__ unsigned short head[AV + 1];
    __shared__ unsigned whist[kAggWarps][kMaxBins];
    __shared__ int nruns_s, nvalid_s;
    __shared__ int wcnt[kAggWarps];
    const int nbx = (d.nx + AX - 1) / AX, nby = (d.ny + AY - 1) / AY, nbz = (d.nz + AZ - 1) / AZ;
    const int64_t nbricks = (int64_t)nbx * nby * nbz;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int B = p.n_bins;
    for (int64_t br = blockIdx.x; br < nbricks; br += gridDim.x) {
        const int bx = (int)(br % nbx), by = (int)((br / nbx) % nby), bz = (int)(br / ((int64_t)nbx * nby));
        const int ox = bx * AX, oy = by * AY, oz = bz * AZ;
        for (int i = tid; i < AV; i += kAggThreads) {
            int lx = i % AX, ly = (i / AX) % AY, lz = i / (AX * AY);
            int gx = ox + lx, gy = oy + ly, gz = oz + lz;
            unsigned long long k = ~0ULL;
            if (gx < d.nx && gy < d.ny && gz < d.nz) {
                int32_t c = cell[gx + (int64_t)d.nx * (gy + (int64_t)d.ny * gz)];
                if (c >= 0 && c < max_sites) k = ((unsigned long long)(uint32_t)c << 32) | (uint32_t)i;
            }
            keys[i] = k;
        }
        block_bitonic_sort(keys, AV);
        // run heads in order
        int carry = 0;
        for (int base = 0; base < AV; base += kAggThreads) {
            int i = base + tid;
            unsigned long long k = keys[i];
            bool h = k != ~0ULL && (i == 0 || (keys[i - 1] >> 32) != (k >> 32));
            unsigned bal = __ballot_sync(0xffffffffu, h);
            if (lane == 0) wcnt[w] = __popc(bal);
            __syncthreads();
            int before = carry;
            for (int q2 = 0; q2 < w; ++q2) before += wcnt[q2];
            if (h) head[before + __popc(bal & lanemask_lt())] = (unsigned short)i;
            for (int q2 = 0; q2 < kAggWarps; ++q2) carry += wcnt[q2];
            if (k != ~0ULL && (i + 1 == AV || keys[i + 1] == ~0ULL)) nvalid_s = i + 1;
            __syncthreads();
        }
        if (tid == 0) {
            nruns_s = carry;
            if (carry == 0) nvalid_s = 0;
        }
        __syncthreads();
        const int nruns = nruns_s;
        if (nruns == 0) continue;
        if (tid == 0) head[nruns] = (unsigned short)nvalid_s;
        __syncthreads();
        // counts
        for (int r = tid; r < nruns; r += kAggThreads) {
            int32_t c = (int32_t)(keys[head[r]] >> 32);
            atomicAdd(&acc.cnt[c], (unsigned long long)(head[r + 1] - head[r]));
        }
        // kAggWarps variables at a time; the warps share the (variable, cell run) items, so a
        // brick with few cells still keeps every warp busy
        for (int j0 = 0; j0 < p.m; j0 += kAggWarps) {
            const int nj = p.m - j0 < kAggWarps ? p.m - j0 : kAggWarps;
            __syncthreads();
            for (int jj = 0; jj < nj; ++jj) {
                const float *x = p.aux[j0 + jj];
                for (int i = tid; i < AV; i += kAggThreads) {
                    int lx = i % AX, ly = (i / AX) % AY, lz = i / (AX * AY);
                    int gx = ox + lx, gy = oy + ly, gz = oz + lz;
                    float v = 0.0f;
                    if (gx < d.nx && gy < d.ny && gz < d.nz)
                        v = __ldcs(x + gx + (int64_t)d.nx * (gy + (int64_t)d.ny * gz));
                    xs[jj * AV + i] = v;
                }
            }
            __syncthreads();
            for (int item = w; item < nruns * nj; item += kAggWarps) {
                const int jj = item % nj, r = item / nj, j = j0 + jj;
                const float *xv = xs + jj * AV;
                const float loj = B ? lo[j] : 0.0f, scj = B ? scale[j] : 0.0f;
                const int s0 = head[r], s1 = head[r + 1];
                const int32_t c = (int32_t)(keys[s0] >> 32);
                const float sh = __ldg(p.aux[j] + site_pos[c]);
                if (B) {
                    for (int b = lane; b < B; b += 32) whist[w][b] = 0;
                    __syncwarp();
                }
                FF a1{0.0f, 0.0f}, a2{0.0f, 0.0f};
                float mn = __int_as_float(0x7f800000), mx = -__int_as_float(0x7f800000);
                bool bad = false;
                for (int t = s0 + lane; t < s1; t += 32) {
                    float v = xv[(uint32_t)keys[t]];
                    if (!isfinite(v)) { bad = true; continue; }
                    mn = fminf(mn, v);
                    mx = fmaxf(mx, v);
                    float dh, dl;
                    two_sum(v, -sh, dh, dl);  // v - sh = dh + dl exactly
                    a1.add(dh);
                    a1.lo = __fadd_rn(a1.lo, dl);
                    float pp = __fmul_rn(dh, dh);
                    float pe = __fmaf_rn(dh, dh, -pp);  // dh^2 = pp + pe exactly
                    a2.add(pp);
                    a2.lo = __fadd_rn(a2.lo, __fadd_rn(pe, __fmul_rn(2.0f, __fmul_rn(dh, dl))));
                    if (B) {
                        float tt = __fmul_rn(__fsub_rn(v, loj), scj);
                        int bin;
                        if (!(tt > 0.0f)) bin = 0;
                        else if (tt >= (float)B) bin = B - 1;
                        else bin = (int)tt;
                        atomicAdd(&whist[w][bin], 1u);
                    }
                }
                if (__any_sync(0xffffffffu, bad)) { if (lane == 0) set_status(status, LSRVT_ERR_NONFINITE); }
                double d1 = (double)a1.hi + (double)a1.lo;
                double d2 = (double)a2.hi + (double)a2.lo;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    d1 += __shfl_xor_sync(0xffffffffu, d1, o);
                    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
                    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
                    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                }
                const int64_t cj = (int64_t)c * p.m + j;
                if (lane == 0) {
                    atomicAdd(&acc.s1[cj], d1);
                    atomicAdd(&acc.s2[cj], d2);
                    atomicMin(&acc.vmin[cj], float_to_ordered(mn));
                    atomicMax(&acc.vmax[cj], float_to_ordered(mx));
                }
                if (B) {
                    __syncwarp();
                    for (int b = lane; b < B; b += 32) {
                        unsigned hcount = whist[w][b];
                        if (hcount) atomicAdd(&hist[cj * B + b], hcount);
                    }
                    __syncwarp();
                }
            }
        }
        __syncthreads();
    }
}

__global__ void aggregate_init_kernel(AggAcc acc, const int32_t *n_sites_dev, int32_t max_sites, int32_t m,
                                      lsrvt_stats out) {
    int32_t ns = max_sites;
    int64_t total = (int64_t)ns * m;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        acc.s1[i] = 0.0;
        acc.s2[i] = 0.0;
        acc.vmin[i] = float_to_ordered(__int_as_float(0x7f800000));
        acc.vmax[i] = float_to_ordered(-__int_as_float(0x7f800000));
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x)
        acc.cnt[i] = 0;
}

__global__ void aggregate_finalize_kernel(AggAcc acc, const int32_t *n_sites_dev, int32_t max_sites, int32_t m,
                                          const __grid_constant__ AggParams p, const int32_t *__restrict__ site_pos,
                                          lsrvt_stats out) {
    int32_t ns = min(*n_sites_dev, max_sites);
    int64_t total = (int64_t)max_sites * m;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = (int32_t)(i / (m > 0 ? m : 1));
        int32_t j = (int32_t)(i - (int64_t)c * m);
        long long n = (long long)acc.cnt[c];
        double mean = 0.0, m2 = 0.0;
        if (n > 0 && c < ns) {
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
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < max_sites; c += (int64_t)gridDim.x * blockDim.x)
        out.count[c] = (int64_t)acc.cnt[c];
}

// ------------------------------------------------------------------ co-moments on tensor cores
// C_ij = sum over the cell (x_i - mean_i)(x_j - mean_j): per 16x8x8 brick the values, centred
// by c = float(mean) of their cell, are split d = hi + lo into two BF16 numbers (lo = the
// exact float remainder rounded to BF16) and staged var-major in shared memory in the brick's
// cell-sorted order.  One warp per cell run accumulates X^T X with mma.sync m16n8k16 (BF16 in,
// FP32 accumulate) over 16-voxel chunks as hi.hi + hi.lo + lo.hi (the lo.lo term is below
// 2^-16 relative), then adds its 32x32 tile into the FP64 totals.  The finalisation removes
// the centring offset exactly: C = C' - n (mean_i - c_i)(mean_j - c_j), and takes the
// diagonal from the float-float M2 of the moments pass.
constexpr int CX = 16, CY = 8, CZ = 8, CV = CX * CY * CZ;  // 1024 voxels
constexpr int kCovVars = 32;
constexpr int kCovStride = CV + 8;  // bf16 elements per variable row (bank offset)
constexpr size_t kCovSmem = (size_t)2 * kCovVars * kCovStride * 2 + (size_t)CV * 8 + (CV + 1) * 2 + 64;

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                               unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// two consecutive bf16 of row `var` at even position p, with elements at or beyond `end` zeroed
__device__ __forceinline__ unsigned frag2(const unsigned short *rows, int var, int p, int end) {
    if (p >= end) return 0u;
    unsigned v = *reinterpret_cast<const unsigned *>(rows + (size_t)var * kCovStride + p);
    if (p + 1 >= end) return v & 0xFFFFu;
    return v;
}

__device__ __forceinline__ unsigned short bf16_bits(float f) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}

__global__ void __launch_bounds__(256) covariance_kernel(const int32_t *__restrict__ cell, Dims d,
                                                         const __grid_constant__ AggParams p,
                                                         const double *__restrict__ mean, int32_t max_sites,
                                                         double *comom) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned short *hi = (unsigned short *)smem_raw;
    unsigned short *lo = hi + kCovVars * kCovStride;
    unsigned long long *keys = (unsigned long long *)(lo + kCovVars * kCovStride);
    unsigned short *inv = (unsigned short *)(keys + CV);  // local index -> sorted position
    __shared__ unsigned short head[CV + 1];
    __shared__ int nruns_s, nvalid_s, wcnt[8];
    const int m = p.m, T = m * (m + 1) / 2;
    const int nbx = (d.nx + CX - 1) / CX, nby = (d.ny + CY - 1) / CY, nbz = (d.nz + CZ - 1) / CZ;
    const int64_t nbricks = (int64_t)nbx * nby * nbz;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    for (int64_t br = blockIdx.x; br < nbricks; br += gridDim.x) {
        const int ox = (int)(br % nbx) * CX, oy = (int)((br / nbx) % nby) * CY, oz = (int)(br / ((int64_t)nbx * nby)) * CZ;
        for (int i = tid; i < CV; i += blockDim.x) {
            int x = ox + i % CX, y = oy + (i / CX) % CY, z = oz + i / (CX * CY);
            unsigned long long k = ~0ULL;
            if (x < d.nx && y < d.ny && z < d.nz) {
                int32_t c = cell[x + (int64_t)d.nx * (y + (int64_t)d.ny * z)];
                if (c >= 0 && c < max_sites) k = ((unsigned long long)(uint32_t)c << 32) | (uint32_t)i;
            }
            keys[i] = k;
        }
        block_bitonic_sort(keys, CV);
        int carry = 0;
        for (int base = 0; base < CV; base += blockDim.x) {
            int i = base + tid;
            unsigned long long k = keys[i];
            if (k != ~0ULL) inv[(uint32_t)k] = (unsigned short)i;
            bool h = k != ~0ULL && (i == 0 || (keys[i - 1] >> 32) != (k >> 32));
            unsigned bal = __ballot_sync(0xffffffffu, h);
            if (lane == 0) wcnt[w] = __popc(bal);
            __syncthreads();
            int before = carry;
            for (int q = 0; q < w; ++q) before += wcnt[q];
            if (h) head[before + __popc(bal & lanemask_lt())] = (unsigned short)i;
            for (int q = 0; q < 8; ++q) carry += wcnt[q];
            if (k != ~0ULL && (i + 1 == CV || keys[i + 1] == ~0ULL)) nvalid_s = i + 1;
            __syncthreads();
        }
        if (tid == 0) {
            nruns_s = carry;
            if (carry == 0) nvalid_s = 0;
            head[carry] = (unsigned short)nvalid_s;
        }
        __syncthreads();
        const int nruns = nruns_s;
        if (nruns == 0) continue;
        // stage centred values, var-major, in sorted order; padding variables are zero
        for (int i = tid; i < CV; i += blockDim.x) {
            int x = ox + i % CX, y = oy + (i / CX) % CY, z = oz + i / (CX * CY);
            if (x >= d.nx || y >= d.ny || z >= d.nz) continue;
            const int64_t gidx = x + (int64_t)d.nx * (y + (int64_t)d.ny * z);
            const int32_t c = cell[gidx];
            if (c < 0 || c >= max_sites) continue;
            const int pos = inv[i];
            for (int j = 0; j < kCovVars; ++j) {
                unsigned short h2 = 0, l2 = 0;
                if (j < m) {
                    float v = __ldcs(p.aux[j] + gidx);
                    float cen = (float)mean[(int64_t)c * m + j];
                    float dd = __fsub_rn(v, cen);
                    h2 = bf16_bits(dd);
                    float hf = __bfloat162float(__ushort_as_bfloat16(h2));
                    l2 = bf16_bits(__fsub_rn(dd, hf));
                }
                hi[(size_t)j * kCovStride + pos] = h2;
                lo[(size_t)j * kCovStride + pos] = l2;
            }
        }
        __syncthreads();
        const int nI = (m + 15) / 16, nJ = (m + 7) / 8;
        for (int r = w; r < nruns; r += 8) {
            const int s0 = head[r], s1 = head[r + 1];
            const int32_t c = (int32_t)(keys[s0] >> 32);
            float acc[2][4][4];
#pragma unroll
            for (int I = 0; I < 2; ++I)
#pragma unroll
                for (int J = 0; J < 4; ++J)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[I][J][e] = 0.0f;
            for (int ch = s0 - (s0 & 1); ch < s1; ch += 16) {
                // positions of this lane's elements: ch + 2t (+1) and ch + 2t + 8 (+1); elements
                // before s0 belong to the previous run and are masked by starting at an even
                // position and zeroing below s0
                const int pa = ch + 2 * t, pb = ch + 2 * t + 8;
#pragma unroll
                for (int I = 0; I < 2; ++I) {
                    if (I >= nI) break;
                    const int vi0 = 16 * I + g, vi1 = vi0 + 8;
                    unsigned ah[4], al[4];
                    auto ld = [&](const unsigned short *rows, int var, int pp) {
                        unsigned v = frag2(rows, var, pp, s1);
                        if (pp < s0) v &= (pp + 1 < s0) ? 0u : 0xFFFF0000u;
                        return v;
                    };
                    ah[0] = ld(hi, vi0, pa); ah[1] = ld(hi, vi1, pa); ah[2] = ld(hi, vi0, pb); ah[3] = ld(hi, vi1, pb);
                    al[0] = ld(lo, vi0, pa); al[1] = ld(lo, vi1, pa); al[2] = ld(lo, vi0, pb); al[3] = ld(lo, vi1, pb);
#pragma unroll
                    for (int J = 0; J < 4; ++J) {
                        if (J >= nJ) break;
                        const int vj = 8 * J + g;
                        unsigned bh0 = ld(hi, vj, pa), bh1 = ld(hi, vj, pb);
                        unsigned bl0 = ld(lo, vj, pa), bl1 = ld(lo, vj, pb);
                        mma_bf16_16816(acc[I][J], ah[0], ah[1], ah[2], ah[3], bh0, bh1);
                        mma_bf16_16816(acc[I][J], ah[0], ah[1], ah[2], ah[3], bl0, bl1);
                        mma_bf16_16816(acc[I][J], al[0], al[1], al[2], al[3], bh0, bh1);
                    }
                }
            }
            // accumulate the upper triangle in FP64
#pragma unroll
            for (int I = 0; I < 2; ++I)
#pragma unroll
                for (int J = 0; J < 4; ++J)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        int i = 16 * I + g + (e >= 2 ? 8 : 0);
                        int j = 8 * J + 2 * t + (e & 1);
                        if (i < m && j < m && i <= j) {
                            int tri = i * m - i * (i - 1) / 2 + (j - i);
                            atomicAdd(&comom[(int64_t)c * T + tri], (double)acc[I][J][e]);
                        }
                    }
        }
        __syncthreads();
    }
}

__global__ void covariance_finalize_kernel(const int64_t *count, const double *mean, const double *m2,
                                           int32_t max_sites, int32_t m, double *comom) {
    const int T = m * (m + 1) / 2;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)max_sites * T;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = idx / T;
        int tri = (int)(idx - c * T);
        int i = 0;
        while (tri >= (i + 1) * m - i * (i + 1) / 2) ++i;  // row of the upper triangle
        int j = i + (tri - (i * m - i * (i - 1) / 2));
        int64_t n = count[c];
        if (n == 0) { comom[idx] = 0.0; continue; }
        if (i == j) { comom[idx] = m2[c * m + i]; continue; }
        double mi = mean[c * m + i], mj = mean[c * m + j];
        double di = mi - (double)(float)mi, dj = mj - (double)(float)mj;
        comom[idx] = comom[idx] - (double)n * di * dj;
    }
}

// ------------------------------------------------------------------ value ranges
__global__ void range_init_kernel(unsigned *lo_bits, unsigned *hi_bits, int32_t m) {
    int j = threadIdx.x + blockIdx.x * blockDim.x;
    if (j < m) {
        lo_bits[j] = float_to_ordered(__int_as_float(0x7f800000));
        hi_bits[j] = float_to_ordered(-__int_as_float(0x7f800000));
    }
}

__global__ void __launch_bounds__(256) range_kernel(const int32_t *__restrict__ cell, const float *__restrict__ x,
                                                    int64_t n, unsigned *lo_bits, unsigned *hi_bits, int32_t *status) {
    float mn = __int_as_float(0x7f800000), mx = -__int_as_float(0x7f800000);
    bool bad = false;
    int64_t n4 = n / 4;
    const int4 *c4 = (const int4 *)cell;
    const float4 *x4 = (const float4 *)x;
    bool vec = (((uintptr_t)cell | (uintptr_t)x) & 15) == 0;
    if (vec) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
            int4 c = __ldcs(c4 + i);
            float4 v = __ldcs(x4 + i);
            float vv[4] = {v.x, v.y, v.z, v.w};
            int cc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (cc[k] >= 0) {
                    if (!isfinite(vv[k])) bad = true;
                    else { mn = fminf(mn, vv[k]); mx = fmaxf(mx, vv[k]); }
                }
        }
    }
    for (int64_t i = (vec ? n4 * 4 : 0) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (cell[i] < 0) continue;
        float v = x[i];
        if (!isfinite(v)) bad = true;
        else { mn = fminf(mn, v); mx = fmaxf(mx, v); }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(lo_bits, float_to_ordered(mn));
        atomicMax(hi_bits, float_to_ordered(mx));
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
};

AggWs carve_agg(void *ws, size_t bytes, int32_t max_sites, int32_t m, size_t *need) {
    Carver c(ws, bytes);
    AggWs w;
    int64_t sm = (int64_t)max_sites * (m > 0 ? m : 1);
    w.acc.s1 = c.take<double>(sm);
    w.acc.s2 = c.take<double>(sm);
    w.acc.vmin = c.take<unsigned>(sm);
    w.acc.vmax = c.take<unsigned>(sm);
    w.acc.cnt = c.take<unsigned long long>(max_sites > 0 ? max_sites : 1);
    *need = c.used;
    return w;
}

}  // namespace

size_t aggregate_workspace(int32_t max_sites, int32_t m) {
    size_t need;
    carve_agg(nullptr, 0, max_sites, m, &need);
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
    range_init_kernel<<<1, 64, 0, s>>>((unsigned *)lo_dev, (unsigned *)scale_dev, n_aux);
    for (int j = 0; j < n_aux; ++j)
        range_kernel<<<grid_for(n / 4 + 1, 256, kSMs * 8), 256, 0, s>>>(cell, aux_host[j], n, (unsigned *)lo_dev + j,
                                                                       (unsigned *)scale_dev + j, status_dev);
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
    AggWs w = carve_agg(ws, ws_bytes, max_sites, n_aux, &need);
    size_t cov_need = 0;
    if (!ws || ws_bytes < need + cov_need || ((uintptr_t)ws & 255)) return LSRVT_ERR_WORKSPACE;
    cudaStream_t s = as_stream(stream);
    Dims d{dd.nx, dd.ny, dd.nz};
    if (want_hist && n_aux > 0)
        cudaMemsetAsync(out.hist, 0, sizeof(uint32_t) * (size_t)max_sites * n_aux * n_bins, s);
    aggregate_init_kernel<<<grid_for((int64_t)max_sites * (n_aux > 0 ? n_aux : 1), 256, kSMs * 8), 256, 0, s>>>(
        w.acc, n_sites_dev, max_sites, n_aux, out);
    int64_t nbricks = (int64_t)((d.nx + AX - 1) / AX) * ((d.ny + AY - 1) / AY) * ((d.nz + AZ - 1) / AZ);
    int occ = 0;
    cudaFuncSetAttribute(aggregate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAggDyn);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, aggregate_kernel, kAggThreads, kAggDyn);
    if (occ < 1) occ = 1;
    int grid = (int)(nbricks < (int64_t)kSMs * occ ? nbricks : (int64_t)kSMs * occ);
    aggregate_kernel<<<grid, kAggThreads, kAggDyn, s>>>(cell, d, p, lo_dev, scale_dev, site_pos, max_sites, w.acc, out.hist,
                                                  status_dev);
    aggregate_finalize_kernel<<<grid_for((int64_t)max_sites * (n_aux > 0 ? n_aux : 1), 256, kSMs * 8), 256, 0, s>>>(
        w.acc, n_sites_dev, max_sites, n_aux, p, site_pos, out);
    if (want_cov && n_aux > 0) {
        const int T = n_aux * (n_aux + 1) / 2;
        cudaMemsetAsync(out.comom, 0, sizeof(double) * (size_t)max_sites * T, s);
        cudaFuncSetAttribute(covariance_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCovSmem);
        int64_t ncb = (int64_t)((d.nx + CX - 1) / CX) * ((d.ny + CY - 1) / CY) * ((d.nz + CZ - 1) / CZ);
        int cg = (int)(ncb < (int64_t)kSMs * 2 ? ncb : (int64_t)kSMs * 2);
        covariance_kernel<<<cg, 256, kCovSmem, s>>>(cell, d, p, out.mean, max_sites, out.comom);
        covariance_finalize_kernel<<<grid_for((int64_t)max_sites * T, 256, kSMs * 8), 256, 0, s>>>(
            out.count, out.mean, out.m2, max_sites, n_aux, out.comom);
    }
    return launch_status();
}
