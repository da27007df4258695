// common.cuh -- shared device helpers of the LSRVT CUDA library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/lsrvt.h"

namespace lsrvt {

constexpr uint8_t kInvalidBand = 0xFF;
constexpr int kSMs = 148;  // B300: 2 dies x 74 SMs

// 16.16 fixed-point Euclidean edge lengths, rounded up: 1, sqrt(2), sqrt(3).
constexpr uint32_t kWFace = 65536u;
constexpr uint32_t kWEdge = 92682u;
constexpr uint32_t kWCorner = 113512u;

struct Dims {
    int32_t nx, ny, nz;
    __host__ __device__ int64_t n() const { return (int64_t)nx * ny * nz; }
};

inline bool dims_ok(lsrvt_dims d) {
    if (d.nx <= 0 || d.ny <= 0 || d.nz <= 0) return false;
    int64_t n = (int64_t)d.nx * d.ny * d.nz;
    return n < (int64_t(1) << 31);
}

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// First data-dependent error wins.
__device__ __forceinline__ void set_status(int32_t *status, int32_t code) {
    if (status) atomicCAS(status, 0, code);
}

inline lsrvt_status launch_status() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LSRVT_OK : LSRVT_ERR_CUDA;
}

// ---------------------------------------------------------------- workspace carving
struct Carver {
    char *base;
    size_t used, cap;
    __host__ Carver(void *b, size_t c) : base((char *)b), used(0), cap(c) {}
    template <class T>
    __host__ T *take(size_t count) {
        size_t off = (used + 255) & ~size_t(255);
        used = off + count * sizeof(T);
        return base ? reinterpret_cast<T *>(base + off) : nullptr;
    }
    __host__ bool ok() const { return used <= cap; }
};

inline int grid_for(int64_t work, int threads, int max_blocks) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

// Division by a divisor fixed for a launch (Granlund & Montgomery 1994, "Division by invariant
// integers using multiplication", the method for unsigned run-time invariant divisors): for
// 1 <= d < 2^31 let l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1, which fits in 32
// bits; then floor(n / d) = (t + ((n - t) >> s1)) >> s2 for every 32-bit n, with t the high word
// of m n, s1 = min(l, 1) and s2 = max(l - 1, 0).
struct InvDiv {
    uint32_t m;
    int s1, s2;
    __device__ __forceinline__ uint32_t div(uint32_t n) const {
        const uint32_t t = __umulhi(m, n);
        return (t + ((n - t) >> s1)) >> s2;
    }
};

inline InvDiv make_invdiv(uint32_t d) {
    int l = 0;
    while ((1ull << l) < d) ++l;
    InvDiv r;
    r.m = (uint32_t)(((((1ull << l) - d) << 32) / d) + 1);
    r.s1 = l < 1 ? l : 1;
    r.s2 = l > 1 ? l - 1 : 0;
    return r;
}

// the coordinates of linear voxel index v (< 2^31) with the two divisions by the volume's
// extents done by InvDiv
struct VoxelCoder {
    InvDiv by_nx, by_ny;
    __device__ __forceinline__ void decode(uint32_t v, Dims d, int &x, int &y, int &z) const {
        const uint32_t r = by_nx.div(v);
        x = (int)(v - r * (uint32_t)d.nx);
        z = (int)by_ny.div(r);
        y = (int)(r - (uint32_t)z * (uint32_t)d.ny);
    }
};

inline VoxelCoder make_coder(Dims d) { return VoxelCoder{make_invdiv((uint32_t)d.nx), make_invdiv((uint32_t)d.ny)}; }

// SMs that grid-wide launches on stream s may size their grids to (the stream's share of the
// GPU, lsrvt_set_stream_share; the whole GPU by default)
int stream_sms(cudaStream_t s);

// ---------------------------------------------------------------- warp helpers
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// float atomics via ordered integer encoding (exact, order independent)
__device__ __forceinline__ unsigned float_to_ordered(float f) {
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ __forceinline__ float ordered_to_float(unsigned u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
#else
    unsigned v = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    float f;
    memcpy(&f, &v, 4);
    return f;
#endif
}

// ---------------------------------------------------------------- scans (scan.cu)
// Exclusive scan of n int64 values in place; `total` (device, nullable) receives the sum.
// Temporary storage: scan_temp_bytes(n).
size_t scan_temp_bytes(int64_t n);
void exclusive_scan_i64(int64_t *data, int64_t n, int64_t *total, void *temp, cudaStream_t s);
// The same over the first *n_dev (device) entries, n_dev <= n; temp sized for n.
void exclusive_scan_i64_dev(int64_t *data, int64_t n, const int64_t *n_dev, int64_t *total, void *temp,
                           cudaStream_t s);

// Stable LSD radix sort of (key, value) uint32 pairs by the low `bits` bits of key.
size_t radix_temp_bytes(int64_t n);
// Sorts keys/vals in place using ping-pong buffers in temp; n_dev (device, nullable)
// overrides n with a device-side count <= n.
void radix_sort_pairs(uint32_t *keys, uint32_t *vals, int64_t n, const int32_t *n_dev, int bits, void *temp,
                      cudaStream_t s);

// ---------------------------------------------------------------- bitonic sort in shared memory
// Sorts n_pow2 uint64 keys in shared memory ascending (all threads of the block call it).
__device__ __forceinline__ void block_bitonic_sort(unsigned long long *k, int n_pow2) {
    for (int size = 2; size <= n_pow2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int i = threadIdx.x; i < (n_pow2 >> 1); i += blockDim.x) {
                int lo = 2 * i - (i & (stride - 1));
                int hi = lo + stride;
                bool up = ((lo & size) == 0);
                unsigned long long a = k[lo], b = k[hi];
                if ((a > b) == up) {
                    k[lo] = b;
                    k[hi] = a;
                }
            }
        }
    }
    __syncthreads();
}

}  // namespace lsrvt
