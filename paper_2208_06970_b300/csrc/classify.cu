// classify.cu -- isoband classification, Sec. 3.1 "Level Sets, Isobands, and Connected
// Components": B_{a,b} = { v : a < f(v) <= b }; band = #{ i : t_i < f(v) }.
//
// HBM-bound sweep: 4 B in, 1 B out per voxel.  Each thread reads 16 floats as four
// 16-byte loads and writes 16 bands as one 16-byte store; the grid is a multiple of the
// SM count and strides over the volume.  The isovalues are staged in shared memory
// padded with +inf to 2^L - 1 entries and each voxel does an L-step branch-free
// lower-bound search (L = 3 for up to 7 isovalues, 8 for 254).
#include "common.cuh"

namespace lsrvt {
namespace {

struct IsoParams {
    float t[256];
    int levels;  // search steps: 2^levels - 1 >= n_iso
};

__device__ __forceinline__ uint8_t band_of(float f, const float *t, int levels) {
    if (f != f) return kInvalidBand;
    int b = 0;
    for (int step = 1 << (levels - 1); step >= 1; step >>= 1)
        if (t[b + step - 1] < f) b += step;
    return (uint8_t)b;
}

__global__ void __launch_bounds__(256) classify_vec_kernel(const float4 *__restrict__ field,
                                                           uint4 *__restrict__ band, int64_t n16,
                                                           const __grid_constant__ IsoParams p) {
    __shared__ float t[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) t[i] = p.t[i];
    __syncthreads();
    const int L = p.levels;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x) {
        float4 a = __ldcs(field + 4 * i + 0);
        float4 b = __ldcs(field + 4 * i + 1);
        float4 c = __ldcs(field + 4 * i + 2);
        float4 d = __ldcs(field + 4 * i + 3);
        float v[16] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w, d.x, d.y, d.z, d.w};
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t r = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) r |= (uint32_t)band_of(v[4 * k + j], t, L) << (8 * j);
            w[k] = r;
        }
        __stcs(band + i, make_uint4(w[0], w[1], w[2], w[3]));
    }
}

__global__ void classify_scalar_kernel(const float *__restrict__ field, uint8_t *__restrict__ band, int64_t begin,
                                       int64_t n, const __grid_constant__ IsoParams p) {
    __shared__ float t[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) t[i] = p.t[i];
    __syncthreads();
    for (int64_t i = begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        band[i] = band_of(field[i], t, p.levels);
}

}  // namespace
}  // namespace lsrvt

using namespace lsrvt;

extern "C" lsrvt_status lsrvt_classify(const float *field, lsrvt_dims d, const float *iso_host, int32_t n_iso,
                                       uint8_t *band, void *stream) {
    if (!dims_ok(d) || !field || !band || n_iso < 0 || n_iso > 254 || (n_iso > 0 && !iso_host))
        return LSRVT_ERR_INVALID_ARG;
    for (int i = 0; i < n_iso; ++i)
        if (iso_host[i] != iso_host[i]) return LSRVT_ERR_NOT_SORTED;
    for (int i = 1; i < n_iso; ++i)
        if (!(iso_host[i - 1] < iso_host[i])) return LSRVT_ERR_NOT_SORTED;
    IsoParams p;
    for (int i = 0; i < 256; ++i) p.t[i] = __builtin_inff();
    for (int i = 0; i < n_iso; ++i) p.t[i] = iso_host[i];
    int L = 1;
    while ((1 << L) - 1 < n_iso) ++L;
    p.levels = L;
    cudaStream_t s = as_stream(stream);
    int64_t n = (int64_t)d.nx * d.ny * d.nz;
    int64_t done = 0;
    bool aligned = ((uintptr_t)field % 16 == 0) && ((uintptr_t)band % 16 == 0);
    if (aligned && n >= 16) {
        int64_t n16 = n / 16;
        int grid = grid_for(n16, 256, kSMs * 8);
        classify_vec_kernel<<<grid, 256, 0, s>>>((const float4 *)field, (uint4 *)band, n16, p);
        done = n16 * 16;
    }
    if (done < n) {
        int grid = grid_for(n - done, 256, kSMs * 8);
        classify_scalar_kernel<<<grid, 256, 0, s>>>(field, band, done, n, p);
    }
    return launch_status();
}
