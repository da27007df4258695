// saliency.cu -- saliency weights m_v (Sec. 3.1 "Centroids or Centers of Mass": the
// weighting function m_v; Sec. 3.3: a second field with attraction gamma rescales it).
// q = max(1, rint(g^gamma * 65535 / gmax)), g = |grad f| by central differences with
// one-sided half differences at the faces.  Every float operation is an explicit
// round-to-nearest intrinsic in a fixed order (no contraction), so the result is
// reproducible bit for bit by any IEEE-754 implementation of the same sequence.
//
// Two HBM sweeps: the first finds gmax (ordered-integer atomicMax), the second
// recomputes g and writes q.  Neighbour reads along y/z come from L1/L2.
#include "common.cuh"

namespace lsrvt {
namespace {

__device__ __forceinline__ float grad_pow(const float *__restrict__ f, Dims d, int32_t x, int32_t y, int32_t z,
                                          int gamma) {
    int32_t xm = x > 0 ? x - 1 : 0, xp = x < d.nx - 1 ? x + 1 : d.nx - 1;
    int32_t ym = y > 0 ? y - 1 : 0, yp = y < d.ny - 1 ? y + 1 : d.ny - 1;
    int32_t zm = z > 0 ? z - 1 : 0, zp = z < d.nz - 1 ? z + 1 : d.nz - 1;
    int64_t row = (int64_t)d.nx * (y + (int64_t)d.ny * z);
    float fxp = f[xp + row], fxm = f[xm + row];
    float fyp = f[x + (int64_t)d.nx * (yp + (int64_t)d.ny * z)];
    float fym = f[x + (int64_t)d.nx * (ym + (int64_t)d.ny * z)];
    float fzp = f[x + (int64_t)d.nx * (y + (int64_t)d.ny * zp)];
    float fzm = f[x + (int64_t)d.nx * (y + (int64_t)d.ny * zm)];
    float dx = __fmul_rn(0.5f, __fsub_rn(fxp, fxm));
    float dy = __fmul_rn(0.5f, __fsub_rn(fyp, fym));
    float dz = __fmul_rn(0.5f, __fsub_rn(fzp, fzm));
    float s = __fmul_rn(dx, dx);
    s = __fadd_rn(s, __fmul_rn(dy, dy));
    s = __fadd_rn(s, __fmul_rn(dz, dz));
    float g = __fsqrt_rn(s);
    float p = g;
    for (int k = 1; k < gamma; ++k) p = __fmul_rn(p, g);
    return p;
}

__global__ void __launch_bounds__(256) saliency_max_kernel(const float *__restrict__ f, Dims d, int gamma,
                                                           unsigned *gmax_bits, VoxelCoder vc) {
    int64_t n = d.n();
    float best = 0.0f;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        vc.decode((uint32_t)v, d, x, y, z);
        float p = grad_pow(f, d, x, y, z, gamma);
        if (isfinite(p) && p > best) best = p;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0 && best > 0.0f) atomicMax(gmax_bits, __float_as_uint(best));
}

__global__ void __launch_bounds__(256) saliency_q_kernel(const float *__restrict__ f, Dims d, int gamma,
                                                         const unsigned *gmax_bits, uint16_t *__restrict__ q,
                                                         VoxelCoder vc) {
    float gmax = __uint_as_float(*gmax_bits);
    float scale = gmax > 0.0f ? __fdiv_rn(65535.0f, gmax) : 0.0f;
    int64_t n = d.n();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        vc.decode((uint32_t)v, d, x, y, z);
        float p = grad_pow(f, d, x, y, z, gamma);
        float t = __fmul_rn(p, scale);
        uint16_t w = 1;
        if (isfinite(p) && t >= 0.5f) {
            float rr = rintf(t);
            if (rr > 65535.0f) rr = 65535.0f;
            w = (uint16_t)rr;
            if (w < 1) w = 1;
        }
        q[v] = w;
    }
}

__global__ void fill_u16_kernel(uint16_t *q, int64_t n, uint16_t val) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        q[v] = val;
}

}  // namespace

size_t saliency_workspace(Dims) { return 256; }

}  // namespace lsrvt

using namespace lsrvt;

extern "C" lsrvt_status lsrvt_saliency_grad(const float *field, lsrvt_dims dd, int32_t gamma, uint16_t *q, void *ws,
                                            size_t ws_bytes, void *stream) {
    if (!dims_ok(dd) || !field || !q || gamma < 0 || gamma > 4) return LSRVT_ERR_INVALID_ARG;
    if (!ws || ws_bytes < saliency_workspace(Dims{dd.nx, dd.ny, dd.nz}) || ((uintptr_t)ws & 255))
        return LSRVT_ERR_WORKSPACE;
    Dims d{dd.nx, dd.ny, dd.nz};
    cudaStream_t s = as_stream(stream);
    int64_t n = d.n();
    int grid = grid_for(n, 256, kSMs * 8);
    if (gamma == 0) {
        fill_u16_kernel<<<grid, 256, 0, s>>>(q, n, 1);
        return launch_status();
    }
    unsigned *gmax = (unsigned *)ws;
    cudaMemsetAsync(gmax, 0, sizeof(unsigned), s);
    const VoxelCoder vc = make_coder(d);
    saliency_max_kernel<<<grid, 256, 0, s>>>(field, d, gamma, gmax, vc);
    saliency_q_kernel<<<grid, 256, 0, s>>>(field, d, gamma, gmax, q, vc);
    return launch_status();
}
