// seed.cu -- stratified random initial sites.  Sec. 3.2 "Stratified Random Initial Site
// Distribution", Eq. (nc), Algorithm 1 (StratifiedRandomSiteDistribution).
//
// Readings (the printed equations are garbled): n_c = max(ceil(|V| m(C) / (P m(V))), 1)
// capped at |C| (alpha = 1/P sites per voxel); strata = component x cubic block of side
// sb aligned to the origin; floor(n_c m_b / m_C) sites per stratum, the remainder by
// largest remainder (ties to the lower block index), capacity caps re-apportioned by the
// same rule; site j of a stratum with k voxels and n_b sites takes the voxel of rank
// floor(j k / n_b) + h_j mod (floor((j+1) k / n_b) - floor(j k / n_b)) in linear order,
// h_j = splitmix64((seed ^ splitmix64(block)) + j).  Site ids: (component, block, j).
//
// GPU design: one CTA per stratification block sorts its (component, local index) keys
// in shared memory (bitonic, <= 4096 keys), so every stratum is a contiguous run with its
// voxels already in linear order.  Stratum records are emitted block by block, sorted
// by component with a stable radix sort (block order is kept inside a component), the
// apportionment runs one CTA per component, and a final per-block pass places sites.
#include "common.cuh"

namespace lsrvt {
namespace {

constexpr int kSeedThreads = 512;
constexpr int kMaxBlockVox = 4096;

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

struct BlockGeom {
    int32_t sb, nbx, nby, nbz;
};

// Load the block's (component << 32 | local index) keys (invalid -> ~0) and sort them.
// Returns the padded power-of-two count; keys[i] for i < npow2 sorted ascending.
__device__ int load_sort_block(const int32_t *__restrict__ comp, Dims d, BlockGeom g, int64_t b,
                               unsigned long long *keys) {
    int sb = g.sb;
    int bx = (int)(b % g.nbx), by = (int)((b / g.nbx) % g.nby), bz = (int)(b / ((int64_t)g.nbx * g.nby));
    int nvox = sb * sb * sb;
    int npow2 = 1;
    while (npow2 < nvox) npow2 <<= 1;
    for (int i = threadIdx.x; i < npow2; i += blockDim.x) {
        unsigned long long k = ~0ULL;
        if (i < nvox) {
            int lx = i % sb, ly = (i / sb) % sb, lz = i / (sb * sb);
            int x = bx * sb + lx, y = by * sb + ly, z = bz * sb + lz;
            if (x < d.nx && y < d.ny && z < d.nz) {
                int32_t c = comp[x + (int64_t)d.nx * (y + (int64_t)d.ny * z)];
                if (c >= 0) k = ((unsigned long long)(uint32_t)c << 32) | (uint32_t)i;
            }
        }
        keys[i] = k;
    }
    __syncthreads();
    // a block inside one component (most of them) is already in (component, index) order
    bool ordered = true;
    for (int i = threadIdx.x; i + 1 < npow2; i += blockDim.x) ordered &= keys[i] <= keys[i + 1];
    if (!__syncthreads_and(ordered)) block_bitonic_sort(keys, npow2);
    return npow2;
}

// The component of block b if every voxel of it lies inside the volume and in that one component
// (the common case away from band boundaries), else -1.  Such a block is one stratum whose
// voxels in (component, index) order are the block's own linear order, so the callers skip the
// sort.  All threads of the CTA call it (it ends with a barrier).
__device__ int32_t uniform_block(const int32_t *__restrict__ comp, Dims d, BlockGeom g, int64_t b) {
    const int sb = g.sb;
    const int bx = (int)(b % g.nbx), by = (int)((b / g.nbx) % g.nby), bz = (int)(b / ((int64_t)g.nbx * g.nby));
    const int x0 = bx * sb, y0 = by * sb, z0 = bz * sb;
    const bool inside = x0 + sb <= d.nx && y0 + sb <= d.ny && z0 + sb <= d.nz;
    const int32_t c0 = inside ? __ldg(comp + x0 + (int64_t)d.nx * (y0 + (int64_t)d.ny * z0)) : -1;
    bool same = inside && c0 >= 0;
    const int nvox = sb * sb * sb;
    for (int i = threadIdx.x; i < nvox && same; i += blockDim.x) {
        const int lx = i % sb, ly = (i / sb) % sb, lz = i / (sb * sb);
        same = __ldg(comp + (x0 + lx) + (int64_t)d.nx * ((y0 + ly) + (int64_t)d.ny * (z0 + lz))) == c0;
    }
    return __syncthreads_and(same) ? c0 : -1;
}

__device__ __forceinline__ int64_t local_to_global(int li, Dims d, BlockGeom g, int64_t b) {
    int sb = g.sb;
    int bx = (int)(b % g.nbx), by = (int)((b / g.nbx) % g.nby), bz = (int)(b / ((int64_t)g.nbx * g.nby));
    int lx = li % sb, ly = (li / sb) % sb, lz = li / (sb * sb);
    return (bx * sb + lx) + (int64_t)d.nx * ((by * sb + ly) + (int64_t)d.ny * (bz * sb + lz));
}

__device__ __forceinline__ bool is_head(const unsigned long long *keys, int i) {
    unsigned long long k = keys[i];
    if (k == ~0ULL) return false;
    return i == 0 || (keys[i - 1] >> 32) != (k >> 32);
}

__global__ void __launch_bounds__(kSeedThreads) seed_block_count_kernel(const int32_t *__restrict__ comp, Dims d,
                                                                         BlockGeom g, int64_t *blk_cnt) {
    __shared__ unsigned long long keys[kMaxBlockVox];
    __shared__ int cnt;
    int64_t nblocks = (int64_t)g.nbx * g.nby * g.nbz;
    for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
        if (uniform_block(comp, d, g, b) >= 0) {
            if (threadIdx.x == 0) blk_cnt[b] = 1;
            continue;
        }
        if (threadIdx.x == 0) cnt = 0;
        int npow2 = load_sort_block(comp, d, g, b, keys);
        int c = 0;
        for (int i = threadIdx.x; i < npow2; i += blockDim.x) c += is_head(keys, i);
        c = __reduce_add_sync(0xffffffffu, (unsigned)c);
        if ((threadIdx.x & 31) == 0 && c) atomicAdd(&cnt, c);
        __syncthreads();
        if (threadIdx.x == 0) blk_cnt[b] = cnt;
        __syncthreads();
    }
}

struct SeedRec {
    uint32_t *comp;   // key for the radix sort
    uint32_t *idx;    // value: record index
    int32_t *block;
    int32_t *k;
    uint64_t *m;
};

// dynamic shared memory: keys[4096] u64 | qpre[4097] u32 | head_pos[4097] u16
constexpr size_t kEmitSmem = kMaxBlockVox * 8 + (kMaxBlockVox + 1) * 4 + (kMaxBlockVox + 1) * 2 + 64;

__global__ void __launch_bounds__(kSeedThreads) seed_block_emit_kernel(const int32_t *__restrict__ comp,
                                                                        const uint16_t *__restrict__ q, Dims d,
                                                                        BlockGeom g, const int64_t *blk_off,
                                                                        int64_t max_rec, SeedRec rec,
                                                                        uint64_t *comp_mass, int64_t *comp_cnt,
                                                                        int64_t *comp_nstr, int32_t max_comp,
                                                                        unsigned long long *totals) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long *keys = (unsigned long long *)smem_raw;
    uint32_t *qpre = (uint32_t *)(keys + kMaxBlockVox);          // exclusive prefix of q in sorted order
    uint16_t *head_pos = (uint16_t *)(qpre + kMaxBlockVox + 1);  // position of the r-th run head
    __shared__ uint32_t warp_q[kSeedThreads / 32];
    __shared__ int warp_h[kSeedThreads / 32];
    int64_t nblocks = (int64_t)g.nbx * g.nby * g.nbz;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
        const int32_t cu = uniform_block(comp, d, g, b);
        if (cu >= 0) {
            // one stratum: all sb^3 voxels, mass = the sum of their weights
            const int nvox = g.sb * g.sb * g.sb;
            unsigned long long qs = 0;
            if (q)
                for (int i = threadIdx.x; i < nvox; i += blockDim.x) qs += q[local_to_global(i, d, g, b)];
            else
                for (int i = threadIdx.x; i < nvox; i += blockDim.x) qs += 1;
            qs = __reduce_add_sync(0xffffffffu, (unsigned)qs);  // at most 4096 x 65535 < 2^32
            if (lane == 0) warp_q[w] = (uint32_t)qs;
            __syncthreads();
            if (threadIdx.x == 0) {
                uint64_t mm = 0;
                for (int k2 = 0; k2 < nw; ++k2) mm += warp_q[k2];
                const int64_t pos = blk_off[b];
                if (pos < max_rec) {
                    rec.comp[pos] = (uint32_t)cu;
                    rec.idx[pos] = (uint32_t)pos;
                    rec.block[pos] = (int32_t)b;
                    rec.k[pos] = nvox;
                    rec.m[pos] = mm;
                }
                if (cu < max_comp) {
                    atomicAdd((unsigned long long *)&comp_mass[cu], (unsigned long long)mm);
                    atomicAdd((unsigned long long *)&comp_cnt[cu], (unsigned long long)nvox);
                    atomicAdd((unsigned long long *)&comp_nstr[cu], 1ULL);
                }
                atomicAdd(&totals[0], (unsigned long long)nvox);
                atomicAdd(&totals[1], (unsigned long long)mm);
            }
            __syncthreads();
            continue;
        }
        int npow2 = load_sort_block(comp, d, g, b, keys);
        // block scan over sorted positions: prefix of q and numbering of run heads
        uint32_t qcarry = 0;
        int hcarry = 0;
        for (int base = 0; base < npow2; base += blockDim.x) {
            int i = base + threadIdx.x;
            unsigned long long k = i < npow2 ? keys[i] : ~0ULL;
            uint32_t qi = 0;
            if (k != ~0ULL) qi = q ? (uint32_t)q[local_to_global((int)(uint32_t)k, d, g, b)] : 1u;
            int h = (i < npow2) ? is_head(keys, i) : 0;
            uint32_t qinc = qi;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t t = __shfl_up_sync(0xffffffffu, qinc, o);
                if (lane >= o) qinc += t;
            }
            unsigned bal = __ballot_sync(0xffffffffu, h);
            if (lane == 31) warp_q[w] = qinc;
            if (lane == 0) warp_h[w] = __popc(bal);
            __syncthreads();
            uint32_t qb = qcarry;
            int hb = hcarry;
            for (int k2 = 0; k2 < w; ++k2) { qb += warp_q[k2]; hb += warp_h[k2]; }
            if (i < npow2) qpre[i] = qb + qinc - qi;
            if (h) head_pos[hb + __popc(bal & lanemask_lt())] = (uint16_t)i;
            for (int k2 = 0; k2 < nw; ++k2) { qcarry += warp_q[k2]; hcarry += warp_h[k2]; }
            __syncthreads();
        }
        int nruns = hcarry;
        // number of valid keys = end of the last run
        __shared__ int nvalid;
        if (threadIdx.x == 0) nvalid = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < npow2; i += blockDim.x)
            if (keys[i] != ~0ULL && (i + 1 == npow2 || keys[i + 1] == ~0ULL)) nvalid = i + 1;
        if (threadIdx.x == 0) qpre[npow2] = qcarry;
        __syncthreads();
        int64_t off = blk_off[b];
        for (int r = threadIdx.x; r < nruns; r += blockDim.x) {
            int s0 = head_pos[r], s1 = (r + 1 < nruns) ? head_pos[r + 1] : nvalid;
            uint32_t c = (uint32_t)(keys[s0] >> 32);
            int32_t kk = s1 - s0;
            uint64_t mm = (uint64_t)(qpre[s1] - qpre[s0]);
            int64_t pos = off + r;
            if (pos < max_rec) {
                rec.comp[pos] = c;
                rec.idx[pos] = (uint32_t)pos;
                rec.block[pos] = (int32_t)b;
                rec.k[pos] = kk;
                rec.m[pos] = mm;
            }
            if ((int32_t)c < max_comp) {
                atomicAdd((unsigned long long *)&comp_mass[c], (unsigned long long)mm);
                atomicAdd((unsigned long long *)&comp_cnt[c], (unsigned long long)kk);
                atomicAdd((unsigned long long *)&comp_nstr[c], 1ULL);
            }
            atomicAdd(&totals[0], (unsigned long long)kk);
            atomicAdd(&totals[1], (unsigned long long)mm);
        }
        __syncthreads();
    }
}

__global__ void seed_check_kernel(const int64_t *n_rec_total, int64_t max_rec, const int32_t *n_comp_dev,
                                  int32_t max_comp, int32_t *n_rec_dev, int32_t *status) {
    int64_t r = *n_rec_total;
    if (r > max_rec) {
        set_status(status, LSRVT_ERR_CAPACITY);
        r = max_rec;
    }
    *n_rec_dev = (int32_t)r;
    if (*n_comp_dev > max_comp) set_status(status, LSRVT_ERR_CAPACITY);
}

__global__ void seed_nc_kernel(const int32_t *n_comp_dev, int32_t max_comp, int64_t P, const uint64_t *comp_mass,
                               const int64_t *comp_cnt, const unsigned long long *totals, int64_t *nc) {
    int32_t ncomp = min(*n_comp_dev, max_comp);
    unsigned __int128 nV = totals[0], mV = totals[1];
    unsigned __int128 den = (unsigned __int128)(uint64_t)P * mV;
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncomp; c += gridDim.x * blockDim.x) {
        unsigned __int128 num = nV * (unsigned __int128)comp_mass[c];
        int64_t k = den ? (int64_t)((num + den - 1) / den) : 1;
        if (k < 1) k = 1;
        if (k > comp_cnt[c]) k = comp_cnt[c];
        nc[c] = k;
    }
}

__global__ void seed_inverse_kernel(const uint32_t *sorted_idx, const int32_t *n_rec_dev, uint32_t *inv) {
    int32_t n = *n_rec_dev;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        inv[sorted_idx[i]] = (uint32_t)i;
}

// ---------------------------------------------------------------- apportionment
constexpr int kApThreads = 128;

template <class T>
__device__ T block_sum(T v, T *red) {
    v = warp_sum(v);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    T s = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    return s;
}

__global__ void __launch_bounds__(kApThreads) seed_apportion_kernel(
    const int32_t *n_comp_dev, int32_t max_comp, const int64_t *nc, const int64_t *cso, const uint32_t *sorted_idx,
    const int32_t *rec_k, const uint64_t *rec_m, int64_t *nb, uint8_t *capped, uint64_t *rem, int32_t *status) {
    __shared__ unsigned long long red_u[kApThreads / 32];
    __shared__ long long red_i[kApThreads / 32];
    int32_t ncomp = min(*n_comp_dev, max_comp);
    for (int32_t c = blockIdx.x; c < ncomp; c += gridDim.x) {
        int64_t s0 = cso[c], s1 = cso[c + 1];
        int64_t n = nc[c];
        if (s1 - s0 == 1) {
            if (threadIdx.x == 0) nb[s0] = n;
            continue;
        }
        for (int64_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) { nb[i] = 0; capped[i] = 0; }
        __syncthreads();
        bool done = false;
        for (int round = 0; round < (1 << 20) && !done; ++round) {
            long long a = 0;
            unsigned long long mA = 0;
            for (int64_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
                a += nb[i];
                if (!capped[i]) mA += rec_m[sorted_idx[i]];
            }
            a = block_sum<long long>(a, red_i);
            mA = block_sum<unsigned long long>(mA, red_u);
            long long remaining = n - a;
            if (remaining <= 0 || mA == 0) break;
            long long given = 0;
            for (int64_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
                if (capped[i]) continue;
                unsigned long long prod = (unsigned long long)remaining * rec_m[sorted_idx[i]];
                unsigned long long fl = prod / mA;
                rem[i] = prod % mA;
                nb[i] += (long long)fl;
                given += (long long)fl;
            }
            given = block_sum<long long>(given, red_i);
            long long left = remaining - given;
            if (left > 0) {
                // largest T with #{uncapped: rem >= T} >= left
                unsigned long long lo = 0, hi = mA;  // invariant: count(lo) >= left, count(hi) < left
                while (hi - lo > 1) {
                    unsigned long long mid = lo + (hi - lo) / 2;
                    long long cnt = 0;
                    for (int64_t i = s0 + threadIdx.x; i < s1; i += blockDim.x)
                        cnt += (!capped[i] && rem[i] >= mid);
                    cnt = block_sum<long long>(cnt, red_i);
                    if (cnt >= left) lo = mid; else hi = mid;
                }
                unsigned long long T = lo;
                long long gt = 0;
                for (int64_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) gt += (!capped[i] && rem[i] > T);
                gt = block_sum<long long>(gt, red_i);
                long long need = left - gt;
                // every uncapped stratum with rem > T gets one; among rem == T the first `need` by position
                long long carry = 0;
                for (int64_t base = s0; base < s1; base += blockDim.x) {
                    int64_t i = base + threadIdx.x;
                    bool inr = i < s1;
                    bool eq = inr && !capped[i] && rem[i] == T;
                    bool g2 = inr && !capped[i] && rem[i] > T;
                    unsigned bal = __ballot_sync(0xffffffffu, eq);
                    __shared__ int wc[kApThreads / 32];
                    int w = threadIdx.x >> 5;
                    if ((threadIdx.x & 31) == 0) wc[w] = __popc(bal);
                    __syncthreads();
                    long long before = carry;
                    for (int k = 0; k < w; ++k) before += wc[k];
                    long long my = before + __popc(bal & lanemask_lt());
                    if (g2 || (eq && my < need)) nb[i] += 1;
                    long long tot = 0;
                    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += wc[k];
                    __syncthreads();
                    carry += tot;
                }
            }
            int any = 0;
            for (int64_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
                int32_t k = rec_k[sorted_idx[i]];
                if (!capped[i] && nb[i] > k) { nb[i] = k; capped[i] = 1; any = 1; }
            }
            any = __syncthreads_or(any);
            if (!any) done = true;
            __syncthreads();
            if (round == (1 << 20) - 1) set_status(status, LSRVT_ERR_TIMEOUT);
        }
        __syncthreads();
    }
}

__global__ void seed_offsets_kernel(const int32_t *n_comp_dev, int32_t max_comp, const int64_t *cso,
                                    const int64_t *site_off, const int64_t *n_sites_total, int32_t *comp_site_off,
                                    int32_t *n_sites_dev, int32_t max_sites, int32_t *status) {
    int32_t ncomp = min(*n_comp_dev, max_comp);
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c <= ncomp; c += gridDim.x * blockDim.x) {
        if (c == ncomp) comp_site_off[c] = (int32_t)min(*n_sites_total, (int64_t)INT32_MAX);
        else comp_site_off[c] = (int32_t)site_off[cso[c]];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int64_t t = *n_sites_total;
        *n_sites_dev = (int32_t)min(t, (int64_t)INT32_MAX);
        if (t > max_sites) set_status(status, LSRVT_ERR_CAPACITY);
    }
}

__global__ void __launch_bounds__(kSeedThreads) seed_place_kernel(const int32_t *__restrict__ comp, Dims d,
                                                                   BlockGeom g, const int64_t *blk_off,
                                                                   int64_t max_rec, const uint32_t *inv,
                                                                   const int32_t *rec_k,
                                                                   const int64_t *nb, const int64_t *site_off,
                                                                   uint64_t seed, int32_t *site_pos,
                                                                   int32_t *site_comp, int32_t max_sites) {
    __shared__ unsigned long long keys[kMaxBlockVox];
    int64_t nblocks = (int64_t)g.nbx * g.nby * g.nbz;
    for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
        int64_t off = blk_off[b];
        uint64_t hb = seed ^ splitmix64((uint64_t)b);
        const int32_t cu = uniform_block(comp, d, g, b);
        if (cu >= 0) {
            // one stratum in the block's linear order: the voxel of rank r is local index r
            const int64_t r = off;
            if (r < max_rec) {
                const int64_t k = rec_k[r];
                const uint32_t pos = inv[r];
                const int64_t n_b = nb[pos], so = site_off[pos];
                for (int64_t j = threadIdx.x; j < n_b; j += blockDim.x) {
                    uint64_t lo = (uint64_t)j * (uint64_t)k / (uint64_t)n_b;
                    uint64_t hi = (uint64_t)(j + 1) * (uint64_t)k / (uint64_t)n_b;
                    uint64_t h2 = splitmix64(hb + (uint64_t)j);
                    uint64_t rank = lo + h2 % (hi - lo);
                    int64_t sid = so + j;
                    if (sid < max_sites) {
                        site_pos[sid] = (int32_t)local_to_global((int)rank, d, g, b);
                        site_comp[sid] = cu;
                    }
                }
            }
            __syncthreads();
            continue;
        }
        int npow2 = load_sort_block(comp, d, g, b, keys);
        // one warp per run head found by scanning positions
        int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        // runs: enumerate heads in order; count heads before each head with a running scan
        int run = 0;
        for (int base = 0; base < npow2; base += 32) {
            int i = base + lane;
            bool h = i < npow2 && is_head(keys, i);
            unsigned bal = __ballot_sync(0xffffffffu, h);
            while (bal) {
                int l = __ffs(bal) - 1;
                bal &= bal - 1;
                int hp = base + l;
                if ((run % nw) == w) {
                    // stratum run starting at hp
                    uint32_t c = (uint32_t)(keys[hp] >> 32);
                    int64_t r = off + run;
                    if (r < max_rec) {
                        int64_t k = rec_k[r];
                        uint32_t pos = inv[r];
                        int64_t n_b = nb[pos], so = site_off[pos];
                        for (int64_t j = lane; j < n_b; j += 32) {
                            uint64_t lo = (uint64_t)j * (uint64_t)k / (uint64_t)n_b;
                            uint64_t hi = (uint64_t)(j + 1) * (uint64_t)k / (uint64_t)n_b;
                            uint64_t h2 = splitmix64(hb + (uint64_t)j);
                            uint64_t rank = lo + h2 % (hi - lo);
                            int li = (int)(uint32_t)keys[hp + rank];
                            int64_t sid = so + j;
                            if (sid < max_sites) {
                                site_pos[sid] = (int32_t)local_to_global(li, d, g, b);
                                site_comp[sid] = (int32_t)c;
                            }
                        }
                    }
                }
                ++run;
            }
        }
        __syncthreads();
    }
}

struct SeedWs {
    int64_t *blk_cnt;     // [nblocks] -> exclusive offsets
    int64_t *rec_total;
    int32_t *n_rec;
    SeedRec rec;
    uint32_t *inv;
    int64_t *nb;          // sorted order
    int64_t *site_off;    // sorted order
    int64_t *n_sites_total;
    uint8_t *capped;
    uint64_t *rem;
    uint64_t *comp_mass;
    int64_t *comp_cnt;
    int64_t *comp_nstr;   // -> exclusive offsets (cso), size max_comp + 1
    int64_t *nc;
    unsigned long long *totals;
    int64_t *cso_total;
    void *scan;
    void *radix;
};

int64_t default_max_strata(Dims d, int32_t sb, int32_t max_comp) {
    int64_t n = d.n();
    int64_t nblocks = (int64_t)((d.nx + sb - 1) / sb) * ((d.ny + sb - 1) / sb) * ((d.nz + sb - 1) / sb);
    int64_t r = 4 * nblocks + (int64_t)max_comp + 1024;
    return r < n ? r : n;
}

SeedWs carve_seed(void *ws, size_t bytes, Dims d, int32_t sb, int32_t max_comp, int64_t max_rec, size_t *need) {
    Carver c(ws, bytes);
    int64_t nblocks = (int64_t)((d.nx + sb - 1) / sb) * ((d.ny + sb - 1) / sb) * ((d.nz + sb - 1) / sb);
    SeedWs w;
    w.blk_cnt = c.take<int64_t>(nblocks + 1);
    w.rec_total = c.take<int64_t>(1);
    w.n_rec = c.take<int32_t>(1);
    w.rec.comp = c.take<uint32_t>(max_rec);
    w.rec.idx = c.take<uint32_t>(max_rec);
    w.rec.block = c.take<int32_t>(max_rec);
    w.rec.k = c.take<int32_t>(max_rec);
    w.rec.m = c.take<uint64_t>(max_rec);
    w.inv = c.take<uint32_t>(max_rec);
    w.nb = c.take<int64_t>(max_rec);
    w.site_off = c.take<int64_t>(max_rec);
    w.n_sites_total = c.take<int64_t>(1);
    w.capped = c.take<uint8_t>(max_rec);
    w.rem = c.take<uint64_t>(max_rec);
    w.comp_mass = c.take<uint64_t>(max_comp + 1);
    w.comp_cnt = c.take<int64_t>(max_comp + 1);
    w.comp_nstr = c.take<int64_t>(max_comp + 1);
    w.nc = c.take<int64_t>(max_comp + 1);
    w.totals = c.take<unsigned long long>(2);
    w.cso_total = c.take<int64_t>(1);
    int64_t scan_n = nblocks + 1;
    if (scan_n < max_rec) scan_n = max_rec;
    if (scan_n < max_comp + 1) scan_n = max_comp + 1;
    w.scan = c.take<char>(scan_temp_bytes(scan_n));
    w.radix = c.take<char>(radix_temp_bytes(max_rec));
    *need = c.used;
    return w;
}

}  // namespace

size_t seed_workspace(Dims d, int32_t sb, int32_t max_comp, int64_t max_rec) {
    size_t need;
    carve_seed(nullptr, 0, d, sb, max_comp, max_rec, &need);
    return need;
}

int64_t seed_default_strata(Dims d, int32_t sb, int32_t max_comp) { return default_max_strata(d, sb, max_comp); }

}  // namespace lsrvt

using namespace lsrvt;

extern "C" lsrvt_status lsrvt_seed(const int32_t *comp, const uint16_t *q, lsrvt_dims dd, const int32_t *n_comp_dev,
                                   int32_t max_comp, lsrvt_seed_params p, int32_t *site_pos, int32_t *site_comp,
                                   int32_t *comp_site_off, int32_t max_sites, int32_t *n_sites_dev, void *ws,
                                   size_t ws_bytes, int32_t *status_dev, void *stream) {
    if (!dims_ok(dd) || !comp || !n_comp_dev || max_comp < 0 || !site_pos || !site_comp || !comp_site_off ||
        max_sites < 0 || !n_sites_dev || p.voxels_per_site < 1 || p.strat_block < 1 || p.strat_block > 16 ||
        p.max_strata < 0)
        return LSRVT_ERR_INVALID_ARG;
    Dims d{dd.nx, dd.ny, dd.nz};
    int32_t sb = p.strat_block;
    int64_t max_rec = p.max_strata > 0 ? p.max_strata : default_max_strata(d, sb, max_comp);
    size_t need;
    SeedWs w = carve_seed(ws, ws_bytes, d, sb, max_comp, max_rec, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) return LSRVT_ERR_WORKSPACE;
    cudaStream_t s = as_stream(stream);
    BlockGeom g{sb, (d.nx + sb - 1) / sb, (d.ny + sb - 1) / sb, (d.nz + sb - 1) / sb};
    int64_t nblocks = (int64_t)g.nbx * g.nby * g.nbz;
    int bgrid = (int)(nblocks < kSMs * 16 ? nblocks : kSMs * 16);
    cudaMemsetAsync(w.comp_mass, 0, sizeof(uint64_t) * (max_comp + 1), s);
    cudaMemsetAsync(w.comp_cnt, 0, sizeof(int64_t) * (max_comp + 1), s);
    cudaMemsetAsync(w.comp_nstr, 0, sizeof(int64_t) * (max_comp + 1), s);
    cudaMemsetAsync(w.totals, 0, sizeof(unsigned long long) * 2, s);
    seed_block_count_kernel<<<bgrid, kSeedThreads, 0, s>>>(comp, d, g, w.blk_cnt);
    exclusive_scan_i64(w.blk_cnt, nblocks, w.rec_total, w.scan, s);
    seed_check_kernel<<<1, 1, 0, s>>>(w.rec_total, max_rec, n_comp_dev, max_comp, w.n_rec, status_dev);
    cudaFuncSetAttribute(seed_block_emit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEmitSmem);
    seed_block_emit_kernel<<<bgrid, kSeedThreads, kEmitSmem, s>>>(comp, q, d, g, w.blk_cnt, max_rec, w.rec, w.comp_mass,
                                                           w.comp_cnt, w.comp_nstr, max_comp, w.totals);
    int cgrid = grid_for(max_comp, 256, kSMs * 8);
    seed_nc_kernel<<<cgrid, 256, 0, s>>>(n_comp_dev, max_comp, p.voxels_per_site, w.comp_mass, w.comp_cnt, w.totals,
                                         w.nc);
    int bits = 1;
    while (bits < 32 && ((int64_t)1 << bits) < (int64_t)max_comp + 1) ++bits;
    radix_sort_pairs(w.rec.comp, w.rec.idx, max_rec, w.n_rec, bits, w.radix, s);
    seed_inverse_kernel<<<grid_for(max_rec, 256, kSMs * 8), 256, 0, s>>>(w.rec.idx, w.n_rec, w.inv);
    // strata offsets per component (comp_nstr -> cso)
    exclusive_scan_i64(w.comp_nstr, (int64_t)max_comp + 1, w.cso_total, w.scan, s);
    cudaMemsetAsync(w.nb, 0, sizeof(int64_t) * max_rec, s);
    seed_apportion_kernel<<<kSMs * 8, kApThreads, 0, s>>>(n_comp_dev, max_comp, w.nc, w.comp_nstr, w.rec.idx,
                                                          w.rec.k, w.rec.m, w.nb, w.capped, w.rem, status_dev);
    // site offsets in sorted (component, block) order
    cudaMemcpyAsync(w.site_off, w.nb, sizeof(int64_t) * max_rec, cudaMemcpyDeviceToDevice, s);
    exclusive_scan_i64(w.site_off, max_rec, w.n_sites_total, w.scan, s);
    seed_offsets_kernel<<<grid_for((int64_t)max_comp + 1, 256, kSMs * 8), 256, 0, s>>>(
        n_comp_dev, max_comp, w.comp_nstr, w.site_off, w.n_sites_total, comp_site_off, n_sites_dev, max_sites,
        status_dev);
    seed_place_kernel<<<bgrid, kSeedThreads, 0, s>>>(comp, d, g, w.blk_cnt, max_rec, w.inv, w.rec.k, w.nb, w.site_off,
                                                      p.rng_seed, site_pos, site_comp, max_sites);
    return launch_status();
}
