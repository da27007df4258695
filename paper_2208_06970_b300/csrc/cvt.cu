// cvt.cu -- Lloyd iterations of the level set restricted CVT (Algorithm 1, LRCVT):
// restricted geodesic Voronoi tessellation (Eq. 1) and geodesically weighted site update
// (Eq. 2), n_iters times, then a final tessellation.
//
// Tessellation.  Every voxel holds a 64-bit key (distance << 32 | site): 16.16 fixed-point
// geodesic distance and site id, compared lexicographically.  The solution of the
// restricted multi-source shortest-path problem under this order is unique, and any
// sequence of valid relaxations that ends with every edge relaxed reaches it, so the
// labels are deterministic whatever the schedule.  B300 design: the volume is cut into
// 16x8x8 bricks; a CTA loads a brick plus a one-voxel halo of keys and bands into shared
// memory, derives the 26-bit edge mask of every voxel (an edge exists when the box it
// spans is in one band), and relaxes in place (pull updates from the 26 neighbours)
// only where a neighbour changed in the previous step (row bitmasks dilated each step),
// until nothing changes.  Improved keys are written back; bricks whose boundary layer
// changed queue their neighbours for the next round (deduplicated by a per-brick tag).
// Rounds run until the queue is empty.
//
// Update (Eq. 2).  One pass over the voxels: a voxel at distance 0 is its site; other
// voxels walk the 6-connected traversal toward their site (line of sight); LOS voxels add
// q * coords to their site's integer sums (warp-aggregated atomics); the rest record
// their parent (first neighbour in (dz,dy,dx) order on a shortest path to the same site)
// and are resolved in a second pass by walking parents to the first LOS voxel (phi).  A
// per-site pass rounds the centroid half up and walks the site toward it, stopping before
// it would leave its band.
#include <cstdio>

#include "common.cuh"

namespace lsrvt {
namespace {

constexpr int RX = 16, RY = 8, RZ = 8, RV = RX * RY * RZ;  // brick 1024 voxels
constexpr int HX = RX + 2, HY = RY + 2, HZ = RZ + 2, HV = HX * HY * HZ;
constexpr int kRelaxThreads = 256;
constexpr int kVPT = RV / kRelaxThreads;  // 4 voxels per thread
constexpr int kRows = RY * RZ;            // 64 x-rows of 16 voxels
constexpr uint32_t kInf32 = 0xFFFFFFFFu;
constexpr unsigned long long kInfKey = ~0ULL;
constexpr int kMaxSteps = 256;  // in-brick relaxation steps per visit (the brick requeues itself past this)

struct BrickGeom {
    int32_t nbx, nby, nbz;
};

// box mask of offset o = (dx,dy,dz): bits of every (ax dx, ay dy, az dz), a in {0,1}^3
__host__ __device__ constexpr uint32_t box_mask(int o) {
    int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
    uint32_t m = 0;
    for (int az = 0; az <= 1; ++az)
        for (int ay = 0; ay <= 1; ++ay)
            for (int ax = 0; ax <= 1; ++ax) m |= 1u << ((az * dz + 1) * 9 + (ay * dy + 1) * 3 + (ax * dx + 1));
    return m;
}

__host__ __device__ constexpr uint32_t weight_of(int o) {
    int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
    int k = (dx != 0) + (dy != 0) + (dz != 0);
    return k == 1 ? kWFace : (k == 2 ? kWEdge : kWCorner);
}

__host__ __device__ constexpr int halo_off(int o) {
    return (o % 3 - 1) + HX * ((o / 3) % 3 - 1 + HY * (o / 9 - 1));
}

// 26-bit edge mask from the 27-bit "same band" mask S (bit 13 = the voxel itself)
__device__ __forceinline__ uint32_t edges_from_same(uint32_t S) {
    uint32_t e = 0;
#pragma unroll
    for (int o = 0; o < 27; ++o) {
        if (o == 13) continue;
        constexpr uint32_t dummy = 0;
        (void)dummy;
        uint32_t bm = box_mask(o);
        if ((S & bm) == bm) e |= 1u << o;
    }
    return e;
}

__global__ void __launch_bounds__(kRelaxThreads) relax_round_kernel(
    const uint8_t *__restrict__ band, Dims d, BrickGeom bg, unsigned long long *key, const int32_t *__restrict__ list_in,
    const int32_t *n_in, int32_t *list_out, int32_t *n_out, uint32_t *flags, uint32_t tag, int32_t *work,
    int32_t *status) {
    // packed keys: one aligned 64-bit access per read/write, so a reader never pairs the
    // distance of one update with the site of another
    __shared__ unsigned long long sk[HV];
    __shared__ uint8_t sb[HV];
    __shared__ uint32_t changed[kRows];
    __shared__ uint32_t dirty[kRows];
    __shared__ uint32_t touch;
    __shared__ int item;
    const int tid = threadIdx.x;
    const int nin = *n_in;
    while (true) {
        if (tid == 0) item = atomicAdd(work, 1);
        __syncthreads();
        const int it = item;
        if (it >= nin) break;
        const int brick = list_in[it];
        const int bx = brick % bg.nbx, by = (brick / bg.nbx) % bg.nby, bz = brick / (bg.nbx * bg.nby);
        const int ox = bx * RX, oy = by * RY, oz = bz * RZ;
        // ---- load halo
        for (int i = tid; i < HV; i += kRelaxThreads) {
            int hx = i % HX, hy = (i / HX) % HY, hz = i / (HX * HY);
            int gx = ox + hx - 1, gy = oy + hy - 1, gz = oz + hz - 1;
            uint8_t b = kInvalidBand;
            unsigned long long k = kInfKey;
            if (gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny && gz >= 0 && gz < d.nz) {
                int64_t g = gx + (int64_t)d.nx * (gy + (int64_t)d.ny * gz);
                b = band[g];
                k = __ldcg(key + g);
            }
            sb[i] = b;
            sk[i] = k;
        }
        if (tid < kRows) {
            changed[tid] = 0;
            dirty[tid] = 0xFFFFu;
        }
        if (tid == 0) touch = 0;
        __syncthreads();
        // ---- edge masks and original keys
        unsigned long long orig[kVPT];
        uint32_t em[kVPT];
#pragma unroll
        for (int j = 0; j < kVPT; ++j) {
            int i = tid + kRelaxThreads * j;
            int lx = i & (RX - 1), ly = (i >> 4) & (RY - 1), lz = i >> 7;
            int h = (lx + 1) + HX * ((ly + 1) + HY * (lz + 1));
            uint8_t b = sb[h];
            uint32_t e = 0;
            if (b != kInvalidBand) {
                uint32_t S = 0;
#pragma unroll
                for (int o = 0; o < 27; ++o) S |= (uint32_t)(sb[h + halo_off(o)] == b) << o;
                e = edges_from_same(S);
            }
            em[j] = e;
            orig[j] = sk[h];
        }
        __syncthreads();
        // ---- relaxation steps
        int step = 0;
        for (; step < kMaxSteps; ++step) {
            int any = 0;
#pragma unroll
            for (int j = 0; j < kVPT; ++j) {
                int i = tid + kRelaxThreads * j;
                int lx = i & (RX - 1), row = i >> 4;
                uint32_t e = em[j];
                if (!e || !((dirty[row] >> lx) & 1u)) continue;
                int ly = row & (RY - 1), lz = row >> 3;
                int h = (lx + 1) + HX * ((ly + 1) + HY * (lz + 1));
                unsigned long long best = sk[h];
                unsigned long long own = best;
#pragma unroll
                for (int o = 0; o < 27; ++o) {
                    if (o == 13) continue;
                    if (!((e >> o) & 1u)) continue;
                    int u = h + halo_off(o);
                    unsigned long long ku = sk[u];
                    uint32_t du = (uint32_t)(ku >> 32);
                    if (du == kInf32) continue;
                    unsigned long long cd = (unsigned long long)du + weight_of(o);
                    if (cd >= kInf32) {
                        set_status(status, LSRVT_ERR_OVERFLOW);
                        continue;
                    }
                    if ((cd << 32) > best) continue;  // distance alone already worse
                    unsigned long long cand = (cd << 32) | (ku & 0xFFFFFFFFull);
                    if (cand < best) best = cand;
                }
                if (best < own) {
                    sk[h] = best;
                    atomicOr(&changed[row], 1u << lx);
                    any = 1;
                }
            }
            if (!__syncthreads_or(any)) break;
            if (tid < kRows) {
                int ly = tid & (RY - 1), lz = tid >> 3;
                uint32_t m = 0;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy) {
                        int y2 = ly + dy, z2 = lz + dz;
                        if (y2 < 0 || y2 >= RY || z2 < 0 || z2 >= RZ) continue;
                        uint32_t c = changed[y2 + RY * z2];
                        m |= c | (c << 1) | (c >> 1);
                    }
                dirty[tid] = m & 0xFFFFu;
            }
            __syncthreads();
            if (tid < kRows) changed[tid] = 0;
            __syncthreads();
        }
        // ---- write back and collect the neighbour bricks to requeue
        uint32_t my_touch = step >= kMaxSteps ? (1u << 13) : 0u;
#pragma unroll
        for (int j = 0; j < kVPT; ++j) {
            int i = tid + kRelaxThreads * j;
            int lx = i & (RX - 1), ly = (i >> 4) & (RY - 1), lz = i >> 7;
            int h = (lx + 1) + HX * ((ly + 1) + HY * (lz + 1));
            unsigned long long nk = sk[h];
            if (nk == orig[j]) continue;
            int gx = ox + lx, gy = oy + ly, gz = oz + lz;
            key[gx + (int64_t)d.nx * (gy + (int64_t)d.ny * gz)] = nk;
            int xs0 = lx == 0 ? -1 : 0, xs1 = lx == RX - 1 ? 1 : 0;
            int ys0 = ly == 0 ? -1 : 0, ys1 = ly == RY - 1 ? 1 : 0;
            int zs0 = lz == 0 ? -1 : 0, zs1 = lz == RZ - 1 ? 1 : 0;
            for (int a = zs0; a <= zs1; ++a)
                for (int b2 = ys0; b2 <= ys1; ++b2)
                    for (int c = xs0; c <= xs1; ++c)
                        if (a || b2 || c) my_touch |= 1u << ((a + 1) * 9 + (b2 + 1) * 3 + (c + 1));
        }
        if (my_touch) atomicOr(&touch, my_touch);
        __syncthreads();
        if (tid < 27 && ((touch >> tid) & 1u)) {
            int nx2 = bx + tid % 3 - 1, ny2 = by + (tid / 3) % 3 - 1, nz2 = bz + tid / 9 - 1;
            if (nx2 >= 0 && nx2 < bg.nbx && ny2 >= 0 && ny2 < bg.nby && nz2 >= 0 && nz2 < bg.nbz) {
                int nb = nx2 + bg.nbx * (ny2 + bg.nby * nz2);
                if (atomicExch(&flags[nb], tag) != tag) {
                    int pos = atomicAdd(n_out, 1);
                    list_out[pos] = nb;
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- closed-form initialisation
// Lower bound: the unconstrained 26-neighbour chamfer distance C(v, s) = (a-b) W1 +
// (b-c) W2 + c W3 (a >= b >= c the sorted |v - s|) never exceeds the restricted geodesic
// gd(v, s).  So min over the same-band sites of (C(v, s), s) is a lexicographic lower
// bound of v's key; if one shortest chamfer path from v to that site s* stays in the band
// (every edge box in band), gd(v, s*) = C(v, s*) is attained and the bound IS the key.
// Sites are binned by brick; a CTA gathers the sites of the bricks within +-1 (x) / +-2
// (y, z) bricks, so any site outside is at Chebyshev distance >= gap(v) and chamfer
// distance >= gap(v) W1; the key is confirmed only when it is below that.  Unconfirmed
// voxels start at +inf and their bricks are relaxed.
constexpr int kSX = 1, kSY = 2, kSZ = 2;
constexpr int kMaxCand = 1024;

__device__ __forceinline__ unsigned long long chamfer(int dx, int dy, int dz) {
    unsigned a = abs(dx), b = abs(dy), c = abs(dz), t;
    if (a < b) { t = a; a = b; b = t; }
    if (b < c) { t = b; b = c; c = t; }
    if (a < b) { t = a; a = b; b = t; }
    return (unsigned long long)(a - b) * kWFace + (unsigned long long)(b - c) * kWEdge +
           (unsigned long long)c * kWCorner;
}

// One shortest chamfer path from v to s (26-connected digital line: the dominant axis
// advances every step, the middle axis by rounded proportion, the smallest axis only on
// middle-axis steps so that no corner move is split); true if every move's box is in band b.
__device__ bool chamfer_path_in_band(const uint8_t *__restrict__ band, Dims d, int vx, int vy, int vz, int sx,
                                     int sy, int sz, uint8_t b) {
    int D[3] = {sx - vx, sy - vy, sz - vz};
    int A[3] = {abs(D[0]), abs(D[1]), abs(D[2])};
    int S[3] = {D[0] < 0 ? -1 : 1, D[1] < 0 ? -1 : 1, D[2] < 0 ? -1 : 1};
    int i = 0, j = 1, k = 2, t;
    if (A[i] < A[j]) { t = i; i = j; j = t; }
    if (A[j] < A[k]) { t = j; j = k; k = t; }
    if (A[i] < A[j]) { t = i; i = j; j = t; }
    const int ai = A[i], aj = A[j], ak = A[k];
    int p[3] = {vx, vy, vz};
    int jc = 0, kc = 0;
    const int64_t sxy = (int64_t)d.nx * d.ny;
    for (int step = 1; step <= ai; ++step) {
        int jt = (int)((2LL * step * aj + ai) / (2LL * ai));
        bool mj = jt > jc;
        bool mk = false;
        if (mj) {
            int kt = (int)((2LL * (jc + 1) * ak + aj) / (2LL * aj));
            mk = kt > kc;
        }
        int m[3] = {0, 0, 0};
        m[i] = S[i];
        if (mj) m[j] = S[j];
        if (mk) m[k] = S[k];
        // every voxel of the box spanned by p and p + m, except p itself
        for (int az = 0; az <= (m[2] != 0); ++az)
            for (int ay = 0; ay <= (m[1] != 0); ++ay)
                for (int ax = 0; ax <= (m[0] != 0); ++ax) {
                    if (!ax && !ay && !az) continue;
                    int64_t g = (p[0] + ax * m[0]) + (int64_t)d.nx * (p[1] + ay * m[1]) + sxy * (p[2] + az * m[2]);
                    if (__ldg(band + g) != b) return false;
                }
        p[0] += m[0]; p[1] += m[1]; p[2] += m[2];
        jc += mj;
        kc += mk;
    }
    return true;
}

__global__ void site_bin_count_kernel(const int32_t *__restrict__ site_pos, const int32_t *n_sites_dev,
                                      int32_t max_sites, Dims d, BrickGeom bg, int64_t *bin_cnt, int32_t *status) {
    int32_t ns = min(*n_sites_dev, max_sites);
    int64_t n = d.n();
    for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
        int32_t p = site_pos[s];
        if (p < 0 || p >= n) {
            set_status(status, LSRVT_ERR_INVALID_ARG);
            continue;
        }
        int32_t x = p % d.nx, y = (p / d.nx) % d.ny, z = p / (d.nx * d.ny);
        atomicAdd((unsigned long long *)&bin_cnt[x / RX + bg.nbx * (y / RY + bg.nby * (z / RZ))], 1ULL);
    }
}

__global__ void site_bin_fill_kernel(const int32_t *__restrict__ site_pos, const int32_t *n_sites_dev,
                                     int32_t max_sites, const uint8_t *__restrict__ band, Dims d, BrickGeom bg,
                                     const int64_t *__restrict__ bin_off, int32_t *cursor, int4 *cand) {
    int32_t ns = min(*n_sites_dev, max_sites);
    int64_t n = d.n();
    for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
        int32_t p = site_pos[s];
        if (p < 0 || p >= n) continue;
        int32_t x = p % d.nx, y = (p / d.nx) % d.ny, z = p / (d.nx * d.ny);
        int b = x / RX + bg.nbx * (y / RY + bg.nby * (z / RZ));
        int64_t pos = bin_off[b] + atomicAdd(&cursor[b], 1);
        cand[pos] = make_int4(s, x, y, z | ((int)band[p] << 24));
    }
}

__global__ void __launch_bounds__(kRelaxThreads) cfi_kernel(const uint8_t *__restrict__ band, Dims d, BrickGeom bg,
                                                            const int64_t *__restrict__ bin_off,
                                                            const int4 *__restrict__ cand, unsigned long long *key,
                                                            int32_t *list_out, int32_t *n_out, uint32_t *flags,
                                                            uint32_t tag) {
    __shared__ int4 cs[kMaxCand];
    __shared__ unsigned long long ck[kMaxCand];
    __shared__ int ncand_s, unknown_s;
    const int tid = threadIdx.x;
    const int64_t nbricks = (int64_t)bg.nbx * bg.nby * bg.nbz;
    for (int64_t brick = blockIdx.x; brick < nbricks; brick += gridDim.x) {
        const int bx = (int)(brick % bg.nbx), by = (int)((brick / bg.nbx) % bg.nby),
                  bz = (int)(brick / ((int64_t)bg.nbx * bg.nby));
        const int ox = bx * RX, oy = by * RY, oz = bz * RZ;
        if (tid == 0) { ncand_s = 0; unknown_s = 0; }
        __syncthreads();
        // gather the sites of the neighbouring bins
        constexpr int NBX = 2 * kSX + 1, NBY = 2 * kSY + 1, NBZ = 2 * kSZ + 1;
        for (int q = tid; q < NBX * NBY * NBZ; q += blockDim.x) {
            int cx = bx + q % NBX - kSX, cy = by + (q / NBX) % NBY - kSY, cz = bz + q / (NBX * NBY) - kSZ;
            if (cx < 0 || cx >= bg.nbx || cy < 0 || cy >= bg.nby || cz < 0 || cz >= bg.nbz) continue;
            int64_t bb = cx + (int64_t)bg.nbx * (cy + (int64_t)bg.nby * cz);
            int64_t a0 = bin_off[bb], a1 = bin_off[bb + 1];
            int cnt = (int)(a1 - a0);
            if (cnt == 0) continue;
            int at = atomicAdd(&ncand_s, cnt);
            for (int r = 0; r < cnt && at + r < kMaxCand; ++r) cs[at + r] = cand[a0 + r];
        }
        __syncthreads();
        const int nc = ncand_s;
        const bool overflow = nc > kMaxCand;
        int npow2 = 1;
        if (!overflow) {
            while (npow2 < nc) npow2 <<= 1;
            for (int i = tid; i < npow2; i += blockDim.x) {
                unsigned long long e = ~0ULL;
                if (i < nc) {
                    int4 c = cs[i];
                    int cz = c.w & 0xFFFFFF;
                    int gx = max(max(ox - c.y, c.y - (ox + RX - 1)), 0);
                    int gy = max(max(oy - c.z, c.z - (oy + RY - 1)), 0);
                    int gz = max(max(oz - cz, cz - (oz + RZ - 1)), 0);
                    unsigned long long lb = (unsigned long long)max(gx, max(gy, gz)) * kWFace;
                    e = (lb << 32) | (unsigned)i;
                }
                ck[i] = e;
            }
            block_bitonic_sort(ck, npow2);
        }
        // search box in voxels and whether it reaches the volume faces
        const int lox = (bx - kSX) * RX, hix = (bx + kSX + 1) * RX - 1;
        const int loy = (by - kSY) * RY, hiy = (by + kSY + 1) * RY - 1;
        const int loz = (bz - kSZ) * RZ, hiz = (bz + kSZ + 1) * RZ - 1;
        int unknown = 0;
#pragma unroll
        for (int j = 0; j < kVPT; ++j) {
            int i = tid + kRelaxThreads * j;
            int lx = i & (RX - 1), ly = (i >> 4) & (RY - 1), lz = i >> 7;
            int x = ox + lx, y = oy + ly, z = oz + lz;
            if (x >= d.nx || y >= d.ny || z >= d.nz) continue;
            int64_t g = x + (int64_t)d.nx * (y + (int64_t)d.ny * z);
            uint8_t b = band[g];
            unsigned long long best = kInfKey;
            int best_i = -1;
            if (b != kInvalidBand && !overflow) {
                for (int t = 0; t < nc; ++t) {
                    unsigned long long e = ck[t];
                    if ((e >> 32) > (best >> 32)) break;
                    int4 c = cs[(unsigned)e];
                    if ((uint8_t)(c.w >> 24) != b) continue;
                    unsigned long long cd = chamfer(c.y - x, c.z - y, (c.w & 0xFFFFFF) - z);
                    if (cd >= kInf32) continue;
                    unsigned long long k2 = (cd << 32) | (unsigned)c.x;
                    if (k2 < best) { best = k2; best_i = (int)(unsigned)e; }
                }
                if (best != kInfKey) {
                    long long gap = 1LL << 40;
                    if (lox > 0) gap = min(gap, (long long)(x - lox + 1));
                    if (hix < d.nx - 1) gap = min(gap, (long long)(hix - x + 1));
                    if (loy > 0) gap = min(gap, (long long)(y - loy + 1));
                    if (hiy < d.ny - 1) gap = min(gap, (long long)(hiy - y + 1));
                    if (loz > 0) gap = min(gap, (long long)(z - loz + 1));
                    if (hiz < d.nz - 1) gap = min(gap, (long long)(hiz - z + 1));
                    bool in_range = (best >> 32) < (unsigned long long)gap * kWFace;
                    bool ok = false;
                    if (in_range) {
                        int4 c = cs[best_i];
                        ok = chamfer_path_in_band(band, d, x, y, z, c.y, c.z, c.w & 0xFFFFFF, b);
                    }
                    if (!ok) best = kInfKey;
                }
                if (best == kInfKey) unknown = 1;
            } else if (b != kInvalidBand) {
                unknown = 1;  // candidate list overflowed: relax the whole brick
            }
            key[g] = best;
        }
        if (unknown) unknown_s = 1;
        __syncthreads();
        // the brick's own sites: distance 0, lowest id (needed where the candidate list overflowed)
        {
            int64_t a0 = bin_off[brick], a1 = bin_off[brick + 1];
            for (int64_t r = a0 + tid; r < a1; r += blockDim.x) {
                int4 c = cand[r];
                int64_t g = c.y + (int64_t)d.nx * (c.z + (int64_t)d.ny * (c.w & 0xFFFFFF));
                atomicMin(key + g, (unsigned long long)(uint32_t)c.x);
            }
        }
        if (tid == 0 && unknown_s) {
            if (atomicExch(&flags[brick], tag) != tag) {
                int pos = atomicAdd(n_out, 1);
                list_out[pos] = (int32_t)brick;
            }
        }
        __syncthreads();
    }
}

// reset the consumed queue (count + work counter) after a round
__global__ void round_advance_kernel(int32_t *n_consumed, int32_t *work_consumed) {
    *n_consumed = 0;
    *work_consumed = 0;
}

// ---------------------------------------------------------------- voxel traversal
// 6-connected Amanatides-Woo traversal of the segment joining the centres of voxels a
// and b, walked from a.  The k-th crossing on axis i is at t = (2k-1)/(2|d_i|); scaled
// by 2 prod(|d_j| != 0) it is the integer (2k-1) P_i with P_i the product of the other
// non-zero |d_j|, so crossing order is decided exactly; ties step x, then y, then z.
// Returns the number of steps whose voxel has band `b` before the first that does not;
// *end receives the last voxel reached.
__device__ int walk(const uint8_t *__restrict__ band, Dims d, int ax, int ay, int az, int bx, int by, int bz,
                    uint8_t b, int *ex, int *ey, int *ez) {
    int Ax = abs(bx - ax), Ay = abs(by - ay), Az = abs(bz - az);
    int sx = bx >= ax ? 1 : -1, sy = by >= ay ? 1 : -1, sz = bz >= az ? 1 : -1;
    unsigned long long fx = Ax ? Ax : 1, fy = Ay ? Ay : 1, fz = Az ? Az : 1;
    unsigned long long Px = fy * fz, Py = fx * fz, Pz = fx * fy;
    const unsigned long long INF = ~0ULL;
    unsigned long long Tx = Ax ? Px : INF, Ty = Ay ? Py : INF, Tz = Az ? Pz : INF;
    int kx = 0, ky = 0, kz = 0;
    int x = ax, y = ay, z = az;
    int steps = 0;
    const int total = Ax + Ay + Az;
    while (steps < total) {
        int axis;
        if (Tx <= Ty && Tx <= Tz) axis = 0;
        else if (Ty <= Tz) axis = 1;
        else axis = 2;
        int nx2 = x, ny2 = y, nz2 = z;
        if (axis == 0) nx2 += sx;
        else if (axis == 1) ny2 += sy;
        else nz2 += sz;
        if (band[nx2 + (int64_t)d.nx * (ny2 + (int64_t)d.ny * nz2)] != b) break;
        x = nx2; y = ny2; z = nz2;
        if (axis == 0) { if (++kx == Ax) Tx = INF; else Tx += 2 * Px; }
        else if (axis == 1) { if (++ky == Ay) Ty = INF; else Ty += 2 * Py; }
        else { if (++kz == Az) Tz = INF; else Tz += 2 * Pz; }
        ++steps;
    }
    *ex = x; *ey = y; *ez = z;
    return steps;
}

__global__ void __launch_bounds__(256) update_voxels_kernel(
    const uint8_t *__restrict__ band, const uint16_t *__restrict__ q, Dims d, const unsigned long long *__restrict__ key,
    const int32_t *__restrict__ site_pos, unsigned long long *sums, uint32_t *los_bits, int32_t *par,
    int32_t *nonlos, int32_t *n_nonlos, bool small_coords) {
    int64_t n = d.n();
    int64_t nw = (n + 31) >> 5;
    int lane = threadIdx.x & 31;
    for (int64_t wv = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wv < nw;
         wv += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int64_t v = wv * 32 + lane;
        bool los = false;
        int32_t s = -1;
        int x = 0, y = 0, z = 0;
        if (v < n) {
            unsigned long long k = key[v];
            if (k != kInfKey) {
                s = (int32_t)(uint32_t)k;
                uint32_t dist = (uint32_t)(k >> 32);
                x = (int)(v % d.nx);
                int64_t r = v / d.nx;
                y = (int)(r % d.ny);
                z = (int)(r / d.ny);
                if (dist == 0) {
                    los = true;
                } else {
                    int32_t p = site_pos[s];
                    int px = p % d.nx, py = (p / d.nx) % d.ny, pz = p / (d.nx * d.ny);
                    int ex, ey, ez;
                    int need = abs(px - x) + abs(py - y) + abs(pz - z);
                    los = walk(band, d, x, y, z, px, py, pz, band[v], &ex, &ey, &ez) == need;
                }
                if (!los) {
                    // parent: first neighbour in (dz,dy,dx) order with an edge, same site and D(u)+w = D(v)
                    uint8_t b = band[v];
                    int32_t parent = -1;
                    for (int o = 0; o < 27 && parent < 0; ++o) {
                        if (o == 13) continue;
                        int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
                        int ux = x + dx, uy = y + dy, uz = z + dz;
                        if (ux < 0 || ux >= d.nx || uy < 0 || uy >= d.ny || uz < 0 || uz >= d.nz) continue;
                        bool ok = true;
                        for (int az = 0; az <= (dz != 0) && ok; ++az)
                            for (int ay = 0; ay <= (dy != 0) && ok; ++ay)
                                for (int ax = 0; ax <= (dx != 0) && ok; ++ax)
                                    ok = band[(x + ax * dx) + (int64_t)d.nx * ((y + ay * dy) + (int64_t)d.ny * (z + az * dz))] == b;
                        if (!ok) continue;
                        int64_t u = ux + (int64_t)d.nx * (uy + (int64_t)d.ny * uz);
                        unsigned long long ku = key[u];
                        if ((int32_t)(uint32_t)ku != s) continue;
                        if ((ku >> 32) + weight_of(o) == (k >> 32)) parent = (int32_t)u;
                    }
                    par[v] = parent;
                    int pos = atomicAdd(n_nonlos, 1);
                    nonlos[pos] = (int32_t)v;
                }
            }
        }
        unsigned bal = __ballot_sync(0xffffffffu, los);
        if (lane == 0 && wv < nw) los_bits[wv] = bal;
        // warp-aggregated integer moment sums of the LOS voxels
        int32_t grp = los ? s : -1;
        unsigned m = __match_any_sync(0xffffffffu, grp);
        unsigned w = los ? (q ? q[v] : 1u) : 0u;
        if (small_coords) {
            unsigned sx = __reduce_add_sync(m, w * (unsigned)x);
            unsigned sy = __reduce_add_sync(m, w * (unsigned)y);
            unsigned sz = __reduce_add_sync(m, w * (unsigned)z);
            unsigned sw = __reduce_add_sync(m, w);
            if (los && (m & lanemask_lt()) == 0) {
                atomicAdd(&sums[4 * (int64_t)s + 0], (unsigned long long)sx);
                atomicAdd(&sums[4 * (int64_t)s + 1], (unsigned long long)sy);
                atomicAdd(&sums[4 * (int64_t)s + 2], (unsigned long long)sz);
                atomicAdd(&sums[4 * (int64_t)s + 3], (unsigned long long)sw);
            }
        } else if (los) {
            atomicAdd(&sums[4 * (int64_t)s + 0], (unsigned long long)w * (unsigned)x);
            atomicAdd(&sums[4 * (int64_t)s + 1], (unsigned long long)w * (unsigned)y);
            atomicAdd(&sums[4 * (int64_t)s + 2], (unsigned long long)w * (unsigned)z);
            atomicAdd(&sums[4 * (int64_t)s + 3], (unsigned long long)w);
        }
    }
}

__global__ void update_nonlos_kernel(const uint16_t *__restrict__ q, Dims d, const unsigned long long *__restrict__ key,
                                     const uint32_t *__restrict__ los_bits, const int32_t *__restrict__ par,
                                     const int32_t *__restrict__ nonlos, const int32_t *n_nonlos,
                                     unsigned long long *sums, int32_t *status) {
    int32_t cnt = *n_nonlos;
    int64_t n = d.n();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        int32_t v = nonlos[i];
        int32_t u = par[v];
        int64_t guard = 0;
        while (u >= 0 && !((los_bits[u >> 5] >> (u & 31)) & 1u)) {
            u = par[u];
            if (++guard > n) { u = -1; break; }
        }
        if (u < 0) {
#ifdef LSRVT_DEBUG
            printf("nonlos fail v=%d par=%d key=%llx losbit=%u cnt=%d i=%d\n", v, par[v], key[v],
                   (los_bits[v >> 5] >> (v & 31)) & 1u, cnt, i);
#endif
            set_status(status, LSRVT_ERR_TIMEOUT);
            continue;
        }
        int32_t s = (int32_t)(uint32_t)key[v];
        unsigned long long w = q ? q[v] : 1u;
        int ux = u % d.nx, uy = (u / d.nx) % d.ny, uz = u / (d.nx * d.ny);
        atomicAdd(&sums[4 * (int64_t)s + 0], w * (unsigned)ux);
        atomicAdd(&sums[4 * (int64_t)s + 1], w * (unsigned)uy);
        atomicAdd(&sums[4 * (int64_t)s + 2], w * (unsigned)uz);
        atomicAdd(&sums[4 * (int64_t)s + 3], w);
    }
}

__global__ void move_sites_kernel(const uint8_t *__restrict__ band, Dims d, int32_t *site_pos, const int32_t *n_sites_dev,
                                  int32_t max_sites, const unsigned long long *__restrict__ sums,
                                  unsigned long long *trace) {
    int32_t ns = min(*n_sites_dev, max_sites);
    for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
        int32_t p = site_pos[s];
        int x = p % d.nx, y = (p / d.nx) % d.ny, z = p / (d.nx * d.ny);
        long long M = (long long)sums[4 * (int64_t)s + 3];
        if (M <= 0) continue;
        long long tx = (2 * (long long)sums[4 * (int64_t)s + 0] + M) / (2 * M);
        long long ty = (2 * (long long)sums[4 * (int64_t)s + 1] + M) / (2 * M);
        long long tz = (2 * (long long)sums[4 * (int64_t)s + 2] + M) / (2 * M);
        // the centroid of in-volume coordinates lies in the volume; clamp only guards bad input
        tx = tx < 0 ? 0 : (tx >= d.nx ? d.nx - 1 : tx);
        ty = ty < 0 ? 0 : (ty >= d.ny ? d.ny - 1 : ty);
        tz = tz < 0 ? 0 : (tz >= d.nz ? d.nz - 1 : tz);
        int ex, ey, ez;
        walk(band, d, x, y, z, (int)tx, (int)ty, (int)tz, band[p], &ex, &ey, &ez);
        int32_t np = ex + d.nx * (ey + d.ny * ez);
        if (np != p) {
            site_pos[s] = np;
            long long ddx = ex - x, ddy = ey - y, ddz = ez - z;
            if (trace) {
                atomicAdd(&trace[0], 1ULL);
                atomicAdd(&trace[1], (unsigned long long)(ddx * ddx + ddy * ddy + ddz * ddz));
            }
        }
    }
}

__global__ void emit_kernel(const unsigned long long *__restrict__ key, int64_t n, int32_t *cell, uint32_t *dist) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long k = key[v];
        bool inf = k == kInfKey;
        cell[v] = inf ? -1 : (int32_t)(uint32_t)k;
        if (dist) dist[v] = inf ? kInf32 : (uint32_t)(k >> 32);
    }
}

struct CvtWs {
    unsigned long long *key;
    int32_t *par;
    uint32_t *los_bits;
    int32_t *nonlos;
    int32_t *counters;  // [0] n_nonlos, [1..2] queue counts, [3..4] work counters
    unsigned long long *sums;
    uint32_t *flags;
    int32_t *list[2];
    int64_t *bin_off;
    int32_t *bin_cursor;
    int4 *cand;
    int64_t *bin_total;
    void *scan;
};

CvtWs carve_cvt(void *ws, size_t bytes, Dims d, int32_t max_sites, size_t *need) {
    Carver c(ws, bytes);
    int64_t n = d.n();
    BrickGeom bg{(d.nx + RX - 1) / RX, (d.ny + RY - 1) / RY, (d.nz + RZ - 1) / RZ};
    int64_t nbricks = (int64_t)bg.nbx * bg.nby * bg.nbz;
    CvtWs w;
    w.key = c.take<unsigned long long>(n);
    w.par = c.take<int32_t>(n);
    w.los_bits = c.take<uint32_t>((n + 31) / 32);
    w.nonlos = c.take<int32_t>(n);
    w.counters = c.take<int32_t>(8);
    w.sums = c.take<unsigned long long>((int64_t)max_sites * 4 + 4);
    w.flags = c.take<uint32_t>(nbricks);
    w.list[0] = c.take<int32_t>(nbricks);
    w.list[1] = c.take<int32_t>(nbricks);
    w.bin_off = c.take<int64_t>(nbricks + 1);
    w.bin_cursor = c.take<int32_t>(nbricks);
    w.cand = c.take<int4>((int64_t)max_sites + 1);
    w.bin_total = c.take<int64_t>(1);
    w.scan = c.take<char>(scan_temp_bytes(nbricks + 1));
    *need = c.used;
    return w;
}

constexpr int kRoundsPerCheck = 8;
constexpr int kMaxRounds = 1 << 16;

}  // namespace

size_t cvt_workspace(Dims d, int32_t max_sites) {
    size_t need;
    carve_cvt(nullptr, 0, d, max_sites, &need);
    return need;
}

}  // namespace lsrvt

using namespace lsrvt;

namespace {

// One tessellation: keys <- restricted geodesic Voronoi assignment of the current sites.
lsrvt_status run_assignment(const uint8_t *band, Dims d, const int32_t *site_pos, const int32_t *n_sites_dev,
                            int32_t max_sites, CvtWs &w, uint32_t &tag, int32_t *status, cudaStream_t s) {
    BrickGeom bg{(d.nx + RX - 1) / RX, (d.ny + RY - 1) / RY, (d.nz + RZ - 1) / RZ};
    int64_t n = d.n();
    int64_t nbricks = (int64_t)bg.nbx * bg.nby * bg.nbz;
    (void)n;
    cudaMemsetAsync(w.counters + 1, 0, sizeof(int32_t) * 4, s);
    cudaMemsetAsync(w.bin_off, 0, sizeof(int64_t) * (nbricks + 1), s);
    cudaMemsetAsync(w.bin_cursor, 0, sizeof(int32_t) * nbricks, s);
    site_bin_count_kernel<<<grid_for(max_sites, 256, kSMs * 4), 256, 0, s>>>(site_pos, n_sites_dev, max_sites, d, bg,
                                                                            w.bin_off, status);
    exclusive_scan_i64(w.bin_off, nbricks + 1, w.bin_total, w.scan, s);
    site_bin_fill_kernel<<<grid_for(max_sites, 256, kSMs * 4), 256, 0, s>>>(site_pos, n_sites_dev, max_sites, band, d,
                                                                           bg, w.bin_off, w.bin_cursor, w.cand);
    ++tag;
    int nb_cfi = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb_cfi, cfi_kernel, kRelaxThreads, 0);
    if (nb_cfi < 1) nb_cfi = 1;
    int cgrid = (int)(nbricks < (int64_t)kSMs * nb_cfi ? nbricks : (int64_t)kSMs * nb_cfi);
    cfi_kernel<<<cgrid, kRelaxThreads, 0, s>>>(band, d, bg, w.bin_off, w.cand, w.key, w.list[0], w.counters + 1,
                                               w.flags, tag);
#ifdef LSRVT_DEBUG
    {
        int32_t q0 = 0;
        cudaMemcpyAsync(&q0, w.counters + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        fprintf(stderr, "cfi: %d of %lld bricks queued\n", q0, (long long)nbricks);
    }
#endif
    int nb_per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb_per_sm, relax_round_kernel, kRelaxThreads, 0);
    if (nb_per_sm < 1) nb_per_sm = 1;
    int grid = kSMs * nb_per_sm;
    int cur = 0;
    for (int r = 0; r < kMaxRounds; ++r) {
        ++tag;
        relax_round_kernel<<<grid, kRelaxThreads, 0, s>>>(band, d, bg, w.key, w.list[cur], w.counters + 1 + cur,
                                                           w.list[1 - cur], w.counters + 1 + (1 - cur), w.flags, tag,
                                                           w.counters + 3 + cur, status);
        round_advance_kernel<<<1, 1, 0, s>>>(w.counters + 1 + cur, w.counters + 3 + cur);
        cur = 1 - cur;
#ifdef LSRVT_DEBUG
        {
            int32_t pend = 0;
            cudaMemcpyAsync(&pend, w.counters + 1 + cur, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
            fprintf(stderr, "round %d next=%d\n", r, pend);
        }
#endif
        if ((r + 1) % kRoundsPerCheck == 0) {
            int32_t pending = 0;
            cudaMemcpyAsync(&pending, w.counters + 1 + cur, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
            if (cudaStreamSynchronize(s) != cudaSuccess) return LSRVT_ERR_CUDA;
            if (pending == 0) return launch_status();
        }
    }
    return LSRVT_ERR_TIMEOUT;
}

}  // namespace

extern "C" lsrvt_status lsrvt_cvt_iterate(const uint8_t *band, const uint16_t *q, lsrvt_dims dd, int32_t *site_pos,
                                          const int32_t *n_sites_dev, int32_t max_sites, int32_t n_iters,
                                          int32_t *cell, uint32_t *dist, int64_t *iter_trace, void *ws,
                                          size_t ws_bytes, int32_t *status_dev, void *stream) {
    if (!dims_ok(dd) || !band || !site_pos || !n_sites_dev || max_sites < 0 || n_iters < 0 || !cell)
        return LSRVT_ERR_INVALID_ARG;
    Dims d{dd.nx, dd.ny, dd.nz};
    size_t need;
    CvtWs w = carve_cvt(ws, ws_bytes, d, max_sites, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) return LSRVT_ERR_WORKSPACE;
    cudaStream_t s = as_stream(stream);
    int64_t n = d.n();
    BrickGeom bg{(d.nx + RX - 1) / RX, (d.ny + RY - 1) / RY, (d.nz + RZ - 1) / RZ};
    int64_t nbricks = (int64_t)bg.nbx * bg.nby * bg.nbz;
    cudaMemsetAsync(w.flags, 0, sizeof(uint32_t) * nbricks, s);
    if (iter_trace && n_iters > 0) cudaMemsetAsync(iter_trace, 0, sizeof(int64_t) * 2 * n_iters, s);
    bool small = d.nx <= 2048 && d.ny <= 2048 && d.nz <= 2048;
    uint32_t tag = 0;
    int vgrid = grid_for((n + 31) / 32 * 32, 256, kSMs * 16);
    for (int32_t it = 0; it < n_iters; ++it) {
        lsrvt_status st = run_assignment(band, d, site_pos, n_sites_dev, max_sites, w, tag, status_dev, s);
        if (st != LSRVT_OK) return st;
        cudaMemsetAsync(w.sums, 0, sizeof(unsigned long long) * ((size_t)max_sites * 4 + 4), s);
        cudaMemsetAsync(w.counters, 0, sizeof(int32_t), s);
        update_voxels_kernel<<<vgrid, 256, 0, s>>>(band, q, d, w.key, site_pos, w.sums, w.los_bits, w.par, w.nonlos,
                                                   w.counters, small);
        update_nonlos_kernel<<<kSMs * 8, 256, 0, s>>>(q, d, w.key, w.los_bits, w.par, w.nonlos, w.counters, w.sums,
                                                      status_dev);
        move_sites_kernel<<<grid_for(max_sites, 256, kSMs * 8), 256, 0, s>>>(
            band, d, site_pos, n_sites_dev, max_sites, w.sums,
            iter_trace ? (unsigned long long *)(iter_trace + 2 * it) : nullptr);
    }
    lsrvt_status st = run_assignment(band, d, site_pos, n_sites_dev, max_sites, w, tag, status_dev, s);
    if (st != LSRVT_OK) return st;
    emit_kernel<<<grid_for(n, 256, kSMs * 16), 256, 0, s>>>(w.key, n, cell, dist);
    return launch_status();
}
