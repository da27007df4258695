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
// changed queue their neighbours (at most once at a time: a per-brick flag) on one
// asynchronous work queue that runs until no queued or running brick is left.
//
// Update (Eq. 2).  One pass over the voxels: a voxel at distance 0 is its site; other
// voxels walk the 6-connected traversal toward their site (line of sight); LOS voxels add
// q * coords to their site's integer sums (warp-aggregated atomics); the rest record
// their parent (first neighbour in (dz,dy,dx) order on a shortest path to the same site)
// and are resolved in a second pass by walking parents to the first LOS voxel (phi).  A
// per-site pass rounds the centroid half up and walks the site toward it, stopping before
// it would leave its band.
#include <climits>
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

// voxel coordinates of a linear index (N < 2^31, so 32-bit unsigned division is exact)
__device__ __forceinline__ void decode_voxel(uint32_t v, Dims d, int &x, int &y, int &z) {
    const uint32_t r = v / (uint32_t)d.nx;
    x = (int)(v - r * (uint32_t)d.nx);
    z = (int)(r / (uint32_t)d.ny);
    y = (int)(r - (uint32_t)z * (uint32_t)d.ny);
}

// CVT energy sum of m_v D(v)^2 (16.16 distances), exact in 128 bits: each thread keeps its
// own sum, a warp folds its lanes' sums at the end of the kernel and adds them to the two
// 64-bit words of the iteration's trace record (low word first, the carry detected from the
// old value the atomic returns).  A term is below 2^16 * 2^64, the total below 2^111.
struct EnergyAcc {
    unsigned long long lo = 0, hi = 0;
    __device__ __forceinline__ void add(unsigned w, uint32_t D) {
        const unsigned long long d2 = (unsigned long long)D * D;
        const unsigned long long l = d2 * w, h = __umul64hi(d2, (unsigned long long)w);
        lo += l;
        hi += h + (lo < l ? 1ull : 0ull);
    }
    // every lane of the warp calls this (full-warp shuffles)
    __device__ __forceinline__ void flush(unsigned long long *out) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long l2 = __shfl_down_sync(0xffffffffu, lo, o);
            const unsigned long long h2 = __shfl_down_sync(0xffffffffu, hi, o);
            lo += l2;
            hi += h2 + (lo < l2 ? 1ull : 0ull);
        }
        if (out && (threadIdx.x & 31) == 0 && (lo | hi)) {
            const unsigned long long old = atomicAdd(out, lo);
            atomicAdd(out + 1, hi + (old + lo < old ? 1ull : 0ull));
        }
    }
};

// ceil(2^16 sqrt(D)) for 0 < D < 2^32: a rounded square root brought to the exact integer by
// comparing squares (the result r is the least with r^2 >= 2^32 D).  D = dx^2 + dy^2 + dz^2 is
// never 2^32 - 1 (7 mod 8: not a sum of three squares), the one value whose r would be 2^32,
// so r < 2^32 and r^2 fits in 64 bits.
__device__ __forceinline__ unsigned long long ceil_q16_length(unsigned long long D) {
    const unsigned long long v = D << 32;
    unsigned long long r = D < (1ull << 16) ? (unsigned long long)(__fsqrt_rn((float)D) * 65536.0f)
                                            : (unsigned long long)(__dsqrt_rn((double)D) * 65536.0);
    while (r * r < v) ++r;
    while (r > 1 && (r - 1) * (r - 1) >= v) --r;
    return r;
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

#ifdef LSRVT_DEBUG
__device__ unsigned long long g_relax_steps[2];  // in-brick steps, brick visits
#endif
// The relaxation: the CTAs of the grid take queued bricks one at a time.
// Only voxels the candidate filter left unsettled can change (settled keys are exact), so
// their exact bits (xmask, brick order) switch the others off, and only bricks holding
// unsettled voxels (hasunk) are ever queued.
// One visit of a brick: load its keys with a one-voxel halo, relax in place until stable, write
// back what changed, and hand every neighbour brick whose shared boundary improved to `queue`
// (called by one thread per neighbour, after the block's writes).  All threads of the CTA call it.
// kMinStore: two visits of the brick may overlap (the asynchronous queue), so a key is written
// with a 64-bit atomic minimum -- keys only decrease, and an older visit must not overwrite what
// a newer one found.
template <bool kMinStore, class Queue>
__device__ __forceinline__ void relax_brick(const uint32_t *__restrict__ emask, const uint32_t *__restrict__ xmask,
                                            const uint8_t *__restrict__ hasunk, Dims d, BrickGeom bg,
                                            unsigned long long *key, const int brick, int32_t *status,
                                            Queue &&queue) {
    // packed keys: one aligned 64-bit access per read/write, so a reader never pairs the
    // distance of one update with the site of another
    __shared__ unsigned long long sk[HV];
    __shared__ uint32_t changed[2][kRows];  // double buffered: written in one step, cleared in the next
    __shared__ uint32_t dirty[kRows];
    __shared__ uint32_t touch;
    const int tid = threadIdx.x;
    {
        const int bx = brick % bg.nbx, by = (brick / bg.nbx) % bg.nby, bz = brick / (bg.nbx * bg.nby);
        const int ox = bx * RX, oy = by * RY, oz = bz * RZ;
        // ---- load halo
        for (int i = tid; i < HV; i += kRelaxThreads) {
            int hx = i % HX, hy = (i / HX) % HY, hz = i / (HX * HY);
            int gx = ox + hx - 1, gy = oy + hy - 1, gz = oz + hz - 1;
            unsigned long long k = kInfKey;
            if (gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny && gz >= 0 && gz < d.nz)
                k = __ldcg(key + gx + (int64_t)d.nx * (gy + (int64_t)d.ny * gz));
            sk[i] = k;
        }
        if (tid < kRows) {
            changed[0][tid] = 0;
            changed[1][tid] = 0;
            dirty[tid] = 0xFFFFu;
        }
        if (tid == 0) touch = 0;
        __syncthreads();
        // ---- edge masks (precomputed per call) and original keys
        unsigned long long orig[kVPT];
        uint32_t em[kVPT];
#pragma unroll
        for (int j = 0; j < kVPT; ++j) {
            int i = tid + kRelaxThreads * j;
            int lx = i & (RX - 1), ly = (i >> 4) & (RY - 1), lz = i >> 7;
            int gx = ox + lx, gy = oy + ly, gz = oz + lz;
            const bool exact = (__ldcg(xmask + (int64_t)brick * 32 + (tid >> 5) + (kRelaxThreads / 32) * j) >> (tid & 31)) & 1u;
            em[j] = (!exact && gx < d.nx && gy < d.ny && gz < d.nz)
                        ? __ldg(emask + gx + (int64_t)d.nx * (gy + (int64_t)d.ny * gz))
                        : 0u;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kVPT; ++j) {
            int i = tid + kRelaxThreads * j;
            int lx = i & (RX - 1), ly = (i >> 4) & (RY - 1), lz = i >> 7;
            orig[j] = sk[(lx + 1) + HX * ((ly + 1) + HY * (lz + 1))];
        }
        // ---- relaxation steps
        int step = 0;
        for (int cur = 0; step < kMaxSteps; ++step, cur ^= 1) {
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
                    // packed keys: (d, s) + (w << 32) = (d + w, s) unless d + w reaches 2^32 - 1
                    const unsigned long long lim = (unsigned long long)(kInf32 - weight_of(o)) << 32;
                    const unsigned long long ku = sk[h + halo_off(o)];
                    if (ku >= lim) {
                        if ((uint32_t)(ku >> 32) != kInf32) set_status(status, LSRVT_ERR_OVERFLOW);
                        continue;
                    }
                    const unsigned long long cand = ku + ((unsigned long long)weight_of(o) << 32);
                    best = cand < best ? cand : best;
                }
                if (best < own) {
                    sk[h] = best;
                    atomicOr(&changed[cur][row], 1u << lx);
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
                        uint32_t c = changed[cur][y2 + RY * z2];
                        m |= c | (c << 1) | (c >> 1);
                    }
                dirty[tid] = m & 0xFFFFu;
                changed[cur ^ 1][tid] = 0;  // last read before the previous barrier
            }
            __syncthreads();
        }
#ifdef LSRVT_DEBUG
        if (tid == 0) {
            atomicAdd(&g_relax_steps[0], (unsigned long long)step);
            atomicAdd(&g_relax_steps[1], 1ULL);
        }
#endif
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
            if (kMinStore) atomicMin(key + gx + (int64_t)d.nx * (gy + (int64_t)d.ny * gz), nk);
            else key[gx + (int64_t)d.nx * (gy + (int64_t)d.ny * gz)] = nk;
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
                if (__ldcg(hasunk + nb)) queue(nb);
            }
        }
        __syncthreads();
    }
}

// The relaxation as one asynchronous work queue (one launch, no rounds).  A ticket counter
// hands out work: tickets below the filter's count read its brick list, later ones a ring of
// bricks queued during the relaxation (capacity = the number of bricks: a brick is in the queue
// at most once at a time -- its flag holds `tag` from the push until the pop).  A CTA pops a
// brick, relaxes it, and pushes every neighbour whose shared boundary improved; `outstanding`
// counts the bricks pushed and not yet finished, so a CTA whose ticket finds nothing leaves once
// it reaches zero.  A brick pushed again while a visit of it is still running can be visited
// twice at once, so keys are written back with an atomic minimum.  Keys only decrease and the
// fixed point is unique, so the result does not depend on the order.  Every wait is bounded: past the limit the status gets TIMEOUT and the
// abort flag empties the queue.
struct RelaxQueue {
    int32_t head;         // next ticket
    int32_t pushed;       // bricks pushed to the ring so far
    int32_t outstanding;  // pushed (or listed) and not yet finished
    int32_t abort;
};

__global__ void relax_queue_init_kernel(RelaxQueue *q, const int32_t *n_list) {
    q->head = 0;
    q->pushed = 0;
    q->outstanding = *n_list;
    q->abort = 0;
}

__global__ void __launch_bounds__(kRelaxThreads) relax_async_kernel(
    const uint32_t *__restrict__ emask, const uint32_t *__restrict__ xmask, const uint8_t *__restrict__ hasunk, Dims d,
    BrickGeom bg, unsigned long long *key, const int32_t *list0, const int32_t *n_list, int32_t *ring, int32_t cap,
    RelaxQueue *q, uint32_t *flags, uint32_t tag, int32_t max_tickets, int32_t *status) {
    __shared__ int item;
    const int n0 = __ldcg(n_list);
    while (true) {
        if (threadIdx.x == 0) {
            int b = -1;
            if (!*(volatile int32_t *)&q->abort) {
                const int t = atomicAdd(&q->head, 1);
                if (t >= max_tickets) {
                    set_status(status, LSRVT_ERR_TIMEOUT);
                    atomicExch(&q->abort, 1);
                } else if (t < n0) {
                    b = __ldcg(list0 + t);
                } else {
                    int32_t *slot = ring + (t - n0) % cap;
                    for (long long spin = 0;; ++spin) {
                        const int v = atomicExch(slot, 0);
                        if (v) {
                            b = v - 1;
                            break;
                        }
                        if (*(volatile int32_t *)&q->outstanding == 0 || *(volatile int32_t *)&q->abort) break;
                        if (spin > (1LL << 24)) {
                            set_status(status, LSRVT_ERR_TIMEOUT);
                            atomicExch(&q->abort, 1);
                            break;
                        }
                        __nanosleep(128);
                    }
                }
                if (b >= 0) {
                    // the pop: pushes from now on queue the brick again; the fence orders the
                    // neighbours' key writes seen through the flag and the ring before our loads
                    atomicExch(&flags[b], 0u);
                    __threadfence();
                }
            }
            item = b;
        }
        __syncthreads();
        const int b = item;
        __syncthreads();  // every thread has read `item` before thread 0 may overwrite it
        if (b < 0) break;
        relax_brick<true>(emask, xmask, hasunk, d, bg, key, b, status, [&](int nb) {
            __threadfence();  // the block's key writes (ordered by the barrier) before the push
            if (atomicExch(&flags[nb], tag) != tag) {
                atomicAdd(&q->outstanding, 1);
                const int pidx = atomicAdd(&q->pushed, 1);
                atomicExch(ring + pidx % cap, nb + 1);
            }
        });
        // relax_brick ends with a barrier: the pushes above are done
        if (threadIdx.x == 0) {
            __threadfence();
            atomicSub(&q->outstanding, 1);
        }
    }
}

// ---------------------------------------------------------------- clearance field
// c(v) = min(K, L-infinity distance from v to the nearest "boundary" voxel), a boundary
// voxel being one with a 26-neighbour of another band or outside the volume.  Every voxel
// within L-infinity distance c(v) of v then has band(v) (the (c-1)-ball holds no boundary
// voxel, so it and its neighbours share one band), so c(v) path moves from v need no band
// test.  The bands never change during the Lloyd iterations, so c is computed once per
// call: S_0 = non-boundary voxels as a bit volume (32 voxels per word along x), S_k+1 =
// S_k eroded by the 3x3x3 cube (shift-and of rows), c = number of sets holding v.
constexpr int kClearLevels = 32;

struct BitGeom {
    int32_t W;  // words per x row
    __host__ __device__ int64_t words(Dims d) const { return (int64_t)W * d.ny * d.nz; }
};

// The bands of a 32 x 8 x 8 tile plus a one-voxel halo in shared memory (16-bit entries:
// kOutside marks positions outside the volume, unequal to every band).  From them, per voxel:
// the 27-bit "same band" mask S (bit 13 the voxel itself); the edge mask (bit o set when the
// move by offset o = (dz+1) 9 + (dy+1) 3 + (dx+1) spans a box that lies in the band, so a path
// move costs one word instead of up to seven band bytes); and S_0, the non-boundary bit
// (a valid voxel whose 26 neighbours all lie in the volume and share its band), packed 32
// voxels to a word along x.  A warp handles a row of the tile, a lane a voxel.
constexpr int kTileX = 32, kTileY = 8, kTileZ = 8;
constexpr int kHX = kTileX + 2, kHY = kTileY + 2, kHZ = kTileZ + 2;
constexpr uint16_t kOutside = 0x100;

__global__ void __launch_bounds__(256) band_masks_kernel(const uint8_t *__restrict__ band, Dims d, BitGeom bgm,
                                                         uint32_t *__restrict__ S0, uint32_t *__restrict__ emask) {
    __shared__ uint16_t t[kHZ][kHY][kHX];
    const int nty = (d.ny + kTileY - 1) / kTileY, ntz = (d.nz + kTileZ - 1) / kTileZ;
    const int64_t ntiles = (int64_t)bgm.W * nty * ntz;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int wx = (int)(tile % bgm.W);
        const int ty = (int)((tile / bgm.W) % nty), tz = (int)(tile / ((int64_t)bgm.W * nty));
        const int x0 = wx * kTileX - 1, y0 = ty * kTileY - 1, z0 = tz * kTileZ - 1;
        for (int i = threadIdx.x; i < kHX * kHY * kHZ; i += blockDim.x) {
            const int hx = i % kHX, hy = (i / kHX) % kHY, hz = i / (kHX * kHY);
            const int x = x0 + hx, y = y0 + hy, z = z0 + hz;
            uint16_t v = kOutside;
            if (x >= 0 && x < d.nx && y >= 0 && y < d.ny && z >= 0 && z < d.nz)
                v = __ldg(band + x + (int64_t)d.nx * (y + (int64_t)d.ny * z));
            t[hz][hy][hx] = v;
        }
        __syncthreads();
        for (int r = w; r < kTileY * kTileZ; r += blockDim.x >> 5) {
            const int ly = r % kTileY, lz = r / kTileY;
            const int x = x0 + 1 + lane, y = y0 + 1 + ly, z = z0 + 1 + lz;
            const bool live = x < d.nx && y < d.ny && z < d.nz;
            const uint16_t b = t[lz + 1][ly + 1][lane + 1];
            uint32_t S = 0;
            if (live && b != kInvalidBand) {
#pragma unroll
                for (int o = 0; o < 27; ++o) {
                    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
                    S |= (uint32_t)(t[lz + 1 + dz][ly + 1 + dy][lane + 1 + dx] == b) << o;
                }
            }
            if (live) emask[x + (int64_t)d.nx * (y + (int64_t)d.ny * z)] = S ? edges_from_same(S) : 0u;
            const unsigned bal = __ballot_sync(0xffffffffu, S == 0x7FFFFFFu);
            if (lane == 0 && y < d.ny && z < d.nz) S0[wx + (int64_t)bgm.W * (y + (int64_t)d.ny * z)] = bal;
        }
        __syncthreads();
    }
}

// x-erosion of word wx of a row (bits outside the row count as 0)
__device__ __forceinline__ uint32_t erode_x3(uint32_t lo, uint32_t w, uint32_t hi) {
    const uint32_t left = (w << 1) | (lo >> 31);   // bit i <- bit i-1
    const uint32_t right = (w >> 1) | (hi << 31);  // bit i <- bit i+1
    return w & left & right;
}

// S_k+1 = S_k eroded by the 3x3x3 cube (a voxel stays when its whole neighbourhood is in S_k;
// words and rows outside the volume count as 0).  A CTA loads 6 words x 10 rows x 10 slabs
// (its 4 x 8 x 8 output words plus a halo) into shared memory.
constexpr int kEW = 4, kEY = 8, kEZ = 8;

__global__ void __launch_bounds__(256) clear_erode_kernel(const uint32_t *__restrict__ Sk, Dims d, BitGeom bgm,
                                                          uint32_t *__restrict__ Sk1) {
    __shared__ uint32_t t[kEZ + 2][kEY + 2][kEW + 2];
    const int ntx = (bgm.W + kEW - 1) / kEW, nty = (d.ny + kEY - 1) / kEY, ntz = (d.nz + kEZ - 1) / kEZ;
    const int64_t ntiles = (int64_t)ntx * nty * ntz;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tx = (int)(tile % ntx), ty = (int)((tile / ntx) % nty), tz = (int)(tile / ((int64_t)ntx * nty));
        const int w0 = tx * kEW - 1, y0 = ty * kEY - 1, z0 = tz * kEZ - 1;
        for (int i = threadIdx.x; i < (kEW + 2) * (kEY + 2) * (kEZ + 2); i += blockDim.x) {
            const int hx = i % (kEW + 2), hy = (i / (kEW + 2)) % (kEY + 2), hz = i / ((kEW + 2) * (kEY + 2));
            const int wx = w0 + hx, y = y0 + hy, z = z0 + hz;
            uint32_t v = 0;
            if (wx >= 0 && wx < bgm.W && y >= 0 && y < d.ny && z >= 0 && z < d.nz)
                v = Sk[wx + (int64_t)bgm.W * (y + (int64_t)d.ny * z)];
            t[hz][hy][hx] = v;
        }
        __syncthreads();
        {
            const int i = threadIdx.x;  // one output word per thread (kEW * kEY * kEZ = 256)
            const int ox = i % kEW, oy = (i / kEW) % kEY, oz = i / (kEW * kEY);
            const int wx = w0 + 1 + ox, y = y0 + 1 + oy, z = z0 + 1 + oz;
            if (wx < bgm.W && y < d.ny && z < d.nz) {
                uint32_t acc = 0xffffffffu;
#pragma unroll
                for (int dz = 0; dz < 3; ++dz)
#pragma unroll
                    for (int dy = 0; dy < 3; ++dy)
                        acc &= erode_x3(t[oz + dz][oy + dy][ox], t[oz + dz][oy + dy][ox + 1], t[oz + dz][oy + dy][ox + 2]);
                Sk1[wx + (int64_t)bgm.W * (y + (int64_t)d.ny * z)] = acc;
            }
        }
        __syncthreads();
    }
}

// c(v) = number of the nested sets S_0 ... S_levels-1 holding v.  A thread per word: the word's
// planes are added into 6-bit counters held bit-sliced (one word per counter bit), stopping
// at the first empty plane (the sets are nested), then each voxel's count is read out.
__global__ void clear_count_kernel(const uint32_t *__restrict__ planes, Dims d, BitGeom bgm, int levels,
                                   uint8_t *__restrict__ clr) {
    const int64_t nw = bgm.words(d);
    for (int64_t wi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; wi < nw; wi += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0, c4 = 0, c5 = 0;
        for (int k = 0; k < levels; ++k) {
            uint32_t carry = planes[(int64_t)k * nw + wi];
            if (!carry) break;
            uint32_t tt;
            tt = c0 & carry; c0 ^= carry; carry = tt;
            tt = c1 & carry; c1 ^= carry; carry = tt;
            tt = c2 & carry; c2 ^= carry; carry = tt;
            tt = c3 & carry; c3 ^= carry; carry = tt;
            tt = c4 & carry; c4 ^= carry; carry = tt;
            c5 ^= carry;
        }
        const int wx = (int)(wi % bgm.W);
        const int64_t row = wi / bgm.W;
        const int xs = wx * 32, xe = min(xs + 32, d.nx);
        uint8_t *out = clr + row * d.nx;
        for (int x = xs; x < xe; ++x) {
            const int bb = x - xs;
            out[x] = (uint8_t)(((c0 >> bb) & 1u) | (((c1 >> bb) & 1u) << 1) | (((c2 >> bb) & 1u) << 2) |
                               (((c3 >> bb) & 1u) << 3) | (((c4 >> bb) & 1u) << 4) | (((c5 >> bb) & 1u) << 5));
        }
    }
}

// ---------------------------------------------------------------- closed-form initialisation
// Lower bound: the unconstrained 26-neighbour chamfer distance C(v, s) = (a-b) W1 +
// (b-c) W2 + c W3 (a >= b >= c the sorted |v - s|) never exceeds the restricted geodesic
// gd(v, s).  So min over the same-band sites of (C(v, s), s) is a lexicographic lower
// bound of v's key; if one shortest chamfer path from v to that site s* stays in the band
// (every edge box in band), gd(v, s*) = C(v, s*) is attained and the bound IS the key.
// Candidates come in stages of growing boxes around the brick: first the bricks within
// +-1 (x) / +-2 (y, z) bricks (fine bins), then shells of 32^3 coarse cells at Chebyshev
// distance 1, 2, ... (coarse bins); only sites whose band occurs in the brick are taken.
// A site outside the current box is at Chebyshev distance >= gap(v) and chamfer distance
// >= gap(v) W1, so a voxel is settled once its best is below that.  Voxels not settled,
// or whose path check fails, start at +inf and their bricks are relaxed.
constexpr int kMaxCand = 1024;
constexpr int kCoarse = 32, kCoarseShift = 5;
constexpr int kMaxRho = 12;

struct CoarseGeom {
    int32_t ncx, ncy, ncz;
};

__device__ __forceinline__ unsigned long long chamfer(int dx, int dy, int dz) {
    unsigned a = abs(dx), b = abs(dy), c = abs(dz), t;
    if (a < b) { t = a; a = b; b = t; }
    if (b < c) { t = b; b = c; c = t; }
    if (a < b) { t = a; a = b; b = t; }
    return (unsigned long long)(a - b) * kWFace + (unsigned long long)(b - c) * kWEdge +
           (unsigned long long)c * kWCorner;
}

// The same distance in 32-bit arithmetic, for differences below 2048 per axis (the whole sum
// stays below 2^28): |d| sorted by three compare-exchanges, then a W1 + b (W2 - W1) + c (W3 - W2)
// for a >= b >= c.
__device__ __forceinline__ unsigned long long chamfer_small(int dx, int dy, int dz) {
    const unsigned a = abs(dx), b = abs(dy), c = abs(dz);
    const unsigned hi = max(a, b), lo = min(a, b);
    const unsigned mid = max(lo, c), low = min(lo, c);
    const unsigned top = max(hi, mid), mid2 = min(hi, mid);
    return top * kWFace + mid2 * (kWEdge - kWFace) + low * (kWCorner - kWEdge);
}

template <bool kSmall>
__device__ __forceinline__ unsigned long long chamfer_t(int dx, int dy, int dz) {
    return kSmall ? chamfer_small(dx, dy, dz) : chamfer(dx, dy, dz);
}

// unsigned division, 32-bit when both operands fit (the common case for volumes <= 2048^3)
__device__ __forceinline__ unsigned long long udiv(unsigned long long a, unsigned long long b) {
    if (((a | b) >> 32) == 0) return (unsigned)a / (unsigned)b;
    return a / b;
}

// floor(a / b) for b >= 1: below 2^22 both operands are exact floats and the float quotient
// a * rcp(b) (two roundings, relative error below 2^-23) is within 0.5 of a / b < 2^22, so its
// truncation is off by at most one and one remainder test corrects it; larger operands take the
// integer division
__device__ __forceinline__ unsigned long long udiv_fast(unsigned long long a, unsigned long long b) {
    if (((a | b) >> 22) != 0) return udiv(a, b);
    const unsigned ua = (unsigned)a, ub = (unsigned)b;
    unsigned q = __float2uint_rz(__fmul_rn((float)ua, __frcp_rn((float)ub)));
    const int r = (int)(ua - q * ub);
    if (r < 0) --q;
    else if (r >= (int)ub) ++q;
    return q;
}

// One shortest chamfer path from v to s (26-connected digital line: the dominant axis i
// advances every move, the middle axis j after move t has advanced round(t aj / ai)
// times, the smallest axis k after m middle-axis advances round(m ak / aj) times, so it
// only moves together with j and no corner move is split).  True if every move's box is
// in band b.  From a voxel p with clearance c >= 1 the next c moves are in band and are
// skipped without tests.  Single moves advance Bresenham error terms (no division).
// Returns 0 if a move leaves the band, 1 if the path is in band, 2 if it is in band with a
// margin of 2: every jump anchor p covered only moves within L-infinity c(p) - 2 of p and
// the walk ended at most c(s) - 2 from s.  The 6-connected traversal of the segment v-s
// stays within L-infinity 2 of the digital path (per axis the rounding errors of the path
// and of the segment's voxel add up to at most 2), so margin 2 also certifies line of sight.
#ifdef LSRVT_DEBUG
__device__ unsigned long long g_path_dbg[12];  // checks cov=0, cov>0, -, -, status 0/1/2, sub-box tubes
                                               // 4x4x4 / 8x4x4 / 2x2x2 that would certify, los upgrades
#endif
// mv_start > 0: the moves before it are already known to be in band with a margin of 2
// (a brick tube certificate covered them); the walk starts there.
__device__ int chamfer_path_in_band(const uint32_t *__restrict__ emask, const uint8_t *__restrict__ clr, Dims d,
                                    int vx, int vy, int vz, int sx, int sy, int sz, int cs, int mv_start) {
    const int D0 = sx - vx, D1 = sy - vy, D2 = sz - vz;
    const int A0 = abs(D0), A1 = abs(D1), A2 = abs(D2);
    // axes sorted by extent: i >= j >= k
    int i = 0, j = 1, k = 2;
    int Ai = A0, Aj = A1, Ak = A2;
    if (Ai < Aj) { int t = i; i = j; j = t; t = Ai; Ai = Aj; Aj = t; }
    if (Aj < Ak) { int t = j; j = k; k = t; t = Aj; Aj = Ak; Ak = t; }
    if (Ai < Aj) { int t = i; i = j; j = t; t = Ai; Ai = Aj; Aj = t; }
    if (Ai == 0) return 2;
    const int64_t sxy = (int64_t)d.nx * d.ny;
    bool margin = true;
    // strides and signs along i, j, k in linear index space
    const int64_t stride[3] = {1, d.nx, sxy};
    const int sgn[3] = {D0 < 0 ? -1 : 1, D1 < 0 ? -1 : 1, D2 < 0 ? -1 : 1};
    const int64_t si = stride[i] * sgn[i], sj = stride[j] * sgn[j], sk = stride[k] * sgn[k];
    const int ow[3] = {1, 3, 9};
    const int oi = 13 + ow[i] * sgn[i], oj = ow[j] * sgn[j], ok = ow[k] * sgn[k];  // edge-mask bit offsets
    const int64_t v0 = vx + (int64_t)d.nx * vy + sxy * vz;
    const unsigned long long ai2 = 2ULL * Ai, aj2 = 2ULL * Aj;
    int mv = 0, jc = 0, kc = 0;
    // error terms: ej = 2 mv aj + ai - 2 ai jc in [0, 2ai); ek = 2 jc ak + aj - 2 aj kc in [0, 2aj)
    long long ej = Ai, ek = Aj;
    int64_t g = v0;
    if (mv_start > 0) {
        mv = mv_start < Ai ? mv_start : Ai;
        unsigned long long nj = 2ULL * mv * Aj + Ai;
        jc = (int)udiv_fast(nj, ai2);
        ej = (long long)(nj - ai2 * jc);
        if (Aj) {
            unsigned long long nk = 2ULL * jc * Ak + Aj;
            kc = (int)udiv_fast(nk, aj2);
            ek = (long long)(nk - aj2 * kc);
        }
        g = v0 + si * mv + sj * jc + sk * kc;
    }
    while (mv < Ai) {
#ifdef LSRVT_DEBUG
        atomicAdd(&g_path_dbg[2], 1ULL);
#endif
        // the rest of the path approaches s monotonically on every axis, so once within the
        // site's own clearance ball it stays in band
        int rem = max(Ai - mv, max(Aj - jc, Ak - kc));
        if (rem <= cs) return (margin && rem <= cs - 2) ? 2 : 1;
        int c = __ldg(clr + g);
        if (c >= 1) {
            int step = c;
            if (c >= 3) step = c - 2;
            else margin = false;
            int mv2 = mv + step < Ai ? mv + step : Ai;
            unsigned long long nj = 2ULL * mv2 * Aj + Ai;
            jc = (int)udiv_fast(nj, ai2);
            ej = (long long)(nj - ai2 * jc);
            if (Aj) {
                unsigned long long nk = 2ULL * jc * Ak + Aj;
                kc = (int)udiv_fast(nk, aj2);
                ek = (long long)(nk - aj2 * kc);
            }
            mv = mv2;
            g = v0 + si * mv + sj * jc + sk * kc;

            continue;
        }

        margin = false;
        ej += 2LL * Aj;
        bool mj = ej >= (long long)ai2;
        if (mj) ej -= (long long)ai2;
        bool mk = false;
        if (mj) {
            ek += 2LL * Ak;
            mk = ek >= (long long)aj2;
            if (mk) ek -= (long long)aj2;
        }
        // the move g -> g + mi + (mj) + (mk) must be an edge (its box in band)
        const int o = oi + (mj ? oj : 0) + (mk ? ok : 0);
        if (!((__ldg(emask + g) >> o) & 1u)) return 0;
        g += si + (mj ? sj : 0) + (mk ? sk : 0);
        ++mv;
        jc += mj;
        kc += mk;
    }
    return margin ? 2 : 1;
}

// Certificate for a whole brick at once.  Let C be the centre of the box [l, h], R its
// largest half extent and P(t) = C + t (s - C).  For a voxel v of the box the point
// v + t (s - v) is within L-infinity (1 - t) R of P(t); the move boxes of v's chamfer path
// (above) and the voxels of v's 6-connected traversal to s lie within L-infinity 2 of the
// points of v's segment.  So if every voxel within (1 - t) R + 2 of P(t), 0 <= t <= 1, is in
// band, every voxel of the box whose winner is s has an exact key and line of sight.  The
// tube is covered by clearance balls: at u = round(P(t_k)) with clearance c, the ball of
// radius c holds the tube over [t_k, t_k + dt] when rho(t_k) + 1/2 + dt |s - C| <= c (rho
// only shrinks along t).  Consecutive balls share a voxel, and the first holds the box's
// voxels of band b, so all of them lie in band b.  Exact integer arithmetic in doubled
// coordinates: k counts half voxels along the dominant axis of s - C (length L2).
// Returns the covered extent: the tube is certified for t <= k / L2 (k >= L2: all of it).
// The sequential walk below serves the debug counters; the kernels run the warp form after it.
#ifdef LSRVT_DEBUG
__device__ int brick_tube_in_band(const uint8_t *__restrict__ clr, Dims d, int lx, int ly, int lz, int hx, int hy,
                                  int hz, int sx, int sy, int sz) {
    const int cx2 = lx + hx, cy2 = ly + hy, cz2 = lz + hz;  // doubled centre
    const int dx2 = 2 * sx - cx2, dy2 = 2 * sy - cy2, dz2 = 2 * sz - cz2;
    const int L2 = max(abs(dx2), max(abs(dy2), abs(dz2)));
    const int R2 = max(hx - lx, max(hy - ly, hz - lz));  // doubled largest half extent
    if (L2 == 0) {
        int c = __ldg(clr + (cx2 >> 1) + (int64_t)d.nx * ((cy2 >> 1) + (int64_t)d.ny * (cz2 >> 1)));
        return 2 * c - 1 - (R2 + 4) >= 1 ? 1 : 0;
    }
    const unsigned den = 2u * (unsigned)L2;
    int k = 0;
    for (int guard = 0; guard < 4 * 4096; ++guard) {
        // round half up of the doubled coordinates (c2 L2 + d2 k) / L2, halved; all >= 0
        const int ux = (int)((unsigned)(cx2 * L2 + dx2 * k + L2) / den);
        const int uy = (int)((unsigned)(cy2 * L2 + dy2 * k + L2) / den);
        const int uz = (int)((unsigned)(cz2 * L2 + dz2 * k + L2) / den);
        const int c = __ldg(clr + ux + (int64_t)d.nx * (uy + (int64_t)d.ny * uz));
        // 2 rho(k), rounded up: R2 (L2 - k) / L2 + 4
        const int two_rho = (int)(((unsigned)R2 * (unsigned)(L2 - k) + (unsigned)L2 - 1u) / (unsigned)L2) + 4;
        const int delta = 2 * c - 1 - two_rho;
        if (delta < 1) return k;
        if (k + delta >= L2) return L2;
        k += delta;
    }
    return k;
}
#endif

// The same walk by a group of G lanes (G a power of two, at most 32, groups aligned within the
// warp): the lanes load the clearance of G consecutive tube points at once, then the group
// follows the sequential walk's jumps through that window with shuffles, so the result is the
// sequential one, with one dependent load per G positions instead of one per jump.  All lanes
// of a group call it with the same arguments.
__device__ int brick_tube_in_band_group(const uint8_t *__restrict__ clr, Dims d, int lx, int ly, int lz, int hx,
                                        int hy, int hz, int sx, int sy, int sz, int G) {
    const int lane = threadIdx.x & 31, gl = lane & (G - 1);
    const unsigned mask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << (lane & ~(G - 1));
    const int cx2 = lx + hx, cy2 = ly + hy, cz2 = lz + hz;
    const int dx2 = 2 * sx - cx2, dy2 = 2 * sy - cy2, dz2 = 2 * sz - cz2;
    const int L2 = max(abs(dx2), max(abs(dy2), abs(dz2)));
    const int R2 = max(hx - lx, max(hy - ly, hz - lz));
    if (L2 == 0) {
        int c = __ldg(clr + (cx2 >> 1) + (int64_t)d.nx * ((cy2 >> 1) + (int64_t)d.ny * (cz2 >> 1)));
        return 2 * c - 1 - (R2 + 4) >= 1 ? 1 : 0;
    }
    const unsigned den = 2u * (unsigned)L2;
    int f = 0;  // the walk's position: every tube point before it is covered
    for (int round = 0; round < 4 * 4096; ++round) {
        const int k = f + gl;
        int delta = 0;
        if (k < L2) {
            const int ux = (int)((unsigned)(cx2 * L2 + dx2 * k + L2) / den);
            const int uy = (int)((unsigned)(cy2 * L2 + dy2 * k + L2) / den);
            const int uz = (int)((unsigned)(cz2 * L2 + dz2 * k + L2) / den);
            const int c = __ldg(clr + ux + (int64_t)d.nx * (uy + (int64_t)d.ny * uz));
            const int two_rho = (int)(((unsigned)R2 * (unsigned)(L2 - k) + (unsigned)L2 - 1u) / (unsigned)L2) + 4;
            delta = 2 * c - 1 - two_rho;
        }
        int cur = f;
        while (cur - f < G) {  // every jump is at least 1: at most G turns
            const int dd = __shfl_sync(mask, delta, cur - f, G);
            if (dd < 1) return cur;
            if (cur + dd >= L2) return L2;
            cur += dd;
        }
        f = cur;
    }
    return f;
}

// site bins: one pass counts, a scan gives offsets, a second pass fills entries
// (site id, x, y, z | band << 24); the fine bins are the bricks, the coarse bins 32^3 cells
__device__ __forceinline__ int64_t fine_bin(int x, int y, int z, BrickGeom bg) {
    return x / RX + (int64_t)bg.nbx * (y / RY + (int64_t)bg.nby * (z / RZ));
}
__device__ __forceinline__ int64_t coarse_bin(int x, int y, int z, CoarseGeom cg) {
    return (x >> kCoarseShift) + (int64_t)cg.ncx * ((y >> kCoarseShift) + (int64_t)cg.ncy * (z >> kCoarseShift));
}

__global__ void site_bin_count_kernel(const int32_t *__restrict__ site_pos, const int32_t *n_sites_dev,
                                      int32_t max_sites, Dims d, BrickGeom bg, CoarseGeom cg, int64_t *fine_cnt,
                                      int64_t *coarse_cnt, int32_t *status) {
    int32_t ns = min(*n_sites_dev, max_sites);
    int64_t n = d.n();
    for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
        int32_t p = site_pos[s];
        if (p < 0 || p >= n) {
            set_status(status, LSRVT_ERR_INVALID_ARG);
            continue;
        }
        int32_t x = p % d.nx, y = (p / d.nx) % d.ny, z = p / (d.nx * d.ny);
        atomicAdd((unsigned long long *)&fine_cnt[fine_bin(x, y, z, bg)], 1ULL);
        atomicAdd((unsigned long long *)&coarse_cnt[coarse_bin(x, y, z, cg)], 1ULL);
    }
}

__global__ void site_bin_fill_kernel(const int32_t *__restrict__ site_pos, const int32_t *n_sites_dev,
                                     int32_t max_sites, const uint8_t *__restrict__ band, Dims d, BrickGeom bg,
                                     CoarseGeom cg, const int64_t *__restrict__ fine_off, int32_t *fine_cur,
                                     int4 *fine_cand, const int64_t *__restrict__ coarse_off, int32_t *coarse_cur,
                                     int4 *coarse_cand, int32_t *status) {
    int32_t ns = min(*n_sites_dev, max_sites);
    int64_t n = d.n();
    for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
        int32_t p = site_pos[s];
        if (p < 0 || p >= n) continue;
        int32_t x = p % d.nx, y = (p / d.nx) % d.ny, z = p / (d.nx * d.ny);
        int4 e = make_int4(s, x, y, z | ((int)band[p] << 24));
        int64_t fb = fine_bin(x, y, z, bg), cb = coarse_bin(x, y, z, cg);
        // the offsets come from a scan of the counts of the same sites, so the slots stay
        // below ns; checked anyway, so that a bad offset is an error status, not a stray write
        const int64_t fpos = fine_off[fb] + atomicAdd(&fine_cur[fb], 1);
        const int64_t cpos = coarse_off[cb] + atomicAdd(&coarse_cur[cb], 1);
        if (fpos < 0 || fpos >= ns || cpos < 0 || cpos >= ns) {
            set_status(status, LSRVT_ERR_CAPACITY);
            continue;
        }
        fine_cand[fpos] = e;
        coarse_cand[cpos] = e;
    }
}

#ifdef LSRVT_DEBUG
__device__ unsigned long long g_phase[12];
__device__ unsigned long long g_cfi_ph[8];  // cfi phase cycles (thread 0 of each CTA)
#define PHASE_T0() long long _t0 = clock64()
#define PHASE_ADD(i) do { if (threadIdx.x == 0) atomicAdd(&g_cfi_ph[i], (unsigned long long)(clock64() - _t0)); _t0 = clock64(); } while (0)
#else
#define PHASE_T0()
#define PHASE_ADD(i)
#endif

// q-th cell of the Chebyshev shell of radius rho (count 2(2rho+1)^2 + 8 rho (2rho-1)):
// the two z faces, then the square rings of the layers in between.
__device__ __forceinline__ void shell_cell(int q, int rho, int &dx, int &dy, int &dz) {
    const int side = 2 * rho + 1, face = side * side;
    if (q < 2 * face) {
        dz = q < face ? -rho : rho;
        int r = q % face;
        dx = r % side - rho;
        dy = r / side - rho;
        return;
    }
    q -= 2 * face;
    const int ring = 8 * rho;
    dz = -rho + 1 + q / ring;
    int r = q % ring;
    if (r < side) { dy = -rho; dx = -rho + r; return; }
    r -= side;
    if (r < side) { dy = rho; dx = -rho + r; return; }
    r -= side;
    const int inner = 2 * rho - 1;
    dx = r < inner ? -rho : rho;
    dy = -rho + 1 + (r % inner);
}

// Line of sight v -> s: the traversal of walk() below, but where the clearance c of the
// current voxel is >= 2 it jumps to the state after the (k + c - 1)-th crossing of the
// dominant axis (all crossings up to that time, ties included, exactly as the stepwise
// walk takes them).  Over that interval each axis crosses at most c times, so every voxel
// passed is within L-infinity distance c and in band: no tests are needed.
// mt_start > 0: the traversal up to the mt_start-th crossing of the dominant axis is known to
// be in band (a brick tube certified the segment that far with a margin of 2); it starts there.
__device__ bool los_clear(const uint8_t *__restrict__ band, const uint8_t *__restrict__ clr, Dims d, int vx, int vy,
                          int vz, int sx, int sy, int sz, int cs, int mt_start = 0) {
    const int A0 = abs(sx - vx), A1 = abs(sy - vy), A2 = abs(sz - vz);
    const int total = A0 + A1 + A2;
    if (total == 0) return true;
    const int64_t sxy = (int64_t)d.nx * d.ny;
    const int64_t st0 = sx >= vx ? 1 : -1, st1 = sy >= vy ? d.nx : -(int64_t)d.nx, st2 = sz >= vz ? sxy : -sxy;
    int m = 0, Am = A0;
    if (A1 > Am) { m = 1; Am = A1; }
    if (A2 > Am) { m = 2; Am = A2; }
    const unsigned long long f0 = A0 ? A0 : 1, f1 = A1 ? A1 : 1, f2 = A2 ? A2 : 1;
    const unsigned long long P0 = f1 * f2, P1 = f0 * f2, P2 = f0 * f1;
    const int64_t v0 = vx + (int64_t)d.nx * vy + sxy * vz;
    const uint8_t b = band[v0];
    const unsigned long long INF = ~0ULL;
    int k0 = 0, k1 = 0, k2 = 0;
    unsigned long long T0 = A0 ? P0 : INF, T1 = A1 ? P1 : INF, T2 = A2 ? P2 : INF;
    int64_t g = v0;
    int done = 0;
    if (mt_start > 0) {
        const long long mt = mt_start < Am ? mt_start : Am;
        const unsigned long long num = 2ULL * mt - 1, den = 2ULL * Am;
        k0 = m == 0 ? (int)mt : (int)udiv_fast(num * A0 + Am, den);
        k1 = m == 1 ? (int)mt : (int)udiv_fast(num * A1 + Am, den);
        k2 = m == 2 ? (int)mt : (int)udiv_fast(num * A2 + Am, den);
        T0 = k0 < A0 ? (2ULL * k0 + 1) * P0 : INF;
        T1 = k1 < A1 ? (2ULL * k1 + 1) * P1 : INF;
        T2 = k2 < A2 ? (2ULL * k2 + 1) * P2 : INF;
        g = v0 + st0 * k0 + st1 * k1 + st2 * k2;
        done = k0 + k1 + k2;
    }
    while (done < total) {
#ifdef LSRVT_DEBUG
        atomicAdd(&g_path_dbg[3], 1ULL);
#endif
        // inside the site's clearance ball the rest of the (monotone) traversal is in band
        if (max(A0 - k0, max(A1 - k1, A2 - k2)) <= cs) return true;
        int c = __ldg(clr + g);
        int km = m == 0 ? k0 : (m == 1 ? k1 : k2);
        if (c >= 2 && km < Am) {
            long long mt = km + c - 1;
            if (mt > Am) mt = Am;
            unsigned long long num = 2ULL * mt - 1, den = 2ULL * Am;
            k0 = m == 0 ? (int)mt : (int)udiv_fast(num * A0 + Am, den);
            k1 = m == 1 ? (int)mt : (int)udiv_fast(num * A1 + Am, den);
            k2 = m == 2 ? (int)mt : (int)udiv_fast(num * A2 + Am, den);
            T0 = k0 < A0 ? (2ULL * k0 + 1) * P0 : INF;
            T1 = k1 < A1 ? (2ULL * k1 + 1) * P1 : INF;
            T2 = k2 < A2 ? (2ULL * k2 + 1) * P2 : INF;
            g = v0 + st0 * k0 + st1 * k1 + st2 * k2;
            done = k0 + k1 + k2;
            continue;
        }
        if (T0 <= T1 && T0 <= T2) {
            g += st0;
            T0 = ++k0 < A0 ? T0 + 2 * P0 : INF;
        } else if (T1 <= T2) {
            g += st1;
            T1 = ++k1 < A1 ? T1 + 2 * P1 : INF;
        } else {
            g += st2;
            T2 = ++k2 < A2 ? T2 + 2 * P2 : INF;
        }
        if (__ldg(band + g) != b) return false;
        ++done;
    }
    return true;
}

// ---------------------------------------------------------------- candidate lists per coarse cell
// For a coarse cell Q (32^3 voxels) and a band b present in Q, let U_b = min over the band-b
// sites s of Cmax(Q, s), the chamfer distance from s to the farthest voxel of Q (a corner:
// the closed form grows with every |delta|).  Every band-b voxel of Q has a site within U_b,
// so a site whose nearest possible distance Cmin(Q, s) (to the clamp of s into Q) exceeds
// U_b can never be the minimum for a voxel of Q.  The list of Q keeps exactly the sites
// with Cmin <= U_band(s); it is complete.  Sites are gathered ring by ring of coarse cells
// (each ring's sites are at Chebyshev distance >= 32 (rho - 1) + 1 from Q) until every
// band present has U_b below that bound; the buffer is pruned as U_b falls.
// Outputs of the geodesically weighted update (Eq. 2) filled while tessellating: integer
// moment sums of line-of-sight voxels, the line-of-sight bit of every voxel, and the
// list of "pending" voxels whose update needs final neighbour keys (no line of sight, or
// key not settled here).  enabled = false for the final tessellation.
struct UpdateOut {
    bool enabled;
    bool small_coords;
    const uint16_t *q;
    const int32_t *site_pos;
    unsigned long long *sums;
    uint32_t *los_bits;
    int32_t *plist;    // pending voxels, appended per brick
    int32_t *n_plist;
    unsigned long long *energy;  // the iteration's energy words (trace record), or null
};

// Voxels whose key needs their own path check (no brick tube covers them), handed from the
// candidate filter to check_paths_kernel: voxel, winning site, first move to walk.
struct CheckList {
    int32_t *v;   // voxel
    int32_t *s;   // winning site
    int32_t *p;   // the site's voxel
    int32_t *mv;  // first move to walk (the tube-covered prefix), low 24 bits; the site's clearance above
    int32_t *n;
};

// Warm start of the relaxation.  From the second tessellation of a call on, the key array
// still holds the previous tessellation's exact keys (d, s), and site s has since moved by
// msteps[s] face steps, all inside its band (Eq. 2's move walks the 6-connected traversal),
// so a path of length d + msteps[s] W1 from s's new position reaches the voxel: an upper
// bound of its new key.  Voxels whose key is not settled by the filter start the relaxation
// there instead of at +inf, which leaves it far less to do when the sites move little.
struct WarmStart {
    bool on;
    const int32_t *msteps;
    __device__ __forceinline__ unsigned long long bound(unsigned long long old) const {
        if (!on || old == kInfKey) return kInfKey;
        const uint32_t s = (uint32_t)old;
        const unsigned long long dd = (old >> 32) + (unsigned long long)__ldg(msteps + s) * kWFace;
        return dd >= kInf32 ? kInfKey : (dd << 32) | s;
    }
};

constexpr int kCellGather = 4096;   // shared buffer while searching
constexpr int kCellList = 2048;     // stored list per coarse cell
constexpr int kCellThreads = 256;

__device__ __forceinline__ unsigned long long chamfer_box_min(int sx, int sy, int sz, int lx, int ly, int lz, int hx,
                                                              int hy, int hz) {
    int cx = min(max(sx, lx), hx), cy = min(max(sy, ly), hy), cz = min(max(sz, lz), hz);
    return chamfer(sx - cx, sy - cy, sz - cz);
}
__device__ __forceinline__ unsigned long long chamfer_box_max(int sx, int sy, int sz, int lx, int ly, int lz, int hx,
                                                              int hy, int hz) {
    return chamfer(max(abs(sx - lx), abs(sx - hx)), max(abs(sy - ly), abs(sy - hy)), max(abs(sz - lz), abs(sz - hz)));
}

__global__ void __launch_bounds__(kCellThreads) cell_bands_kernel(const uint8_t *__restrict__ band, Dims d,
                                                                  CoarseGeom cg, uint32_t *cell_bands) {
    __shared__ uint32_t m[8];
    const int64_t ncell = (int64_t)cg.ncx * cg.ncy * cg.ncz;
    for (int64_t cell = blockIdx.x; cell < ncell; cell += gridDim.x) {
        if (threadIdx.x < 8) m[threadIdx.x] = 0;
        __syncthreads();
        const int x0 = (int)(cell % cg.ncx) * kCoarse, y0 = (int)((cell / cg.ncx) % cg.ncy) * kCoarse,
                  z0 = (int)(cell / ((int64_t)cg.ncx * cg.ncy)) * kCoarse;
        for (int i = threadIdx.x; i < kCoarse * kCoarse * kCoarse; i += blockDim.x) {
            int x = x0 + (i & 31), y = y0 + ((i >> 5) & 31), z = z0 + (i >> 10);
            if (x >= d.nx || y >= d.ny || z >= d.nz) continue;
            uint8_t b = band[x + (int64_t)d.nx * (y + (int64_t)d.ny * z)];
            if (b != kInvalidBand) atomicOr(&m[b >> 5], 1u << (b & 31));
        }
        __syncthreads();
        if (threadIdx.x < 8) cell_bands[cell * 8 + threadIdx.x] = m[threadIdx.x];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kCellThreads) cell_list_kernel(Dims d, CoarseGeom cg, const uint32_t *cell_bands,
                                                                 const int64_t *__restrict__ coarse_off,
                                                                 const int4 *__restrict__ coarse_cand,
                                                                 int4 *cell_list, int32_t *cell_count) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int4 *buf = (int4 *)smem_raw;                      // kCellGather
    __shared__ unsigned long long U[256];
    __shared__ uint32_t present[8];
    __shared__ int nbuf_s, overflow_s, gscan[kCellThreads / 32], gstart[kCellThreads], gsrc[kCellThreads];
    const int tid = threadIdx.x;
    const int64_t ncell = (int64_t)cg.ncx * cg.ncy * cg.ncz;
    for (int64_t cell = blockIdx.x; cell < ncell; cell += gridDim.x) {
        const int ccx = (int)(cell % cg.ncx), ccy = (int)((cell / cg.ncx) % cg.ncy),
                  ccz = (int)(cell / ((int64_t)cg.ncx * cg.ncy));
        const int lx = ccx * kCoarse, ly = ccy * kCoarse, lz = ccz * kCoarse;
        const int hx = min(lx + kCoarse, d.nx) - 1, hy = min(ly + kCoarse, d.ny) - 1, hz = min(lz + kCoarse, d.nz) - 1;
        if (tid < 8) present[tid] = cell_bands[cell * 8 + tid];
        for (int b = tid; b < 256; b += blockDim.x) U[b] = ~0ULL;
        if (tid == 0) { nbuf_s = 0; overflow_s = 0; }
        __syncthreads();
        bool any_band = false;
        for (int k = 0; k < 8; ++k) any_band |= present[k] != 0;
        for (int rho = 0; any_band && rho <= kMaxRho; ++rho) {
            const int nshell = rho == 0 ? 1 : 2 * (2 * rho + 1) * (2 * rho + 1) + 8 * rho * (2 * rho - 1);
            for (int base = 0; base < nshell; base += kCellThreads) {
                const int q = base + tid;
                int a0 = 0, cnt = 0;
                if (q < nshell) {
                    int dx = 0, dy = 0, dz = 0;
                    if (rho > 0) shell_cell(q, rho, dx, dy, dz);
                    int cx = ccx + dx, cy = ccy + dy, cz = ccz + dz;
                    if (cx >= 0 && cx < cg.ncx && cy >= 0 && cy < cg.ncy && cz >= 0 && cz < cg.ncz) {
                        int64_t cb = cx + (int64_t)cg.ncx * (cy + (int64_t)cg.ncy * cz);
                        a0 = (int)coarse_off[cb];
                        cnt = (int)(coarse_off[cb + 1] - a0);
                    }
                }
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int t2 = __shfl_up_sync(0xffffffffu, incl, o);
                    if ((tid & 31) >= o) incl += t2;
                }
                if ((tid & 31) == 31) gscan[tid >> 5] = incl;
                __syncthreads();
                int wbase = 0, total = 0;
                for (int w2 = 0; w2 < kCellThreads / 32; ++w2) {
                    if (w2 < (tid >> 5)) wbase += gscan[w2];
                    total += gscan[w2];
                }
                gstart[tid] = wbase + incl - cnt;
                gsrc[tid] = a0;
                __syncthreads();
                for (int e = tid; e < total; e += kCellThreads) {
                    int lo2 = 0, hi2 = kCellThreads - 1;
                    while (lo2 < hi2) {
                        int mid = (lo2 + hi2 + 1) >> 1;
                        if (gstart[mid] <= e) lo2 = mid; else hi2 = mid - 1;
                    }
                    int4 c = coarse_cand[gsrc[lo2] + (e - gstart[lo2])];
                    int b = c.w >> 24, sz = c.w & 0xFFFFFF;
                    if (!((present[b >> 5] >> (b & 31)) & 1u)) continue;
                    if (chamfer_box_min(c.y, c.z, sz, lx, ly, lz, hx, hy, hz) > U[b]) continue;
                    atomicMin(&U[b], chamfer_box_max(c.y, c.z, sz, lx, ly, lz, hx, hy, hz));
                    int at = atomicAdd(&nbuf_s, 1);
                    if (at < kCellGather) buf[at] = c;
                    else overflow_s = 1;
                }
                __syncthreads();
            }
            if (overflow_s) break;
            // prune the buffer with the current bounds (in place, order kept not needed)
            {
                int n0 = nbuf_s;
                __syncthreads();
                if (tid == 0) nbuf_s = 0;
                __syncthreads();
                for (int base = 0; base < n0; base += kCellThreads) {
                    int i = base + tid;
                    int4 c = make_int4(0, 0, 0, 0);
                    bool keep = false;
                    if (i < n0) {
                        c = buf[i];
                        int b = c.w >> 24;
                        keep = chamfer_box_min(c.y, c.z, c.w & 0xFFFFFF, lx, ly, lz, hx, hy, hz) <= U[b];
                    }
                    __syncthreads();
                    if (keep) buf[atomicAdd(&nbuf_s, 1)] = c;
                    __syncthreads();
                }
            }
            // done when every present band has a site and the next ring cannot beat its bound
            const unsigned long long next_min = (unsigned long long)(rho * kCoarse + 1) * kWFace;
            int pending = 0;
            for (int b = tid; b < 256; b += blockDim.x)
                if (((present[b >> 5] >> (b & 31)) & 1u) && U[b] >= next_min) pending = 1;
            bool covers = (ccx - rho) <= 0 && (ccx + rho) >= cg.ncx - 1 && (ccy - rho) <= 0 &&
                          (ccy + rho) >= cg.ncy - 1 && (ccz - rho) <= 0 && (ccz + rho) >= cg.ncz - 1;
            if (!__syncthreads_or(pending) || covers) break;
        }
        // store the list; bands without any site keep U = inf and their voxels are relaxed
        const int n = nbuf_s;
        const bool bad = overflow_s || n > kCellList;
        for (int i = tid; i < n && !bad; i += blockDim.x) cell_list[cell * kCellList + i] = buf[i];
        if (tid == 0) cell_count[cell] = bad ? -1 : n;
        __syncthreads();
    }
}

// Brick pass: the brick re-prunes its coarse cell's list with its own box (the same
// argument at brick scale), sorts the survivors by (band, chamfer distance from the brick
// centre), and every voxel scans its band's segment until C(centre, s) - R exceeds its
// best (triangle inequality; R = the brick's chamfer radius).  Keys are exact where one
// shortest chamfer path to the winner stays in band; elsewhere +inf and the brick is queued.
template <bool kSmall>
__global__ void __launch_bounds__(kRelaxThreads, 3) cfi_kernel(const uint8_t *__restrict__ band,
                                                            const uint8_t *__restrict__ clr,
                                                            const uint32_t *__restrict__ emask, Dims d, BrickGeom bg,
                                                            CoarseGeom cg, const int4 *__restrict__ cell_list,
                                                            const int32_t *__restrict__ cell_count,
                                                            const int64_t *__restrict__ fine_off,
                                                            const int4 *__restrict__ fine_cand, unsigned long long *key,
                                                            int32_t *list_out, int32_t *n_out, uint32_t *flags,
                                                            uint32_t *xmask, uint8_t *hasunk, uint32_t tag,
                                                            UpdateOut up, CheckList chk, WarmStart warm) {
    __shared__ int4 cs[kMaxCand];
    __shared__ unsigned long long ck[kMaxCand];
    __shared__ unsigned long long Ub[256];
    __shared__ uint32_t present[8];
    __shared__ short band_start[257];
    __shared__ int ncand_s, unknown_s, pcount_s, pbase_s, ccount_s, cbase_s;
    __shared__ uint8_t csclr[kMaxCand];       // per winning candidate: the clearance at its site
    __shared__ unsigned long long vbest[RV];  // per voxel: best chamfer key
    __shared__ short vwin[RV];                // per voxel: index of the winner in cs (-1 none)
    __shared__ uint8_t wcert[kMaxCand];       // per candidate: 1 = wins a voxel, 2 = brick certificate holds
    __shared__ int wcov[kMaxCand];            // per candidate: tube extent certified (half voxels)
    const int tid = threadIdx.x;
    const int64_t nbricks = (int64_t)bg.nbx * bg.nby * bg.nbz;
    EnergyAcc eacc;
    for (int64_t brick = blockIdx.x; brick < nbricks; brick += gridDim.x) {
        const int bx = (int)(brick % bg.nbx), by = (int)((brick / bg.nbx) % bg.nby),
                  bz = (int)(brick / ((int64_t)bg.nbx * bg.nby));
        const int ox = bx * RX, oy = by * RY, oz = bz * RZ;
        const int lx = ox, ly = oy, lz = oz;
        const int hx = min(ox + RX, d.nx) - 1, hy = min(oy + RY, d.ny) - 1, hz = min(oz + RZ, d.nz) - 1;
        const int64_t cell = (ox >> kCoarseShift) + (int64_t)cg.ncx * ((oy >> kCoarseShift) + (int64_t)cg.ncy * (oz >> kCoarseShift));
        PHASE_T0();
        // the coarse cell's list (when complete): this thread's first entry is loaded now, so its
        // latency overlaps the initialisation and the band loads
        const int nl = cell_count[cell];
        const int4 *L = cell_list + cell * kCellList;
        const bool has_reg = tid < nl;
        int4 c_reg = make_int4(0, 0, 0, 0);
        if (has_reg) c_reg = L[tid];
        if (tid < 8) present[tid] = 0;
        for (int b = tid; b < 256; b += blockDim.x) Ub[b] = ~0ULL;
        for (int c2 = tid; c2 < kMaxCand / 4; c2 += blockDim.x) reinterpret_cast<uint32_t *>(wcert)[c2] = 0u;
        if (tid == 0) { unknown_s = 0; ncand_s = 0; pcount_s = 0; ccount_s = 0; }
        __syncthreads();
        uint8_t vb[kVPT];
#pragma unroll
        for (int j = 0; j < kVPT; ++j) {
            int i = tid + kRelaxThreads * j;
            int x = ox + (i & (RX - 1)), y = oy + ((i >> 4) & (RY - 1)), z = oz + (i >> 7);
            uint8_t b = kInvalidBand;
            if (x < d.nx && y < d.ny && z < d.nz) b = band[x + (int64_t)d.nx * (y + (int64_t)d.ny * z)];
            vb[j] = b;
            if (b != kInvalidBand) atomicOr(&present[b >> 5], 1u << (b & 31));
        }
        // complete = the coarse cell's list is usable (it holds every site that can win);
        // otherwise (dense regions overflow it) the brick takes the sites of the bricks within
        // +-1 (x) / +-2 (y, z) bricks and settles a voxel only when its best is closer than
        // any site outside that box can be
        const bool complete = nl >= 0;
        constexpr int FX = 1, FY = 2, FZ = 2, NFX = 2 * FX + 1, NFY = 2 * FY + 1, NFZ = 2 * FZ + 1;
        // brick-level bounds Ub (every band, present or not: a bound of an absent band is never
        // read), then the survivors of the present bands
        auto bound = [&](const int4 &c) {
            atomicMin(&Ub[c.w >> 24], chamfer_box_max(c.y, c.z, c.w & 0xFFFFFF, lx, ly, lz, hx, hy, hz));
        };
        auto keep = [&](const int4 &c) {
            int b = c.w >> 24;
            if (!((present[b >> 5] >> (b & 31)) & 1u)) return;
            if (chamfer_box_min(c.y, c.z, c.w & 0xFFFFFF, lx, ly, lz, hx, hy, hz) <= Ub[b]) {
                int at = atomicAdd(&ncand_s, 1);
                if (at < kMaxCand) cs[at] = c;
            }
        };
        if (complete) {
            if (has_reg) bound(c_reg);
            for (int i = tid + blockDim.x; i < nl; i += blockDim.x) bound(L[i]);
            __syncthreads();
            if (has_reg) keep(c_reg);
            for (int i = tid + blockDim.x; i < nl; i += blockDim.x) keep(L[i]);
            __syncthreads();
        } else {
            for (int pass = 0; pass < 2; ++pass) {
                for (int qb = tid; qb < NFX * NFY * NFZ; qb += blockDim.x) {
                    int cx = bx + qb % NFX - FX, cy = by + (qb / NFX) % NFY - FY, cz = bz + qb / (NFX * NFY) - FZ;
                    if (cx < 0 || cx >= bg.nbx || cy < 0 || cy >= bg.nby || cz < 0 || cz >= bg.nbz) continue;
                    int64_t bb = cx + (int64_t)bg.nbx * (cy + (int64_t)bg.nby * cz);
                    for (int64_t r = fine_off[bb]; r < fine_off[bb + 1]; ++r) {
                        if (pass == 0) bound(fine_cand[r]);
                        else keep(fine_cand[r]);
                    }
                }
                __syncthreads();
            }
        }
        PHASE_ADD(0);
        // a brick without a voxel of any band (NaN regions, the gaps between the blocks of a
        // packed batch): every voxel keeps +inf and counts as exact; nothing else to do
        if (!(present[0] | present[1] | present[2] | present[3] | present[4] | present[5] | present[6] |
              present[7])) {
#pragma unroll
            for (int j = 0; j < kVPT; ++j) {
                const int i = tid + kRelaxThreads * j;
                const int x = ox + (i & (RX - 1)), y = oy + ((i >> 4) & (RY - 1)), z = oz + (i >> 7);
                if (x < d.nx && y < d.ny && z < d.nz) key[x + (int64_t)d.nx * (y + (int64_t)d.ny * z)] = kInfKey;
                if ((tid & 31) == 0) xmask[brick * 32 + (tid >> 5) + (kRelaxThreads / 32) * j] = 0xFFFFFFFFu;
            }
            if (tid == 0) hasunk[brick] = 0;
            __syncthreads();
            continue;
        }
        const int nc = ncand_s;
        const bool ok_list = nc <= kMaxCand;
#ifdef LSRVT_DEBUG
        if (tid == 0) { atomicAdd(&g_phase[0], (unsigned long long)max(nl, 0)); atomicAdd(&g_phase[1], (unsigned long long)nc); atomicAdd(&g_phase[3], 1ULL); }
#endif
        // fine search box in voxels (used only when !complete)
        const int flx = (bx - FX) * RX, fhx = (bx + FX + 1) * RX - 1;
        const int fly = (by - FY) * RY, fhy = (by + FY + 1) * RY - 1;
        const int flz = (bz - FZ) * RZ, fhz = (bz + FZ + 1) * RZ - 1;
        int npow2 = 1;
        if (ok_list && nc <= kRelaxThreads) {
            // one key per thread, placed at its rank among the others (keys are distinct): one
            // barrier instead of the sorting network's log^2 stages
            unsigned long long e = ~0ULL;
            if (tid < nc) {
                const int4 c = cs[tid];
                unsigned long long cc = chamfer(c.y - (ox + RX / 2), c.z - (oy + RY / 2), (c.w & 0xFFFFFF) - (oz + RZ / 2));
                if (cc > (1ULL << 36) - 1) cc = (1ULL << 36) - 1;
                e = ((unsigned long long)(uint32_t)(c.w >> 24) << 56) | (cc << 12) | (unsigned)tid;
                vbest[tid] = e;  // staging (vbest is written again only in the scan below)
            }
            __syncthreads();
            if (tid < nc) {
                int r = 0;
                for (int f = 0; f < nc; ++f) r += vbest[f] < e;
                ck[r] = e;
            }
        } else if (ok_list) {
            while (npow2 < nc) npow2 <<= 1;
            for (int i = tid; i < npow2; i += blockDim.x) {
                unsigned long long e = ~0ULL;
                if (i < nc) {
                    int4 c = cs[i];
                    unsigned long long cc = chamfer(c.y - (ox + RX / 2), c.z - (oy + RY / 2), (c.w & 0xFFFFFF) - (oz + RZ / 2));
                    if (cc > (1ULL << 36) - 1) cc = (1ULL << 36) - 1;
                    e = ((unsigned long long)(uint32_t)(c.w >> 24) << 56) | (cc << 12) | (unsigned)i;
                }
                ck[i] = e;
            }
            if (npow2 > 1) block_bitonic_sort(ck, npow2);
        }
        __syncthreads();
        if (ok_list) {
            for (int b2 = tid; b2 <= 256; b2 += blockDim.x) {
                int lo2 = 0, hi2 = nc;
                while (lo2 < hi2) {
                    int mid = (lo2 + hi2) >> 1;
                    if ((int)(ck[mid] >> 56) < b2) lo2 = mid + 1;
                    else hi2 = mid;
                }
                band_start[b2] = (short)lo2;
            }
        }
        __syncthreads();
        PHASE_ADD(1);
        // (1) per voxel: the smallest chamfer key over the candidates of its band.  Triangle
        // inequality of the chamfer metric: C(v, s) >= C(c, s) - C(c, v) for the sort centre c,
        // so a voxel's scan ends once C(c, s) - C(c, v) exceeds its best; C(c, s) never decreases
        // along a band's segment and the best only falls, so a voxel that stops never restarts.
        // When a thread's voxels share one band they scan its segment together: each candidate
        // is loaded once and evaluated for every voxel still scanning (4 independent chains).
        {
            unsigned long long bestv[kVPT], cvv[kVPT];
            int bidxv[kVPT], xv[kVPT], yv[kVPT], zv[kVPT];
            bool scanv[kVPT];
            bool same = true;
            int b0 = -1;
#pragma unroll
            for (int j = 0; j < kVPT; ++j) {
                const int i = tid + kRelaxThreads * j;
                xv[j] = ox + (i & (RX - 1));
                yv[j] = oy + ((i >> 4) & (RY - 1));
                zv[j] = oz + (i >> 7);
                const bool inb = xv[j] < d.nx && yv[j] < d.ny && zv[j] < d.nz;
                scanv[j] = inb && vb[j] != kInvalidBand && ok_list && Ub[vb[j]] != ~0ULL;
                bestv[j] = kInfKey;
                bidxv[j] = -1;
                cvv[j] = chamfer(xv[j] - (ox + RX / 2), yv[j] - (oy + RY / 2), zv[j] - (oz + RZ / 2));
                if (scanv[j]) {
                    if (b0 < 0) b0 = vb[j];
                    else if (vb[j] != b0) same = false;
                }
            }
            if (same && b0 >= 0) {
                const int t0 = band_start[b0], t1 = band_start[b0 + 1];
                for (int t = t0; t < t1; ++t) {
                    const unsigned long long e = ck[t];
                    const unsigned long long dc = (e >> 12) & ((1ULL << 36) - 1);
                    bool act[kVPT], any = false;
#pragma unroll
                    for (int j = 0; j < kVPT; ++j) {
                        act[j] = scanv[j] && dc <= (bestv[j] >> 32) + cvv[j];
                        any |= act[j];
                    }
                    if (!any) break;
                    const int4 c = cs[(unsigned)(e & 0xFFF)];
                    const int cz = c.w & 0xFFFFFF;
#ifdef LSRVT_DEBUG
                    atomicAdd(&g_phase[10], 1ULL);
#endif
#pragma unroll
                    for (int j = 0; j < kVPT; ++j) {
                        if (!act[j]) continue;
                        const unsigned long long cd = chamfer_t<kSmall>(c.y - xv[j], c.z - yv[j], cz - zv[j]);
                        if (!kSmall && cd >= kInf32) continue;
                        const unsigned long long k2 = (cd << 32) | (unsigned)c.x;
                        if (k2 < bestv[j]) { bestv[j] = k2; bidxv[j] = (int)(e & 0xFFF); }
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < kVPT; ++j) {
                    if (!scanv[j]) continue;
                    const int t0 = band_start[vb[j]], t1 = band_start[vb[j] + 1];
                    for (int t = t0; t < t1; ++t) {
                        const unsigned long long e = ck[t];
                        if (((e >> 12) & ((1ULL << 36) - 1)) > (bestv[j] >> 32) + cvv[j]) break;
#ifdef LSRVT_DEBUG
                        atomicAdd(&g_phase[11], 1ULL);
#endif
                        const int4 c = cs[(unsigned)(e & 0xFFF)];
                        const unsigned long long cd =
                            chamfer_t<kSmall>(c.y - xv[j], c.z - yv[j], (c.w & 0xFFFFFF) - zv[j]);
                        if (!kSmall && cd >= kInf32) continue;
                        const unsigned long long k2 = (cd << 32) | (unsigned)c.x;
                        if (k2 < bestv[j]) { bestv[j] = k2; bidxv[j] = (int)(e & 0xFFF); }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < kVPT; ++j) {
                const int i = tid + kRelaxThreads * j;
                const int x = xv[j], y = yv[j], z = zv[j];
                unsigned long long best = bestv[j];
                int bidx = bidxv[j];
                if (!complete && best != kInfKey) {
                    long long gap = 1LL << 40;
                    if (flx > 0) gap = min(gap, (long long)(x - flx + 1));
                    if (fhx < d.nx - 1) gap = min(gap, (long long)(fhx - x + 1));
                    if (fly > 0) gap = min(gap, (long long)(y - fly + 1));
                    if (fhy < d.ny - 1) gap = min(gap, (long long)(fhy - y + 1));
                    if (flz > 0) gap = min(gap, (long long)(z - flz + 1));
                    if (fhz < d.nz - 1) gap = min(gap, (long long)(fhz - z + 1));
                    if ((best >> 32) >= (unsigned long long)gap * kWFace) best = kInfKey;  // not settled
                }
                if (best == kInfKey) bidx = -1;
                vbest[i] = best;
                vwin[i] = (short)bidx;
                if (bidx >= 0) wcert[bidx] = 1;
            }
        }
        __syncthreads();
        PHASE_ADD(2);
        // (2) one tube certificate per (brick, winning site), a group of G lanes per candidate
        // that wins: whole warps for at most 8 candidates, narrower groups for more, so that
        // the block's threads cover the candidates in one pass
        if (ok_list) {
            int G = 32;
            while (G > 1 && nc * G > kRelaxThreads) G >>= 1;
            for (int c2 = tid / G; c2 < nc; c2 += kRelaxThreads / G) {
                if (wcert[c2] != 1) continue;  // uniform over the group
                const int4 c = cs[c2];
                const int cz = c.w & 0xFFFFFF;
                const int cov = brick_tube_in_band_group(clr, d, lx, ly, lz, hx, hy, hz, c.y, c.z, cz, G);
                if ((tid & (G - 1)) == 0) {
                    csclr[c2] = __ldg(clr + c.y + (int64_t)d.nx * (c.z + (int64_t)d.ny * cz));
                    const int L2 = max(abs(2 * c.y - lx - hx), max(abs(2 * c.z - ly - hy), abs(2 * cz - lz - hz)));
                    wcov[c2] = cov;
                    // L2 = 0 (a clipped edge brick centred on the site): the walk returns its answer, 0 or 1
                    if (cov >= max(L2, 1)) wcert[c2] = 2;
                }
            }
        }
        __syncthreads();
        PHASE_ADD(4);
        // (3) per voxel: keys and update outputs; voxels that need their own path check are
        // handed to check_paths_kernel (full warps, no barriers) with a tentative exact key
        int unknown = 0;
        uint32_t pmask = 0, cmask = 0;
        int cmv[kVPT];
#pragma unroll
        for (int j = 0; j < kVPT; ++j) {
            int i = tid + kRelaxThreads * j;
            int x = ox + (i & (RX - 1)), y = oy + ((i >> 4) & (RY - 1)), z = oz + (i >> 7);
            const bool inb = x < d.nx && y < d.ny && z < d.nz;
            const int64_t g = inb ? x + (int64_t)d.nx * (y + (int64_t)d.ny * z) : 0;
            const unsigned long long best = vbest[i];
            const int bidx = vwin[i];
            const int4 bs = bidx >= 0 ? cs[bidx] : make_int4(0, 0, 0, 0);
            unsigned long long k = kInfKey;
            bool los = false, pend = false, exactv = false;
            cmv[j] = 0;
            if (inb && vb[j] != kInvalidBand) {
                int status = 0;
                const int bsz = bs.w & 0xFFFFFF;
                if (best != kInfKey) {
                    if (wcert[bidx] == 2 || (best >> 32) == 0) {
                        status = 2;
#ifdef LSRVT_DEBUG
                        atomicAdd(&g_phase[5], 1ULL);
#endif
                    } else {
                        // skip the moves the brick's tube already covers: t <= cov / L2
                        int mv0 = 0;
                        const int cov = wcov[bidx];
                        if (cov > 0) {
                            const int L2 = max(abs(2 * bs.y - lx - hx),
                                               max(abs(2 * bs.z - ly - hy), abs(2 * bsz - lz - hz)));
                            const int Av = max(abs(bs.y - x), max(abs(bs.z - y), abs(bsz - z)));
                            mv0 = (int)(((long long)cov * Av) / L2);
                        }
                        cmv[j] = mv0;
                        cmask |= 1u << j;
                        status = -1;  // tentative: exact key, no outputs until checked
                    }
                }
                if (status < 0) {
                    // the path check writes the exact key; until then the warm bound
                    k = warm.bound(key[g]);
                } else if (status) {
                    k = best;
                    if (up.enabled) {
                        // O(1) line-of-sight certificates only; other voxels are walked in the pending pass
                        los = (best >> 32) == 0 || status == 2;
                        pend = !los;
                    }
                } else {
                    k = warm.bound(key[g]);
                    unknown = 1;
                    pend = up.enabled;
                }
                key[g] = k;
                exactv = status != 0;
            } else if (inb) {
                key[g] = k;
            }
            if (pend) pmask |= 1u << j;
            {
                // exact keys never change in the relaxation: one bit per voxel in brick order
                // (a failed path check clears its bit)
                const bool exact = !(inb && vb[j] != kInvalidBand) || exactv;
                const unsigned xb = __ballot_sync(0xffffffffu, exact);
                if ((tid & 31) == 0) xmask[brick * 32 + (tid >> 5) + (kRelaxThreads / 32) * j] = xb;
            }
            if (up.enabled) {
                {
                    // one atomic per distinct bit-array word in the warp
                    const int64_t word = inb ? (g >> 5) : -1;
                    const unsigned bit = inb ? (1u << (g & 31)) : 0u;
                    unsigned mw = __match_any_sync(0xffffffffu, word);
                    unsigned lb = __reduce_or_sync(mw, los ? bit : 0u);
                    if (inb && (mw & lanemask_lt()) == 0 && lb) atomicOr(&up.los_bits[word], lb);
                }
                // warp-aggregated integer moment sums of the line-of-sight voxels (Eq. 2, phi(v) = v)
                const int32_t sid = los ? bs.x : -1;
                const unsigned w = los ? (up.q ? up.q[g] : 1u) : 0u;
                if (los) eacc.add(w, (uint32_t)(best >> 32));
                if (up.small_coords) {
                    unsigned m = __match_any_sync(0xffffffffu, sid);
                    unsigned sx = __reduce_add_sync(m, w * (unsigned)x);
                    unsigned sy = __reduce_add_sync(m, w * (unsigned)y);
                    unsigned sz = __reduce_add_sync(m, w * (unsigned)z);
                    unsigned sw = __reduce_add_sync(m, w);
                    if (los && (m & lanemask_lt()) == 0) {
                        atomicAdd(&up.sums[4 * (int64_t)sid + 0], (unsigned long long)sx);
                        atomicAdd(&up.sums[4 * (int64_t)sid + 1], (unsigned long long)sy);
                        atomicAdd(&up.sums[4 * (int64_t)sid + 2], (unsigned long long)sz);
                        atomicAdd(&up.sums[4 * (int64_t)sid + 3], (unsigned long long)sw);
                    }
                } else if (los) {
                    atomicAdd(&up.sums[4 * (int64_t)sid + 0], (unsigned long long)w * (unsigned)x);
                    atomicAdd(&up.sums[4 * (int64_t)sid + 1], (unsigned long long)w * (unsigned)y);
                    atomicAdd(&up.sums[4 * (int64_t)sid + 2], (unsigned long long)w * (unsigned)z);
                    atomicAdd(&up.sums[4 * (int64_t)sid + 3], (unsigned long long)w);
                }
            }
        }
        if (unknown) unknown_s = 1;
#ifdef LSRVT_DEBUG
        __syncthreads();
        PHASE_ADD(3);
#endif
        {
            // append the brick's pending voxels and path checks: warp offsets in shared memory,
            // one global atomic per list per brick (entry order varies between runs; every use
            // is order-free)
            const int lane = tid & 31;
            unsigned bal[kVPT], cbal[kVPT];
            int wtot = 0, ctot = 0;
#pragma unroll
            for (int j = 0; j < kVPT; ++j) {
                bal[j] = __ballot_sync(0xffffffffu, (pmask >> j) & 1u);
                cbal[j] = __ballot_sync(0xffffffffu, (cmask >> j) & 1u);
                wtot += __popc(bal[j]);
                ctot += __popc(cbal[j]);
            }
            int wbase = 0, cbase = 0;
            if (lane == 0 && wtot) wbase = atomicAdd(&pcount_s, wtot);
            if (lane == 0 && ctot) cbase = atomicAdd(&ccount_s, ctot);
            wbase = __shfl_sync(0xffffffffu, wbase, 0);
            cbase = __shfl_sync(0xffffffffu, cbase, 0);
            __syncthreads();
            if (tid == 0) pbase_s = pcount_s ? atomicAdd(up.n_plist, pcount_s) : 0;
            if (tid == 32) cbase_s = ccount_s ? atomicAdd(chk.n, ccount_s) : 0;
            __syncthreads();
            int off = pbase_s + wbase, coff = cbase_s + cbase;
#pragma unroll
            for (int j = 0; j < kVPT; ++j) {
                int i = tid + kRelaxThreads * j;
                int x = ox + (i & (RX - 1)), y = oy + ((i >> 4) & (RY - 1)), z = oz + (i >> 7);
                const int32_t g32 = (int32_t)(x + (int64_t)d.nx * (y + (int64_t)d.ny * z));
                if ((pmask >> j) & 1u) up.plist[off + __popc(bal[j] & lanemask_lt())] = g32;
                if ((cmask >> j) & 1u) {
                    const int at = coff + __popc(cbal[j] & lanemask_lt());
                    const int w2 = vwin[i];
                    const int4 cw = cs[w2];
                    chk.v[at] = g32;
                    chk.s[at] = cw.x;
                    chk.p[at] = (int32_t)(cw.y + (int64_t)d.nx * (cw.z + (int64_t)d.ny * (cw.w & 0xFFFFFF)));
                    chk.mv[at] = min(cmv[j], 0xFFFFFF) | ((int)csclr[w2] << 24);
                }
                off += __popc(bal[j]);
                coff += __popc(cbal[j]);
            }
        }
        __syncthreads();
        PHASE_ADD(5);
        // the brick's own sites: distance 0, lowest id (also where the list was unusable)
        for (int64_t r = fine_off[brick] + tid; r < fine_off[brick + 1]; r += blockDim.x) {
            int4 c = fine_cand[r];
            int64_t g = c.y + (int64_t)d.nx * (c.z + (int64_t)d.ny * (c.w & 0xFFFFFF));
            atomicMin(key + g, (unsigned long long)(uint32_t)c.x);
        }
        if (tid == 0) {
            hasunk[brick] = (uint8_t)(unknown_s != 0);
            if (unknown_s && atomicExch(&flags[brick], tag) != tag) {
                int pos = atomicAdd(n_out, 1);
                list_out[pos] = (int32_t)brick;
            }
        }
        __syncthreads();
    }
    if (up.enabled) eacc.flush(up.energy);
}


// Path checks of the voxels the brick tubes did not cover, one thread per voxel in whole
// warps: status 0 (the path leaves the band) makes the key unknown (+inf, exact bit cleared,
// brick queued for the relaxation); status 2 certifies line of sight (moments added);
// status 1 (exact key, no margin) walks Eq. 2's traversal here, and only voxels without
// line of sight go to the pending pass (their parents need the final keys).
__global__ void __launch_bounds__(256, 3) check_paths_kernel(
    const uint8_t *__restrict__ band, const uint32_t *__restrict__ emask, const uint8_t *__restrict__ clr, Dims d,
    BrickGeom bg,
    const int32_t *__restrict__ site_pos, unsigned long long *key, uint32_t *xmask, uint8_t *hasunk, uint32_t *flags,
    uint32_t tag, int32_t *list_out, int32_t *n_out, CheckList chk, UpdateOut up, VoxelCoder vc) {
    const int32_t cnt = *chk.n;
    const int lane = threadIdx.x & 31;
    EnergyAcc eacc;
    // whole warps step through the list together (warp-level reductions and appends below)
    for (int32_t bstart = blockIdx.x * blockDim.x; bstart < cnt; bstart += gridDim.x * blockDim.x) {
        const int32_t i = bstart + threadIdx.x;
        const bool valid = i < cnt;
        int status = 2;
        int x = 0, y = 0, z = 0, px = 0, py = 0, pz = 0;
        int32_t s = -1;
        int64_t g = -1;
        if (valid) {
            g = __ldg(chk.v + i);
            s = __ldg(chk.s + i);
            const int32_t p = __ldg(chk.p + i);
            const int mvw = __ldg(chk.mv + i);
            const int mv0 = mvw & 0xFFFFFF, cs = (int)((unsigned)mvw >> 24);
            vc.decode((uint32_t)g, d, x, y, z);
            vc.decode((uint32_t)p, d, px, py, pz);
            status = chamfer_path_in_band(emask, clr, d, x, y, z, px, py, pz, cs, mv0);
#ifdef LSRVT_DEBUG
            atomicAdd(&g_path_dbg[mv0 > 0 ? 1 : 0], 1ULL);
            atomicAdd(&g_path_dbg[4 + status], 1ULL);
            for (int sb = 0; sb < 3; ++sb) {
                const int mx = sb == 0 ? 3 : (sb == 1 ? 7 : 1), myz = sb == 2 ? 1 : 3;
                const int lx = x & ~mx, ly = y & ~myz, lz = z & ~myz;
                const int hx = min(lx + mx, d.nx - 1), hy = min(ly + myz, d.ny - 1), hz = min(lz + myz, d.nz - 1);
                const int cov = brick_tube_in_band(clr, d, lx, ly, lz, hx, hy, hz, px, py, pz);
                const int L2 = max(abs(2 * px - lx - hx), max(abs(2 * py - ly - hy), abs(2 * pz - lz - hz)));
                if (cov >= max(L2, 1)) atomicAdd(&g_path_dbg[7 + sb], 1ULL);
            }
#endif
            // an exact key without the margin certificate: walk Eq. 2's traversal now (the
            // update pass keeps only the voxels without line of sight, for their parents)
            if (status == 1 && up.enabled && los_clear(band, clr, d, x, y, z, px, py, pz, cs, mv0)) {
                status = 2;
#ifdef LSRVT_DEBUG
                atomicAdd(&g_path_dbg[10], 1ULL);
#endif
            }
            if (status != 0) {
                // exact: the chamfer distance to the site (the filter left the warm bound here)
                key[g] = ((unsigned long long)chamfer(px - x, py - y, pz - z) << 32) | (uint32_t)s;
            } else {
                const int64_t brick = x / RX + (int64_t)bg.nbx * (y / RY + (int64_t)bg.nby * (z / RZ));
                const int li = (x & (RX - 1)) + RX * ((y & (RY - 1)) + RY * (z & (RZ - 1)));
                atomicAnd(&xmask[brick * 32 + (li >> 5)], ~(1u << (li & 31)));
                hasunk[brick] = 1;
                if (atomicExch(&flags[brick], tag) != tag) {
                    int pos = atomicAdd(n_out, 1);
                    list_out[pos] = (int32_t)brick;
                }
            }
        }
        if (!up.enabled) continue;  // uniform over the launch
        const bool los = valid && status == 2;
        const bool pend = valid && status != 2;
        {
            // one atomic per distinct bit-array word in the warp
            const int64_t word = valid ? (g >> 5) : -1;
            const unsigned bit = valid ? (1u << (g & 31)) : 0u;
            unsigned mw = __match_any_sync(0xffffffffu, word);
            unsigned lb = __reduce_or_sync(mw, los ? bit : 0u);
            if (valid && (mw & lanemask_lt()) == 0 && lb) atomicOr(&up.los_bits[word], lb);
        }
        // warp-aggregated integer moment sums of the line-of-sight voxels (Eq. 2, phi(v) = v)
        const int32_t sid = los ? s : -1;
        const unsigned w = los ? (up.q ? up.q[g] : 1u) : 0u;
        if (los) eacc.add(w, (uint32_t)chamfer(px - x, py - y, pz - z));  // the checked key: chamfer distance
        if (up.small_coords) {
            unsigned m = __match_any_sync(0xffffffffu, sid);
            unsigned sx = __reduce_add_sync(m, w * (unsigned)x);
            unsigned sy = __reduce_add_sync(m, w * (unsigned)y);
            unsigned sz = __reduce_add_sync(m, w * (unsigned)z);
            unsigned sw = __reduce_add_sync(m, w);
            if (los && (m & lanemask_lt()) == 0) {
                atomicAdd(&up.sums[4 * (int64_t)sid + 0], (unsigned long long)sx);
                atomicAdd(&up.sums[4 * (int64_t)sid + 1], (unsigned long long)sy);
                atomicAdd(&up.sums[4 * (int64_t)sid + 2], (unsigned long long)sz);
                atomicAdd(&up.sums[4 * (int64_t)sid + 3], (unsigned long long)sw);
            }
        } else if (los) {
            atomicAdd(&up.sums[4 * (int64_t)sid + 0], (unsigned long long)w * (unsigned)x);
            atomicAdd(&up.sums[4 * (int64_t)sid + 1], (unsigned long long)w * (unsigned)y);
            atomicAdd(&up.sums[4 * (int64_t)sid + 2], (unsigned long long)w * (unsigned)z);
            atomicAdd(&up.sums[4 * (int64_t)sid + 3], (unsigned long long)w);
        }
        // pending voxels: one atomic per warp, 32 consecutive entries in entry order (spatially
        // coherent runs for the update pass)
        const unsigned pb = __ballot_sync(0xffffffffu, pend);
        int wbase = 0;
        if (lane == 0 && pb) wbase = atomicAdd(up.n_plist, __popc(pb));
        wbase = __shfl_sync(0xffffffffu, wbase, 0);
        if (pend) up.plist[wbase + __popc(pb & lanemask_lt())] = (int32_t)g;
    }
    if (up.enabled) eacc.flush(up.energy);
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
    const int32_t *__restrict__ site_pos, const uint8_t *__restrict__ clr, unsigned long long *sums,
    uint32_t *los_bits, int32_t *par, int32_t *nonlos, int32_t *n_nonlos, const int32_t *__restrict__ plist,
    const int32_t *n_plist, bool small_coords, const int32_t *__restrict__ src, unsigned long long *energy,
    const uint32_t *__restrict__ emask, VoxelCoder vc) {
    // plist == nullptr: every voxel (N < 2^31); src != nullptr: the path's next node is the
    // voxel's source (any-angle tessellation) instead of the chamfer parent
    const int32_t cnt = plist ? *n_plist : (int32_t)d.n();
    EnergyAcc eacc;
    // whole warps step through the list together (the warp-level reductions below need them)
    for (int32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; base < cnt; base += gridDim.x * blockDim.x) {
        const int32_t i = base + (threadIdx.x & 31);
#ifdef LSRVT_DEBUG
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&g_phase[2], 1ULL);
            atomicAdd(&g_phase[4], (unsigned long long)min(32, cnt - base));
        }
#endif
        const int64_t v = i < cnt ? (plist ? __ldg(plist + i) : i) : -1;
        const int64_t wv = v >> 5;
        bool los = false;
        int32_t s = -1;
        int x = 0, y = 0, z = 0;
        if (v >= 0) {
            unsigned long long k = key[v];
            if (k != kInfKey) {
                s = (int32_t)(uint32_t)k;
                uint32_t dist = (uint32_t)(k >> 32);
                vc.decode((uint32_t)v, d, x, y, z);
                if (dist == 0) {
                    los = true;
                } else {
#ifdef LSRVT_DEBUG
                    long long _u0 = clock64();
#endif
                    int32_t p = site_pos[s];
                    int px, py, pz;
                    vc.decode((uint32_t)p, d, px, py, pz);
                    los = los_clear(band, clr, d, x, y, z, px, py, pz, __ldg(clr + p));
#ifdef LSRVT_DEBUG
                    atomicAdd(&g_phase[6], (unsigned long long)(clock64() - _u0));
                    if (los) atomicAdd(&g_phase[9], 1ULL);
#endif
                }
                if (!los) {
                    // parent: first neighbour in (dz,dy,dx) order with an edge (the edge mask: the
                    // spanned box lies in the band), same site and D(u)+w = D(v)
                    int32_t parent = src ? __ldg(src + v) : -1;
                    const uint32_t e = src ? 0u : __ldg(emask + v);
                    for (int o = 0; o < 27 && parent < 0 && !src; ++o) {
                        if (o == 13 || !((e >> o) & 1u)) continue;
                        int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
                        int64_t u = (x + dx) + (int64_t)d.nx * ((y + dy) + (int64_t)d.ny * (z + dz));
                        unsigned long long ku = key[u];
                        if ((int32_t)(uint32_t)ku != s) continue;
                        if ((ku >> 32) + weight_of(o) == (k >> 32)) parent = (int32_t)u;
                    }
                    par[v] = parent;
#ifdef LSRVT_DEBUG
                    atomicAdd(&g_phase[7], 1ULL);
#endif
                }
            }
        }
        {
            // voxels without line of sight, for the phi pass: one atomic per warp
            const bool nl = v >= 0 && s >= 0 && !los;
            const unsigned nb2 = __ballot_sync(0xffffffffu, nl);
            int nbase = 0;
            if ((threadIdx.x & 31) == 0 && nb2) nbase = atomicAdd(n_nonlos, __popc(nb2));
            nbase = __shfl_sync(0xffffffffu, nbase, 0);
            if (nl) nonlos[nbase + __popc(nb2 & lanemask_lt())] = (int32_t)v;
        }
        {
            // one atomic per distinct bit-array word in the warp
            const unsigned bit = v >= 0 ? (1u << (v & 31)) : 0u;
            unsigned mw = __match_any_sync(0xffffffffu, wv);
            unsigned lb = __reduce_or_sync(mw, los ? bit : 0u);
            if (v >= 0 && (mw & lanemask_lt()) == 0 && lb) atomicOr(&los_bits[wv], lb);
        }
        // warp-aggregated integer moment sums of the LOS voxels
        int32_t grp = los ? s : -1;
        unsigned m = __match_any_sync(0xffffffffu, grp);
        unsigned w = los ? (q ? q[v] : 1u) : 0u;
        if (los) eacc.add(w, (uint32_t)(key[v] >> 32));
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
    eacc.flush(energy);
}

__global__ void update_nonlos_kernel(const uint16_t *__restrict__ q, Dims d, const unsigned long long *__restrict__ key,
                                     const uint32_t *__restrict__ los_bits, const int32_t *__restrict__ par,
                                     const int32_t *__restrict__ nonlos, const int32_t *n_nonlos,
                                     unsigned long long *sums, int32_t *status, unsigned long long *energy) {
    int32_t cnt = *n_nonlos;
    int64_t n = d.n();
    EnergyAcc eacc;
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
        const unsigned long long kv = key[v];
        int32_t s = (int32_t)(uint32_t)kv;
        unsigned long long w = q ? q[v] : 1u;
        eacc.add((unsigned)w, (uint32_t)(kv >> 32));
        int ux, uy, uz;
        decode_voxel((uint32_t)u, d, ux, uy, uz);
        atomicAdd(&sums[4 * (int64_t)s + 0], w * (unsigned)ux);
        atomicAdd(&sums[4 * (int64_t)s + 1], w * (unsigned)uy);
        atomicAdd(&sums[4 * (int64_t)s + 2], w * (unsigned)uz);
        atomicAdd(&sums[4 * (int64_t)s + 3], w);
    }
    eacc.flush(energy);
}

__global__ void move_sites_kernel(const uint8_t *__restrict__ band, Dims d, int32_t *site_pos, const int32_t *n_sites_dev,
                                  int32_t max_sites, const unsigned long long *__restrict__ sums,
                                  unsigned long long *trace, int32_t *msteps) {
    int32_t ns = min(*n_sites_dev, max_sites);
    for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
        int32_t p = site_pos[s];
        int x = p % d.nx, y = (p / d.nx) % d.ny, z = p / (d.nx * d.ny);
        long long M = (long long)sums[4 * (int64_t)s + 3];
        if (msteps) msteps[s] = 0;
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
            // the walk's face steps: a path of this many W1 edges joins the old and new position
            if (msteps) msteps[s] = (int32_t)(llabs(ddx) + llabs(ddy) + llabs(ddz));
            if (trace) {
                const unsigned long long D2 = (unsigned long long)(ddx * ddx + ddy * ddy + ddz * ddz);
                atomicAdd(&trace[0], 1ULL);
                atomicAdd(&trace[1], D2);
                atomicAdd(&trace[2], ceil_q16_length(D2));  // d_s in 16.16, rounded up
            }
        }
    }
}

// the moment sums of the live sites (4 words each) and the 4 words after them, cleared before
// each update: the count is read on the device, so the work follows the sites, not the capacity
__global__ void zero_sums_kernel(unsigned long long *sums, const int32_t *__restrict__ n_sites_dev, int32_t max_sites) {
    const int64_t words = 4 * (int64_t)min(max(*n_sites_dev, 0), max_sites) + 4;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x)
        sums[i] = 0ull;
}

__global__ void emit_kernel(const unsigned long long *__restrict__ key, int64_t n, int32_t *cell, uint32_t *dist) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long k = key[v];
        bool inf = k == kInfKey;
        cell[v] = inf ? -1 : (int32_t)(uint32_t)k;
        if (dist) dist[v] = inf ? kInf32 : (uint32_t)(k >> 32);
    }
}

// Edge masks and the clearance field, once per call (the bands never change during the Lloyd
// iterations): S_0 and the edge masks from band tiles, kClearLevels - 1 tiled erosions, then
// the per-voxel count of sets.
void clearance_and_edges(const uint8_t *band, Dims d, uint32_t *planes, uint8_t *clr, uint32_t *emask,
                         cudaStream_t s) {
    BitGeom bgm{(d.nx + 31) / 32};
    const int64_t nw = bgm.words(d);
    const int64_t mt = (int64_t)bgm.W * ((d.ny + kTileY - 1) / kTileY) * ((d.nz + kTileZ - 1) / kTileZ);
    band_masks_kernel<<<(int)(mt < kSMs * 8 ? mt : kSMs * 8), 256, 0, s>>>(band, d, bgm, planes, emask);
    const int64_t et = (int64_t)((bgm.W + kEW - 1) / kEW) * ((d.ny + kEY - 1) / kEY) * ((d.nz + kEZ - 1) / kEZ);
    for (int k = 1; k < kClearLevels; ++k)
        clear_erode_kernel<<<(int)(et < kSMs * 8 ? et : kSMs * 8), 256, 0, s>>>(planes + (int64_t)(k - 1) * nw, d, bgm,
                                                                                planes + (int64_t)k * nw);
    clear_count_kernel<<<grid_for(nw, 256, kSMs * 16), 256, 0, s>>>(planes, d, bgm, kClearLevels, clr);
}

struct CvtWs {
    unsigned long long *key;
    int32_t *par;
    uint32_t *los_bits;
    int32_t *nonlos;
    int32_t *counters;  // [0] n_nonlos, [1..2] queue counts, [3..4] work counters, [5] n_plist, [6] checks
    unsigned long long *sums;
    uint32_t *flags;
    int32_t *list[2];
    RelaxQueue *rq;
    int64_t *fine_off, *coarse_off;
    int32_t *fine_cur, *coarse_cur;
    int4 *fine_cand, *coarse_cand;
    int64_t *bin_total;
    uint8_t *clr;
    uint32_t *emask;
    uint32_t *xmask;   // per brick 32 words: exact-key bits written by the candidate filter
    uint8_t *hasunk;   // per brick: unsettled voxels left by the candidate filter
    uint32_t *planes;
    uint32_t *cell_bands;
    int4 *cell_list;
    int32_t *cell_count;
    int32_t *plist;
    int32_t *chk_p;    // path checks: the site's voxel
    int32_t *msteps;   // per site: face steps of its last move (warm start)
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
    CoarseGeom cg{(d.nx + kCoarse - 1) / kCoarse, (d.ny + kCoarse - 1) / kCoarse, (d.nz + kCoarse - 1) / kCoarse};
    int64_t ncoarse = (int64_t)cg.ncx * cg.ncy * cg.ncz;
    w.fine_off = c.take<int64_t>(nbricks + 1);
    w.coarse_off = c.take<int64_t>(ncoarse + 1);
    w.fine_cur = c.take<int32_t>(nbricks);
    w.coarse_cur = c.take<int32_t>(ncoarse);
    w.fine_cand = c.take<int4>((int64_t)max_sites + 1);
    w.coarse_cand = c.take<int4>((int64_t)max_sites + 1);
    w.bin_total = c.take<int64_t>(2);
    w.clr = c.take<uint8_t>(n);
    w.emask = c.take<uint32_t>(n);
    w.xmask = c.take<uint32_t>(nbricks * 32);
    w.hasunk = c.take<uint8_t>(nbricks);
    BitGeom bgm{(d.nx + 31) / 32};
    w.planes = c.take<uint32_t>(bgm.words(d) * kClearLevels);
    w.cell_bands = c.take<uint32_t>(ncoarse * 8);
    w.cell_list = c.take<int4>(ncoarse * kCellList);
    w.cell_count = c.take<int32_t>(ncoarse);
    w.plist = c.take<int32_t>(n);
    w.chk_p = c.take<int32_t>(n);
    w.msteps = c.take<int32_t>((int64_t)max_sites + 1);
    w.rq = c.take<RelaxQueue>(1);
    w.scan = c.take<char>(scan_temp_bytes((nbricks > ncoarse ? nbricks : ncoarse) + 1));
    *need = c.used;
    return w;
}

// ---------------------------------------------------------------- any-angle tessellation
// Sec. 3.2 region growing: each voxel v polls the neighbours w it has an edge with and weighs
// the paths (v, P_w), length |x_v - x_w| + d[w], and (v, P_src(w)), length |x_v - x_src(w)| +
// d[src(w)], the latter only when the traversal v -> src(w) stays in v's band; v also
// re-evaluates its own path (v, P_src(v)) with the current d[src(v)].  Updates take effect in
// the next round (synchronous rounds, double-buffered state), so the result does not depend
// on thread order.  The new state is the lexicographic minimum of (length, site, d[src], src);
// the re-evaluated own path is never worse than the old state, so states only decrease and
// the rounds end.  Lengths are ceil(2^16 |.|) integers, so sums are exact.
// State: key (length << 32 | site) and src (voxel index, -1 unreached).

__device__ __forceinline__ bool aa_less(unsigned long long ka, uint32_t dpa, int32_t pa, unsigned long long kb,
                                        uint32_t dpb, int32_t pb) {
    if (ka != kb) return ka < kb;
    if (dpa != dpb) return dpa < dpb;
    return pa < pb;
}

__global__ void aa_timeout_kernel(int32_t *status) { set_status(status, LSRVT_ERR_TIMEOUT); }

__global__ void aa_init_kernel(int64_t n, unsigned long long *k0, int32_t *p0, unsigned long long *k1, int32_t *p1) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        k0[v] = kInfKey;
        k1[v] = kInfKey;
        p0[v] = -1;
        p1[v] = -1;
    }
}

// sites at distance 0, the lowest id on a shared voxel, in both state buffers
__global__ void aa_sites_kernel(const uint8_t *__restrict__ band, Dims d, const int32_t *__restrict__ site_pos,
                                const int32_t *n_sites_dev, int32_t max_sites, unsigned long long *k0, int32_t *p0,
                                unsigned long long *k1, int32_t *p1, int32_t *status) {
    const int32_t ns = min(*n_sites_dev, max_sites);
    const int64_t n = d.n();
    for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
        const int32_t p = site_pos[s];
        if (p < 0 || p >= n || band[p] == kInvalidBand) {
            set_status(status, LSRVT_ERR_INVALID_ARG);
            continue;
        }
        atomicMin(&k0[p], (unsigned long long)(uint32_t)s);
        atomicMin(&k1[p], (unsigned long long)(uint32_t)s);
        p0[p] = p;
        p1[p] = p;
    }
}

__device__ __forceinline__ bool test_bit(const uint32_t *__restrict__ bits, int64_t i) {
    return (__ldg(bits + (i >> 5)) >> (i & 31)) & 1u;
}

// One synchronous round r: reads (k0, p0), writes (k1, p1); c1 receives the voxels whose
// state changed (one bitmap word per warp of 32 consecutive voxels) and flags[r] = 1 if any
// did.  A voxel whose inputs -- its own state, its source's, and the states of its edge
// neighbours and of their sources -- did not change in round r-1 (c0) gets the candidates of
// round r-1 again, so its state stays; it is skipped and not written, since both buffers
// already hold that state (the sites start in both buffers, and every evaluated voxel is
// written, so a voxel unchanged in the round that last evaluated it is equal in both).  A round after one that
// changed nothing returns at once (both buffers then hold the fixed point).
__global__ void __launch_bounds__(256) aa_round_kernel(const uint8_t *__restrict__ band,
                                                       const uint8_t *__restrict__ clr,
                                                       const uint32_t *__restrict__ emask, Dims d,
                                                       const unsigned long long *__restrict__ k0,
                                                       const int32_t *__restrict__ p0, unsigned long long *k1,
                                                       int32_t *p1, const uint32_t *__restrict__ c0, uint32_t *c1,
                                                       uint32_t *flags, int32_t round, int32_t *status,
                                                       VoxelCoder vc) {
    if (round > 0 && __ldcg(flags + round - 1) == 0) return;
    const int64_t n = d.n();
    const int64_t nwords = (n + 31) >> 5;
    const int64_t sxy = (int64_t)d.nx * d.ny;
    const int lane = threadIdx.x & 31;
    bool any = false;
    for (int64_t wi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wi < nwords;
         wi += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t v = wi * 32 + lane;
        bool changed = false;
        const uint8_t b = v < n ? band[v] : kInvalidBand;
        if (b != kInvalidBand) {  // NaN voxels stay unreached in both buffers
            const uint32_t em = emask[v];
            const int32_t pv = p0[v];
            bool active = round == 0 || test_bit(c0, v) || (pv >= 0 && test_bit(c0, pv));
            if (!active) {
                // all 26 tests issued without an early exit, so their loads overlap
                uint32_t hit = 0u;
#pragma unroll
                for (int o = 0; o < 27; ++o) {
                    if (o == 13 || !((em >> o) & 1u)) continue;
                    const int64_t w = v + (o % 3 - 1) + d.nx * (int64_t)((o / 3) % 3 - 1) + sxy * (o / 9 - 1);
                    const int32_t t = __ldg(p0 + w);
                    hit |= (uint32_t)test_bit(c0, w) | (t >= 0 ? (uint32_t)test_bit(c0, t) : 0u);
                }
                active = hit != 0u;
            }
            if (active) {
                int x, y, z;
                vc.decode((uint32_t)v, d, x, y, z);
                const unsigned long long kv = k0[v];
                unsigned long long bk = kInfKey;
                uint32_t bdp = kInf32;
                int32_t bp = INT32_MAX;
                // a candidate through source t (t != v): (d[t] + |x_v - x_t|, site(t), d[t], t)
                auto through = [&](int32_t t, unsigned long long &ck, uint32_t &cdp) -> bool {
                    const unsigned long long kt = k0[t];
                    if (kt == kInfKey) return false;
                    int tx, ty, tz;
                    vc.decode((uint32_t)t, d, tx, ty, tz);
                    const long long dx = x - tx, dy = y - ty, dz = z - tz;
                    const unsigned long long D = (unsigned long long)(dx * dx + dy * dy + dz * dz);
                    if (D >= (1ull << 32)) return false;
                    const unsigned long long tot = (kt >> 32) + ceil_q16_length(D);
                    if (tot > 0xFFFFFFFEull) {
                        set_status(status, LSRVT_ERR_OVERFLOW);
                        return false;
                    }
                    ck = (tot << 32) | (kt & 0xFFFFFFFFull);
                    cdp = (uint32_t)(kt >> 32);
                    return true;
                };
                if (pv == v) {  // a site keeps (0, s, 0, v)
                    bk = kv;
                    bdp = 0;
                    bp = pv;
                } else if (pv >= 0) {
                    unsigned long long ck;
                    uint32_t cdp;
                    if (through(pv, ck, cdp)) { bk = ck; bdp = cdp; bp = pv; }
                }
                // a source already weighed (the own one, the last one, the last rejected) gives
                // the same candidate again, which cannot beat the best so far
                int32_t last = pv, rejected = -1;
                for (int o = 0; o < 27; ++o) {
                    if (!((em >> o) & 1u)) continue;
                    const int64_t w = v + (o % 3 - 1) + d.nx * (int64_t)((o / 3) % 3 - 1) + sxy * (o / 9 - 1);
                    const unsigned long long kw = k0[w];
                    if (kw == kInfKey) continue;
                    {
                        const unsigned long long tot = (kw >> 32) + weight_of(o);
                        if (tot > 0xFFFFFFFEull) {
                            set_status(status, LSRVT_ERR_OVERFLOW);
                        } else {
                            const unsigned long long ck = (tot << 32) | (kw & 0xFFFFFFFFull);
                            if (aa_less(ck, (uint32_t)(kw >> 32), (int32_t)w, bk, bdp, bp)) {
                                bk = ck;
                                bdp = (uint32_t)(kw >> 32);
                                bp = (int32_t)w;
                            }
                        }
                    }
                    const int32_t t = p0[w];
                    if (t < 0 || t == w || t == v || t == last || t == pv || t == rejected) continue;
                    last = t;
                    unsigned long long ck;
                    uint32_t cdp;
                    if (!through(t, ck, cdp) || !aa_less(ck, cdp, t, bk, bdp, bp)) continue;  // cannot win: no ray
                    int tx, ty, tz;
                    vc.decode((uint32_t)t, d, tx, ty, tz);
                    const int cs = band[t] == b ? __ldg(clr + t) : 0;
                    if (los_clear(band, clr, d, x, y, z, tx, ty, tz, cs)) {
                        bk = ck;
                        bdp = cdp;
                        bp = t;
                    } else {
                        rejected = t;
                    }
                }
                const int32_t np = bk == kInfKey ? -1 : bp;
                changed = (bk != kv) || (np != pv);
                // written even when unchanged: the other buffer may still hold the state before
                // the last change
                k1[v] = bk;
                p1[v] = np;
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, changed);
        if (lane == 0) c1[wi] = bal;
        any |= bal != 0u;
    }
    if (__syncthreads_or(any) && threadIdx.x == 0) flags[round] = 1u;
}

}  // namespace

size_t cvt_workspace(Dims d, int32_t max_sites) {
    size_t need;
    carve_cvt(nullptr, 0, d, max_sites, &need);
    return need;
}

namespace {

struct AaWs {
    unsigned long long *key[2];
    int32_t *src[2];
    uint8_t *clr;
    uint32_t *emask;
    uint32_t *planes;
    uint32_t *los_bits;
    int32_t *par;
    int32_t *nonlos;
    int32_t *counters;  // [0] n_nonlos
    unsigned long long *sums;
    uint32_t *flags;  // one per round
    uint32_t *chg[2];  // voxels changed in the last round, ping-pong
};

AaWs carve_aa(void *ws, size_t bytes, Dims d, int32_t max_sites, int32_t max_rounds, size_t *need) {
    Carver c(ws, bytes);
    const int64_t n = d.n();
    AaWs w;
    w.key[0] = c.take<unsigned long long>(n);
    w.key[1] = c.take<unsigned long long>(n);
    w.src[0] = c.take<int32_t>(n);
    w.src[1] = c.take<int32_t>(n);
    w.clr = c.take<uint8_t>(n);
    w.emask = c.take<uint32_t>(n);
    BitGeom bgm{(d.nx + 31) / 32};
    w.planes = c.take<uint32_t>(bgm.words(d) * kClearLevels);
    w.los_bits = c.take<uint32_t>((n + 31) / 32);
    w.par = c.take<int32_t>(n);
    w.nonlos = c.take<int32_t>(n);
    w.counters = c.take<int32_t>(8);
    w.sums = c.take<unsigned long long>((int64_t)max_sites * 4 + 4);
    w.flags = c.take<uint32_t>(max_rounds > 0 ? max_rounds : 1);
    w.chg[0] = c.take<uint32_t>((n + 31) / 32);
    w.chg[1] = c.take<uint32_t>((n + 31) / 32);
    *need = c.used;
    return w;
}

}  // namespace

size_t cvt_anyangle_workspace(Dims d, int32_t max_sites, int32_t max_rounds) {
    size_t need;
    carve_aa(nullptr, 0, d, max_sites, max_rounds, &need);
    return need;
}

}  // namespace lsrvt

using namespace lsrvt;

namespace {

// One tessellation: keys <- restricted geodesic Voronoi assignment of the current sites.
lsrvt_status run_assignment(const uint8_t *band, Dims d, const int32_t *site_pos, const int32_t *n_sites_dev,
                            int32_t max_sites, CvtWs &w, uint32_t &tag, int32_t *status, cudaStream_t s,
                            UpdateOut up, bool warm) {
    BrickGeom bg{(d.nx + RX - 1) / RX, (d.ny + RY - 1) / RY, (d.nz + RZ - 1) / RZ};
    int64_t n = d.n();
    int64_t nbricks = (int64_t)bg.nbx * bg.nby * bg.nbz;
    (void)n;
    CoarseGeom cg{(d.nx + kCoarse - 1) / kCoarse, (d.ny + kCoarse - 1) / kCoarse, (d.nz + kCoarse - 1) / kCoarse};
    int64_t ncoarse = (int64_t)cg.ncx * cg.ncy * cg.ncz;
    const int sms = stream_sms(s);  // this stream's share of the SMs
    cudaMemsetAsync(w.counters + 1, 0, sizeof(int32_t) * 4, s);
    cudaMemsetAsync(w.counters + 6, 0, sizeof(int32_t), s);
    cudaMemsetAsync(w.fine_off, 0, sizeof(int64_t) * (nbricks + 1), s);
    // the path-check list lives in buffers that are idle while the assignment runs: the
    // erosion planes (used once per call for the clearance, >= 4 bytes per voxel), and the
    // parent and non-LOS arrays (written only by the update pass afterwards)
    CheckList chk{reinterpret_cast<int32_t *>(w.planes), w.par, w.chk_p, w.nonlos, w.counters + 6};
    cudaMemsetAsync(w.coarse_off, 0, sizeof(int64_t) * (ncoarse + 1), s);
    cudaMemsetAsync(w.fine_cur, 0, sizeof(int32_t) * nbricks, s);
    cudaMemsetAsync(w.coarse_cur, 0, sizeof(int32_t) * ncoarse, s);
    site_bin_count_kernel<<<grid_for(max_sites, 256, kSMs * 4), 256, 0, s>>>(site_pos, n_sites_dev, max_sites, d, bg,
                                                                            cg, w.fine_off, w.coarse_off, status);
    exclusive_scan_i64(w.fine_off, nbricks + 1, w.bin_total, w.scan, s);
    exclusive_scan_i64(w.coarse_off, ncoarse + 1, w.bin_total + 1, w.scan, s);
    site_bin_fill_kernel<<<grid_for(max_sites, 256, kSMs * 4), 256, 0, s>>>(site_pos, n_sites_dev, max_sites, band, d,
                                                                           bg, cg, w.fine_off, w.fine_cur, w.fine_cand,
                                                                           w.coarse_off, w.coarse_cur, w.coarse_cand,
                                                                           status);
    {
        size_t smem = kCellGather * sizeof(int4);
        cudaFuncSetAttribute(cell_list_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int cgrid2 = (int)(ncoarse < (int64_t)sms * 4 ? ncoarse : (int64_t)sms * 4);
        cell_list_kernel<<<cgrid2, kCellThreads, smem, s>>>(d, cg, w.cell_bands, w.coarse_off, w.coarse_cand,
                                                            w.cell_list, w.cell_count);
    }
    ++tag;
    int nb_cfi = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb_cfi, cfi_kernel<true>, kRelaxThreads, 0);
    if (nb_cfi < 1) nb_cfi = 1;
    int cgrid = (int)(nbricks < (int64_t)sms * nb_cfi ? nbricks : (int64_t)sms * nb_cfi);
    // differences of coordinates below 2048 per axis: the scan's distances in 32-bit arithmetic
    if (d.nx <= 2048 && d.ny <= 2048 && d.nz <= 2048)
        cfi_kernel<true><<<cgrid, kRelaxThreads, 0, s>>>(band, w.clr, w.emask, d, bg, cg, w.cell_list, w.cell_count,
                                                         w.fine_off, w.fine_cand, w.key, w.list[0], w.counters + 1,
                                                         w.flags, w.xmask, w.hasunk, tag, up, chk,
                                                         WarmStart{warm, w.msteps});
    else
        cfi_kernel<false><<<cgrid, kRelaxThreads, 0, s>>>(band, w.clr, w.emask, d, bg, cg, w.cell_list, w.cell_count,
                                                          w.fine_off, w.fine_cand, w.key, w.list[0], w.counters + 1,
                                                          w.flags, w.xmask, w.hasunk, tag, up, chk,
                                                          WarmStart{warm, w.msteps});
    check_paths_kernel<<<sms * 16, 256, 0, s>>>(band, w.emask, w.clr, d, bg, site_pos, w.key, w.xmask, w.hasunk, w.flags,
                                                 tag, w.list[0], w.counters + 1, chk, up, make_coder(d));
#ifdef LSRVT_DEBUG
    {
        int32_t q0 = 0;
        cudaMemcpyAsync(&q0, w.counters + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        fprintf(stderr, "cfi: %d of %lld bricks queued", q0, (long long)nbricks);
    }
#endif
    int nb_per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb_per_sm, relax_async_kernel, kRelaxThreads, 0);
    if (nb_per_sm < 1) nb_per_sm = 1;
    const int nsm = sms;
    // at most one CTA per brick: small volumes leave the rest of the GPU to concurrent work
    int grid = (int)((int64_t)nsm * nb_per_sm < nbricks ? (int64_t)nsm * nb_per_sm : nbricks);
    relax_queue_init_kernel<<<1, 1, 0, s>>>(w.rq, w.counters + 1);
    cudaMemsetAsync(w.list[1], 0, sizeof(int32_t) * (size_t)nbricks, s);
    const int32_t max_tickets = (int32_t)(int64_t(1) << 30);
    relax_async_kernel<<<grid, kRelaxThreads, 0, s>>>(w.emask, w.xmask, w.hasunk, d, bg, w.key, w.list[0],
                                                      w.counters + 1, w.list[1], (int32_t)nbricks, w.rq, w.flags,
                                                      tag, max_tickets, status);
    tag += 1u;
#ifdef LSRVT_DEBUG
    {
        RelaxQueue hq;
        cudaStreamSynchronize(s);
        cudaMemcpy(&hq, w.rq, sizeof(hq), cudaMemcpyDeviceToHost);
        unsigned long long rs[2], rz[2] = {0, 0};
        cudaMemcpyFromSymbol(rs, g_relax_steps, sizeof(rs));
        cudaMemcpyToSymbol(g_relax_steps, rz, sizeof(rz));
        fprintf(stderr, " | relax brick visits %llu (pushed %d) steps/visit %.1f\n", rs[1], hq.pushed,
                rs[1] ? (double)rs[0] / rs[1] : 0.0);
    }
#endif
    return launch_status();
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
    if (iter_trace && n_iters > 0) cudaMemsetAsync(iter_trace, 0, sizeof(int64_t) * LSRVT_TRACE * n_iters, s);
    bool small = d.nx <= 2048 && d.ny <= 2048 && d.nz <= 2048;
    {
        clearance_and_edges(band, d, w.planes, w.clr, w.emask, s);
        CoarseGeom cg{(d.nx + kCoarse - 1) / kCoarse, (d.ny + kCoarse - 1) / kCoarse, (d.nz + kCoarse - 1) / kCoarse};
        int64_t ncoarse = (int64_t)cg.ncx * cg.ncy * cg.ncz;
        cell_bands_kernel<<<(int)(ncoarse < kSMs * 8 ? ncoarse : kSMs * 8), kCellThreads, 0, s>>>(band, d, cg,
                                                                                                w.cell_bands);
    }
    uint32_t tag = 0;
    const int sms = stream_sms(s);
    int vgrid = grid_for((n + 31) / 32 * 32, 256, sms * 16);
    UpdateOut up{true, small, q, site_pos, w.sums, w.los_bits, w.plist, w.counters + 5, nullptr};
    UpdateOut no_up{false, small, q, site_pos, nullptr, nullptr, nullptr, nullptr, nullptr};
    const int64_t nwords = (n + 31) / 32;
    for (int32_t it = 0; it < n_iters; ++it) {
        unsigned long long *rec = iter_trace ? (unsigned long long *)(iter_trace + (int64_t)LSRVT_TRACE * it) : nullptr;
        up.energy = rec ? rec + 3 : nullptr;
        zero_sums_kernel<<<sms * 2, 256, 0, s>>>(w.sums, n_sites_dev, max_sites);
        cudaMemsetAsync(w.los_bits, 0, sizeof(uint32_t) * nwords, s);
        cudaMemsetAsync(w.counters, 0, sizeof(int32_t), s);
        cudaMemsetAsync(w.counters + 5, 0, sizeof(int32_t), s);
        // from the second tessellation on, the keys of the last one bound the new ones
        lsrvt_status st = run_assignment(band, d, site_pos, n_sites_dev, max_sites, w, tag, status_dev, s, up, it > 0);
        if (st != LSRVT_OK) return st;
        update_voxels_kernel<<<vgrid, 256, 0, s>>>(band, q, d, w.key, site_pos, w.clr, w.sums, w.los_bits, w.par,
                                                   w.nonlos, w.counters, w.plist, w.counters + 5, small, nullptr,
                                                   up.energy, w.emask, make_coder(d));
        update_nonlos_kernel<<<sms * 8, 256, 0, s>>>(q, d, w.key, w.los_bits, w.par, w.nonlos, w.counters, w.sums,
                                                      status_dev, up.energy);
        move_sites_kernel<<<grid_for(max_sites, 256, kSMs * 8), 256, 0, s>>>(band, d, site_pos, n_sites_dev,
                                                                            max_sites, w.sums, rec, w.msteps);
    }
    lsrvt_status st = run_assignment(band, d, site_pos, n_sites_dev, max_sites, w, tag, status_dev, s, no_up,
                                     n_iters > 0);
    if (st != LSRVT_OK) return st;
    emit_kernel<<<grid_for(n, 256, kSMs * 16), 256, 0, s>>>(w.key, n, cell, dist);
#ifdef LSRVT_DEBUG
    {
        unsigned long long ph[12];
        cudaMemcpyFromSymbol(ph, g_phase, sizeof(ph));
        fprintf(stderr, "cfi tube-certified voxels %llu own path checks %llu\n", ph[5], ph[8]);
        unsigned long long pd[12], pz[12] = {0};
        cudaMemcpyFromSymbol(pd, g_path_dbg, sizeof(pd));
        cudaMemcpyToSymbol(g_path_dbg, pz, sizeof(pz));
        fprintf(stderr, "walk loop turns: path %llu los %llu\n", pd[2], pd[3]);
        fprintf(stderr, "path checks: from start %llu after tube prefix %llu | status0 %llu status1 %llu status2 %llu "
                "| sub-box tubes 4x4x4 %llu 8x4x4 %llu 2x2x2 %llu | los upgrades %llu\n", pd[0], pd[1], pd[4], pd[5],
                pd[6], pd[7], pd[8], pd[9], pd[10]);
        fprintf(stderr, "cfi bricks %llu coarse-list entries %llu brick candidates %llu | scan steps same-band %llu mixed %llu\n",
                ph[3], ph[0], ph[1], ph[10], ph[11]);
        fprintf(stderr, "cfi chamfer-evals %llu | update: pending warps %llu pending voxels %llu los-walks true %llu "
                "nonlos %llu los-cycles %.3g\n", ph[10], ph[2], ph[4], ph[9], ph[7], (double)ph[6]);
        unsigned long long cp[8], cz[8] = {0};
        cudaMemcpyFromSymbol(cp, g_cfi_ph, sizeof(cp));
        cudaMemcpyToSymbol(g_cfi_ph, cz, sizeof(cz));
        fprintf(stderr, "cfi phases (cycles, thread 0 of each CTA): gather %.3g sort %.3g scan %.3g tube %.3g "
                "paths+outputs %.3g compaction %.3g\n", (double)cp[0], (double)cp[1], (double)cp[2], (double)cp[4],
                (double)cp[3], (double)cp[5]);
        unsigned long long z[12] = {0};
        cudaMemcpyToSymbol(g_phase, z, sizeof(z));
    }
#endif
    return launch_status();
}

namespace {

// One any-angle tessellation: synchronous rounds from the sites until a round changes
// nothing (the fixed point is then in both buffers).  The host reads the change flags once
// per chunk of rounds; rounds launched after convergence return at once.
lsrvt_status aa_assignment(const uint8_t *band, Dims d, const int32_t *site_pos, const int32_t *n_sites_dev,
                           int32_t max_sites, int32_t max_rounds, AaWs &w, int32_t *status, cudaStream_t s,
                           int32_t *rounds_out) {
    const int64_t n = d.n();
    const int sms = stream_sms(s);
    aa_init_kernel<<<grid_for(n, 256, sms * 16), 256, 0, s>>>(n, w.key[0], w.src[0], w.key[1], w.src[1]);
    aa_sites_kernel<<<grid_for(max_sites, 256, kSMs * 4), 256, 0, s>>>(band, d, site_pos, n_sites_dev, max_sites,
                                                                      w.key[0], w.src[0], w.key[1], w.src[1],
                                                                      status);
    cudaMemsetAsync(w.flags, 0, sizeof(uint32_t) * (size_t)max_rounds, s);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, aa_round_kernel, 256, 0);
    if (nb < 1) nb = 1;
    const int grid = grid_for((n + 31) / 32 * 32, 256, sms * nb);
    constexpr int kChunk = 8;
    uint32_t h[kChunk];
    int32_t r = 0, done = -1;
    while (r < max_rounds && done < 0) {
        const int32_t r0 = r, r1 = r + kChunk < max_rounds ? r + kChunk : max_rounds;
        for (; r < r1; ++r)
            aa_round_kernel<<<grid, 256, 0, s>>>(band, w.clr, w.emask, d, w.key[r & 1], w.src[r & 1],
                                                 w.key[(r + 1) & 1], w.src[(r + 1) & 1], w.chg[r & 1],
                                                 w.chg[(r + 1) & 1], w.flags, r, status, make_coder(d));
        if (cudaMemcpyAsync(h, w.flags + r0, sizeof(uint32_t) * (size_t)(r1 - r0), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return LSRVT_ERR_CUDA;
        for (int32_t j = 0; j < r1 - r0; ++j)
            if (h[j] == 0) { done = r0 + j + 1; break; }
    }
    if (done < 0) {
        // the host knows the limit was hit: record it and stop the whole call here
        aa_timeout_kernel<<<1, 1, 0, s>>>(status);
        if (rounds_out) *rounds_out = max_rounds;
        const lsrvt_status ls = launch_status();
        return ls != LSRVT_OK ? ls : LSRVT_ERR_TIMEOUT;
    }
    if (rounds_out) *rounds_out = done;
    return launch_status();
}

}  // namespace

extern "C" lsrvt_status lsrvt_cvt_iterate_anyangle(const uint8_t *band, const uint16_t *q, lsrvt_dims dd,
                                                   int32_t *site_pos, const int32_t *n_sites_dev, int32_t max_sites,
                                                   int32_t n_iters, int32_t max_rounds, int32_t *cell, uint32_t *dist,
                                                   int32_t *src, int64_t *iter_trace, int32_t *rounds_host, void *ws,
                                                   size_t ws_bytes, int32_t *status_dev, void *stream) {
    if (!dims_ok(dd) || !band || !site_pos || !n_sites_dev || max_sites < 0 || n_iters < 0 || max_rounds < 1 ||
        !cell)
        return LSRVT_ERR_INVALID_ARG;
    Dims d{dd.nx, dd.ny, dd.nz};
    size_t need;
    AaWs w = carve_aa(ws, ws_bytes, d, max_sites, max_rounds, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) return LSRVT_ERR_WORKSPACE;
    cudaStream_t s = as_stream(stream);
    const int64_t n = d.n();
    const int sms = stream_sms(s);
    if (iter_trace && n_iters > 0) cudaMemsetAsync(iter_trace, 0, sizeof(int64_t) * LSRVT_TRACE * n_iters, s);
    const bool small = d.nx <= 2048 && d.ny <= 2048 && d.nz <= 2048;
    clearance_and_edges(band, d, w.planes, w.clr, w.emask, s);
    const int vgrid = grid_for((n + 31) / 32 * 32, 256, sms * 16);
    const int64_t nwords = (n + 31) / 32;
    // a tessellation that hits the round limit ends the call: its last round's state (in the
    // buffer that round wrote) is emitted unconverged, no update or further tessellation runs
    auto stop_at_limit = [&]() {
        const int b = max_rounds & 1;
        emit_kernel<<<grid_for(n, 256, kSMs * 16), 256, 0, s>>>(w.key[b], n, cell, dist);
        if (src) cudaMemcpyAsync(src, w.src[b], sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
        const lsrvt_status ls = launch_status();
        return ls != LSRVT_OK ? ls : LSRVT_ERR_TIMEOUT;
    };
    for (int32_t it = 0; it < n_iters; ++it) {
        lsrvt_status st = aa_assignment(band, d, site_pos, n_sites_dev, max_sites, max_rounds, w, status_dev, s,
                                        rounds_host ? rounds_host + it : nullptr);
        if (st == LSRVT_ERR_TIMEOUT) return stop_at_limit();
        if (st != LSRVT_OK) return st;
        unsigned long long *rec = iter_trace ? (unsigned long long *)(iter_trace + (int64_t)LSRVT_TRACE * it) : nullptr;
        zero_sums_kernel<<<sms * 2, 256, 0, s>>>(w.sums, n_sites_dev, max_sites);
        cudaMemsetAsync(w.los_bits, 0, sizeof(uint32_t) * nwords, s);
        cudaMemsetAsync(w.counters, 0, sizeof(int32_t), s);
        update_voxels_kernel<<<vgrid, 256, 0, s>>>(band, q, d, w.key[0], site_pos, w.clr, w.sums, w.los_bits, w.par,
                                                   w.nonlos, w.counters, nullptr, nullptr, small, w.src[0],
                                                   rec ? rec + 3 : nullptr, w.emask, make_coder(d));
        update_nonlos_kernel<<<sms * 8, 256, 0, s>>>(q, d, w.key[0], w.los_bits, w.par, w.nonlos, w.counters, w.sums,
                                                      status_dev, rec ? rec + 3 : nullptr);
        move_sites_kernel<<<grid_for(max_sites, 256, kSMs * 8), 256, 0, s>>>(band, d, site_pos, n_sites_dev,
                                                                            max_sites, w.sums, rec, nullptr);
    }
    lsrvt_status st = aa_assignment(band, d, site_pos, n_sites_dev, max_sites, max_rounds, w, status_dev, s,
                                    rounds_host ? rounds_host + n_iters : nullptr);
    if (st == LSRVT_ERR_TIMEOUT) return stop_at_limit();
    if (st != LSRVT_OK) return st;
    emit_kernel<<<grid_for(n, 256, kSMs * 16), 256, 0, s>>>(w.key[0], n, cell, dist);
    if (src) cudaMemcpyAsync(src, w.src[0], sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
    return launch_status();
}
