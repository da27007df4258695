/*
 * lsrvt.h -- C ABI of the B300 (sm_103a) Level Set Restricted Voronoi Tessellation
 * hot path.
 *
 * Method: Neuroth et al., "Level Set Restricted Voronoi Tessellation for Large scale
 * Spatial Statistical Analysis" (arXiv 2208.06970).  Each entry point below cites the
 * section / equation / algorithm of the paper that defines the operation.
 *
 * Conventions shared by every entry point
 *  - Volumes are dense 3D grids (nx, ny, nz), linear index i = x + nx*(y + ny*z), x
 *    fastest, N = nx*ny*nz < 2^31 voxels.
 *  - Arrays named *_host are host memory.  Every other array is device memory owned
 *    by the caller; the library never allocates, frees or retains device memory.
 *    Scratch memory comes from a caller workspace `ws` of at least
 *    lsrvt_workspace_bytes(step, ...) bytes, 256-byte aligned.  A workspace may be
 *    reused by later calls on the same stream once they are ordered after this one.
 *  - All calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL =
 *    the legacy default stream).  Argument errors (bad dims, NULL pointers, isovalues
 *    not strictly increasing, too small a workspace) return synchronously and launch
 *    nothing.  Errors that depend on the data (capacity exceeded, distance overflow,
 *    non-finite statistics input, a bounded wait or loop that ran out) are written to the caller's
 *    device status word `status_dev` (int32, first error wins; 0 = OK); the caller
 *    clears it and reads it after synchronising.  LSRVT_ERR_CUDA reports a failed
 *    kernel launch (cudaGetLastError) on return.
 *  - Integer results (bands, components, sites, cells, distances, counts, min, max,
 *    histograms) are deterministic and bit-identical from run to run.
 *  - Voxels whose field value is NaN are not graph nodes: band 0xFF, component -1,
 *    cell -1.
 */
#ifndef LSRVT_H
#define LSRVT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Columns of a Lloyd-iteration trace record (lsrvt_cvt_iterate, lsrvt_cvt_iterate_anyangle). */
#define LSRVT_TRACE 5

typedef enum {
    LSRVT_OK = 0,
    LSRVT_ERR_INVALID_ARG = 1, /* bad dims / NULL pointer / parameter out of range       */
    LSRVT_ERR_NOT_SORTED = 2,  /* isovalues not strictly increasing (or NaN)             */
    LSRVT_ERR_CAPACITY = 3,    /* more components / sites / strata than the capacity     */
    LSRVT_ERR_NONFINITE = 4,   /* a statistics input is NaN or infinite                  */
    LSRVT_ERR_TIMEOUT = 5,     /* a bounded device loop hit its limit                    */
    LSRVT_ERR_OVERFLOW = 6,    /* a geodesic distance reached 2^32 (65536 voxel widths)  */
    LSRVT_ERR_CUDA = 7,        /* a CUDA launch failed                                   */
    LSRVT_ERR_WORKSPACE = 8    /* workspace NULL, misaligned or too small                */
} lsrvt_status;

typedef struct {
    int32_t nx, ny, nz;
} lsrvt_dims;

/* Steps, for lsrvt_workspace_bytes. */
typedef enum {
    LSRVT_STEP_CLASSIFY = 0,
    LSRVT_STEP_LABEL = 1,
    LSRVT_STEP_SALIENCY = 2,
    LSRVT_STEP_SEED = 3,
    LSRVT_STEP_CVT = 4,
    LSRVT_STEP_AGGREGATE = 5,
    LSRVT_STEP_MERGE = 6,
    LSRVT_STEP_LAYOUT = 7,
    LSRVT_STEP_JOINT = 8, /* max_sites = range capacity, max_comp, n_aux = variables; dims: positions */
    LSRVT_STEP_GRAPH = 9, /* site graph of a volume of dims d */
    LSRVT_STEP_CVT_ANYANGLE = 10 /* max_sites; n_aux = max_rounds of the any-angle tessellation */
} lsrvt_step;

/* Seeding parameters (Sec. 3.2 "Stratified Random Initial Site Distribution", Eq. nc;
 * Sec. 3.3 "Role and Choice of Parameters"). */
typedef struct {
    int64_t voxels_per_site; /* P = 1/alpha, the site density parameter as voxels per site (>= 1) */
    int32_t strat_block;     /* side of the cubic stratification blocks, 1..16 (default 16); part
                                of the result, not a tuning knob */
    int32_t max_strata;      /* capacity of the (component x block) stratum table; 0 = default   */
    uint64_t rng_seed;       /* seed of the SplitMix64 placement hash                            */
} lsrvt_seed_params;

/* Statistics records (Sec. 3.3 "Aggregation"): one row per cell / component / band.
 * All arrays are device memory with `rows` rows; m = number of variables, B = bins.
 *   count[rows]            int64  voxels
 *   mean[rows][m]          double mean
 *   m2[rows][m]            double sum of squared deviations (population variance = m2/count)
 *   vmin, vmax[rows][m]    float  exact min / max (+inf / -inf for empty rows)
 *   hist[rows][m][B]       uint32 histogram (may be NULL when B = 0)
 *   comom[rows][m(m+1)/2]  double co-moment sums C_ij = sum (x_i-mean_i)(x_j-mean_j),
 *                          upper triangle row-major (NULL unless LSRVT_STATS_COV)   */
typedef struct {
    int64_t *count;
    double *mean;
    double *m2;
    float *vmin;
    float *vmax;
    uint32_t *hist;
    double *comom;
} lsrvt_stats;

/* Joint central moments of up to 8 variables (orders 2..4): one row per region.
 *   count[rows] int64; mean[rows][m] double;
 *   m2[rows][m(m+1)/2]          sum d_i d_j            (i <= j)
 *   m3[rows][m(m+1)(m+2)/6]     sum d_i d_j d_k        (i <= j <= k; coskewness sums)
 *   m4[rows][m(m+1)(m+2)(m+3)/24] sum d_i d_j d_k d_l  (i <= j <= k <= l; cokurtosis sums)
 * with d = x - mean over the region's voxels; index tuples in lexicographic order. */
typedef struct {
    int64_t *count;
    double *mean;
    double *m2;
    double *m3;
    double *m4;
} lsrvt_joint;

#define LSRVT_STATS_HIST 1u
#define LSRVT_STATS_COV 2u

/* Human-readable name of a status code (static string). */
const char *lsrvt_status_string(lsrvt_status s);

/* Library version: major*10000 + minor*100 + patch. */
int32_t lsrvt_version(void);

/* Workspace bytes needed by `step` for a volume of dims `d` with the given capacities
 * (max_comp components, max_sites sites, n_aux statistics variables; pass 0 where the
 * step does not use a capacity).  Returns 0 for invalid dims. */
size_t lsrvt_workspace_bytes(lsrvt_step step, lsrvt_dims d, int32_t max_comp, int32_t max_sites,
                             int32_t n_aux);

/* Isoband classification.  Sec. 3.1 "Level Sets, Isobands, and Connected Components":
 * B_{a,b} = { v : a < f(v) <= b }.  With strictly increasing isovalues t_1 < ... < t_K
 * (0 <= K <= 254, host array) the band of a voxel is #{ i : t_i < f(v) }: band 0 is
 * (-inf, t_1] and band K is (t_K, inf).  NaN -> 0xFF.  -0 and +0 compare equal.
 *   field [N] float (in), band [N] uint8 (out).
 * Errors: INVALID_ARG (dims, NULL, K > 254), NOT_SORTED. */
lsrvt_status lsrvt_classify(const float *field, lsrvt_dims d, const float *iso_host, int32_t n_iso,
                            uint8_t *band, void *stream);

/* Connected components of each isoband.  Sec. 3.1: an isoband is split into components
 * C^k with no voxel of one adjacent to a voxel of another; 6-adjacency.  Component ids
 * are dense and canonical: ordered by (band, smallest linear index).
 *   band [N] uint8 (in); comp [N] int32 (out, -1 for NaN voxels);
 *   comp_band [max_comp] uint8, comp_size [max_comp] int64, comp_first [max_comp] int32
 *   (out: band, voxel count, smallest linear index of each component);
 *   n_comp_dev [1] int32 (out: number of components, also when it exceeds max_comp).
 * If the count exceeds max_comp, CAPACITY is written to status_dev and the tables hold
 * only the first max_comp entries; comp[] is complete. */
lsrvt_status lsrvt_label_components(const uint8_t *band, lsrvt_dims d, int32_t *comp, uint8_t *comp_band,
                                    int64_t *comp_size, int32_t *comp_first, int32_t max_comp,
                                    int32_t *n_comp_dev, void *ws, size_t ws_bytes, int32_t *status_dev,
                                    void *stream);

/* Allocation-free variant of lsrvt_label_components, for callers that cannot allocate
 * device memory or pass a workspace (for example a simulation that embeds the library for
 * in-situ analysis and owns all device memory through its own pool, or a host program that
 * loads it as a plug-in without exposing its allocator).  The paper has no counterpart:
 * this is a deployment form of the same labelling.  Same arguments and results as
 * lsrvt_label_components without `ws`/`ws_bytes`.
 *  - Scratch lives in a fixed device array inside the library (1.25 MiB, held by every
 *    GPU that loads the library until the process exits); volumes of more than 2^18
 *    voxels (64^3) are rejected with LSRVT_ERR_WORKSPACE and nothing is launched.
 *  - Each call made outside stream capture looks up that array's device address on the
 *    current device (so a device reset, which moves the array, is followed); a call made
 *    while its stream is being captured uses the address the last uncaptured call on that
 *    device found.  Make the first call on a device before any stream capture.
 *  - It calls no cudaMalloc, cudaFree or allocating library routine.
 *  - Every call shares the one array: calls that may overlap on the GPU (different streams
 *    without ordering, or several host threads) race and corrupt each other's results;
 *    order them on one stream.  Each call overwrites what the previous call left. */
lsrvt_status lsrvt_label_components_static(const uint8_t *band, lsrvt_dims d, int32_t *comp, uint8_t *comp_band,
                                           int64_t *comp_size, int32_t *comp_first, int32_t max_comp,
                                           int32_t *n_comp_dev, int32_t *status_dev, void *stream);

/* Saliency weights m_v (Sec. 3.1 "Centroids or Centers of Mass": m_v; Sec. 3.3: the
 * second field and the attraction gamma).  q = max(1, rint(g^gamma * 65535 / gmax)),
 * g = |grad f| by central differences (one-sided half differences at the faces),
 * evaluated in IEEE float in a fixed order; gmax = largest finite g^gamma.  gamma is an
 * integer 0..4 (0 gives q = 1 everywhere).
 *   field [N] float (in), q [N] uint16 (out). */
lsrvt_status lsrvt_saliency_grad(const float *field, lsrvt_dims d, int32_t gamma, uint16_t *q, void *ws,
                                 size_t ws_bytes, void *stream);

/* Stratified random initial sites.  Sec. 3.2 "Stratified Random Initial Site
 * Distribution", Eq. (nc), Algorithm 1 (StratifiedRandomSiteDistribution).
 *   n_c = max(ceil(|V| m(C) / (P m(V))), 1) capped at |C|   (m = sum of q; q NULL = 1)
 * apportioned to strata (component x cubic block) by largest remainder with capacity
 * caps; inside a stratum the k voxels in linear order are split into n_b rank ranges
 * and site j takes rank lo_j + splitmix64((seed ^ splitmix64(block)) + j) mod width.
 * Site ids are ordered by (component, block, j).
 *   comp [N] int32 (in, from lsrvt_label_components); n_comp_dev (in);
 *   site_pos [max_sites] int32 (out, linear voxel index), site_comp [max_sites] int32
 *   (out), comp_site_off [max_comp+1] int32 (out: sites of component c are
 *   [off[c], off[c+1])), n_sites_dev [1] int32 (out).
 * CAPACITY (status_dev) if sites > max_sites or strata > the stratum capacity. */
lsrvt_status lsrvt_seed(const int32_t *comp, const uint16_t *q, lsrvt_dims d, const int32_t *n_comp_dev,
                        int32_t max_comp, lsrvt_seed_params p, int32_t *site_pos, int32_t *site_comp,
                        int32_t *comp_site_off, int32_t max_sites, int32_t *n_sites_dev, void *ws,
                        size_t ws_bytes, int32_t *status_dev, void *stream);

/* Lloyd iterations of the level set restricted CVT.  Algorithm 1 (LRCVT) after
 * seeding: n_iters x (restricted geodesic Voronoi tessellation, Eq. 1; geodesically
 * weighted update, Eq. 2) followed by a final tessellation.
 *  Tessellation: cell(v) = the site s of v's component minimising (gd(v, s), s)
 *   lexicographically, gd = shortest path on the graph of 26-neighbour edges whose
 *   spanned box lies in one band, edge lengths 65536, 92682, 113512 (16.16 fixed
 *   point Euclidean lengths rounded up).
 *  Update: phi(v) = v if the voxel traversal v -> site stays in the band, else
 *   phi(parent(v)); target = round-half-up(sum q_v x_phi(v) / sum q_v) per axis; the
 *   site walks the traversal toward the target and stops before leaving its band.
 *   band [N] uint8, q [N] uint16 or NULL (uniform weight) (in);
 *   site_pos [max_sites] int32 (in/out), n_sites_dev (in);
 *   cell [N] int32 (out, site id, -1 for NaN voxels); dist [N] uint32 (out, optional:
 *   16.16 geodesic distance to the site, 0xFFFFFFFF for NaN voxels);
 *   iter_trace [n_iters][LSRVT_TRACE] int64 (out, optional), one record per iteration:
 *     [0] sites moved, [1] sum of squared moves (voxels^2), [2] sum over moved sites of
 *     ceil(2^16 |move|) (the paper's convergence measure, Fig. "convergence": mean d_s =
 *     [2] / 2^16 / n_sites), [3], [4] the CVT energy of the iteration's assignment,
 *     E = sum over assigned voxels of q_v D(v)^2 with D the 16.16 distance, an exact
 *     unsigned 128-bit integer: [3] its low 64 bits, [4] its high 64 bits.  Recorded
 *     only: E is not guaranteed to fall (the geodesic update of Eq. 2 is not Lloyd's
 *     centroid step), and nothing depends on it.
 * OVERFLOW if a distance reaches 2^32; TIMEOUT if a bounded wait of the relaxation's work queue
 * runs out (about a second without progress) or a parent chain of the update is broken. */
lsrvt_status lsrvt_cvt_iterate(const uint8_t *band, const uint16_t *q, lsrvt_dims d, int32_t *site_pos,
                               const int32_t *n_sites_dev, int32_t max_sites, int32_t n_iters, int32_t *cell,
                               uint32_t *dist, int64_t *iter_trace, void *ws, size_t ws_bytes,
                               int32_t *status_dev, void *stream);

/* Lloyd iterations with the any-angle tessellation of Sec. 3.2 ("Discrete Restricted Geodesic
 * Voronoi Tessellation": region growing where each voxel v polls its neighbours w and weighs
 * the paths (v, P_w), of length |x_v - x_w| + d[w], and (v, P_src(w)), of length
 * |x_v - x_src(w)| + d[src(w)], the latter only when the ray v -> src(w) stays in the band;
 * updates take effect in the next round).  Algorithm 1 as lsrvt_cvt_iterate otherwise.
 *  Rounds are synchronous (round r+1 reads only round r), so the labels do not depend on the
 *   schedule.  v polls the 26-neighbours it has an edge with (spanned box in its band) and
 *   also re-evaluates its own path (v, P_src(v)); its new state is the lexicographic minimum
 *   of (length, site, d[src], src) over these candidates.  Lengths are ceil(2^16 |.|)
 *   integers; the ray is the 6-connected traversal of lsrvt_cvt_iterate's update walked from
 *   v.  At the fixed point d[v] = |x_v - x_src(v)| + d[src(v)] and src chains end at v's site.
 *  Update (Eq. 2): phi(v) = v if v sees its site, else phi(src(v)); target and move as in
 *   lsrvt_cvt_iterate.
 *   band, q, site_pos, n_sites_dev, cell, dist, iter_trace as lsrvt_cvt_iterate (dist: the
 *   any-angle length); src [N] int32 (out, optional: the source of each voxel's path, -1 for
 *   NaN or unreached voxels); rounds_host [n_iters + 1] int32 (HOST, out, optional: the
 *   rounds of each tessellation, the last one, which changed nothing, included).
 *  max_rounds (>= 1) bounds the rounds of one tessellation.  A tessellation that does not
 *   settle within it ends the call at once: TIMEOUT goes to status_dev, cell/dist/src receive
 *   the state of its last round (not converged), no update or further tessellation runs (the
 *   sites keep their positions from before that tessellation), rounds_host gets max_rounds
 *   for it and stays untouched after it, and the call returns LSRVT_ERR_TIMEOUT.
 *  The call synchronises the stream once per 8 rounds to read the change flags, so it cannot
 *   be captured in a CUDA graph (lsrvt_cvt_iterate can).
 *  Workspace: lsrvt_workspace_bytes(LSRVT_STEP_CVT_ANYANGLE, d, 0, max_sites, max_rounds). */
lsrvt_status lsrvt_cvt_iterate_anyangle(const uint8_t *band, const uint16_t *q, lsrvt_dims d, int32_t *site_pos,
                                        const int32_t *n_sites_dev, int32_t max_sites, int32_t n_iters,
                                        int32_t max_rounds, int32_t *cell, uint32_t *dist, int32_t *src,
                                        int64_t *iter_trace, int32_t *rounds_host, void *ws, size_t ws_bytes,
                                        int32_t *status_dev, void *stream);

/* Per-variable histogram range: lo_j = min, scale_j = float(n_bins) / (max - min) (0 if
 * max == min) over voxels with cell >= 0 (Sec. 3.3 "Aggregation": histograms).
 *   cell [N] int32; aux_host[n_aux] = device pointers to [N] float; lo_dev, scale_dev
 *   [n_aux] float (out).  NONFINITE if an input value is NaN or infinite. */
lsrvt_status lsrvt_aux_range(const int32_t *cell, const float *const *aux_host, int32_t n_aux, lsrvt_dims d,
                             int32_t n_bins, float *lo_dev, float *scale_dev, int32_t *status_dev, void *stream);

/* Per-cell statistics of n_aux variables (Sec. 3.3 "Aggregation"; introduction:
 * statistics aggregated within segments).  count, mean, m2, min, max always; an n_bins
 * histogram with bin = clamp((int)((x - lo_j) * scale_j), 0, n_bins-1) in IEEE float if
 * flags & LSRVT_STATS_HIST; co-moments if flags & LSRVT_STATS_COV.  Sums are
 * accumulated in float-float (about 44 significant bits) per brick and combined in
 * FP64; co-moments use BF16 split products on tensor cores with FP32 accumulation.
 *   cell [N] int32 (in); aux_host[n_aux] device pointers to [N] float (in);
 *   lo_dev, scale_dev [n_aux] float (in, device; e.g. from lsrvt_aux_range);
 *   out: rows = max_sites, of which rows < *n_sites_dev are written (the rest are left
 *   untouched, so the row capacity costs memory but no traffic).  NONFINITE if a value is NaN
 *   or infinite. */
lsrvt_status lsrvt_aggregate(const int32_t *cell, const float *const *aux_host, int32_t n_aux, lsrvt_dims d,
                             const float *lo_dev, const float *scale_dev, int32_t n_bins, uint32_t flags,
                             const int32_t *site_pos, const int32_t *n_sites_dev, int32_t max_sites,
                             lsrvt_stats out, void *ws, size_t ws_bytes, int32_t *status_dev, void *stream);

/* Merge statistics up the hierarchy cell -> component -> band -> volume (introduction
 * and Sec. 3.2 "Data Reduction and Structured Data Layout": aggregates merged over
 * cells, components and isobands).  Counts, histograms, min, max combine exactly;
 * means, m2 and co-moments combine in FP64 by the pairwise formulas of Chan, Golub &
 * LeVeque (1979) evaluated as sum n_i mean_i / n and sum (m2_i + n_i (mean_i-mean)^2).
 *   cells (rows max_sites, n_sites_dev valid); comp_site_off [n_comp+1] (from
 *   lsrvt_seed); comp_band [n_comp]; n_bands = number of isovalues + 1;
 *   comps (rows max_comp; rows < *n_comp_dev written), bands (rows n_bands), volume
 *   (1 row) (out).  Cell rows < *n_sites_dev are read. */
lsrvt_status lsrvt_merge_hierarchy(lsrvt_stats cells, const int32_t *n_sites_dev, int32_t max_sites,
                                   int32_t n_aux, int32_t n_bins, uint32_t flags,
                                   const int32_t *comp_site_off, const uint8_t *comp_band,
                                   const int32_t *n_comp_dev, int32_t max_comp, int32_t n_bands,
                                   lsrvt_stats comps, lsrvt_stats bands, lsrvt_stats volume, void *ws,
                                   size_t ws_bytes, void *stream);

/* Structured hierarchical data layout (Sec. 3.2 "Data Reduction and Structured Data Layout",
 * Fig. hierarchy): the voxels of the kept isobands ordered by (band, component, cell) and,
 * inside a cell, by linear index, so that every band, component and cell is one contiguous,
 * directly indexable range, with the raw variables extracted in the same order (one
 * coordinate -- the linear index -- plus n_aux values per kept voxel).
 * Site ids must be grouped by component in ascending order and components ordered by band,
 * as lsrvt_label_components and lsrvt_seed number them.
 *   cell [N] int32 (in; -1 = not a node; 16-byte aligned);
 *   comp_site_off [n_comp+1] int32 (from lsrvt_seed), comp_band [n_comp] uint8 (in);
 *   band_mask_host [8] uint32 (host; bit b%32 of word b/32 keeps band b; NULL = all bands);
 *   aux_host[n_aux] device pointers to [N] float (in); values_host[n_aux] device pointers to
 *   [N] float (out; entries < *n_kept_dev written), n_aux <= 64;
 *   order [N] int32 (out): linear voxel index of each layout position (entries < *n_kept_dev
 *   written);
 *   cell_off [max_sites+1], comp_off [max_comp+1] int64 (out): cell s occupies
 *   [cell_off[s], cell_off[s+1]), component c [comp_off[c], comp_off[c+1]); entries
 *   <= *n_sites_dev / *n_comp_dev written;
 *   band_off [257] int64 (out): band b occupies [band_off[b], band_off[b+1]);
 *   n_kept_dev [1] int64 (out): number of voxels in the layout;
 *   cell_out [N] int32 (out, nullable): the cell of each layout position, -1 past the kept
 *   voxels -- a label array in layout order, so the statistics steps can run on the layout
 *   (every cell then a contiguous run of positions).
 * Deterministic (stable sort).  Errors: INVALID_ARG synchronously (dims, NULL, cell not
 * 16-byte aligned, n_aux), and in status_dev when a cell id has no site or the numbering is
 * not hierarchical. */
lsrvt_status lsrvt_structured_layout(const int32_t *cell, lsrvt_dims d, const int32_t *n_sites_dev,
                                     int32_t max_sites, const int32_t *comp_site_off, const uint8_t *comp_band,
                                     const int32_t *n_comp_dev, int32_t max_comp, const uint32_t *band_mask_host,
                                     const float *const *aux_host, int32_t n_aux, float *const *values_host,
                                     int32_t *order, int64_t *cell_off, int64_t *comp_off, int64_t *band_off,
                                     int64_t *n_kept_dev, int32_t *cell_out, void *ws, size_t ws_bytes,
                                     int32_t *status_dev, void *stream);

/* Joint central moments of orders 2..4 of m (1..8) variables over contiguous ranges of
 * voxel records: cells, components or bands of a structured layout (the joint-plot section
 * compares mean, covariance, coskewness and cokurtosis of summaries and raw data; Sec. 3.3).
 *   values_host[m]: device pointers to the variables in layout order (n_positions each);
 *   range_off [max_ranges+1] int64 (device): range r is [range_off[r], range_off[r+1]);
 *   n_ranges_dev (device, nullable = max_ranges): live ranges; rows < it are written.
 * FP32 products summed over at most 32 voxels, then FP64; central moments from exact FP64
 * shift formulas around a per-range shift (the mean of the range's first 32 voxels).
 * Workspace: lsrvt_workspace_bytes(LSRVT_STEP_JOINT, {n_positions, 1, 1}, 0, max_ranges, m). */
lsrvt_status lsrvt_joint_moments(const float *const *values_host, int32_t m, int64_t n_positions,
                                 const int64_t *range_off, const int32_t *n_ranges_dev, int32_t max_ranges,
                                 lsrvt_joint out, void *ws, size_t ws_bytes, void *stream);

/* Merge joint-moment records cell -> component -> band -> volume by the pairwise formulas of
 * Pebay (2008) in FP64, children in id order (arguments as lsrvt_merge_hierarchy; rows < *n_comp_dev
 * of comps, n_bands rows of bands, 1 row of volume written).  Two levels per merge: blocks of 64
 * children merged in parallel, then each parent's blocks in order.  Workspace:
 * lsrvt_workspace_bytes(LSRVT_STEP_JOINT, dims, max_comp, max_sites, m). */
lsrvt_status lsrvt_merge_joint_hierarchy(lsrvt_joint cells, const int32_t *n_sites_dev, int32_t max_sites,
                                         int32_t m, const int32_t *comp_site_off, const uint8_t *comp_band,
                                         const int32_t *n_comp_dev, int32_t max_comp, int32_t n_bands,
                                         lsrvt_joint comps, lsrvt_joint bands, lsrvt_joint volume, void *ws,
                                         size_t ws_bytes, void *stream);

/* Voronoi site graph ("Voronoi Cell Views" section: site connectivity from region adjacency):
 * cells a and b are adjacent when a voxel of each are face neighbours of one band; the edge
 * weighs ceil(2^16 ||x_a - x_b||_2) (exact integer; path lengths are exact sums).
 *   cell [N] int32, band [N] uint8 (in); site_pos [max_sites] int32 (in);
 *   adj_off [max_sites+1] int64 (out): CSR rows (both directions, neighbours increasing);
 *   adj [max_arcs] int32, adj_w [max_arcs] uint32 (out); *n_edges_dev (out, int64): undirected
 *   edges (arcs = 2x).  CAPACITY in status_dev when the arcs exceed max_arcs or the candidate
 *   list overflows.  Workspace: lsrvt_workspace_bytes(LSRVT_STEP_GRAPH, d, 0, 0, 0). */
lsrvt_status lsrvt_site_graph(const int32_t *cell, const uint8_t *band, lsrvt_dims d, const int32_t *site_pos,
                              const int32_t *n_sites_dev, int32_t max_sites, int64_t *adj_off, int32_t *adj,
                              uint32_t *adj_w, int64_t max_arcs, int64_t *n_edges_dev, void *ws, size_t ws_bytes,
                              int32_t *status_dev, void *stream);

/* Geodesic site distances within the sites [s0, s1) (a union of components, closed under
 * adjacency): dist[i][j] (k x k, k = s1 - s0, uint32 weight units, 0xFFFFFFFF = no path) by
 * Bellman-Ford per source over frontier bitmaps, exact; optionally ratio[i][j] =
 * ||x_i - x_j|| / gd(s_i, s_j) (float; 1 on the diagonal, c_far where no path exists), the
 * distance of the "Voronoi Cell Views" section.  INVALID_ARG in status_dev when an arc leaves
 * the range, OVERFLOW when a path reaches 2^32 - 1, TIMEOUT past k rounds.
 * Workspace: 2 * min(k, 4 * SMs) * ceil(k / 32) * 4 + 512 bytes (see the Python binding). */
lsrvt_status lsrvt_site_geodesics(const int64_t *adj_off, const int32_t *adj, const uint32_t *adj_w,
                                  const int32_t *site_pos, lsrvt_dims d, int32_t s0, int32_t s1, uint32_t *dist,
                                  float *ratio, float c_far, void *ws, size_t ws_bytes, int32_t *status_dev,
                                  void *stream);

/* Packed batches of independent blocks (Discussion "Block Based Distributed Parallelism":
 * the blocks of a volume are decomposed independently, their boundaries acting as
 * restrictions).  Many blocks are placed in one packed volume, each at its own origin, apart
 * from each other by at least one voxel of band 0xFF (a voxel that is no graph node), so that
 * one lsrvt_cvt_iterate over the packed volume runs every launch of the Lloyd loop over the
 * bricks of all blocks at once.  No restricted geodesic, voxel traversal or site walk can
 * cross the gap, every block's sites keep their order, and the update's rounding
 * (round-half-up of sum q x / sum q) commutes with translation by the block's origin, so each
 * block's cells, distances and sites are the ones lsrvt_cvt_iterate gives for the block alone;
 * only the iteration trace is summed over the blocks.
 *   Blocks are given as a host array of descriptors whose pointers are device memory of the
 *   block's own arrays (the layout lsrvt_cvt_iterate takes for the block alone). */
#define LSRVT_MAX_PACK_BLOCKS 128

typedef struct {
    lsrvt_dims d;            /* the block's extent */
    int32_t x0, y0, z0;      /* the block's origin in the packed volume */
    const uint8_t *band;     /* [N_b] isoband indices (pack: in) */
    const uint16_t *q;       /* [N_b] weights (pack: in, read only when the packed q is given) */
    int32_t *site_pos;       /* [n_sites_b] linear voxel indices within the block (pack: in; unpack: out) */
    const int32_t *n_sites;  /* the block's site count, device int32 (pack: in) */
    int32_t *cell;           /* [N_b] the block's cells, its own site ids, -1 for NaN (unpack: out) or NULL */
    uint32_t *dist;          /* [N_b] 16.16 geodesic distances (unpack: out) or NULL */
} lsrvt_block;

/* Pack n_blocks (1..LSRVT_MAX_PACK_BLOCKS) blocks into one volume of extent `packed`:
 *   band [N] (out): 0xFF everywhere, each block's bands at its origin;
 *   q [N] (out, optional): 0 everywhere, each block's weights at its origin (NULL: uniform);
 *   site_pos [max_sites] (out): block b's site i at packed id site_base[b] + i, as a packed
 *     linear index; n_sites_dev (out): the total; site_base [n_blocks + 1] (out, device
 *     int32): the exclusive prefix sums of the blocks' counts.
 * INVALID_ARG (synchronously) for a block outside the packed volume or two blocks whose boxes,
 * each widened by one voxel, overlap (their voxels would touch); CAPACITY (status_dev) if the
 * total count exceeds max_sites (then nothing is packed for the sites). */
lsrvt_status lsrvt_pack_blocks(const lsrvt_block *blocks_host, int32_t n_blocks, lsrvt_dims packed, uint8_t *band,
                               uint16_t *q, int32_t *site_pos, int32_t max_sites, int32_t *n_sites_dev,
                               int32_t *site_base, int32_t *status_dev, void *stream);

/* The inverse for the results of lsrvt_cvt_iterate over a packed volume: per block, its cells
 * (packed site ids less site_base[b]; -1 stays -1), its distances, and its sites as linear
 * indices within the block.  cell and dist [N] are the packed results (dist may be NULL, then
 * the blocks' dist are not written); site_pos the packed sites; site_base from the packing. */
lsrvt_status lsrvt_unpack_blocks(const lsrvt_block *blocks_host, int32_t n_blocks, lsrvt_dims packed,
                                 const int32_t *cell, const uint32_t *dist, const int32_t *site_pos,
                                 const int32_t *site_base, void *stream);

/* Execution resources (the execution forms of Sec. 3.2 "Parallel Algorithm": independent
 * blocks processed side by side).  Kernels launched on `stream` size their grids to `percent`
 * of the GPU's SMs (1..100; 100 restores the whole GPU), so decompositions running
 * concurrently on several streams share the GPU instead of each taking all of it.  Results
 * do not depend on the share.  The setting is host-side, process-wide, and applies to
 * launches made after the call; INVALID_ARG if percent is outside 1..100. */
lsrvt_status lsrvt_set_stream_share(void *stream, int32_t percent);

#ifdef __cplusplus
}
#endif

#endif /* LSRVT_H */
