/*
 * lsrvt_oracle.c -- plain, slow, single-threaded CPU oracle of the LSRVT hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code, header,
 * table or constant generator with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Method: Neuroth et al., "Level Set Restricted Voronoi Tessellation for Large
 * scale Spatial Statistical Analysis", arXiv 2208.06970.  Every function cites the
 * section / equation / algorithm it follows.  Where the paper is silent, garbled or
 * ambiguous the reading taken is stated beside the code (the same readings are
 * listed in the design notes of the repository).
 *
 * Conventions: volume dims (nx, ny, nz), linear index i = x + nx*(y + ny*z), x fastest.
 * All integer results are exact.  Floating point follows IEEE-754 single or double
 * precision with round-to-nearest and no contraction (build with -ffp-contract=off).
 *
 * Build: gcc -O2 -std=gnu11 -ffp-contract=off -fPIC -shared -o liboracle.so lsrvt_oracle.c -lm
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* return codes (oracle-private numbering) */
#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOTSORTED -2
#define ORC_ECAPACITY -3
#define ORC_ENOMEM -4
#define ORC_EOVERFLOW -5
#define ORC_ENONFINITE -6
#define ORC_ETIMEOUT -7

#define INVALID_BAND 0xFF

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------- */
/* Isoband classification.  Sec. 3.1 "Level Sets, Isobands, and Connected    */
/* Components": B_{a,b} = { v : a < f(v) <= b }.                             */
/* Reading: isovalues t_1 < ... < t_K split the line into K+1 bands; band    */
/* index = #{ i : t_i < f(v) }, so band 0 = (-inf, t_1] and band K = (t_K,   */
/* inf).  NaN voxels are not graph nodes (the `node` bit of Sec. 3.2) and get */
/* band 0xFF.                                                                 */
/* ------------------------------------------------------------------------- */
int orc_classify(const float *field, int64_t n, const float *iso, int32_t n_iso, uint8_t *band)
{
    if (n < 0 || n_iso < 0 || n_iso > 254) return ORC_EINVAL;
    for (int32_t i = 0; i < n_iso; ++i)
        if (isnan(iso[i])) return ORC_ENOTSORTED;
    for (int32_t i = 1; i < n_iso; ++i)
        if (!(iso[i - 1] < iso[i])) return ORC_ENOTSORTED;
    for (int64_t v = 0; v < n; ++v) {
        float f = field[v];
        if (isnan(f)) { band[v] = INVALID_BAND; continue; }
        int b = 0;
        for (int32_t i = 0; i < n_iso; ++i)
            if (iso[i] < f) ++b;
        band[v] = (uint8_t)b;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Connected components of each isoband.  Sec. 3.1: an isoband is the union   */
/* of components C^k such that no voxel of one is adjacent to a voxel of      */
/* another.  Reading: 6-adjacency.  The paper fixes no labelling, so ids are  */
/* made canonical: ordered by (band, smallest linear index in the component). */
/* Algorithm: breadth-first flood fill started from voxels in linear order.   */
/* ------------------------------------------------------------------------- */
int orc_label_components(const uint8_t *band, int32_t nx, int32_t ny, int32_t nz,
                         int32_t *comp, uint8_t *comp_band, int64_t *comp_size,
                         int32_t *comp_first, int32_t max_comp, int32_t *n_comp_out)
{
    if (nx <= 0 || ny <= 0 || nz <= 0) return ORC_EINVAL;
    int64_t n = (int64_t)nx * ny * nz;
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *raw_first = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!queue || !raw_first) { free(queue); free(raw_first); return ORC_ENOMEM; }
    for (int64_t v = 0; v < n; ++v) comp[v] = -1;
    int32_t n_raw = 0;
    /* pass 1: raw ids in order of discovery = order of smallest linear index */
    for (int64_t s = 0; s < n; ++s) {
        if (band[s] == INVALID_BAND || comp[s] >= 0) continue;
        int32_t id = n_raw++;
        raw_first[id] = (int32_t)s;
        int64_t head = 0, tail = 0;
        queue[tail++] = (int32_t)s;
        comp[s] = id;
        while (head < tail) {
            int32_t v = queue[head++];
            int32_t x = v % nx, y = (v / nx) % ny, z = v / (nx * ny);
            int32_t nb[6]; int k = 0;
            if (x > 0) nb[k++] = v - 1;
            if (x < nx - 1) nb[k++] = v + 1;
            if (y > 0) nb[k++] = v - nx;
            if (y < ny - 1) nb[k++] = v + nx;
            if (z > 0) nb[k++] = v - nx * ny;
            if (z < nz - 1) nb[k++] = v + nx * ny;
            for (int i = 0; i < k; ++i) {
                int32_t u = nb[i];
                if (comp[u] < 0 && band[u] == band[s]) { comp[u] = id; queue[tail++] = u; }
            }
        }
    }
    /* pass 2: stable re-numbering by band */
    int64_t band_count[256];
    memset(band_count, 0, sizeof(band_count));
    for (int32_t r = 0; r < n_raw; ++r) band_count[band[raw_first[r]]]++;
    int64_t band_off[256];
    int64_t acc = 0;
    for (int b = 0; b < 256; ++b) { band_off[b] = acc; acc += band_count[b]; }
    int32_t *remap = queue; /* reuse */
    for (int32_t r = 0; r < n_raw; ++r) remap[r] = (int32_t)(band_off[band[raw_first[r]]]++);
    *n_comp_out = n_raw;
    int over = n_raw > max_comp;
    for (int64_t v = 0; v < n; ++v)
        if (comp[v] >= 0) comp[v] = remap[comp[v]];
    if (!over) {
        for (int32_t r = 0; r < n_raw; ++r) {
            int32_t c = remap[r];
            comp_band[c] = band[raw_first[r]];
            comp_first[c] = raw_first[r];
            comp_size[c] = 0;
        }
        for (int64_t v = 0; v < n; ++v)
            if (comp[v] >= 0) comp_size[comp[v]]++;
    }
    free(queue); free(raw_first);
    return over ? ORC_ECAPACITY : ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Saliency weights m_v.  Sec. 3.1 "Centroids" (m_v, the weighting function)  */
/* and Sec. 3.3 "Role and Choice of Parameters" (the second field, attraction */
/* gamma).  The paper gives no formula; reading: m_v = |grad f|^gamma with    */
/* central differences (one-sided half differences at the faces), evaluated   */
/* in float in the order written below, then quantised to 16-bit integers     */
/* q = max(1, rint(g^gamma * 65535/gmax)).  gamma must be an integer 0..4.    */
/* ------------------------------------------------------------------------- */
int orc_saliency(const float *f, int32_t nx, int32_t ny, int32_t nz, int32_t gamma, uint16_t *q)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || gamma < 0 || gamma > 4) return ORC_EINVAL;
    int64_t n = (int64_t)nx * ny * nz;
    if (gamma == 0) { for (int64_t v = 0; v < n; ++v) q[v] = 1; return ORC_OK; }
    float *gp = (float *)malloc(sizeof(float) * (size_t)n);
    if (!gp) return ORC_ENOMEM;
    float gmax = 0.0f;
    for (int32_t z = 0; z < nz; ++z)
        for (int32_t y = 0; y < ny; ++y)
            for (int32_t x = 0; x < nx; ++x) {
                int64_t v = x + (int64_t)nx * (y + (int64_t)ny * z);
                int32_t xm = x > 0 ? x - 1 : 0, xp = x < nx - 1 ? x + 1 : nx - 1;
                int32_t ym = y > 0 ? y - 1 : 0, yp = y < ny - 1 ? y + 1 : ny - 1;
                int32_t zm = z > 0 ? z - 1 : 0, zp = z < nz - 1 ? z + 1 : nz - 1;
                float fxp = f[xp + (int64_t)nx * (y + (int64_t)ny * z)];
                float fxm = f[xm + (int64_t)nx * (y + (int64_t)ny * z)];
                float fyp = f[x + (int64_t)nx * (yp + (int64_t)ny * z)];
                float fym = f[x + (int64_t)nx * (ym + (int64_t)ny * z)];
                float fzp = f[x + (int64_t)nx * (y + (int64_t)ny * zp)];
                float fzm = f[x + (int64_t)nx * (y + (int64_t)ny * zm)];
                float dx = 0.5f * (fxp - fxm);
                float dy = 0.5f * (fyp - fym);
                float dz = 0.5f * (fzp - fzm);
                float s = dx * dx;
                s = s + dy * dy;
                s = s + dz * dz;
                float g = sqrtf(s);
                float p = g;
                for (int32_t k = 1; k < gamma; ++k) p = p * g;
                gp[v] = p;
                if (isfinite(p) && p > gmax) gmax = p;
            }
    float scale = gmax > 0.0f ? 65535.0f / gmax : 0.0f;
    for (int64_t v = 0; v < n; ++v) {
        float p = gp[v];
        float t = p * scale;
        uint16_t w = 1;
        if (isfinite(p) && t >= 0.5f) {
            float r = rintf(t); /* round half to even */
            if (r > 65535.0f) r = 65535.0f;
            w = (uint16_t)r;
            if (w < 1) w = 1;
        }
        q[v] = w;
    }
    free(gp);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number       */
/* generators", OOPSLA 2014): one step of the generator whose state advances  */
/* by the golden gamma 0x9e3779b97f4a7c15, i.e. the output for state x.       */
/* ------------------------------------------------------------------------- */
uint64_t orc_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

typedef struct { int32_t comp; int32_t block; int64_t k; uint64_t m; int64_t nb; } orc_stratum;

static int stratum_cmp(const void *a, const void *b)
{
    const orc_stratum *p = (const orc_stratum *)a, *r = (const orc_stratum *)b;
    if (p->comp != r->comp) return p->comp < r->comp ? -1 : 1;
    if (p->block != r->block) return p->block < r->block ? -1 : 1;
    return 0;
}

/* Apportion n sites over the strata st[0..ns) of one component.  Sec. 3.2     */
/* "Stratified Random Initial Site Distribution": first floor(n m_b / m_C) per */
/* stratum, then the remainder to the most under-represented strata.  The      */
/* printed ur(b) is garbled (it equals 1 for every stratum after the first    */
/* pass); reading: largest remainder (Hamilton) -- the remaining sites go one */
/* each to the strata with the largest (n m_b) mod m_C, ties to the lower     */
/* stratum position.  A stratum never receives more sites than voxels: if a   */
/* stratum exceeds its voxel count it is capped and the surplus is             */
/* re-apportioned by the same rule over the strata not yet capped.             */
static void apportion(orc_stratum *st, int64_t ns, int64_t n)
{
    uint8_t *capped = (uint8_t *)calloc((size_t)ns, 1);
    u128 *rem = (u128 *)malloc(sizeof(u128) * (size_t)ns);
    uint8_t *chosen = (uint8_t *)calloc((size_t)ns, 1);
    for (int64_t i = 0; i < ns; ++i) st[i].nb = 0;
    for (;;) {
        int64_t assigned = 0;
        for (int64_t i = 0; i < ns; ++i) assigned += st[i].nb;
        int64_t remaining = n - assigned;
        if (remaining <= 0) break;
        u128 mA = 0;
        for (int64_t i = 0; i < ns; ++i) if (!capped[i]) mA += st[i].m;
        if (mA == 0) break; /* cannot happen: q >= 1 */
        int64_t given = 0;
        for (int64_t i = 0; i < ns; ++i) {
            chosen[i] = 0;
            if (capped[i]) continue;
            u128 prod = (u128)(uint64_t)remaining * st[i].m;
            int64_t fl = (int64_t)(prod / mA);
            rem[i] = prod % mA;
            st[i].nb += fl;
            given += fl;
        }
        int64_t left = remaining - given;
        /* hand out `left` single sites by (remainder desc, position asc) */
        for (int64_t t = 0; t < left; ++t) {
            int64_t best = -1;
            for (int64_t i = 0; i < ns; ++i) {
                if (capped[i] || chosen[i]) continue;
                if (best < 0 || rem[i] > rem[best]) best = i;
            }
            if (best < 0) break;
            chosen[best] = 1;
            st[best].nb += 1;
        }
        int any = 0;
        for (int64_t i = 0; i < ns; ++i)
            if (!capped[i] && st[i].nb > st[i].k) { st[i].nb = st[i].k; capped[i] = 1; any = 1; }
        if (!any) break;
    }
    free(capped); free(rem); free(chosen);
}

/* ------------------------------------------------------------------------- */
/* Initial sites.  Sec. 3.2 "Stratified Random Initial Site Distribution",    */
/* Eq. (nc), Algorithm 1 (StratifiedRandomSiteDistribution).                  */
/* Eq. (nc) as printed reduces to ceil(alpha); reading (alpha = ratio of      */
/* sites to voxels, Sec. 3.3): n_c = max(ceil(|V| m(C) / (P m(V))), 1),        */
/* capped at |C|, with P = 1/alpha voxels per site, |V| the valid voxels and  */
/* m(.) the sum of the weights q.  Strata = component x cubic block of side   */
/* `sb` aligned to the origin; block index = linear index of the block.       */
/* Placement (the paper only says "random"): the stratum's k voxels in linear */
/* order are split into n_b contiguous rank ranges [floor(jk/n), floor((j+1)k */
/* /n)); site j takes rank lo_j + h_j mod (hi_j - lo_j) with                  */
/* h_j = splitmix64((seed ^ splitmix64(block)) + j).                           */
/* Site ids are ordered by (component, block, j).                             */
/* ------------------------------------------------------------------------- */
int orc_seed(const int32_t *comp, const uint16_t *q, int32_t nx, int32_t ny, int32_t nz,
             int32_t n_comp, int64_t voxels_per_site, int32_t sb, uint64_t seed,
             int32_t *site_pos, int32_t *site_comp, int32_t *comp_site_off,
             int32_t max_sites, int32_t *n_sites_out, int64_t *n_site_comp /* nullable, n_c per comp */)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || voxels_per_site < 1 || sb < 1 || n_comp < 0) return ORC_EINVAL;
    int64_t n = (int64_t)nx * ny * nz;
    int64_t *csize = (int64_t *)calloc((size_t)(n_comp + 1), sizeof(int64_t));
    uint64_t *cmass = (uint64_t *)calloc((size_t)(n_comp + 1), sizeof(uint64_t));
    int64_t *nc = (int64_t *)calloc((size_t)(n_comp + 1), sizeof(int64_t));
    if (!csize || !cmass || !nc) { free(csize); free(cmass); free(nc); return ORC_ENOMEM; }
    int64_t nV = 0; uint64_t mV = 0;
    for (int64_t v = 0; v < n; ++v) {
        int32_t c = comp[v];
        if (c < 0) continue;
        if (c >= n_comp) { free(csize); free(cmass); free(nc); return ORC_EINVAL; }
        uint64_t w = q ? q[v] : 1;
        nV++; mV += w; csize[c]++; cmass[c] += w;
    }
    for (int32_t c = 0; c < n_comp; ++c) {
        u128 num = (u128)(uint64_t)nV * cmass[c];
        u128 den = (u128)(uint64_t)voxels_per_site * mV;
        int64_t k = den ? (int64_t)((num + den - 1) / den) : 1;
        if (k < 1) k = 1;
        if (k > csize[c]) k = csize[c];
        nc[c] = k;
        if (n_site_comp) n_site_comp[c] = k;
    }
    /* enumerate strata block by block */
    int32_t nbx = (nx + sb - 1) / sb, nby = (ny + sb - 1) / sb, nbz = (nz + sb - 1) / sb;
    int64_t cap = 1024, ns = 0;
    orc_stratum *st = (orc_stratum *)malloc(sizeof(orc_stratum) * (size_t)cap);
    for (int32_t bz = 0; bz < nbz; ++bz)
        for (int32_t by = 0; by < nby; ++by)
            for (int32_t bx = 0; bx < nbx; ++bx) {
                int32_t b = bx + nbx * (by + nby * bz);
                int64_t first = ns;
                for (int32_t z = bz * sb; z < nz && z < (bz + 1) * sb; ++z)
                    for (int32_t y = by * sb; y < ny && y < (by + 1) * sb; ++y)
                        for (int32_t x = bx * sb; x < nx && x < (bx + 1) * sb; ++x) {
                            int64_t v = x + (int64_t)nx * (y + (int64_t)ny * z);
                            int32_t c = comp[v];
                            if (c < 0) continue;
                            int64_t i;
                            for (i = first; i < ns; ++i) if (st[i].comp == c) break;
                            if (i == ns) {
                                if (ns == cap) { cap *= 2; st = (orc_stratum *)realloc(st, sizeof(orc_stratum) * (size_t)cap); }
                                st[ns].comp = c; st[ns].block = b; st[ns].k = 0; st[ns].m = 0; st[ns].nb = 0;
                                ++ns;
                            }
                            st[i].k++;
                            st[i].m += q ? q[v] : 1;
                        }
            }
    qsort(st, (size_t)ns, sizeof(orc_stratum), stratum_cmp);
    /* apportion per component */
    int64_t i0 = 0;
    while (i0 < ns) {
        int64_t i1 = i0;
        while (i1 < ns && st[i1].comp == st[i0].comp) ++i1;
        apportion(st + i0, i1 - i0, nc[st[i0].comp]);
        i0 = i1;
    }
    int64_t total = 0;
    for (int64_t i = 0; i < ns; ++i) total += st[i].nb;
    *n_sites_out = (int32_t)(total > 0x7fffffff ? 0x7fffffff : total);
    if (total > max_sites) { free(st); free(csize); free(cmass); free(nc); return ORC_ECAPACITY; }
    /* comp_site_off */
    {
        int64_t acc = 0;
        int64_t j = 0;
        for (int32_t c = 0; c < n_comp; ++c) {
            comp_site_off[c] = (int32_t)acc;
            while (j < ns && st[j].comp == c) { acc += st[j].nb; ++j; }
        }
        comp_site_off[n_comp] = (int32_t)acc;
    }
    /* placement */
    int32_t *vox = (int32_t *)malloc(sizeof(int32_t) * (size_t)sb * sb * sb);
    int64_t sid = 0;
    for (int64_t i = 0; i < ns; ++i) {
        int32_t b = st[i].block, c = st[i].comp;
        int32_t bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
        int64_t k = 0;
        for (int32_t z = bz * sb; z < nz && z < (bz + 1) * sb; ++z)
            for (int32_t y = by * sb; y < ny && y < (by + 1) * sb; ++y)
                for (int32_t x = bx * sb; x < nx && x < (bx + 1) * sb; ++x) {
                    int64_t v = x + (int64_t)nx * (y + (int64_t)ny * z);
                    if (comp[v] == c) vox[k++] = (int32_t)v;
                }
        uint64_t hb = seed ^ orc_splitmix64((uint64_t)b);
        int64_t nb = st[i].nb;
        for (int64_t j = 0; j < nb; ++j) {
            uint64_t lo = (uint64_t)j * (uint64_t)k / (uint64_t)nb;
            uint64_t hi = (uint64_t)(j + 1) * (uint64_t)k / (uint64_t)nb;
            uint64_t h = orc_splitmix64(hb + (uint64_t)j);
            uint64_t r = lo + h % (hi - lo);
            site_pos[sid] = vox[r];
            site_comp[sid] = c;
            ++sid;
        }
    }
    free(vox); free(st); free(csize); free(cmass); free(nc);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Restricted graph.  Eq. 1 and Sec. 3.2 "Discrete Restricted Geodesic        */
/* Voronoi Tessellation": voxels are nodes and no edge crosses a boundary.    */
/* Reading: an edge joins 26-neighbours u, v when every voxel of the          */
/* axis-aligned box spanned by u and v has the band of v (so no edge cuts a   */
/* level set, and the edge graph's components are the 6-connected ones).     */
/* Edge lengths are the Euclidean lengths in 16.16 fixed point, rounded up.   */
/* ------------------------------------------------------------------------- */
#define W_FACE 65536u
#define W_EDGE 92682u
#define W_CORNER 113512u

static uint32_t edge_weight(int dx, int dy, int dz)
{
    int k = (dx != 0) + (dy != 0) + (dz != 0);
    return k == 1 ? W_FACE : (k == 2 ? W_EDGE : W_CORNER);
}

/* does the edge v -> v+(dx,dy,dz) exist?  (x,y,z) = coords of v */
static int has_edge(const uint8_t *band, int32_t nx, int32_t ny, int32_t nz,
                    int32_t x, int32_t y, int32_t z, int dx, int dy, int dz)
{
    int32_t ux = x + dx, uy = y + dy, uz = z + dz;
    if (ux < 0 || ux >= nx || uy < 0 || uy >= ny || uz < 0 || uz >= nz) return 0;
    uint8_t b = band[x + (int64_t)nx * (y + (int64_t)ny * z)];
    if (b == INVALID_BAND) return 0;
    for (int az = 0; az <= (dz != 0); ++az)
        for (int ay = 0; ay <= (dy != 0); ++ay)
            for (int ax = 0; ax <= (dx != 0); ++ax) {
                int32_t px = x + ax * dx, py = y + ay * dy, pz = z + az * dz;
                if (band[px + (int64_t)nx * (py + (int64_t)ny * pz)] != b) return 0;
            }
    return 1;
}

/* binary heap of (dist, site, voxel), lexicographic */
typedef struct { uint64_t d; int32_t s; int32_t v; } hent;
typedef struct { hent *a; int64_t n, cap; } heap;

static int hless(const hent *p, const hent *q)
{
    if (p->d != q->d) return p->d < q->d;
    if (p->s != q->s) return p->s < q->s;
    return p->v < q->v;
}

static int hpush(heap *h, hent e)
{
    if (h->n == h->cap) {
        int64_t nc = h->cap ? h->cap * 2 : 1024;
        hent *na = (hent *)realloc(h->a, sizeof(hent) * (size_t)nc);
        if (!na) return ORC_ENOMEM;
        h->a = na; h->cap = nc;
    }
    int64_t i = h->n++;
    h->a[i] = e;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!hless(&h->a[i], &h->a[p])) break;
        hent t = h->a[i]; h->a[i] = h->a[p]; h->a[p] = t;
        i = p;
    }
    return ORC_OK;
}

static hent hpop(heap *h)
{
    hent top = h->a[0];
    h->a[0] = h->a[--h->n];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < h->n && hless(&h->a[l], &h->a[m])) m = l;
        if (r < h->n && hless(&h->a[r], &h->a[m])) m = r;
        if (m == i) break;
        hent t = h->a[i]; h->a[i] = h->a[m]; h->a[m] = t;
        i = m;
    }
    return top;
}

/* ------------------------------------------------------------------------- */
/* Restricted geodesic Voronoi assignment, Eq. 1: each voxel v of component C */
/* belongs to the site of S_C with the smallest graph-geodesic distance.      */
/* Ties (equal distance) go to the lowest site id, so the label is the        */
/* lexicographic minimum of (gd, site).  Multi-source Dijkstra on             */
/* (distance, site).  Unreached / invalid voxels: cell -1, dist 0xFFFFFFFF.   */
/* Distances are 16.16 fixed point and must stay below 2^32.                  */
/* ------------------------------------------------------------------------- */
int orc_assign(const uint8_t *band, int32_t nx, int32_t ny, int32_t nz,
               const int32_t *site_pos, int32_t n_sites, int32_t *cell, uint32_t *dist)
{
    int64_t n = (int64_t)nx * ny * nz;
    uint64_t *kd = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    if (!kd) return ORC_ENOMEM;
    for (int64_t v = 0; v < n; ++v) { kd[v] = UINT64_MAX; cell[v] = -1; }
    heap h = {0, 0, 0};
    int rc = ORC_OK;
    for (int32_t s = 0; s < n_sites; ++s) {
        int32_t p = site_pos[s];
        if (p < 0 || p >= n || band[p] == INVALID_BAND) { rc = ORC_EINVAL; goto done; }
        if (kd[p] == 0 && cell[p] <= s) continue; /* lower id already there */
        kd[p] = 0; cell[p] = s;
        hent e = {0, s, p};
        if (hpush(&h, e)) { rc = ORC_ENOMEM; goto done; }
    }
    while (h.n > 0) {
        hent e = hpop(&h);
        if (e.d != kd[e.v] || e.s != cell[e.v]) continue; /* stale */
        int32_t v = e.v, x = v % nx, y = (v / nx) % ny, z = v / (nx * ny);
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!dx && !dy && !dz) continue;
                    if (!has_edge(band, nx, ny, nz, x, y, z, dx, dy, dz)) continue;
                    int64_t u = (x + dx) + (int64_t)nx * ((y + dy) + (int64_t)ny * (z + dz));
                    uint64_t nd = e.d + edge_weight(dx, dy, dz);
                    if (nd > 0xFFFFFFFFull) { rc = ORC_EOVERFLOW; goto done; }
                    if (nd < kd[u] || (nd == kd[u] && e.s < cell[u])) {
                        kd[u] = nd; cell[u] = e.s;
                        hent f = {nd, e.s, (int32_t)u};
                        if (hpush(&h, f)) { rc = ORC_ENOMEM; goto done; }
                    }
                }
    }
    for (int64_t v = 0; v < n; ++v) dist[v] = kd[v] == UINT64_MAX ? 0xFFFFFFFFu : (uint32_t)kd[v];
done:
    free(h.a); free(kd);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Discrete line of sight.  Eq. 2 (los(v, s)) and Sec. 3.2 "Geodesically      */
/* Weighted Voronoi Site Update" (ray cast toward the centroid).  Reading:    */
/* the 6-connected voxel traversal of Amanatides & Woo (1987) of the segment  */
/* joining the centres of voxels a and b, walked from a toward b.  The k-th   */
/* crossing on axis i happens at t = (2k-1) / (2|d_i|); the next axis to step */
/* is the one with the earliest crossing, compared exactly by cross-          */
/* multiplication; simultaneous crossings step x, then y, then z.             */
/* walk_traversal returns the number of steps taken before the first voxel   */
/* whose band differs from `b` (all steps if none), and the reached voxel.    */
/* ------------------------------------------------------------------------- */
static int64_t walk_traversal(const uint8_t *band, int32_t nx, int32_t ny,
                              int32_t ax0, int32_t ay0, int32_t az0,
                              int32_t bx, int32_t by, int32_t bz, uint8_t b,
                              int32_t *ex, int32_t *ey, int32_t *ez)
{
    int64_t d[3] = {bx - ax0, by - ay0, bz - az0};
    int64_t A[3], S[3], k[3] = {0, 0, 0};
    for (int i = 0; i < 3; ++i) { A[i] = d[i] < 0 ? -d[i] : d[i]; S[i] = d[i] < 0 ? -1 : 1; }
    int32_t p[3] = {ax0, ay0, az0};
    int64_t steps = 0;
    for (;;) {
        int best = -1;
        for (int i = 0; i < 3; ++i) {
            if (k[i] >= A[i]) continue;
            if (best < 0) { best = i; continue; }
            /* t_i = (2k_i+1)/(2A_i) < t_best = (2k_b+1)/(2A_b) ? (strictly earlier wins; ties keep lower axis) */
            if ((2 * k[i] + 1) * A[best] < (2 * k[best] + 1) * A[i]) best = i;
        }
        if (best < 0) break;
        int32_t np[3] = {p[0], p[1], p[2]};
        np[best] += (int32_t)S[best];
        if (band[np[0] + (int64_t)nx * (np[1] + (int64_t)ny * np[2])] != b) break;
        p[0] = np[0]; p[1] = np[1]; p[2] = np[2];
        k[best]++;
        steps++;
    }
    *ex = p[0]; *ey = p[1]; *ez = p[2];
    return steps;
}

int orc_los(const uint8_t *band, int32_t nx, int32_t ny, int32_t nz,
            int32_t v, int32_t s)
{
    (void)nz;
    int32_t vx = v % nx, vy = (v / nx) % ny, vz = v / (nx * ny);
    int32_t sx = s % nx, sy = (s / nx) % ny, sz = s / (nx * ny);
    int32_t ex, ey, ez;
    int64_t need = (int64_t)abs(sx - vx) + abs(sy - vy) + abs(sz - vz);
    int64_t got = walk_traversal(band, nx, ny, vx, vy, vz, sx, sy, sz, band[v], &ex, &ey, &ez);
    return got == need;
}

/* ------------------------------------------------------------------------- */
/* Geodesically weighted site update, Eq. 2 and Sec. 3.2 "Geodesically        */
/* Weighted Voronoi Site Update".                                             */
/*  parent(v) (the src map of Sec. 3.2): reading -- the first 26-neighbour u  */
/*   in offset order (dz,dy,dx) = (-1,-1,-1) ... (1,1,1) with an edge to v,    */
/*   the same site, and D(u) + w(u,v) = D(v); a site voxel is its own parent. */
/*  phi(v) = v if los(v, site(v)) else phi(parent(v))            (Eq. 2)     */
/*  x'_c = sum_v m_v x_phi(v) / sum_v m_v   (integer sums, exact)  (Eq. 2)     */
/*  target = per-axis floor((2 S + M) / (2 M))  (round half up)               */
/*  move: walk the traversal from the site toward the target and stop at the */
/*   last voxel of the site's band (move only as far as possible before      */
/*   crossing the boundary).  Cells with M = 0 do not move.                   */
/* stats[0] = sites moved, stats[1] = sum of squared displacements,          */
/* stats[2] = sum of ceil(2^16 |displacement|).                                */
/* parent_out / los_out / phi_out / sums_out are optional (NULL) diagnostics. */
/* ------------------------------------------------------------------------- */
/* site_sel (optional, one byte per site): when given, only the voxels of the  */
/* selected cells are visited and only the selected sites move.  A cell's     */
/* parents, line-of-sight tests and phi never leave the cell, so the selected */
/* sites get exactly the positions of the full update; this lets one full-    */
/* size replay check a sample of cells.                                       */
/* Per-axis target of Eq. 2: the centroid S / M rounded half up, floor((2S + M) / (2M)),   */
/* for M > 0 and S >= 0 (coordinates are non-negative, so C division is the floor).        */
static int32_t centroid_round(int64_t S, int64_t M)
{
    return (int32_t)((2 * S + M) / (2 * M));
}

/* ceil(2^16 sqrt(D)) of an integer D (declared here, defined with the site graph).        */
uint32_t orc_site_weight(int32_t dx, int32_t dy, int32_t dz);

static int update_impl(const uint8_t *band, const uint16_t *q, int32_t nx, int32_t ny, int32_t nz,
                       const int32_t *cell, const uint32_t *dist, const int32_t *site_pos, int32_t n_sites,
                       const uint8_t *site_sel, const int32_t *src_in, int32_t *new_pos, int64_t *stats,
                       int32_t *parent_out, uint8_t *los_out, int32_t *phi_out, int64_t *sums_out)
{
    int64_t n = (int64_t)nx * ny * nz;
    int32_t *parent = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int8_t *los = (int8_t *)malloc((size_t)n);
    int32_t *phi = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *S = (int64_t *)calloc((size_t)n_sites * 4 + 1, sizeof(int64_t));
    if (!parent || !los || !phi || !S) { free(parent); free(los); free(phi); free(S); return ORC_ENOMEM; }
    int rc = ORC_OK;
    for (int64_t v = 0; v < n; ++v) {
        parent[v] = -1; los[v] = 0; phi[v] = -1;
        int32_t s = cell[v];
        if (s < 0) continue;
        if (site_sel && !site_sel[s]) continue;
        int32_t x = (int32_t)(v % nx), y = (int32_t)((v / nx) % ny), z = (int32_t)(v / ((int64_t)nx * ny));
        if (dist[v] == 0) { parent[v] = (int32_t)v; }
        else if (src_in) {
            /* any-angle paths: the path's next node is the voxel's source */
            parent[v] = src_in[v];
            if (parent[v] < 0 || parent[v] >= n || cell[parent[v]] != s) { rc = ORC_EINVAL; goto done; }
        } else {
            for (int dz = -1; dz <= 1 && parent[v] < 0; ++dz)
                for (int dy = -1; dy <= 1 && parent[v] < 0; ++dy)
                    for (int dx = -1; dx <= 1 && parent[v] < 0; ++dx) {
                        if (!dx && !dy && !dz) continue;
                        if (!has_edge(band, nx, ny, nz, x, y, z, dx, dy, dz)) continue;
                        int64_t u = (x + dx) + (int64_t)nx * ((y + dy) + (int64_t)ny * (z + dz));
                        if (cell[u] != s) continue;
                        if ((uint64_t)dist[u] + edge_weight(dx, dy, dz) == (uint64_t)dist[v]) parent[v] = (int32_t)u;
                    }
            if (parent[v] < 0) { rc = ORC_EINVAL; goto done; } /* not a shortest-path labelling */
        }
        los[v] = (int8_t)orc_los(band, nx, ny, nz, (int32_t)v, site_pos[s]);
    }
    for (int64_t v = 0; v < n; ++v) {
        if (cell[v] < 0) continue;
        if (site_sel && !site_sel[cell[v]]) continue;
        int64_t u = v;
        int64_t guard = 0;
        while (!los[u]) {
            u = parent[u];
            if (++guard > n) { rc = ORC_EINVAL; goto done; }
        }
        phi[v] = (int32_t)u;
        int64_t w = q ? q[v] : 1;
        int32_t s = cell[v];
        int64_t px = u % nx, py = (u / nx) % ny, pz = u / ((int64_t)nx * ny);
        S[4 * s + 0] += w * px;
        S[4 * s + 1] += w * py;
        S[4 * s + 2] += w * pz;
        S[4 * s + 3] += w;
    }
    int64_t moved = 0, sumsq = 0, sumlen = 0;
    for (int32_t s = 0; s < n_sites; ++s) {
        int32_t p = site_pos[s];
        int32_t x = p % nx, y = (p / nx) % ny, z = p / (nx * ny);
        int64_t M = S[4 * s + 3];
        int32_t nxp = x, nyp = y, nzp = z;
        if (M > 0) {
            int32_t tx = centroid_round(S[4 * s + 0], M);
            int32_t ty = centroid_round(S[4 * s + 1], M);
            int32_t tz = centroid_round(S[4 * s + 2], M);
            walk_traversal(band, nx, ny, x, y, z, tx, ty, tz, band[p], &nxp, &nyp, &nzp);
        }
        new_pos[s] = nxp + nx * (nyp + ny * nzp);
        if (new_pos[s] != p) {
            moved++;
            int64_t ddx = nxp - x, ddy = nyp - y, ddz = nzp - z;
            sumsq += ddx * ddx + ddy * ddy + ddz * ddz;
            /* d_s = |new - old| in 16.16 fixed point, rounded up (Fig. "convergence": mean d_s) */
            sumlen += orc_site_weight((int32_t)ddx, (int32_t)ddy, (int32_t)ddz);
        }
    }
    stats[0] = moved; stats[1] = sumsq; stats[2] = sumlen;
    if (parent_out) memcpy(parent_out, parent, sizeof(int32_t) * (size_t)n);
    if (los_out) for (int64_t v = 0; v < n; ++v) los_out[v] = (uint8_t)los[v];
    if (phi_out) memcpy(phi_out, phi, sizeof(int32_t) * (size_t)n);
    if (sums_out) memcpy(sums_out, S, sizeof(int64_t) * (size_t)n_sites * 4);
done:
    free(parent); free(los); free(phi); free(S);
    return rc;
}

int orc_update(const uint8_t *band, const uint16_t *q, int32_t nx, int32_t ny, int32_t nz,
               const int32_t *cell, const uint32_t *dist, const int32_t *site_pos, int32_t n_sites,
               int32_t *new_pos, int64_t *stats,
               int32_t *parent_out, uint8_t *los_out, int32_t *phi_out, int64_t *sums_out)
{
    return update_impl(band, q, nx, ny, nz, cell, dist, site_pos, n_sites, NULL, NULL, new_pos, stats,
                       parent_out, los_out, phi_out, sums_out);
}

/* The same update with the any-angle path representation: a voxel's next path */
/* node is its source src[v] (from orc_anyangle_assign) instead of the chamfer */
/* parent, so phi(v) = v if los(v, site(v)) else phi(src(v)).                  */
int orc_update_src(const uint8_t *band, const uint16_t *q, int32_t nx, int32_t ny, int32_t nz,
                   const int32_t *cell, const uint32_t *dist, const int32_t *src, const int32_t *site_pos,
                   int32_t n_sites, int32_t *new_pos, int64_t *stats,
                   int32_t *parent_out, uint8_t *los_out, int32_t *phi_out, int64_t *sums_out)
{
    if (!src) return ORC_EINVAL;
    return update_impl(band, q, nx, ny, nz, cell, dist, site_pos, n_sites, NULL, src, new_pos, stats,
                       parent_out, los_out, phi_out, sums_out);
}

/* Update of the selected sites only (new_pos and sums_out hold all sites;   */
/* unselected ones keep their position and zero sums).                        */
int orc_update_selected(const uint8_t *band, const uint16_t *q, int32_t nx, int32_t ny, int32_t nz,
                        const int32_t *cell, const uint32_t *dist, const int32_t *site_pos, int32_t n_sites,
                        const uint8_t *site_sel, int32_t *new_pos, int64_t *sums_out)
{
    int64_t stats[3];
    return update_impl(band, q, nx, ny, nz, cell, dist, site_pos, n_sites, site_sel, NULL, new_pos, stats,
                       NULL, NULL, NULL, sums_out);
}

/* ------------------------------------------------------------------------- */
/* CVT energy of an assignment, the quantity Lloyd's method lowers:          */
/* E = sum over assigned voxels of m_v D(v)^2 (Sec. 3.1 "Centroids or Centers */
/* of Mass": m_v; Eq. 1: D = the tessellation's distance to the voxel's      */
/* site, 16.16 fixed point), exact in 128 bits: out[0] = low 64 bits,        */
/* out[1] = high 64 bits.  Recorded per iteration, never used in control.    */
/* ------------------------------------------------------------------------- */
void orc_energy(const uint16_t *q, const int32_t *cell, const uint32_t *dist, int64_t n, uint64_t *out)
{
    u128 e = 0;
    for (int64_t v = 0; v < n; ++v) {
        if (cell[v] < 0) continue;
        u128 d = dist[v];
        e += (u128)(q ? q[v] : 1u) * d * d;
    }
    out[0] = (uint64_t)e;
    out[1] = (uint64_t)(e >> 64);
}

/* One Lloyd iteration's trace record: sites moved, sum of |d|^2, sum of      */
/* ceil(2^16 |d|) (mean d_s = that / 2^16 / n_sites), and the energy of the  */
/* iteration's assignment (low, high 64 bits).                                */
#define ORC_TRACE 5

static void trace_record(int64_t *trace, int32_t it, const int64_t *st, const uint16_t *q, const int32_t *cell,
                         const uint32_t *dist, int64_t n)
{
    uint64_t e[2];
    orc_energy(q, cell, dist, n, e);
    int64_t *t = trace + (int64_t)ORC_TRACE * it;
    t[0] = st[0]; t[1] = st[1]; t[2] = st[2];
    t[3] = (int64_t)e[0]; t[4] = (int64_t)e[1];
}

/* ------------------------------------------------------------------------- */
/* Textbook Lloyd iteration on the integer lattice of a box, Euclidean       */
/* metric (the CVT setting of Sec. 2 without restriction), used to pin the   */
/* centroid rounding of Eq. 2 by a theorem: every voxel goes to its nearest  */
/* site (squared distance, ties to the lowest id), then every site with a    */
/* non-empty cell moves to its cell's centroid rounded half up per axis --   */
/* the same centroid_round as the update.  That rounding is a nearest lattice */
/* point to the centroid, and sum |v - p|^2 over a cell = sum |v - c|^2 +    */
/* n |c - p|^2, so neither step can raise E = sum |v - site(v)|^2.           */
/* energy[k], k = 0..n_iters: E of the k-th assignment; site_pos in/out.     */
/* ------------------------------------------------------------------------- */
int orc_lattice_lloyd(int32_t nx, int32_t ny, int32_t nz, int32_t *site_pos, int32_t n_sites, int32_t n_iters,
                      int64_t *energy)
{
    int64_t n = (int64_t)nx * ny * nz;
    if (n <= 0 || n_sites <= 0 || n_iters < 0) return ORC_EINVAL;
    for (int32_t s = 0; s < n_sites; ++s)
        if (site_pos[s] < 0 || site_pos[s] >= n) return ORC_EINVAL;
    int32_t *cell = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *S = (int64_t *)malloc(sizeof(int64_t) * 4 * (size_t)n_sites);
    if (!cell || !S) { free(cell); free(S); return ORC_ENOMEM; }
    for (int32_t it = 0; it <= n_iters; ++it) {
        int64_t E = 0;
        for (int64_t v = 0; v < n; ++v) {
            int64_t x = v % nx, y = (v / nx) % ny, z = v / ((int64_t)nx * ny);
            int64_t best = -1;
            int32_t bs = -1;
            for (int32_t s = 0; s < n_sites; ++s) {
                int64_t p = site_pos[s];
                int64_t dx = x - p % nx, dy = y - (p / nx) % ny, dz = z - p / ((int64_t)nx * ny);
                int64_t d2 = dx * dx + dy * dy + dz * dz;
                if (bs < 0 || d2 < best) { best = d2; bs = s; }
            }
            cell[v] = bs;
            E += best;
        }
        energy[it] = E;
        if (it == n_iters) break;
        memset(S, 0, sizeof(int64_t) * 4 * (size_t)n_sites);
        for (int64_t v = 0; v < n; ++v) {
            int32_t s = cell[v];
            S[4 * s + 0] += v % nx;
            S[4 * s + 1] += (v / nx) % ny;
            S[4 * s + 2] += v / ((int64_t)nx * ny);
            S[4 * s + 3] += 1;
        }
        for (int32_t s = 0; s < n_sites; ++s) {
            int64_t M = S[4 * s + 3];
            if (M == 0) continue;
            site_pos[s] = centroid_round(S[4 * s + 0], M) +
                          nx * (centroid_round(S[4 * s + 1], M) + ny * centroid_round(S[4 * s + 2], M));
        }
    }
    free(cell); free(S);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1 (LRCVT) after seeding: n_iters x (restricted geodesic VT,      */
/* geodesically weighted update), then a final VT.  The paper loops until    */
/* converged (mean d_s below a tolerance, Fig. "scaling"/Table 1); here the  */
/* count is given.  trace[ORC_TRACE*it ...] = the iteration's record          */
/* (trace_record: moved, sum |d|^2, sum ceil(2^16 |d|), energy low, high).    */
/* ------------------------------------------------------------------------- */
int orc_cvt_iterate(const uint8_t *band, const uint16_t *q, int32_t nx, int32_t ny, int32_t nz,
                    int32_t *site_pos, int32_t n_sites, int32_t n_iters,
                    int32_t *cell, uint32_t *dist, int64_t *trace)
{
    int32_t *np = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_sites > 0 ? n_sites : 1));
    if (!np) return ORC_ENOMEM;
    int rc = ORC_OK;
    for (int32_t it = 0; it < n_iters; ++it) {
        rc = orc_assign(band, nx, ny, nz, site_pos, n_sites, cell, dist);
        if (rc) goto done;
        int64_t st[3];
        rc = orc_update(band, q, nx, ny, nz, cell, dist, site_pos, n_sites, np, st, 0, 0, 0, 0);
        if (rc) goto done;
        memcpy(site_pos, np, sizeof(int32_t) * (size_t)n_sites);
        if (trace) trace_record(trace, it, st, q, cell, dist, (int64_t)nx * ny * nz);
    }
    rc = orc_assign(band, nx, ny, nz, site_pos, n_sites, cell, dist);
done:
    free(np);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Any-angle restricted geodesic Voronoi tessellation, Sec. 3.2 "Discrete     */
/* Restricted Geodesic Voronoi Tessellation".  Region growing: each voxel v   */
/* polls its neighbours w and weighs two paths, (v, P_w) of length            */
/* |x_v - x_w| + d[w] and the shortcut (v, P_src(w)) of length                */
/* |x_v - x_src(w)| + d[src(w)]; the shortcut only when the ray from v to     */
/* src(w) stays in the band.  Updates take effect in the next invocation      */
/* (synchronous rounds: round r+1 reads only the state of round r), and the   */
/* rounds repeat until one changes nothing.                                   */
/* Readings:                                                                  */
/*  - a length |x_a - x_b| is ceil(2^16 |x_a - x_b|) (16.16 fixed point, an   */
/*    integer), so path lengths are exact sums;                               */
/*  - v polls the 26-neighbours it has an edge with (the box they span lies   */
/*    in v's band, as for the chamfer metric); the ray is the 6-connected     */
/*    traversal walked from v (orc_los);                                      */
/*  - v also re-evaluates its own path (v, P_src(v)) with the current          */
/*    d[src(v)], so at the fixed point d[v] = |x_v - x_src(v)| + d[src(v)]    */
/*    holds everywhere and every src chain ends at the voxel's own site;     */
/*  - v's new state is the lexicographic minimum of (length, site, d[src],    */
/*    src) over these candidates: equal lengths go to the lower site id, then */
/*    to the source nearer its site (the longer straight segment), then to   */
/*    the lower voxel index.  The re-evaluated own path is never worse than   */
/*    the previous state, so states only decrease and the rounds end.         */
/* Sites start at (0, s, 0, p_s) (the lowest id on a shared voxel), every     */
/* other voxel unreached.  Unreached / invalid voxels: cell -1, dist          */
/* 0xFFFFFFFF, src -1.  *rounds = rounds run, the last (unchanged) included.  */
/* ------------------------------------------------------------------------- */
typedef struct { uint64_t d; int32_t s; uint64_t dp; int32_t p; } aa_cand;

static int aa_less(const aa_cand *a, const aa_cand *b)
{
    if (a->d != b->d) return a->d < b->d;
    if (a->s != b->s) return a->s < b->s;
    if (a->dp != b->dp) return a->dp < b->dp;
    return a->p < b->p;
}

/* ceil(2^16 |x_a - x_b|); UINT64_MAX beyond the 32-bit distance range */
static uint64_t seg_length(int32_t nx, int32_t ny, int64_t a, int64_t b)
{
    int64_t dx = a % nx - b % nx, dy = (a / nx) % ny - (b / nx) % ny, dz = a / ((int64_t)nx * ny) - b / ((int64_t)nx * ny);
    if ((uint64_t)(dx * dx + dy * dy + dz * dz) >= ((uint64_t)1 << 32)) return UINT64_MAX;
    return orc_site_weight((int32_t)dx, (int32_t)dy, (int32_t)dz);
}

int orc_anyangle_assign(const uint8_t *band, int32_t nx, int32_t ny, int32_t nz,
                        const int32_t *site_pos, int32_t n_sites, int32_t max_rounds,
                        int32_t *cell, uint32_t *dist, int32_t *src, int32_t *rounds)
{
    const uint32_t INF = 0xFFFFFFFFu;
    int64_t n = (int64_t)nx * ny * nz;
    uint32_t *D[2];
    int32_t *S[2], *Q[2];
    D[0] = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n); D[1] = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    S[0] = (int32_t *)malloc(sizeof(int32_t) * (size_t)n); S[1] = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    Q[0] = (int32_t *)malloc(sizeof(int32_t) * (size_t)n); Q[1] = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int rc = ORC_OK, cur = 0;
    int32_t r = 0;
    if (!D[0] || !D[1] || !S[0] || !S[1] || !Q[0] || !Q[1]) { rc = ORC_ENOMEM; goto done; }
    for (int64_t v = 0; v < n; ++v) { D[0][v] = INF; S[0][v] = -1; Q[0][v] = -1; }
    for (int32_t s = 0; s < n_sites; ++s) {
        int32_t p = site_pos[s];
        if (p < 0 || p >= n || band[p] == INVALID_BAND) { rc = ORC_EINVAL; goto done; }
        if (D[0][p] == 0) continue; /* a lower id holds this voxel */
        D[0][p] = 0; S[0][p] = s; Q[0][p] = p;
    }
    for (;;) {
        if (r >= max_rounds) { rc = ORC_ETIMEOUT; goto done; }
        ++r;
        const uint32_t *d0 = D[cur];
        const int32_t *s0 = S[cur], *q0 = Q[cur];
        uint32_t *d1 = D[cur ^ 1];
        int32_t *s1 = S[cur ^ 1], *q1 = Q[cur ^ 1];
        int changed = 0;
        for (int64_t v = 0; v < n; ++v) {
            aa_cand best = {UINT64_MAX, INT32_MAX, UINT64_MAX, INT32_MAX};
            if (band[v] != INVALID_BAND) {
                int32_t x = (int32_t)(v % nx), y = (int32_t)((v / nx) % ny), z = (int32_t)(v / ((int64_t)nx * ny));
                /* own path, re-evaluated */
                int32_t u = q0[v];
                if (u >= 0) {
                    uint64_t L = u == v ? 0 : seg_length(nx, ny, v, u);
                    if (L != UINT64_MAX) { aa_cand c = {d0[u] + L, s0[u], d0[u], u}; best = c; }
                }
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            if (!dx && !dy && !dz) continue;
                            if (!has_edge(band, nx, ny, nz, x, y, z, dx, dy, dz)) continue;
                            int64_t w = (x + dx) + (int64_t)nx * ((y + dy) + (int64_t)ny * (z + dz));
                            if (d0[w] == INF) continue;
                            /* (v, P_w) */
                            aa_cand c = {(uint64_t)d0[w] + edge_weight(dx, dy, dz), s0[w], d0[w], (int32_t)w};
                            if (aa_less(&c, &best)) best = c;
                            /* (v, P_src(w)): a shortcut that cannot win needs no ray cast */
                            int32_t t = q0[w];
                            if (t < 0 || t == w || t == v) continue;
                            uint64_t L = seg_length(nx, ny, v, t);
                            if (L == UINT64_MAX) continue;
                            aa_cand c2 = {(uint64_t)d0[t] + L, s0[t], d0[t], t};
                            if (aa_less(&c2, &best) && orc_los(band, nx, ny, nz, (int32_t)v, t)) best = c2;
                        }
            }
            if (best.d != UINT64_MAX && best.d > 0xFFFFFFFEull) { rc = ORC_EOVERFLOW; goto done; }
            uint32_t nd = best.d == UINT64_MAX ? INF : (uint32_t)best.d;
            int32_t ns = best.d == UINT64_MAX ? -1 : best.s, np = best.d == UINT64_MAX ? -1 : best.p;
            if (nd != d0[v] || ns != s0[v] || np != q0[v]) changed = 1;
            d1[v] = nd; s1[v] = ns; q1[v] = np;
        }
        cur ^= 1;
        if (!changed) break;
    }
    for (int64_t v = 0; v < n; ++v) { cell[v] = S[cur][v]; dist[v] = D[cur][v]; if (src) src[v] = Q[cur][v]; }
    if (rounds) *rounds = r;
done:
    free(D[0]); free(D[1]); free(S[0]); free(S[1]); free(Q[0]); free(Q[1]);
    return rc;
}

/* Algorithm 1 with the any-angle tessellation: n_iters x (tessellation, Eq. 2  */
/* update with phi following the src chain), then a final tessellation.       */
/* rounds[it] = synchronous rounds of tessellation it (n_iters + 1 entries).   */
int orc_cvt_iterate_anyangle(const uint8_t *band, const uint16_t *q, int32_t nx, int32_t ny, int32_t nz,
                             int32_t *site_pos, int32_t n_sites, int32_t n_iters, int32_t max_rounds,
                             int32_t *cell, uint32_t *dist, int32_t *src, int64_t *trace, int32_t *rounds)
{
    if (!src) return ORC_EINVAL;
    int32_t *np = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_sites > 0 ? n_sites : 1));
    if (!np) return ORC_ENOMEM;
    int rc = ORC_OK;
    for (int32_t it = 0; it < n_iters; ++it) {
        rc = orc_anyangle_assign(band, nx, ny, nz, site_pos, n_sites, max_rounds, cell, dist, src,
                                 rounds ? rounds + it : NULL);
        if (rc) goto done;
        int64_t st[3];
        rc = orc_update_src(band, q, nx, ny, nz, cell, dist, src, site_pos, n_sites, np, st, 0, 0, 0, 0);
        if (rc) goto done;
        memcpy(site_pos, np, sizeof(int32_t) * (size_t)n_sites);
        if (trace) trace_record(trace, it, st, q, cell, dist, (int64_t)nx * ny * nz);
    }
    rc = orc_anyangle_assign(band, nx, ny, nz, site_pos, n_sites, max_rounds, cell, dist, src,
                             rounds ? rounds + n_iters : NULL);
done:
    free(np);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Per-variable value range over valid voxels (cell >= 0), used as the        */
/* default histogram range, and the float bin scale B / (hi - lo).            */
/* ------------------------------------------------------------------------- */
int orc_aux_range(const int32_t *cell, const float *aux, int32_t m, int64_t n, int32_t n_bins,
                  float *lo, float *hi, float *scale)
{
    for (int32_t j = 0; j < m; ++j) {
        float a = INFINITY, b = -INFINITY;
        const float *x = aux + (int64_t)j * n;
        for (int64_t v = 0; v < n; ++v) {
            if (cell[v] < 0) continue;
            if (!isfinite(x[v])) return ORC_ENONFINITE;
            if (x[v] < a) a = x[v];
            if (x[v] > b) b = x[v];
        }
        if (a > b) { a = 0.0f; b = 0.0f; }
        lo[j] = a; hi[j] = b;
        float w = b - a;
        scale[j] = (w > 0.0f) ? (float)n_bins / w : 0.0f;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Statistical aggregation per Voronoi cell.  Sec. 3.3 "Aggregation" and the  */
/* introduction (statistics aggregated within segments, e.g. histograms and  */
/* Gaussians).  Per cell s and variable j: count, mean, M2 = sum (x-mean)^2   */
/* (population variance = M2 / n), min, max, an n_bins histogram on          */
/* [lo_j, lo_j + n_bins/scale_j] with bin = (int)((x - lo) * scale) clamped,  */
/* and optionally the co-moment sums C_ij = sum (x_i-mean_i)(x_j-mean_j)      */
/* (upper triangle, row-major).  Two passes, FP64: the textbook definition.  */
/* Empty cells: count 0, mean 0, M2 0, min +inf, max -inf.                    */
/* ------------------------------------------------------------------------- */
int orc_aggregate(const int32_t *cell, const float *aux, int32_t m, int64_t n, int32_t n_cells,
                  const float *lo, const float *scale, int32_t n_bins, int32_t want_cov,
                  int64_t *count, double *mean, double *m2, float *vmin, float *vmax,
                  uint32_t *hist, double *comom)
{
    int32_t T = m * (m + 1) / 2;
    for (int32_t s = 0; s < n_cells; ++s) {
        count[s] = 0;
        for (int32_t j = 0; j < m; ++j) {
            mean[(int64_t)s * m + j] = 0.0; m2[(int64_t)s * m + j] = 0.0;
            vmin[(int64_t)s * m + j] = INFINITY; vmax[(int64_t)s * m + j] = -INFINITY;
            for (int32_t b = 0; b < n_bins; ++b) hist[((int64_t)s * m + j) * n_bins + b] = 0;
        }
        if (want_cov) for (int32_t t = 0; t < T; ++t) comom[(int64_t)s * T + t] = 0.0;
    }
    double *sum = (double *)calloc((size_t)n_cells * (size_t)(m > 0 ? m : 1), sizeof(double));
    if (!sum) return ORC_ENOMEM;
    for (int64_t v = 0; v < n; ++v) {
        int32_t s = cell[v];
        if (s < 0) continue;
        if (s >= n_cells) { free(sum); return ORC_EINVAL; }
        count[s]++;
        for (int32_t j = 0; j < m; ++j) {
            float x = aux[(int64_t)j * n + v];
            if (!isfinite(x)) { free(sum); return ORC_ENONFINITE; }
            int64_t k = (int64_t)s * m + j;
            sum[k] += (double)x;
            if (x < vmin[k]) vmin[k] = x;
            if (x > vmax[k]) vmax[k] = x;
            if (n_bins > 0) {
                float t = (x - lo[j]) * scale[j];
                int32_t bin;
                if (!(t > 0.0f)) bin = 0;
                else if (t >= (float)n_bins) bin = n_bins - 1;
                else bin = (int32_t)t;
                hist[k * n_bins + bin]++;
            }
        }
    }
    for (int32_t s = 0; s < n_cells; ++s)
        for (int32_t j = 0; j < m; ++j)
            if (count[s] > 0) mean[(int64_t)s * m + j] = sum[(int64_t)s * m + j] / (double)count[s];
    for (int64_t v = 0; v < n; ++v) {
        int32_t s = cell[v];
        if (s < 0) continue;
        int32_t t = 0;
        for (int32_t i = 0; i < m; ++i) {
            double di = (double)aux[(int64_t)i * n + v] - mean[(int64_t)s * m + i];
            m2[(int64_t)s * m + i] += di * di;
            if (want_cov)
                for (int32_t j = i; j < m; ++j) {
                    double dj = (double)aux[(int64_t)j * n + v] - mean[(int64_t)s * m + j];
                    comom[(int64_t)s * T + t] += di * dj;
                    ++t;
                }
        }
    }
    free(sum);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Merging statistics up the hierarchy cell -> component -> isoband ->        */
/* volume (introduction: aggregations may be merged over cells, components   */
/* and isobands).  Pairwise update of Chan, Golub & LeVeque (1979) in FP64,   */
/* merging children in increasing id order:                                   */
/*   n = na + nb, d = mean_b - mean_a, mean = mean_a + d nb / n,              */
/*   M2 = M2a + M2b + d^2 na nb / n, C_ij = Ca + Cb + d_i d_j na nb / n.       */
/* Counts, histograms, min and max combine exactly.  `parent` maps each of    */
/* the n_child records to its parent record in [0, n_parent).                  */
/* ------------------------------------------------------------------------- */
int orc_merge(int32_t n_child, const int32_t *parent, int32_t n_parent, int32_t m, int32_t n_bins, int32_t want_cov,
              const int64_t *c_count, const double *c_mean, const double *c_m2, const float *c_min,
              const float *c_max, const uint32_t *c_hist, const double *c_comom,
              int64_t *p_count, double *p_mean, double *p_m2, float *p_min, float *p_max,
              uint32_t *p_hist, double *p_comom)
{
    int32_t T = m * (m + 1) / 2;
    for (int32_t p = 0; p < n_parent; ++p) {
        p_count[p] = 0;
        for (int32_t j = 0; j < m; ++j) {
            p_mean[(int64_t)p * m + j] = 0.0; p_m2[(int64_t)p * m + j] = 0.0;
            p_min[(int64_t)p * m + j] = INFINITY; p_max[(int64_t)p * m + j] = -INFINITY;
            for (int32_t b = 0; b < n_bins; ++b) p_hist[((int64_t)p * m + j) * n_bins + b] = 0;
        }
        if (want_cov) for (int32_t t = 0; t < T; ++t) p_comom[(int64_t)p * T + t] = 0.0;
    }
    double *d = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    if (!d) return ORC_ENOMEM;
    for (int32_t c = 0; c < n_child; ++c) {
        int32_t p = parent[c];
        if (p < 0 || p >= n_parent) { free(d); return ORC_EINVAL; }
        int64_t nb = c_count[c];
        if (nb == 0) continue;
        int64_t na = p_count[p];
        for (int32_t j = 0; j < m; ++j) {
            int64_t kp = (int64_t)p * m + j, kc = (int64_t)c * m + j;
            if (c_min[kc] < p_min[kp]) p_min[kp] = c_min[kc];
            if (c_max[kc] > p_max[kp]) p_max[kp] = c_max[kc];
            for (int32_t b = 0; b < n_bins; ++b) p_hist[kp * n_bins + b] += c_hist[kc * n_bins + b];
        }
        if (na == 0) {
            for (int32_t j = 0; j < m; ++j) {
                p_mean[(int64_t)p * m + j] = c_mean[(int64_t)c * m + j];
                p_m2[(int64_t)p * m + j] = c_m2[(int64_t)c * m + j];
            }
            if (want_cov) for (int32_t t = 0; t < T; ++t) p_comom[(int64_t)p * T + t] = c_comom[(int64_t)c * T + t];
            p_count[p] = nb;
            continue;
        }
        double nn = (double)(na + nb);
        double f = (double)na * (double)nb / nn;
        for (int32_t j = 0; j < m; ++j) d[j] = c_mean[(int64_t)c * m + j] - p_mean[(int64_t)p * m + j];
        if (want_cov) {
            int32_t t = 0;
            for (int32_t i = 0; i < m; ++i)
                for (int32_t j = i; j < m; ++j) {
                    p_comom[(int64_t)p * T + t] = p_comom[(int64_t)p * T + t] + c_comom[(int64_t)c * T + t] + d[i] * d[j] * f;
                    ++t;
                }
        }
        for (int32_t j = 0; j < m; ++j) {
            int64_t kp = (int64_t)p * m + j, kc = (int64_t)c * m + j;
            p_m2[kp] = p_m2[kp] + c_m2[kc] + d[j] * d[j] * f;
            p_mean[kp] = p_mean[kp] + d[j] * ((double)nb / nn);
        }
        p_count[p] = na + nb;
    }
    free(d);
    return ORC_OK;
}

/* ========================================================================= */
/* Checkers used by the tests (not part of the method).                      */
/* ========================================================================= */

/* Bellman certificate of an assignment: with positive edge weights the      */
/* lexicographic key K(v) = min_s (D_s(v), s) is the unique solution of       */
/*   K(v) = min( (0, s) for sites s at v,  min_edges (K(u).d + w, K(u).s) ),  */
/* so checking this equation at every voxel certifies (cell, dist) exactly.  */
/* Returns the number of voxels that violate it (0 = certified).             */
int64_t orc_certify(const uint8_t *band, int32_t nx, int32_t ny, int32_t nz,
                    const int32_t *site_pos, int32_t n_sites, const int32_t *cell, const uint32_t *dist)
{
    int64_t n = (int64_t)nx * ny * nz;
    int32_t *own = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!own) return -1;
    for (int64_t v = 0; v < n; ++v) own[v] = -1;
    for (int32_t s = n_sites - 1; s >= 0; --s) {
        int32_t p = site_pos[s];
        if (p < 0 || p >= n) { free(own); return -1; }
        own[p] = s; /* lowest id wins */
    }
    int64_t bad = 0;
    for (int64_t v = 0; v < n; ++v) {
        int32_t x = (int32_t)(v % nx), y = (int32_t)((v / nx) % ny), z = (int32_t)(v / ((int64_t)nx * ny));
        uint64_t bd = UINT64_MAX; int64_t bs = INT64_MAX;
        if (band[v] != INVALID_BAND) {
            if (own[v] >= 0) { bd = 0; bs = own[v]; }
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (!dx && !dy && !dz) continue;
                        if (!has_edge(band, nx, ny, nz, x, y, z, dx, dy, dz)) continue;
                        int64_t u = (x + dx) + (int64_t)nx * ((y + dy) + (int64_t)ny * (z + dz));
                        if (cell[u] < 0) continue;
                        uint64_t cd = (uint64_t)dist[u] + edge_weight(dx, dy, dz);
                        if (cd < bd || (cd == bd && cell[u] < bs)) { bd = cd; bs = cell[u]; }
                    }
        }
        int ok;
        if (bd == UINT64_MAX) ok = (cell[v] == -1);
        else ok = (cell[v] == bs && (uint64_t)dist[v] == bd);
        if (!ok) ++bad;
    }
    free(own);
    return bad;
}

/* Single-source Dijkstra (distances only), used by the brute-force check    */
/* "per-seed shortest paths, then lexicographic minimum".                     */
int orc_sssp(const uint8_t *band, int32_t nx, int32_t ny, int32_t nz, int32_t src, uint64_t *d)
{
    int64_t n = (int64_t)nx * ny * nz;
    for (int64_t v = 0; v < n; ++v) d[v] = UINT64_MAX;
    heap h = {0, 0, 0};
    d[src] = 0;
    hent e0 = {0, 0, src};
    if (hpush(&h, e0)) return ORC_ENOMEM;
    while (h.n > 0) {
        hent e = hpop(&h);
        if (e.d != d[e.v]) continue;
        int32_t v = e.v, x = v % nx, y = (v / nx) % ny, z = v / (nx * ny);
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!dx && !dy && !dz) continue;
                    if (!has_edge(band, nx, ny, nz, x, y, z, dx, dy, dz)) continue;
                    int64_t u = (x + dx) + (int64_t)nx * ((y + dy) + (int64_t)ny * (z + dz));
                    uint64_t nd = e.d + edge_weight(dx, dy, dz);
                    if (nd < d[u]) {
                        d[u] = nd;
                        hent f = {nd, 0, (int32_t)u};
                        if (hpush(&h, f)) { free(h.a); return ORC_ENOMEM; }
                    }
                }
    }
    free(h.a);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Structured data layout.  Sec. 3.2 "Data Reduction and Structured Data      */
/* Layout" and Fig. hierarchy: the kept data is ordered hierarchically by     */
/* layer (isoband) and connected component so that each layer and component  */
/* is contiguous and directly indexable through offsets; the raw values are   */
/* extracted next to one coordinate per voxel.                                */
/* Readings: a voxel is kept when the band of its cell's component is in the  */
/* caller's band set; the order is (band, component, cell, linear index), the */
/* coordinate is the linear index, and offsets are given for bands,           */
/* components and cells (the position where each would start, also when it   */
/* holds no kept voxel).  The keys are compared as tuples, so the result does */
/* not depend on how the ids happen to be numbered.                           */
/* ------------------------------------------------------------------------- */
typedef struct { int32_t band, comp, cell, v; } orc_lkey;

static int lkey_cmp(const void *a, const void *b)
{
    const orc_lkey *p = (const orc_lkey *)a, *q = (const orc_lkey *)b;
    if (p->band != q->band) return p->band < q->band ? -1 : 1;
    if (p->comp != q->comp) return p->comp < q->comp ? -1 : 1;
    if (p->cell != q->cell) return p->cell < q->cell ? -1 : 1;
    if (p->v != q->v) return p->v < q->v ? -1 : 1;
    return 0;
}

int orc_layout(const int32_t *cell, int64_t n, const int32_t *site_comp, int32_t n_sites,
               const uint8_t *comp_band, int32_t n_comp, const uint32_t *band_mask,
               const float *aux, int32_t m, int32_t *order, float *values,
               int64_t *cell_off, int64_t *comp_off, int64_t *band_off, int64_t *n_kept)
{
    if (n < 0 || n_sites < 0 || n_comp < 0 || m < 0) return ORC_EINVAL;
    for (int32_t s = 0; s < n_sites; ++s)
        if (site_comp[s] < 0 || site_comp[s] >= n_comp) return ORC_EINVAL;
    orc_lkey *keys = (orc_lkey *)malloc(sizeof(orc_lkey) * (size_t)(n > 0 ? n : 1));
    int64_t *ccnt = (int64_t *)calloc((size_t)n_sites + 1, sizeof(int64_t));
    int64_t *kcnt = (int64_t *)calloc((size_t)n_comp + 1, sizeof(int64_t));
    orc_lkey *cells = (orc_lkey *)malloc(sizeof(orc_lkey) * ((size_t)n_sites + 1));
    orc_lkey *comps = (orc_lkey *)malloc(sizeof(orc_lkey) * ((size_t)n_comp + 1));
    if (!keys || !ccnt || !kcnt || !cells || !comps) {
        free(keys); free(ccnt); free(kcnt); free(cells); free(comps);
        return ORC_ENOMEM;
    }
    int64_t r = 0, bcnt[257];
    memset(bcnt, 0, sizeof(bcnt));
    for (int64_t v = 0; v < n; ++v) {
        int32_t s = cell[v];
        if (s < 0) continue;
        if (s >= n_sites) {
            free(keys); free(ccnt); free(kcnt); free(cells); free(comps);
            return ORC_EINVAL;
        }
        int32_t c = site_comp[s];
        int32_t b = comp_band[c];
        if (!((band_mask[b >> 5] >> (b & 31)) & 1u)) continue;
        keys[r].band = b; keys[r].comp = c; keys[r].cell = s; keys[r].v = (int32_t)v;
        ++r;
        ++ccnt[s]; ++kcnt[c]; ++bcnt[b];
    }
    qsort(keys, (size_t)r, sizeof(orc_lkey), lkey_cmp);
    for (int64_t p = 0; p < r; ++p) {
        order[p] = keys[p].v;
        for (int32_t j = 0; j < m; ++j) values[(int64_t)j * n + p] = aux[(int64_t)j * n + keys[p].v];
    }
    /* cells in layout order: (band, component, cell) */
    for (int32_t s = 0; s < n_sites; ++s) {
        cells[s].band = comp_band[site_comp[s]]; cells[s].comp = site_comp[s]; cells[s].cell = s; cells[s].v = 0;
    }
    qsort(cells, (size_t)n_sites, sizeof(orc_lkey), lkey_cmp);
    int64_t run = 0;
    for (int32_t k = 0; k < n_sites; ++k) { cell_off[cells[k].cell] = run; run += ccnt[cells[k].cell]; }
    cell_off[n_sites] = r;
    for (int32_t c = 0; c < n_comp; ++c) { comps[c].band = comp_band[c]; comps[c].comp = c; comps[c].cell = 0; comps[c].v = 0; }
    qsort(comps, (size_t)n_comp, sizeof(orc_lkey), lkey_cmp);
    run = 0;
    for (int32_t k = 0; k < n_comp; ++k) { comp_off[comps[k].comp] = run; run += kcnt[comps[k].comp]; }
    comp_off[n_comp] = r;
    run = 0;
    for (int b = 0; b < 256; ++b) { band_off[b] = run; run += bcnt[b]; }
    band_off[256] = r;
    *n_kept = r;
    free(keys); free(ccnt); free(kcnt); free(cells); free(comps);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Joint central moments of orders 2..4 (Sec. 3.3 and the joint-plot section: */
/* mean, covariance, coskewness and cokurtosis of the variables of a region,  */
/* compared between summaries and raw data).  For a set of n voxels with      */
/* means mu and deviations d = x - mu (m <= 8 variables):                     */
/*   M2[i<=j] = sum d_i d_j, M3[i<=j<=k] = sum d_i d_j d_k,                   */
/*   M4[i<=j<=k<=l] = sum d_i d_j d_k d_l,                                    */
/* tuples in lexicographic order.  Two passes in FP64 (mean, then sums).      */
/* Regions are the ranges [off[r], off[r+1]) of a list of voxel indices (a    */
/* structured layout), so cells, components and bands use the same code.      */
/* ------------------------------------------------------------------------- */
static int64_t binom_small(int64_t a, int64_t b)
{
    int64_t r = 1;
    for (int64_t i = 1; i <= b; ++i) r = r * (a - b + i) / i;
    return r;
}

int orc_joint_ranges(const float *aux, int32_t m, int64_t n, const int32_t *order, const int64_t *off,
                     int32_t n_ranges, int64_t *count, double *mean, double *m2, double *m3, double *m4)
{
    if (m < 1 || m > 8 || n < 0 || n_ranges < 0) return ORC_EINVAL;
    int64_t T2 = binom_small(m + 1, 2), T3 = binom_small(m + 2, 3), T4 = binom_small(m + 3, 4);
    for (int32_t r = 0; r < n_ranges; ++r) {
        int64_t lo = off[r], hi = off[r + 1];
        double mu[8] = {0};
        for (int64_t p = lo; p < hi; ++p)
            for (int32_t j = 0; j < m; ++j) mu[j] += (double)aux[(int64_t)j * n + order[p]];
        int64_t c = hi - lo;
        for (int32_t j = 0; j < m; ++j) mu[j] = c ? mu[j] / (double)c : 0.0;
        double *o2 = m2 + (int64_t)r * T2, *o3 = m3 + (int64_t)r * T3, *o4 = m4 + (int64_t)r * T4;
        for (int64_t t = 0; t < T2; ++t) o2[t] = 0.0;
        for (int64_t t = 0; t < T3; ++t) o3[t] = 0.0;
        for (int64_t t = 0; t < T4; ++t) o4[t] = 0.0;
        for (int64_t p = lo; p < hi; ++p) {
            double d[8];
            for (int32_t j = 0; j < m; ++j) d[j] = (double)aux[(int64_t)j * n + order[p]] - mu[j];
            int64_t t2 = 0, t3 = 0, t4 = 0;
            for (int i = 0; i < m; ++i)
                for (int j = i; j < m; ++j) {
                    o2[t2++] += d[i] * d[j];
                    for (int k = j; k < m; ++k) {
                        o3[t3++] += d[i] * d[j] * d[k];
                        for (int l = k; l < m; ++l) o4[t4++] += d[i] * d[j] * d[k] * d[l];
                    }
                }
        }
        count[r] = c;
        for (int32_t j = 0; j < m; ++j) mean[(int64_t)r * m + j] = mu[j];
    }
    return ORC_OK;
}

/* index of a sorted tuple in the lexicographic list of non-decreasing tuples of length q over m */
static int64_t tuple_index(const int *t, int q, int m)
{
    /* count the tuples that come before t: for each position, the tuples with a smaller
       value there and the same prefix */
    int64_t idx = 0;
    int prev = 0;
    for (int pos = 0; pos < q; ++pos) {
        for (int v = prev; v < t[pos]; ++v) idx += binom_small(m - v + (q - pos - 1) - 1, q - pos - 1);
        prev = t[pos];
    }
    return idx;
}

static double get_sym(const double *a, int q, int m, int i, int j, int k, int l)
{
    int t[4] = {i, j, k, l};
    /* sort the first q indices */
    for (int x = 1; x < q; ++x)
        for (int y = x; y > 0 && t[y - 1] > t[y]; --y) { int s = t[y]; t[y] = t[y - 1]; t[y - 1] = s; }
    return a[tuple_index(t, q, m)];
}

/* Pairwise merge of two joint-moment records (Pebay, "Formulas for robust, one-pass parallel
   computation of covariances and arbitrary-order statistical moments", Sandia SAND2008-6212,
   2008): with n = nA + nB and delta = muB - muA,
     M2 = M2A + M2B + dd nA nB / n
     M3 = M3A + M3B + ddd nA nB (nA - nB) / n^2 + (1/n) sum_3 d_i (nA M2B_jk - nB M2A_jk)
     M4 = M4A + M4B + dddd nA nB (nA^2 - nA nB + nB^2) / n^3
          + (1/n^2) sum_6 d_i d_j (nA^2 M2B_kl + nB^2 M2A_kl) + (1/n) sum_4 d_i (nA M3B_jkl - nB M3A_jkl)
   the sums running over the distinct ways to split the index tuple. */
static void joint_merge_into(int m, int64_t *nA_, double *muA, double *A2, double *A3, double *A4, int64_t nB_,
                             const double *muB, const double *B2, const double *B3, const double *B4)
{
    if (nB_ == 0) return;
    int64_t T2 = binom_small(m + 1, 2), T3 = binom_small(m + 2, 3), T4 = binom_small(m + 3, 4);
    if (*nA_ == 0) {
        *nA_ = nB_;
        for (int j = 0; j < m; ++j) muA[j] = muB[j];
        for (int64_t t = 0; t < T2; ++t) A2[t] = B2[t];
        for (int64_t t = 0; t < T3; ++t) A3[t] = B3[t];
        for (int64_t t = 0; t < T4; ++t) A4[t] = B4[t];
        return;
    }
    double nA = (double)*nA_, nB = (double)nB_, n = nA + nB;
    double d[8];
    for (int j = 0; j < m; ++j) d[j] = muB[j] - muA[j];
    double *N2 = (double *)malloc(sizeof(double) * (size_t)(T2 + T3 + T4));
    double *N3 = N2 + T2, *N4 = N3 + T3;
    int64_t t2 = 0, t3 = 0, t4 = 0;
    for (int i = 0; i < m; ++i)
        for (int j = i; j < m; ++j) {
            N2[t2] = A2[t2] + B2[t2] + d[i] * d[j] * nA * nB / n;
            ++t2;
            for (int k = j; k < m; ++k) {
                double s3 = d[i] * (nA * get_sym(B2, 2, m, j, k, 0, 0) - nB * get_sym(A2, 2, m, j, k, 0, 0)) +
                            d[j] * (nA * get_sym(B2, 2, m, i, k, 0, 0) - nB * get_sym(A2, 2, m, i, k, 0, 0)) +
                            d[k] * (nA * get_sym(B2, 2, m, i, j, 0, 0) - nB * get_sym(A2, 2, m, i, j, 0, 0));
                N3[t3] = A3[t3] + B3[t3] + d[i] * d[j] * d[k] * nA * nB * (nA - nB) / (n * n) + s3 / n;
                ++t3;
                for (int l = k; l < m; ++l) {
                    int ix[4] = {i, j, k, l};
                    double s6 = 0.0, s4 = 0.0;
                    for (int a = 0; a < 4; ++a)
                        for (int b = a + 1; b < 4; ++b) {
                            int rest[2], q = 0;
                            for (int c = 0; c < 4; ++c)
                                if (c != a && c != b) rest[q++] = ix[c];
                            s6 += d[ix[a]] * d[ix[b]] *
                                  (nA * nA * get_sym(B2, 2, m, rest[0], rest[1], 0, 0) +
                                   nB * nB * get_sym(A2, 2, m, rest[0], rest[1], 0, 0));
                        }
                    for (int a = 0; a < 4; ++a) {
                        int rest[3], q = 0;
                        for (int c = 0; c < 4; ++c)
                            if (c != a) rest[q++] = ix[c];
                        s4 += d[ix[a]] * (nA * get_sym(B3, 3, m, rest[0], rest[1], rest[2], 0) -
                                          nB * get_sym(A3, 3, m, rest[0], rest[1], rest[2], 0));
                    }
                    N4[t4] = A4[t4] + B4[t4] +
                             d[i] * d[j] * d[k] * d[l] * nA * nB * (nA * nA - nA * nB + nB * nB) / (n * n * n) +
                             s6 / (n * n) + s4 / n;
                    ++t4;
                }
            }
        }
    for (int j = 0; j < m; ++j) muA[j] += d[j] * nB / n;
    for (int64_t t = 0; t < T2; ++t) A2[t] = N2[t];
    for (int64_t t = 0; t < T3; ++t) A3[t] = N3[t];
    for (int64_t t = 0; t < T4; ++t) A4[t] = N4[t];
    *nA_ += nB_;
    free(N2);
}

/* Merge child records into parents: parent p takes the children [child_off[p], child_off[p+1])
   in id order. */
int orc_joint_merge(int32_t m, int32_t n_parent, const int64_t *child_off, const int64_t *count,
                    const double *mean, const double *m2, const double *m3, const double *m4, int64_t *pcount,
                    double *pmean, double *pm2, double *pm3, double *pm4)
{
    if (m < 1 || m > 8 || n_parent < 0) return ORC_EINVAL;
    int64_t T2 = binom_small(m + 1, 2), T3 = binom_small(m + 2, 3), T4 = binom_small(m + 3, 4);
    for (int32_t p = 0; p < n_parent; ++p) {
        int64_t n = 0;
        double *mu = pmean + (int64_t)p * m, *A2 = pm2 + (int64_t)p * T2, *A3 = pm3 + (int64_t)p * T3,
               *A4 = pm4 + (int64_t)p * T4;
        for (int j = 0; j < m; ++j) mu[j] = 0.0;
        for (int64_t t = 0; t < T2; ++t) A2[t] = 0.0;
        for (int64_t t = 0; t < T3; ++t) A3[t] = 0.0;
        for (int64_t t = 0; t < T4; ++t) A4[t] = 0.0;
        for (int64_t c = child_off[p]; c < child_off[p + 1]; ++c)
            joint_merge_into(m, &n, mu, A2, A3, A4, count[c], mean + c * m, m2 + c * T2, m3 + c * T3,
                             m4 + c * T4);
        pcount[p] = n;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Voronoi site graph and geodesic site distances (Sec. "Voronoi Cell Views": */
/* the connectivity of the sites from region adjacency, then shortest paths   */
/* between adjacent sites, restricted to the component, and the distance      */
/* ||x_i - x_j|| / gd(s_i, s_j), or c when no path exists).                   */
/* Readings: two cells are adjacent when a voxel of one and a voxel of the    */
/* other are face neighbours (6-adjacency, as for the components; such voxels */
/* share a band, so edges never leave a component); the edge between sites a  */
/* and b weighs ceil(2^16 ||x_a - x_b||_2), an integer, so path lengths are   */
/* exact sums and every shortest-path algorithm gives the same numbers.       */
/* ------------------------------------------------------------------------- */
static uint64_t isqrt_floor_u64(uint64_t v)
{
    uint64_t lo = 0, hi = (uint64_t)1 << 32;  /* hi^2 > v for v < 2^64 */
    while (hi - lo > 1) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (mid * mid <= v) lo = mid;
        else hi = mid;
    }
    return lo;
}

uint32_t orc_site_weight(int32_t dx, int32_t dy, int32_t dz)
{
    uint64_t D = (uint64_t)((int64_t)dx * dx + (int64_t)dy * dy + (int64_t)dz * dz);
    uint64_t v = D << 32;  /* (2^16)^2 D */
    uint64_t r = isqrt_floor_u64(v);
    return (uint32_t)(r * r == v ? r : r + 1);
}

static int pair_cmp(const void *a, const void *b)
{
    const int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Undirected edges (a < b) in increasing (a, b) order; returns the count (or < 0). */
int64_t orc_site_edges(const int32_t *cell, const uint8_t *band, int32_t nx, int32_t ny, int32_t nz,
                       int64_t max_edges, int32_t *ea, int32_t *eb)
{
    int64_t n = (int64_t)nx * ny * nz, cnt = 0, cap = 1024;
    int64_t *pairs = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    if (!pairs) return ORC_ENOMEM;
    for (int64_t v = 0; v < n; ++v) {
        int32_t x = (int32_t)(v % nx), y = (int32_t)((v / nx) % ny), z = (int32_t)(v / ((int64_t)nx * ny));
        if (cell[v] < 0) continue;
        int64_t nb[3] = {x + 1 < nx ? v + 1 : -1, y + 1 < ny ? v + nx : -1, z + 1 < nz ? v + (int64_t)nx * ny : -1};
        for (int k = 0; k < 3; ++k) {
            int64_t u = nb[k];
            if (u < 0 || cell[u] < 0 || cell[u] == cell[v] || band[u] != band[v]) continue;
            int32_t a = cell[v] < cell[u] ? cell[v] : cell[u], b = cell[v] < cell[u] ? cell[u] : cell[v];
            if (cnt == cap) {
                cap *= 2;
                int64_t *np = (int64_t *)realloc(pairs, sizeof(int64_t) * (size_t)cap);
                if (!np) { free(pairs); return ORC_ENOMEM; }
                pairs = np;
            }
            pairs[cnt++] = ((int64_t)a << 32) | (int64_t)b;
        }
    }
    qsort(pairs, (size_t)cnt, sizeof(int64_t), pair_cmp);
    int64_t m = 0;
    for (int64_t i = 0; i < cnt; ++i) {
        if (i > 0 && pairs[i] == pairs[i - 1]) continue;
        if (m >= max_edges) { free(pairs); return ORC_ECAPACITY; }
        ea[m] = (int32_t)(pairs[i] >> 32);
        eb[m] = (int32_t)(pairs[i] & 0xffffffff);
        ++m;
    }
    free(pairs);
    return m;
}

/* Dijkstra from `src` over the undirected site graph given as a CSR (both directions):
   dist[t] = shortest path length in weight units, UINT64_MAX if unreachable. */
int orc_site_sssp(int32_t n_sites, const int64_t *off, const int32_t *dst, const uint32_t *w, int32_t src,
                  uint64_t *dist)
{
    if (src < 0 || src >= n_sites) return ORC_EINVAL;
    for (int32_t i = 0; i < n_sites; ++i) dist[i] = UINT64_MAX;
    uint8_t *done = (uint8_t *)calloc((size_t)n_sites + 1, 1);
    /* binary heap of (dist, node) */
    int64_t cap = 64, hn = 0;
    uint64_t *hd = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)cap);
    int32_t *hv = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    if (!done || !hd || !hv) { free(done); free(hd); free(hv); return ORC_ENOMEM; }
    dist[src] = 0;
    hd[0] = 0; hv[0] = src; hn = 1;
    while (hn > 0) {
        uint64_t d = hd[0];
        int32_t u = hv[0];
        --hn;
        /* sift the last entry down from the root */
        {
            uint64_t kd = hd[hn];
            int32_t kv = hv[hn];
            int64_t i = 0;
            for (;;) {
                int64_t c = 2 * i + 1;
                if (c >= hn) break;
                if (c + 1 < hn && (hd[c + 1] < hd[c] || (hd[c + 1] == hd[c] && hv[c + 1] < hv[c]))) ++c;
                if (hd[c] < kd || (hd[c] == kd && hv[c] < kv)) { hd[i] = hd[c]; hv[i] = hv[c]; i = c; }
                else break;
            }
            hd[i] = kd; hv[i] = kv;
        }
        if (done[u] || d != dist[u]) continue;
        done[u] = 1;
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
            int32_t t = dst[e];
            uint64_t nd = d + w[e];
            if (nd < dist[t]) {
                dist[t] = nd;
                if (hn == cap) {
                    cap *= 2;
                    uint64_t *a = (uint64_t *)realloc(hd, sizeof(uint64_t) * (size_t)cap);
                    int32_t *b = (int32_t *)realloc(hv, sizeof(int32_t) * (size_t)cap);
                    if (!a || !b) { free(done); free(a ? a : hd); free(b ? b : hv); return ORC_ENOMEM; }
                    hd = a; hv = b;
                }
                int64_t i = hn++;
                while (i > 0) {
                    int64_t p = (i - 1) / 2;
                    if (hd[p] < nd || (hd[p] == nd && hv[p] <= t)) break;
                    hd[i] = hd[p]; hv[i] = hv[p]; i = p;
                }
                hd[i] = nd; hv[i] = t;
            }
        }
    }
    free(done); free(hd); free(hv);
    return ORC_OK;
}
