/*
 * nl_oracle.c -- plain, slow, obviously-correct CPU oracle for the compressed
 * cluster neighbor list of "GPU-Native Compressed Neighbor Lists with a
 * Space-Filling-Curve Data Layout" (Thaler & Keller) and for the SPH / LJ
 * neighborhood passes that consume it.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference leg of bench.py use it.  It shares no code, header, table or
 * constant generator with the CUDA library; the two only agree because both
 * follow the same written definitions (the paper's Sec. II plus the readings
 * listed below).
 *
 * Arithmetic: FP64 for every sum (density, forces, energies, MLP).  The pair
 * predicate is the one canonical definition in IEEE binary32 round-to-nearest
 * with no FMA contraction (compile with -ffp-contract=off), because the
 * neighbor *set* is defined by it and must match the GPU bit for bit.
 *
 * Readings of the paper (where it is silent or ambiguous):
 *  - keys: 21 bits per axis, 63-bit Morton (x in the highest bit of every
 *    triple) or Skilling's Hilbert transpose (J. Skilling, "Programming the
 *    Hilbert curve", AIP Conf. Proc. 707, 2004), quantised in FP32 as
 *    q = min(trunc((x-lo) * (2^21/(hi-lo))), 2^21-1).
 *  - sort: stable by key, equal keys keep the original index order.
 *  - clusters of M consecutive SFC particles, super-clusters of 8 clusters
 *    (Sec. II-A); the tail simply ends at n (no particle beyond n exists).
 *  - pair predicate (Sec. II-A, "compare individual particle-particle
 *    distances"; "always compute the periodic distances"):
 *        dx = xj - xi; periodic: if dx > L/2: dx -= L elif dx < -L/2: dx += L
 *        d2 = (dx*dx + dy*dy) + dz*dz ; r = support*h
 *        symmetric: i != j && d2 < max(ri,rj)^2 ; gather: i != j && d2 < ri^2
 *  - octree leaves: maximal key-prefix cells holding <= B particles (cells at
 *    level 21 are leaves whatever their count); only non-empty cells exist.
 *  - list record per super-cluster (Sec. II-A/B/C):
 *        u32 count | count x u8 masks, zero-padded to 4 bytes |
 *        nibble stream (compressed) or count x u32 (uncompressed),
 *        zero-padded to 4 bytes.
 *    Differences d0 = J0 + 1, dk = Jk - J(k-1).  Blocks of w values: a w-bit
 *    mask whose bit k is set iff dk != 1 (Table 1 marks the non-ones), then one
 *    info nibble per set bit (v+6 for v in [2,9], else n_nibbles-1), then the
 *    data nibbles of every value >= 10, most significant nibble first.
 *    Nibble p of the stream is byte p/2, low half when p is even.
 *  - SPH kernel: the M4 cubic spline with support 2h, W = w(r/h)/(pi h^3).
 *    Density includes the self term m_i W(0,h_i) (Sec. II-D, rho_i = sum_j).
 *  - pressure force: the symmetric form
 *        a_i = -sum_j m_j [P_i/rho_i^2 grad_i W(r_ij,h_i) + P_j/rho_j^2 grad_i W(r_ij,h_j)]
 *    over the symmetric neighbor set.
 *  - LJ: F_i = sum_j 24 eps (2 s^12/r^14 - s^6/r^8) (x_i - x_j), no shift.
 *  - LJ + Coulomb (Sec. III-B): the LJ term plus kc q_i q_j (x_i - x_j)/r^3
 *    over the pairs within the interaction cutoff rc, plain cutoff (no shift,
 *    no reaction field); the list is built at a larger radius (Verlet buffer)
 *    and the interaction set is the gather set at rc.
 *
 * The paper's Fig. 2 cluster-overhead values are not printed, so the overhead
 * is pinned by closed forms (1x1 clusters, all pairs in range, isolated
 * clusters), not by the paper's numbers.
 */
#define _DEFAULT_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_KEY_BITS 21
#define ORC_MAX_LEVEL 21
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Box                                                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    float lo[3];
    float hi[3];
    int32_t periodic[3];
} orc_box;

static float box_len32(const orc_box *b, int a) { return b->hi[a] - b->lo[a]; }

/* ------------------------------------------------------------------------ */
/* SFC keys (Sec. II-A: Hilbert-ordered particle data)                      */
/* ------------------------------------------------------------------------ */

/* FP32 quantisation of one coordinate to 21 bits. */
uint32_t orc_quantize(float x, float lo, float hi)
{
    float len = hi - lo;
    float s = 2097152.0f / len;
    float t = (x - lo) * s;
    uint32_t q;
    if (!(t > 0.0f)) return 0u;
    if (t >= 2097151.0f) return 2097151u;
    q = (uint32_t)t;
    return q > 2097151u ? 2097151u : q;
}

/* Morton: bit b of x, y, z goes to key bits 3b+2, 3b+1, 3b. */
uint64_t orc_morton3(uint32_t qx, uint32_t qy, uint32_t qz)
{
    uint64_t key = 0;
    for (int b = ORC_KEY_BITS - 1; b >= 0; --b) {
        key = (key << 3) | ((uint64_t)((qx >> b) & 1u) << 2) |
              ((uint64_t)((qy >> b) & 1u) << 1) | (uint64_t)((qz >> b) & 1u);
    }
    return key;
}

/* Skilling's AxestoTranspose for n = 3 dimensions, `bits` bits per axis,
 * followed by reading the transposed bits out MSB first, X[0] first. */
uint64_t orc_hilbert3(uint32_t qx, uint32_t qy, uint32_t qz, int bits)
{
    uint32_t X[3] = {qx, qy, qz};
    uint32_t M = 1u << (bits - 1);
    /* inverse undo */
    for (uint32_t Q = M; Q > 1; Q >>= 1) {
        uint32_t P = Q - 1;
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;
            } else {
                uint32_t t = (X[0] ^ X[i]) & P;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    /* Gray encode */
    for (int i = 1; i < 3; ++i) X[i] ^= X[i - 1];
    uint32_t t = 0;
    for (uint32_t Q = M; Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    for (int i = 0; i < 3; ++i) X[i] ^= t;
    /* interleave transposed bits */
    uint64_t key = 0;
    for (int b = bits - 1; b >= 0; --b) {
        for (int i = 0; i < 3; ++i) key = (key << 1) | ((X[i] >> b) & 1u);
    }
    return key;
}

/* Skilling's TransposetoAxes (the inverse), used only by the self-tests. */
void orc_hilbert3_inverse(uint64_t key, int bits, uint32_t *q)
{
    uint32_t X[3] = {0, 0, 0};
    for (int b = bits - 1; b >= 0; --b) {
        for (int i = 0; i < 3; ++i) {
            int pos = 3 * b + (2 - i);
            X[i] |= (uint32_t)((key >> pos) & 1u) << b;
        }
    }
    uint32_t N = 2u << (bits - 1);
    /* Gray decode */
    uint32_t t = X[2] >> 1;
    for (int i = 2; i > 0; --i) X[i] ^= X[i - 1];
    X[0] ^= t;
    /* undo excess work */
    for (uint32_t Q = 2; Q != N; Q <<= 1) {
        uint32_t P = Q - 1;
        for (int i = 2; i >= 0; --i) {
            if (X[i] & Q) {
                X[0] ^= P;
            } else {
                uint32_t tt = (X[0] ^ X[i]) & P;
                X[0] ^= tt;
                X[i] ^= tt;
            }
        }
    }
    q[0] = X[0];
    q[1] = X[1];
    q[2] = X[2];
}

/* kind 0 = Morton, 1 = Hilbert */
void orc_keys(int64_t n, const float *x, const float *y, const float *z, const orc_box *box,
              int kind, uint64_t *keys)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        uint32_t qx = orc_quantize(x[i], box->lo[0], box->hi[0]);
        uint32_t qy = orc_quantize(y[i], box->lo[1], box->hi[1]);
        uint32_t qz = orc_quantize(z[i], box->lo[2], box->hi[2]);
        keys[i] = kind == 0 ? orc_morton3(qx, qy, qz) : orc_hilbert3(qx, qy, qz, ORC_KEY_BITS);
    }
}

/* ------------------------------------------------------------------------ */
/* Stable sort: order by (key, original index)                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t key;
    int64_t idx;
} keyidx;

static int cmp_keyidx(const void *a, const void *b)
{
    const keyidx *u = (const keyidx *)a, *v = (const keyidx *)b;
    if (u->key != v->key) return u->key < v->key ? -1 : 1;
    if (u->idx != v->idx) return u->idx < v->idx ? -1 : 1;
    return 0;
}

/* perm[k] = original index of the particle at sorted position k */
int orc_sort(int64_t n, const uint64_t *keys, int64_t *perm)
{
    keyidx *t = (keyidx *)malloc((size_t)(n > 0 ? n : 1) * sizeof(keyidx));
    if (!t) return -1;
    for (int64_t i = 0; i < n; ++i) {
        t[i].key = keys[i];
        t[i].idx = i;
    }
    qsort(t, (size_t)n, sizeof(keyidx), cmp_keyidx);
    for (int64_t i = 0; i < n; ++i) perm[i] = t[i].idx;
    free(t);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Octree from sorted keys (Sec. II-A traversal structure)                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    const uint64_t *keys;
    int bucket;
    int64_t cap, count;
    int32_t *level;
    int64_t *first, *end;
    int32_t *leaf;
} octctx;

static void oct_rec(octctx *c, int level, int64_t a, int64_t b)
{
    int is_leaf = (b - a <= c->bucket) || level == ORC_MAX_LEVEL;
    if (c->count < c->cap) {
        c->level[c->count] = level;
        c->first[c->count] = a;
        c->end[c->count] = b;
        c->leaf[c->count] = is_leaf;
    }
    c->count++;
    if (is_leaf) return;
    int shift = 63 - 3 * (level + 1);
    int64_t s = a;
    while (s < b) {
        uint64_t child = c->keys[s] >> shift;
        int64_t e = s;
        while (e < b && (c->keys[e] >> shift) == child) ++e;
        oct_rec(c, level + 1, s, e);
        s = e;
    }
}

/* Pre-order list of the non-empty cells.  Returns the node count; arrays are
 * filled up to `cap` entries. */
int64_t orc_octree(int64_t n, const uint64_t *sorted_keys, int bucket, int32_t *level,
                   int64_t *first, int64_t *end, int32_t *leaf, int64_t cap)
{
    octctx c = {sorted_keys, bucket, cap, 0, level, first, end, leaf};
    if (n <= 0) return 0;
    oct_rec(&c, 0, 0, n);
    return c.count;
}

/* ------------------------------------------------------------------------ */
/* Canonical FP32 pair predicate                                            */
/* ------------------------------------------------------------------------ */
static inline float wrap32(float d, float len, int periodic)
{
    if (periodic) {
        float half = 0.5f * len;
        if (d > half)
            d = d - len;
        else if (d < -half)
            d = d + len;
    }
    return d;
}

static inline float dist2_32(const float *xs, const float *ys, const float *zs, int64_t i,
                             int64_t j, const orc_box *b)
{
    float dx = wrap32(xs[j] - xs[i], box_len32(b, 0), b->periodic[0]);
    float dy = wrap32(ys[j] - ys[i], box_len32(b, 1), b->periodic[1]);
    float dz = wrap32(zs[j] - zs[i], box_len32(b, 2), b->periodic[2]);
    float xx = dx * dx;
    float yy = dy * dy;
    float zz = dz * dz;
    float s = xx + yy;
    return s + zz;
}

/* mode 0: gather (d2 < ri^2), mode 1: symmetric (d2 < max(ri,rj)^2) */
static inline int pred32(const float *xs, const float *ys, const float *zs, const float *hs,
                         float support, int64_t i, int64_t j, const orc_box *b, int mode)
{
    if (i == j) return 0;
    float d2 = dist2_32(xs, ys, zs, i, j, b);
    float ri = support * hs[i];
    float r = ri;
    if (mode == 1) {
        float rj = support * hs[j];
        if (rj > r) r = rj;
    }
    float r2 = r * r;
    return d2 < r2;
}

/* exposed for the self-tests (bitwise symmetry) */
int orc_pred(const float *xs, const float *ys, const float *zs, const float *hs, float support,
             int64_t i, int64_t j, const orc_box *b, int mode)
{
    return pred32(xs, ys, zs, hs, support, i, j, b, mode);
}

float orc_dist2(const float *xs, const float *ys, const float *zs, int64_t i, int64_t j,
                const orc_box *b)
{
    return dist2_32(xs, ys, zs, i, j, b);
}

/* ------------------------------------------------------------------------ */
/* CSR container                                                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    int64_t *off; /* n+1 */
    int32_t *idx; /* off[n] */
} orc_csr;

int64_t orc_csr_nnz(const orc_csr *c) { return c->off[c->n]; }

void orc_csr_copy(const orc_csr *c, int64_t *off, int32_t *idx)
{
    memcpy(off, c->off, (size_t)(c->n + 1) * sizeof(int64_t));
    if (c->off[c->n]) memcpy(idx, c->idx, (size_t)c->off[c->n] * sizeof(int32_t));
}

void orc_csr_free(orc_csr *c)
{
    if (!c) return;
    free(c->off);
    free(c->idx);
    free(c);
}

static orc_csr *csr_alloc(int64_t n, int64_t nnz)
{
    orc_csr *c = (orc_csr *)calloc(1, sizeof(orc_csr));
    if (!c) return NULL;
    c->n = n;
    c->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    c->idx = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    if (!c->off || !c->idx) {
        orc_csr_free(c);
        return NULL;
    }
    return c;
}

/* Copy a CSR given as arrays (used to hand sampled rows back in). */
orc_csr *orc_csr_from(int64_t n, const int64_t *off, const int32_t *idx)
{
    orc_csr *c = csr_alloc(n, off[n]);
    if (!c) return NULL;
    memcpy(c->off, off, (size_t)(n + 1) * sizeof(int64_t));
    if (off[n]) memcpy(c->idx, idx, (size_t)off[n] * sizeof(int32_t));
    return c;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t u = *(const int32_t *)a, v = *(const int32_t *)b;
    return (u > v) - (u < v);
}

/* ------------------------------------------------------------------------ */
/* Brute force neighbor sets of selected particles: O(n) per query          */
/* ------------------------------------------------------------------------ */
orc_csr *orc_brute_neighbors(int64_t n, const float *xs, const float *ys, const float *zs,
                             const float *hs, const orc_box *b, float support, int mode,
                             int64_t nq, const int64_t *queries)
{
    int64_t *cnt = (int64_t *)calloc((size_t)nq + 1, sizeof(int64_t));
    if (!cnt) return NULL;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nq; ++q) {
        int64_t i = queries[q], c = 0;
        for (int64_t j = 0; j < n; ++j) c += pred32(xs, ys, zs, hs, support, i, j, b, mode);
        cnt[q] = c;
    }
    int64_t nnz = 0;
    for (int64_t q = 0; q < nq; ++q) nnz += cnt[q];
    orc_csr *out = csr_alloc(nq, nnz);
    if (!out) {
        free(cnt);
        return NULL;
    }
    for (int64_t q = 0; q < nq; ++q) out->off[q + 1] = out->off[q] + cnt[q];
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nq; ++q) {
        int64_t i = queries[q], p = out->off[q];
        for (int64_t j = 0; j < n; ++j)
            if (pred32(xs, ys, zs, hs, support, i, j, b, mode)) out->idx[p++] = (int32_t)j;
    }
    free(cnt);
    return out;
}

/* ------------------------------------------------------------------------ */
/* FP64 multi-level cell list: gather sets G_i of every particle            */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t cell;
    int32_t idx;
} cellent;

static int cmp_cellent(const void *a, const void *b)
{
    const cellent *u = (const cellent *)a, *v = (const cellent *)b;
    if (u->cell != v->cell) return u->cell < v->cell ? -1 : 1;
    return (u->idx > v->idx) - (u->idx < v->idx);
}

typedef struct {
    double cs[3];  /* cell size per axis (>= the level's radius) */
    int64_t nc[3]; /* cells per axis */
    cellent *ent;  /* all particles sorted by cell */
    int64_t n;
} grid;

static uint64_t cell_pack(int64_t ix, int64_t iy, int64_t iz)
{
    return ((uint64_t)ix << 42) | ((uint64_t)iy << 21) | (uint64_t)iz;
}

static int64_t cell_coord(double x, double lo, double cs, int64_t nc)
{
    int64_t c = (int64_t)floor((x - lo) / cs);
    if (c < 0) c = 0;
    if (c > nc - 1) c = nc - 1;
    return c;
}

static int grid_build(grid *g, int64_t n, const float *xs, const float *ys, const float *zs,
                      const orc_box *b, double c)
{
    const float *p[3] = {xs, ys, zs};
    for (int a = 0; a < 3; ++a) {
        double len = (double)b->hi[a] - (double)b->lo[a];
        int64_t nc = (int64_t)floor(len / c);
        if (nc < 1) nc = 1;
        if (nc > (1 << 20)) nc = 1 << 20;
        g->nc[a] = nc;
        g->cs[a] = len / (double)nc;
    }
    g->n = n;
    g->ent = (cellent *)malloc((size_t)(n > 0 ? n : 1) * sizeof(cellent));
    if (!g->ent) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t ic[3];
        for (int a = 0; a < 3; ++a)
            ic[a] = cell_coord((double)p[a][i], (double)b->lo[a], g->cs[a], g->nc[a]);
        g->ent[i].cell = cell_pack(ic[0], ic[1], ic[2]);
        g->ent[i].idx = (int32_t)i;
    }
    qsort(g->ent, (size_t)n, sizeof(cellent), cmp_cellent);
    return 0;
}

static void grid_range(const grid *g, uint64_t cell, int64_t *a, int64_t *e)
{
    int64_t lo = 0, hi = g->n;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (g->ent[mid].cell < cell) lo = mid + 1; else hi = mid;
    }
    *a = lo;
    hi = g->n;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (g->ent[mid].cell <= cell) lo = mid + 1; else hi = mid;
    }
    *e = lo;
}

/* neighbor cell coordinates along one axis, without duplicates */
static int axis_cells(int64_t c, int64_t nc, int periodic, int64_t *out)
{
    int k = 0;
    for (int64_t d = -1; d <= 1; ++d) {
        int64_t v = c + d;
        if (periodic) {
            v = ((v % nc) + nc) % nc;
        } else if (v < 0 || v >= nc) {
            continue;
        }
        int dup = 0;
        for (int t = 0; t < k; ++t) dup |= out[t] == v;
        if (!dup) out[k++] = v;
    }
    return k;
}

/* Visit the gather set of particle i in grid g.  Returns the count; writes
 * the (unsorted) members to out when out != NULL. */
static int64_t grid_gather(const grid *g, int64_t i, const float *xs, const float *ys,
                           const float *zs, const float *hs, float support, const orc_box *b,
                           int32_t *out)
{
    const float *p[3] = {xs, ys, zs};
    int64_t cand[3][3];
    int ncand[3];
    for (int a = 0; a < 3; ++a) {
        int64_t c = cell_coord((double)p[a][i], (double)b->lo[a], g->cs[a], g->nc[a]);
        ncand[a] = axis_cells(c, g->nc[a], b->periodic[a], cand[a]);
    }
    int64_t cnt = 0;
    for (int u = 0; u < ncand[0]; ++u)
        for (int v = 0; v < ncand[1]; ++v)
            for (int w = 0; w < ncand[2]; ++w) {
                int64_t a0, a1;
                grid_range(g, cell_pack(cand[0][u], cand[1][v], cand[2][w]), &a0, &a1);
                for (int64_t t = a0; t < a1; ++t) {
                    int64_t j = g->ent[t].idx;
                    if (pred32(xs, ys, zs, hs, support, i, j, b, 0)) {
                        if (out) out[cnt] = (int32_t)j;
                        ++cnt;
                    }
                }
            }
    return cnt;
}

/* Gather sets G_i = {j != i : d2_ij < r_i^2} of all particles, rows sorted.
 * Level l has cells of size >= c0 * 2^l with c0 slightly above min r; every
 * particle queries the 27 cells of the first level whose cell size covers
 * its own radius, so the candidates always include every j within r_i. */
orc_csr *orc_gather_all(int64_t n, const float *xs, const float *ys, const float *zs,
                        const float *hs, const orc_box *b, float support)
{
    if (n <= 0) return csr_alloc(0, 0);
    double rmin = INFINITY, rmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double r = (double)(support * hs[i]);
        if (r < rmin) rmin = r;
        if (r > rmax) rmax = r;
    }
    double c0 = rmin * (1.0 + 1e-5);
    int nlev = 1;
    while (c0 * ldexp(1.0, nlev - 1) < rmax * (1.0 + 1e-5)) ++nlev;
    int *lev = (int *)malloc((size_t)n * sizeof(int));
    int *used = (int *)calloc((size_t)nlev, sizeof(int));
    grid *gs = (grid *)calloc((size_t)nlev, sizeof(grid));
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!lev || !used || !gs || !cnt) return NULL;
    for (int64_t i = 0; i < n; ++i) {
        double r = (double)(support * hs[i]) * (1.0 + 1e-5);
        int l = 0;
        while (c0 * ldexp(1.0, l) < r) ++l;
        lev[i] = l;
        used[l] = 1;
    }
    for (int l = 0; l < nlev; ++l)
        if (used[l] && grid_build(&gs[l], n, xs, ys, zs, b, c0 * ldexp(1.0, l)) != 0)
            return NULL;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i)
        cnt[i] = grid_gather(&gs[lev[i]], i, xs, ys, zs, hs, support, b, NULL);
    int64_t nnz = 0;
    for (int64_t i = 0; i < n; ++i) nnz += cnt[i];
    orc_csr *out = csr_alloc(n, nnz);
    if (!out) return NULL;
    for (int64_t i = 0; i < n; ++i) out->off[i + 1] = out->off[i] + cnt[i];
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        int32_t *row = out->idx + out->off[i];
        grid_gather(&gs[lev[i]], i, xs, ys, zs, hs, support, b, row);
        qsort(row, (size_t)cnt[i], sizeof(int32_t), cmp_i32);
    }
    for (int l = 0; l < nlev; ++l) free(gs[l].ent);
    free(gs);
    free(used);
    free(lev);
    free(cnt);
    return out;
}

/* Symmetric sets P_i = G_i U {j : i in G_j}: the union of a CSR and its
 * transpose (pred_sym(i,j) <=> d2 < ri^2 or d2 < rj^2). */
orc_csr *orc_symmetrize(const orc_csr *g)
{
    int64_t n = g->n, nnz = g->off[n];
    int64_t *toff = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *tidx = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    int64_t *pos = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!toff || !tidx || !pos || !cnt) return NULL;
    for (int64_t t = 0; t < nnz; ++t) toff[g->idx[t] + 1]++;
    for (int64_t i = 0; i < n; ++i) toff[i + 1] += toff[i];
    for (int64_t i = 0; i < n; ++i) pos[i] = toff[i];
    for (int64_t i = 0; i < n; ++i)
        for (int64_t t = g->off[i]; t < g->off[i + 1]; ++t) tidx[pos[g->idx[t]]++] = (int32_t)i;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t a = g->off[i], ae = g->off[i + 1], c = toff[i], ce = toff[i + 1], k = 0;
        while (a < ae || c < ce) {
            if (c >= ce || (a < ae && g->idx[a] < tidx[c])) ++a;
            else if (a >= ae || tidx[c] < g->idx[a]) ++c;
            else { ++a; ++c; }
            ++k;
        }
        cnt[i] = k;
    }
    int64_t tot = 0;
    for (int64_t i = 0; i < n; ++i) tot += cnt[i];
    orc_csr *out = csr_alloc(n, tot);
    if (!out) return NULL;
    for (int64_t i = 0; i < n; ++i) out->off[i + 1] = out->off[i] + cnt[i];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t a = g->off[i], ae = g->off[i + 1], c = toff[i], ce = toff[i + 1];
        int64_t p = out->off[i];
        while (a < ae || c < ce) {
            if (c >= ce || (a < ae && g->idx[a] < tidx[c])) out->idx[p++] = g->idx[a++];
            else if (a >= ae || tidx[c] < g->idx[a]) out->idx[p++] = tidx[c++];
            else { out->idx[p++] = g->idx[a++]; ++c; }
        }
    }
    free(toff);
    free(tidx);
    free(pos);
    free(cnt);
    return out;
}

/* ------------------------------------------------------------------------ */
/* Canonical cluster list (Sec. II-A): per super-cluster the ascending       */
/* j-clusters J having a pair with one of its 8 i-clusters, with an 8-bit    */
/* mask of those i-clusters.                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t nsc;
    int64_t *off;   /* nsc+1 */
    int32_t *J;     /* off[nsc] */
    uint8_t *mask;  /* off[nsc] */
} orc_clist;

int64_t orc_clist_nnz(const orc_clist *c) { return c->off[c->nsc]; }

void orc_clist_copy(const orc_clist *c, int64_t *off, int32_t *J, uint8_t *mask)
{
    memcpy(off, c->off, (size_t)(c->nsc + 1) * sizeof(int64_t));
    if (c->off[c->nsc]) {
        memcpy(J, c->J, (size_t)c->off[c->nsc] * sizeof(int32_t));
        memcpy(mask, c->mask, (size_t)c->off[c->nsc]);
    }
}

void orc_clist_free(orc_clist *c)
{
    if (!c) return;
    free(c->off);
    free(c->J);
    free(c->mask);
    free(c);
}

typedef struct {
    int32_t J;
    int32_t bit;
} jbit;

static int cmp_jbit(const void *a, const void *b)
{
    const jbit *u = (const jbit *)a, *v = (const jbit *)b;
    if (u->J != v->J) return (u->J > v->J) - (u->J < v->J);
    return (u->bit > v->bit) - (u->bit < v->bit);
}

/* P: symmetric neighbor sets of the rows listed in `rows` (rows[k] = sorted
 * particle index of CSR row k), over particles [0,n).  i-clusters hold
 * `cluster` particles (8 per super-cluster, one mask bit each), j-clusters
 * `jcluster` particles (the unit of the stored indices).  The super-clusters
 * built are those whose particles all appear in rows (rows covering whole
 * super-clusters, e.g. all of [0,n)).  sc_ids[t] = super-cluster index of the
 * t-th output record, in ascending order. */
orc_clist *orc_cluster_lists(int64_t n, int cluster, int jcluster, const orc_csr *P,
                             const int64_t *rows, int64_t nsc_out, const int64_t *sc_ids)
{
    const int64_t sp = (int64_t)cluster * 8;
    orc_clist *c = (orc_clist *)calloc(1, sizeof(orc_clist));
    c->nsc = nsc_out;
    c->off = (int64_t *)calloc((size_t)nsc_out + 1, sizeof(int64_t));
    /* row of each particle, -1 if absent */
    int64_t *rowof = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) rowof[i] = -1;
    for (int64_t k = 0; k < P->n; ++k) rowof[rows[k]] = k;
    int64_t *cnt = (int64_t *)calloc((size_t)nsc_out + 1, sizeof(int64_t));
    jbit **tmp = (jbit **)calloc((size_t)nsc_out + 1, sizeof(jbit *));
    int64_t *tmpn = (int64_t *)calloc((size_t)nsc_out + 1, sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < nsc_out; ++t) {
        int64_t s = sc_ids[t];
        int64_t a = s * sp, e = a + sp < n ? a + sp : n, tot = 0;
        for (int64_t i = a; i < e; ++i) {
            int64_t r = rowof[i];
            if (r >= 0) tot += P->off[r + 1] - P->off[r];
        }
        jbit *v = (jbit *)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(jbit));
        int64_t m = 0;
        for (int64_t i = a; i < e; ++i) {
            int64_t r = rowof[i];
            if (r < 0) continue;
            for (int64_t q = P->off[r]; q < P->off[r + 1]; ++q) {
                v[m].J = (int32_t)(P->idx[q] / jcluster);
                v[m].bit = (int32_t)((i - a) / cluster);
                ++m;
            }
        }
        qsort(v, (size_t)m, sizeof(jbit), cmp_jbit);
        int64_t u = 0;
        for (int64_t q = 0; q < m; ++q)
            if (q == 0 || v[q].J != v[q - 1].J) ++u;
        tmp[t] = v;
        tmpn[t] = m;
        cnt[t] = u;
    }
    for (int64_t t = 0; t < nsc_out; ++t) c->off[t + 1] = c->off[t] + cnt[t];
    int64_t nnz = c->off[nsc_out];
    c->J = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    c->mask = (uint8_t *)calloc((size_t)(nnz > 0 ? nnz : 1), 1);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < nsc_out; ++t) {
        int64_t p = c->off[t] - 1;
        for (int64_t q = 0; q < tmpn[t]; ++q) {
            if (q == 0 || tmp[t][q].J != tmp[t][q - 1].J) {
                ++p;
                c->J[p] = tmp[t][q].J;
            }
            c->mask[p] |= (uint8_t)(1u << tmp[t][q].bit);
        }
        free(tmp[t]);
    }
    free(tmp);
    free(tmpn);
    free(cnt);
    free(rowof);
    return c;
}

/* ------------------------------------------------------------------------ */
/* Nibble VLE codec (Sec. II-B, Tables 1 and 2; layout Sec. II-C)            */
/* ------------------------------------------------------------------------ */

/* number of hexadecimal digits of v >= 1 */
static int hex_digits(uint32_t v)
{
    int k = 0;
    while (v) {
        ++k;
        v >>= 4;
    }
    return k;
}

/* Encode one block of nv <= w differences (all >= 1).  Outputs the mask
 * (bit k <=> d_k != 1), the info nibbles and the data nibbles in stream
 * order.  Returns through ninfo / ndata. */
void orc_encode_block(int nv, const uint32_t *d, uint64_t *mask, uint8_t *info, int *ninfo,
                      uint8_t *data, int *ndata)
{
    uint64_t m = 0;
    int ni = 0, nd = 0;
    for (int k = 0; k < nv; ++k) {
        uint32_t v = d[k];
        if (v == 1) continue;
        m |= 1ull << k;
        if (v <= 9) {
            info[ni++] = (uint8_t)(v + 6);
        } else {
            int nn = hex_digits(v);
            info[ni++] = (uint8_t)(nn - 1);
            for (int t = nn - 1; t >= 0; --t) data[nd++] = (uint8_t)((v >> (4 * t)) & 0xF);
        }
    }
    *mask = m;
    *ninfo = ni;
    *ndata = nd;
}

static void put_nibble(uint8_t *s, int64_t p, uint8_t v)
{
    if (p & 1) s[p >> 1] |= (uint8_t)(v << 4);
    else s[p >> 1] |= (uint8_t)(v & 0xF);
}

static uint8_t get_nibble(const uint8_t *s, int64_t p)
{
    return (p & 1) ? (uint8_t)(s[p >> 1] >> 4) : (uint8_t)(s[p >> 1] & 0xF);
}

static int64_t pad4(int64_t b) { return (b + 3) & ~(int64_t)3; }

/* Size in nibbles of the compressed stream of `count` ascending indices. */
int64_t orc_stream_nibbles(int64_t count, const int32_t *J, int w)
{
    int64_t nib = 0, prev = -1;
    for (int64_t k = 0; k < count; ++k) {
        if (k % w == 0) nib += w / 4;
        uint32_t v = (uint32_t)(J[k] - prev);
        prev = J[k];
        if (v == 1) continue;
        nib += 1;
        if (v > 9) nib += hex_digits(v);
    }
    return nib;
}

/* Record bytes for one super-cluster. */
int64_t orc_record_bytes(int64_t count, const int32_t *J, int w, int compress)
{
    int64_t body = compress ? (orc_stream_nibbles(count, J, w) + 1) / 2 : 4 * count;
    return 4 + pad4(count) + pad4(body);
}

/* Write the record into out (zero-filled here).  Returns bytes written. */
int64_t orc_encode_record(int64_t count, const int32_t *J, const uint8_t *mask, int w,
                          int compress, uint8_t *out)
{
    int64_t bytes = orc_record_bytes(count, J, w, compress);
    memset(out, 0, (size_t)bytes);
    uint32_t c32 = (uint32_t)count;
    out[0] = (uint8_t)(c32 & 0xFF);
    out[1] = (uint8_t)((c32 >> 8) & 0xFF);
    out[2] = (uint8_t)((c32 >> 16) & 0xFF);
    out[3] = (uint8_t)((c32 >> 24) & 0xFF);
    for (int64_t k = 0; k < count; ++k) out[4 + k] = mask[k];
    uint8_t *body = out + 4 + pad4(count);
    if (!compress) {
        for (int64_t k = 0; k < count; ++k) {
            uint32_t v = (uint32_t)J[k];
            for (int t = 0; t < 4; ++t) body[4 * k + t] = (uint8_t)((v >> (8 * t)) & 0xFF);
        }
        return bytes;
    }
    uint32_t d[64];
    uint8_t info[64], data[64 * 8];
    int64_t p = 0, prev = -1;
    for (int64_t b0 = 0; b0 < count; b0 += w) {
        int nv = (int)(count - b0 < w ? count - b0 : w);
        for (int k = 0; k < nv; ++k) {
            d[k] = (uint32_t)(J[b0 + k] - prev);
            prev = J[b0 + k];
        }
        uint64_t m;
        int ni, nd;
        orc_encode_block(nv, d, &m, info, &ni, data, &nd);
        for (int t = 0; t < w / 4; ++t) put_nibble(body, p++, (uint8_t)((m >> (4 * t)) & 0xF));
        for (int t = 0; t < ni; ++t) put_nibble(body, p++, info[t]);
        for (int t = 0; t < nd; ++t) put_nibble(body, p++, data[t]);
    }
    return bytes;
}

/* Decode a record.  Returns count; J/mask written when non-NULL. */
int64_t orc_decode_record(const uint8_t *rec, int w, int compress, int32_t *J, uint8_t *mask)
{
    int64_t count = (int64_t)rec[0] | ((int64_t)rec[1] << 8) | ((int64_t)rec[2] << 16) |
                    ((int64_t)rec[3] << 24);
    if (mask)
        for (int64_t k = 0; k < count; ++k) mask[k] = rec[4 + k];
    const uint8_t *body = rec + 4 + pad4(count);
    if (!J) return count;
    if (!compress) {
        for (int64_t k = 0; k < count; ++k)
            J[k] = (int32_t)((uint32_t)body[4 * k] | ((uint32_t)body[4 * k + 1] << 8) |
                             ((uint32_t)body[4 * k + 2] << 16) | ((uint32_t)body[4 * k + 3] << 24));
        return count;
    }
    int64_t p = 0, prev = -1;
    for (int64_t b0 = 0; b0 < count; b0 += w) {
        int nv = (int)(count - b0 < w ? count - b0 : w);
        uint64_t m = 0;
        for (int t = 0; t < w / 4; ++t) m |= (uint64_t)get_nibble(body, p++) << (4 * t);
        int ni = 0;
        for (int k = 0; k < nv; ++k) ni += (int)((m >> k) & 1u);
        int64_t pinfo = p, pdata = p + ni;
        for (int k = 0; k < nv; ++k) {
            uint32_t v = 1;
            if ((m >> k) & 1u) {
                uint8_t inf = get_nibble(body, pinfo++);
                if (inf >= 8) {
                    v = (uint32_t)inf - 6;
                } else {
                    v = 0;
                    for (int t = 0; t <= inf; ++t) v = (v << 4) | get_nibble(body, pdata++);
                }
            }
            prev += v;
            J[b0 + k] = (int32_t)prev;
        }
        p = pdata;
    }
    return count;
}

/* ------------------------------------------------------------------------ */
/* SPH cubic spline (M4), support 2h, 3-D normalisation 1/(pi h^3)          */
/* ------------------------------------------------------------------------ */
double orc_w(double q)
{
    if (q < 1.0) return 1.0 - 1.5 * q * q + 0.75 * q * q * q;
    if (q < 2.0) {
        double t = 2.0 - q;
        return 0.25 * t * t * t;
    }
    return 0.0;
}

double orc_dw(double q)
{
    if (q < 1.0) return -3.0 * q + 2.25 * q * q;
    if (q < 2.0) {
        double t = 2.0 - q;
        return -0.75 * t * t;
    }
    return 0.0;
}

double orc_W(double r, double h) { return orc_w(r / h) / (M_PI * h * h * h); }

/* FP64 position difference x_j - x_i with the same wrap decision as the
 * FP32 predicate (the wrap is decided on the FP32 difference). */
static inline double dx64(const float *p, int64_t i, int64_t j, const orc_box *b, int a)
{
    double d = (double)p[j] - (double)p[i];
    if (b->periodic[a]) {
        float len = box_len32(b, a);
        float d32 = p[j] - p[i];
        float half = 0.5f * len;
        if (d32 > half) d -= (double)len;
        else if (d32 < -half) d += (double)len;
    }
    return d;
}

/* rho_i = m_i W(0,h_i) + sum_{j in G_i} m_j W(r_ij, h_i) for the rows of G
 * (row k is particle rows[k]). */
void orc_density(const float *xs, const float *ys, const float *zs, const float *hs,
                 const float *ms, const orc_box *b, const orc_csr *G, const int64_t *rows,
                 double *rho)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < G->n; ++k) {
        int64_t i = rows[k];
        double h = (double)hs[i];
        double s = (double)ms[i] * orc_W(0.0, h);
        for (int64_t t = G->off[k]; t < G->off[k + 1]; ++t) {
            int64_t j = G->idx[t];
            double dx = dx64(xs, i, j, b, 0), dy = dx64(ys, i, j, b, 1), dz = dx64(zs, i, j, b, 2);
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            s += (double)ms[j] * orc_W(r, h);
        }
        rho[k] = s;
    }
}

/* a_i = -sum_{j in P_i} m_j [P_i/rho_i^2 gW(r_ij,h_i) + P_j/rho_j^2 gW(r_ij,h_j)],
 * gW(r,h) = grad_i W = (x_i - x_j)/r * w'(r/h)/(pi h^4). */
void orc_sph_force(const float *xs, const float *ys, const float *zs, const float *hs,
                   const float *ms, const double *rho, const double *pres, const orc_box *b,
                   const orc_csr *P, const int64_t *rows, double *ax, double *ay, double *az,
                   double *fabs_sum)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < P->n; ++k) {
        int64_t i = rows[k];
        double hi = (double)hs[i];
        double ci = pres[i] / (rho[i] * rho[i]);
        double fx = 0, fy = 0, fz = 0, fa = 0;
        for (int64_t t = P->off[k]; t < P->off[k + 1]; ++t) {
            int64_t j = P->idx[t];
            double dx = dx64(xs, i, j, b, 0), dy = dx64(ys, i, j, b, 1), dz = dx64(zs, i, j, b, 2);
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (r == 0.0) continue;
            double hj = (double)hs[j];
            double cj = pres[j] / (rho[j] * rho[j]);
            double gi = orc_dw(r / hi) / (M_PI * hi * hi * hi * hi);
            double gj = orc_dw(r / hj) / (M_PI * hj * hj * hj * hj);
            double s = (double)ms[j] * (ci * gi + cj * gj) / r;
            /* x_i - x_j = -dx */
            fx -= s * (-dx);
            fy -= s * (-dy);
            fz -= s * (-dz);
            fa += fabs(s) * r;
        }
        ax[k] = fx;
        ay[k] = fy;
        az[k] = fz;
        if (fabs_sum) fabs_sum[k] = fa;
    }
}

/* Lennard-Jones 12/6: F_i = sum_j 24 eps (2 s^12/r^14 - s^6/r^8)(x_i - x_j). */
void orc_lj_force(const float *xs, const float *ys, const float *zs, const orc_box *b,
                  double eps, double sigma, const orc_csr *P, const int64_t *rows, double *fx,
                  double *fy, double *fz, double *fabs_sum)
{
    double s6 = pow(sigma, 6.0), s12 = s6 * s6;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < P->n; ++k) {
        int64_t i = rows[k];
        double ax = 0, ay = 0, az = 0, fa = 0;
        for (int64_t t = P->off[k]; t < P->off[k + 1]; ++t) {
            int64_t j = P->idx[t];
            double dx = dx64(xs, i, j, b, 0), dy = dx64(ys, i, j, b, 1), dz = dx64(zs, i, j, b, 2);
            double r2 = dx * dx + dy * dy + dz * dz;
            double r4 = r2 * r2, r8 = r4 * r4, r14 = r8 * r4 * r2;
            double c = 24.0 * eps * (2.0 * s12 / r14 - s6 / r8);
            ax += c * (-dx);
            ay += c * (-dy);
            az += c * (-dz);
            fa += fabs(c) * sqrt(r2);
        }
        fx[k] = ax;
        fy[k] = ay;
        fz[k] = az;
        if (fabs_sum) fabs_sum[k] = fa;
    }
}

/* E = sum_{i<j, j in P_i} 4 eps ((s/r)^12 - (s/r)^6) for a full-row CSR. */
double orc_lj_energy(const float *xs, const float *ys, const float *zs, const orc_box *b,
                     double eps, double sigma, const orc_csr *P)
{
    double e = 0.0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : e)
    for (int64_t i = 0; i < P->n; ++i) {
        for (int64_t t = P->off[i]; t < P->off[i + 1]; ++t) {
            int64_t j = P->idx[t];
            if (j <= i) continue;
            double dx = dx64(xs, i, j, b, 0), dy = dx64(ys, i, j, b, 1), dz = dx64(zs, i, j, b, 2);
            double sr2 = sigma * sigma / (dx * dx + dy * dy + dz * dz);
            double sr6 = sr2 * sr2 * sr2;
            e += 4.0 * eps * (sr6 * sr6 - sr6);
        }
    }
    return e;
}

/* Lennard-Jones 12/6 plus Coulomb with a plain cutoff (Sec. III-B names the
 * two interactions; the cutoff form is our reading): over the pairs of P (the
 * interaction set, i.e. the gather set at the interaction radius rc),
 *   F_i = sum_j [24 eps (2 s^12/r^14 - s^6/r^8) + kc q_i q_j / r^3] (x_i - x_j),
 * the negative gradient of
 *   E = sum_{i<j} [4 eps ((s/r)^12 - (s/r)^6) + kc q_i q_j / r].
 * q may be NULL (no Coulomb term).  fabs_sum[k] = sum_j |f_ij|. */
void orc_ljc_force(const float *xs, const float *ys, const float *zs, const orc_box *b,
                   double eps, double sigma, const float *q, double kc, const orc_csr *P,
                   const int64_t *rows, double *fx, double *fy, double *fz, double *fabs_sum)
{
    double s6 = pow(sigma, 6.0), s12 = s6 * s6;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < P->n; ++k) {
        int64_t i = rows[k];
        double ax = 0, ay = 0, az = 0, fa = 0;
        for (int64_t t = P->off[k]; t < P->off[k + 1]; ++t) {
            int64_t j = P->idx[t];
            double dx = dx64(xs, i, j, b, 0), dy = dx64(ys, i, j, b, 1), dz = dx64(zs, i, j, b, 2);
            double r2 = dx * dx + dy * dy + dz * dz;
            double r = sqrt(r2);
            double r4 = r2 * r2, r8 = r4 * r4, r14 = r8 * r4 * r2;
            double c = 24.0 * eps * (2.0 * s12 / r14 - s6 / r8);
            if (q) c += kc * (double)q[i] * (double)q[j] / (r2 * r);
            /* x_i - x_j = -(dx, dy, dz) */
            ax += c * (-dx);
            ay += c * (-dy);
            az += c * (-dz);
            fa += fabs(c) * r;
        }
        fx[k] = ax;
        fy[k] = ay;
        fz[k] = az;
        if (fabs_sum) fabs_sum[k] = fa;
    }
}

double orc_ljc_energy(const float *xs, const float *ys, const float *zs, const orc_box *b,
                      double eps, double sigma, const float *q, double kc, const orc_csr *P)
{
    double e = 0.0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : e)
    for (int64_t i = 0; i < P->n; ++i) {
        for (int64_t t = P->off[i]; t < P->off[i + 1]; ++t) {
            int64_t j = P->idx[t];
            if (j <= i) continue;
            double dx = dx64(xs, i, j, b, 0), dy = dx64(ys, i, j, b, 1), dz = dx64(zs, i, j, b, 2);
            double r2 = dx * dx + dy * dy + dz * dz;
            double sr2 = sigma * sigma / r2;
            double sr6 = sr2 * sr2 * sr2;
            e += 4.0 * eps * (sr6 * sr6 - sr6);
            if (q) e += kc * (double)q[i] * (double)q[j] / sqrt(r2);
        }
    }
    return e;
}

/* Distance from particle k to its nearest member of the interaction set
 * P_k (the pair function of Sec. II-D with a minimum reduction), FP64 from
 * the FP32 coordinates with the canonical periodic wrap; +inf for an empty
 * set.  Rows are particles 0..n-1. */
void orc_nearest(const float *xs, const float *ys, const float *zs, const orc_box *b,
                 const orc_csr *P, double *out)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < P->n; ++i) {
        double best = INFINITY;
        for (int64_t t = P->off[i]; t < P->off[i + 1]; ++t) {
            int64_t j = P->idx[t];
            double dx = dx64(xs, i, j, b, 0), dy = dx64(ys, i, j, b, 1), dz = dx64(zs, i, j, b, 2);
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (r < best) best = r;
        }
        out[i] = best;
    }
}

/* Computed pairs of a cluster list (Sec. III-A): every listed tile, i.e.
 * every set mask bit, costs its M x MJ particle pairs.  The cluster overhead
 * is this count divided by the pairs the list serves (ordered neighbor pairs
 * plus one self term per particle). */
int64_t orc_computed_pairs(int64_t nnz, const uint8_t *mask, int cluster, int jcluster)
{
    int64_t s = 0;
    for (int64_t t = 0; t < nnz; ++t) s += __builtin_popcount(mask[t]);
    return s * (int64_t)cluster * (int64_t)jcluster;
}

/* ------------------------------------------------------------------------ */
/* Smoothing-length window: count of gather neighbors of every query with   */
/* the canonical FP32 predicate (the h-iteration's acceptance test).         */
/* ------------------------------------------------------------------------ */
void orc_gather_counts_brute(int64_t n, const float *xs, const float *ys, const float *zs,
                             const float *hs, const orc_box *b, float support, int64_t nq,
                             const int64_t *queries, int64_t *counts)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nq; ++q) {
        int64_t i = queries[q], c = 0;
        for (int64_t j = 0; j < n; ++j) c += pred32(xs, ys, zs, hs, support, i, j, b, 0);
        counts[q] = c;
    }
}

/* Squared distances (FP32 canonical) from query i to every particle, used to
 * pin the h window with k-th neighbor distances. */
void orc_dist2_row(int64_t n, const float *xs, const float *ys, const float *zs,
                   const orc_box *b, int64_t i, float *d2)
{
    for (int64_t j = 0; j < n; ++j) d2[j] = dist2_32(xs, ys, zs, i, j, b);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Smoothing-length MLP (not in the paper): F=8 inputs, three hidden layers */
/* of 64 with SiLU, one output; loss = mean squared error.  Plain FP64.     */
/* Weight layout (row-major, out x in): W1 64x8, W2 64x64, W3 64x64, W4 1x64 */
/* packed as W1 b1 W2 b2 W3 b3 W4 b4 (orc_mlp_nparams values).              */
/* ------------------------------------------------------------------------ */
#define MLP_F 8
#define MLP_H 64

int64_t orc_mlp_nparams(void)
{
    return (int64_t)MLP_H * MLP_F + MLP_H + 2 * ((int64_t)MLP_H * MLP_H + MLP_H) + MLP_H + 1;
}

static double silu(double z) { return z / (1.0 + exp(-z)); }

static double dsilu(double z)
{
    double s = 1.0 / (1.0 + exp(-z));
    return s * (1.0 + z * (1.0 - s));
}

/* One dense layer: out[o] = b[o] + sum_i W[o][i] in[i]. */
static void dense(int nout, int nin, const double *W, const double *b, const double *in,
                  double *out)
{
    for (int o = 0; o < nout; ++o) {
        double s = b[o];
        for (int i = 0; i < nin; ++i) s += W[(int64_t)o * nin + i] * in[i];
        out[o] = s;
    }
}

/* Forward for n samples; X n x 8; pred n. */
void orc_mlp_forward(int64_t n, const double *X, const double *P, double *pred)
{
    const double *W1 = P, *b1 = W1 + MLP_H * MLP_F, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H;
    const double *W3 = b2 + MLP_H, *b3 = W3 + MLP_H * MLP_H, *W4 = b3 + MLP_H, *b4 = W4 + MLP_H;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n; ++r) {
        double z1[MLP_H], h1[MLP_H], z2[MLP_H], h2[MLP_H], z3[MLP_H], h3[MLP_H], y;
        dense(MLP_H, MLP_F, W1, b1, X + r * MLP_F, z1);
        for (int k = 0; k < MLP_H; ++k) h1[k] = silu(z1[k]);
        dense(MLP_H, MLP_H, W2, b2, h1, z2);
        for (int k = 0; k < MLP_H; ++k) h2[k] = silu(z2[k]);
        dense(MLP_H, MLP_H, W3, b3, h2, z3);
        for (int k = 0; k < MLP_H; ++k) h3[k] = silu(z3[k]);
        dense(1, MLP_H, W4, b4, h3, &y);
        pred[r] = y;
    }
}

/* Loss = (1/n) sum_r (pred_r - t_r)^2 and its gradient G (same packing as
 * P) by reverse-mode differentiation of the forward above.  Returns loss. */
double orc_mlp_loss_grad(int64_t n, const double *X, const double *t, const double *P, double *G)
{
    const int64_t np = orc_mlp_nparams();
    const double *W1 = P, *b1 = W1 + MLP_H * MLP_F, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H;
    const double *W3 = b2 + MLP_H, *b3 = W3 + MLP_H * MLP_H, *W4 = b3 + MLP_H, *b4 = W4 + MLP_H;
    for (int64_t k = 0; k < np; ++k) G[k] = 0.0;
    double *gW1 = G, *gb1 = gW1 + MLP_H * MLP_F, *gW2 = gb1 + MLP_H, *gb2 = gW2 + MLP_H * MLP_H;
    double *gW3 = gb2 + MLP_H, *gb3 = gW3 + MLP_H * MLP_H, *gW4 = gb3 + MLP_H, *gb4 = gW4 + MLP_H;
    double loss = 0.0;
    for (int64_t r = 0; r < n; ++r) {
        const double *x = X + r * MLP_F;
        double z1[MLP_H], h1[MLP_H], z2[MLP_H], h2[MLP_H], z3[MLP_H], h3[MLP_H], y;
        dense(MLP_H, MLP_F, W1, b1, x, z1);
        for (int k = 0; k < MLP_H; ++k) h1[k] = silu(z1[k]);
        dense(MLP_H, MLP_H, W2, b2, h1, z2);
        for (int k = 0; k < MLP_H; ++k) h2[k] = silu(z2[k]);
        dense(MLP_H, MLP_H, W3, b3, h2, z3);
        for (int k = 0; k < MLP_H; ++k) h3[k] = silu(z3[k]);
        dense(1, MLP_H, W4, b4, h3, &y);
        double e = y - t[r];
        loss += e * e;
        double dy = 2.0 * e / (double)n;
        double d3[MLP_H], d2[MLP_H], d1[MLP_H];
        gb4[0] += dy;
        for (int k = 0; k < MLP_H; ++k) {
            gW4[k] += dy * h3[k];
            d3[k] = dy * W4[k] * dsilu(z3[k]);
        }
        for (int o = 0; o < MLP_H; ++o) {
            gb3[o] += d3[o];
            for (int i = 0; i < MLP_H; ++i) gW3[o * MLP_H + i] += d3[o] * h2[i];
        }
        for (int i = 0; i < MLP_H; ++i) {
            double s = 0.0;
            for (int o = 0; o < MLP_H; ++o) s += d3[o] * W3[o * MLP_H + i];
            d2[i] = s * dsilu(z2[i]);
        }
        for (int o = 0; o < MLP_H; ++o) {
            gb2[o] += d2[o];
            for (int i = 0; i < MLP_H; ++i) gW2[o * MLP_H + i] += d2[o] * h1[i];
        }
        for (int i = 0; i < MLP_H; ++i) {
            double s = 0.0;
            for (int o = 0; o < MLP_H; ++o) s += d2[o] * W2[o * MLP_H + i];
            d1[i] = s * dsilu(z1[i]);
        }
        for (int o = 0; o < MLP_H; ++o) {
            gb1[o] += d1[o];
            for (int i = 0; i < MLP_F; ++i) gW1[o * MLP_F + i] += d1[o] * x[i];
        }
    }
    return loss / (double)n;
}

/* ------------------------------------------------------------------------ */
/* Learned-start inputs (not in the paper; the features are this project's  */
/* own proposal).  One system in SFC-sorted order, n particles, clusters of */
/* M = `cluster` consecutive particles, super-clusters of 8 clusters; the   */
/* tail cluster slots beyond n hold no particle.  With e(B) the largest     */
/* side of box B (floored at 1e-7 L), e8 the box of the cluster's real      */
/* particles, e64 the box of its super-cluster, e512 / e4096 the boxes of    */
/* super-clusters s-3..s+4 / s-31..s+32 clipped to the system, L the largest */
/* side of the system box and N_s its particle count, cluster c gets        */
/*   log(e8/e64), log(e512/e64), log(e4096/e64), log(ex/e8), log(ey/e8),     */
/*   log(ez/e8), log(count/M), log(e64/L) + log(N_s)/3                       */
/* and an empty cluster gets zeros.  Plain FP64 on the FP32 inputs.          */
/* ------------------------------------------------------------------------ */
typedef struct {
    double lo[3], hi[3];
} dbox;

static void dbox_empty(dbox *b)
{
    for (int a = 0; a < 3; ++a) {
        b->lo[a] = INFINITY;
        b->hi[a] = -INFINITY;
    }
}

static void dbox_add_box(dbox *b, const dbox *o)
{
    for (int a = 0; a < 3; ++a) {
        if (o->lo[a] < b->lo[a]) b->lo[a] = o->lo[a];
        if (o->hi[a] > b->hi[a]) b->hi[a] = o->hi[a];
    }
}

static double dbox_side(const dbox *b, int a, double floor_len)
{
    double e = b->hi[a] - b->lo[a];
    return e > floor_len ? e : floor_len;
}

static double dbox_extent(const dbox *b, double floor_len)
{
    double e = dbox_side(b, 0, floor_len);
    for (int a = 1; a < 3; ++a) {
        double v = dbox_side(b, a, floor_len);
        if (v > e) e = v;
    }
    return e;
}

int orc_mlp_features(int64_t n, const float *xs, const float *ys, const float *zs,
                     const orc_box *box, int cluster, double *X, double *e64)
{
    const int64_t M = cluster, scp = 8 * (int64_t)cluster;
    const int64_t nsc = (n + scp - 1) / scp, ncl = 8 * nsc;
    double L = 0.0;
    for (int a = 0; a < 3; ++a) {
        double len = (double)box->hi[a] - (double)box->lo[a];
        if (len > L) L = len;
    }
    const double fl = 1e-7 * L;
    dbox *cb = (dbox *)malloc((size_t)(ncl > 0 ? ncl : 1) * sizeof(dbox));
    dbox *sb = (dbox *)malloc((size_t)(nsc > 0 ? nsc : 1) * sizeof(dbox));
    int64_t *cnt = (int64_t *)calloc((size_t)(ncl > 0 ? ncl : 1), sizeof(int64_t));
    if (!cb || !sb || !cnt) return -1;
    const float *p[3] = {xs, ys, zs};
    for (int64_t c = 0; c < ncl; ++c) {
        dbox_empty(&cb[c]);
        for (int64_t i = c * M; i < (c + 1) * M && i < n; ++i) {
            for (int a = 0; a < 3; ++a) {
                double v = (double)p[a][i];
                if (v < cb[c].lo[a]) cb[c].lo[a] = v;
                if (v > cb[c].hi[a]) cb[c].hi[a] = v;
            }
            cnt[c]++;
        }
    }
    for (int64_t s = 0; s < nsc; ++s) {
        dbox_empty(&sb[s]);
        for (int k = 0; k < 8; ++k) dbox_add_box(&sb[s], &cb[8 * s + k]);
        e64[s] = dbox_extent(&sb[s], fl);
    }
    for (int64_t s = 0; s < nsc; ++s) {
        dbox r8, r64;
        dbox_empty(&r8);
        dbox_empty(&r64);
        for (int64_t t = s - 3; t < s + 5; ++t)
            if (t >= 0 && t < nsc) dbox_add_box(&r8, &sb[t]);
        for (int64_t t = s - 31; t < s + 33; ++t)
            if (t >= 0 && t < nsc) dbox_add_box(&r64, &sb[t]);
        const double e512 = dbox_extent(&r8, fl), e4096 = dbox_extent(&r64, fl);
        const double dens = log(e64[s] / L) + log((double)n) / 3.0;
        for (int k = 0; k < 8; ++k) {
            const int64_t c = 8 * s + k;
            double *x = X + c * 8;
            if (cnt[c] == 0) {
                for (int f = 0; f < 8; ++f) x[f] = 0.0;
                continue;
            }
            const double ex = dbox_side(&cb[c], 0, fl), ey = dbox_side(&cb[c], 1, fl);
            const double ez = dbox_side(&cb[c], 2, fl);
            const double e8 = dbox_extent(&cb[c], fl);
            x[0] = log(e8 / e64[s]);
            x[1] = log(e512 / e64[s]);
            x[2] = log(e4096 / e64[s]);
            x[3] = log(ex / e8);
            x[4] = log(ey / e8);
            x[5] = log(ez / e8);
            x[6] = log((double)cnt[c] / (double)M);
            x[7] = dens;
        }
    }
    free(cb);
    free(sb);
    free(cnt);
    return 0;
}

/* Targets of the learned start: y[c] = log(mean h of the real particles of
 * cluster c / e64 of its super-cluster), w[c] = 1; empty clusters y = w = 0.
 * hs in SFC-sorted order. */
void orc_mlp_targets(int64_t n, const float *hs, int cluster, const double *e64, double *y,
                     double *w)
{
    const int64_t M = cluster, scp = 8 * (int64_t)cluster;
    const int64_t ncl = 8 * ((n + scp - 1) / scp);
    for (int64_t c = 0; c < ncl; ++c) {
        double s = 0.0;
        int64_t k = 0;
        for (int64_t i = c * M; i < (c + 1) * M && i < n; ++i, ++k) s += (double)hs[i];
        y[c] = k ? log(s / (double)k / e64[c / 8]) : 0.0;
        w[c] = k ? 1.0 : 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* Smoothing lengths at exactly k gather neighbors (the centre of the h     */
/* iteration's window, which is not in the paper): for particle i, with      */
/* d2_(k) <= d2_(k+1) its k-th and (k+1)-th smallest canonical FP32 squared  */
/* distances to the other particles, h_i = sqrt((d2_(k) + d2_(k+1)) / 2) /   */
/* support, rounded once to FP32, so #{j != i : d2_ij < (support h_i)^2} = k */
/* unless distances tie within a rounding.  The k+1 nearest come from an     */
/* exact nearest-neighbor descent of the octree of the sorted keys (node     */
/* boxes in FP64, pruning only where the whole node lies beyond the current  */
/* (k+1)-th distance with a margin far above the FP32 rounding).  Inputs in  */
/* SFC-sorted order with their sorted keys; returns 0, or -1 when n <= k or  */
/* memory runs out.                                                         */
/* ------------------------------------------------------------------------ */
static double gap1(double x, double lo, double hi)
{
    return x < lo ? lo - x : (x > hi ? x - hi : 0.0);
}

static double box_gap2(const dbox *bx, const double *x, const orc_box *b)
{
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        double g = gap1(x[a], bx->lo[a], bx->hi[a]);
        if (b->periodic[a] && g > 0.0) {
            double L = (double)b->hi[a] - (double)b->lo[a];
            double g1 = gap1(x[a] - L, bx->lo[a], bx->hi[a]);
            double g2 = gap1(x[a] + L, bx->lo[a], bx->hi[a]);
            if (g1 < g) g = g1;
            if (g2 < g) g = g2;
        }
        s += g * g;
    }
    return s;
}

/* max-heap of floats: push while not full, else replace the maximum */
static void heap_offer(float *hp, int *size, int cap, float v)
{
    int i;
    if (*size < cap) {
        i = (*size)++;
        while (i > 0 && hp[(i - 1) / 2] < v) {
            hp[i] = hp[(i - 1) / 2];
            i = (i - 1) / 2;
        }
        hp[i] = v;
        return;
    }
    if (!(v < hp[0])) return;
    i = 0;
    for (;;) {
        int l = 2 * i + 1, r = l + 1, m = i;
        float big = v;
        if (l < cap && hp[l] > big) { m = l; big = hp[l]; }
        if (r < cap && hp[r] > big) { m = r; }
        if (m == i) break;
        hp[i] = hp[m];
        i = m;
    }
    hp[i] = v;
}

int orc_h_at_count(int64_t n, const float *xs, const float *ys, const float *zs,
                   const uint64_t *sorted_keys, const orc_box *b, float support, int k,
                   float *hout)
{
    if (n <= k || k < 1) return -1;
    const int bucket = 64;
    int64_t cap = 4 * n / bucket * 22 + 64;
    int32_t *level = NULL, *leaf = NULL;
    int64_t *first = NULL, *end = NULL, cnt = 0;
    for (;;) {
        level = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
        leaf = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
        first = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
        end = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
        if (!level || !leaf || !first || !end) return -1;
        cnt = orc_octree(n, sorted_keys, bucket, level, first, end, leaf, cap);
        if (cnt <= cap) break;
        free(level), free(leaf), free(first), free(end);
        cap = cnt;
    }
    int64_t *skip = (int64_t *)malloc((size_t)cnt * sizeof(int64_t));
    dbox *nb = (dbox *)malloc((size_t)cnt * sizeof(dbox));
    if (!skip || !nb) return -1;
    for (int64_t t = cnt - 1; t >= 0; --t) {
        int64_t c = t + 1;
        if (!leaf[t])
            while (c < cnt && first[c] < end[t]) c = skip[c];
        skip[t] = c;
    }
    const float *p[3] = {xs, ys, zs};
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < cnt; ++t) {
        dbox_empty(&nb[t]);
        for (int64_t i = first[t]; i < end[t]; ++i)
            for (int a = 0; a < 3; ++a) {
                double v = (double)p[a][i];
                if (v < nb[t].lo[a]) nb[t].lo[a] = v;
                if (v > nb[t].hi[a]) nb[t].hi[a] = v;
            }
    }
    int fail = 0;
#pragma omp parallel
    {
        float *hp = (float *)malloc((size_t)(k + 1) * sizeof(float));
        int64_t *stack = (int64_t *)malloc((size_t)(8 * (ORC_MAX_LEVEL + 2)) * sizeof(int64_t));
        if (!hp || !stack) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; ++i) {
            if (!hp || !stack) continue;
            const double x[3] = {(double)xs[i], (double)ys[i], (double)zs[i]};
            int size = 0, top = 0;
            stack[top++] = 0;
            while (top > 0) {
                const int64_t t = stack[--top];
                if (size == k + 1 && box_gap2(&nb[t], x, b) * (1.0 - 1e-5) > (double)hp[0])
                    continue;
                if (leaf[t]) {
                    for (int64_t j = first[t]; j < end[t]; ++j)
                        if (j != i) heap_offer(hp, &size, k + 1, dist2_32(xs, ys, zs, i, j, b));
                    continue;
                }
                /* children, pushed farthest first so the nearest is visited first */
                int64_t ch[8];
                double cd[8];
                int nc = 0;
                for (int64_t c = t + 1; c < cnt && first[c] < end[t]; c = skip[c]) {
                    double d = box_gap2(&nb[c], x, b);
                    int q = nc++;
                    while (q > 0 && cd[q - 1] < d) {
                        ch[q] = ch[q - 1];
                        cd[q] = cd[q - 1];
                        --q;
                    }
                    ch[q] = c;
                    cd[q] = d;
                }
                for (int q = 0; q < nc; ++q) stack[top++] = ch[q];
            }
            /* hp[0] = d2_(k+1); the k-th is the larger of the root's children */
            float dk1 = hp[0], dk = hp[1];
            if (k + 1 > 2 && hp[2] > dk) dk = hp[2];
            hout[i] = (float)(sqrt(0.5 * ((double)dk + (double)dk1)) / (double)support);
        }
        free(hp);
        free(stack);
    }
    free(level), free(leaf), free(first), free(end), free(skip), free(nb);
    return fail ? -1 : 0;
}
