/*
 * sj_oracle.c -- CPU oracle for the Euclidean epsilon self-join.
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark load this code.  The
 * CUDA library never includes, links or calls it, and it includes nothing
 * from the library: the two implementations share no code.
 *
 * What it computes (Gowanlock & Karsin, "GPU Accelerated Self-join for the
 * Distance Similarity Metric", Section III): for a database D of |D| points in
 * n dimensions, every ordered pair (i, j) with dist(p_i, p_j) <= epsilon,
 * where dist is the Euclidean distance.  Self-pairs (i, i) are members
 * (distance 0), and (i, j) is a member exactly when (j, i) is.
 *
 * The predicate is fixed bit-exactly (reading of Section III, see `within`):
 *     s = 0; for j in 0..n-1: t = x_i[j] - x_j[j]; s = s + t*t    (FP64, RN)
 *     member  <=>  s <= fl(eps*eps)
 * each operation rounded separately: no fused multiply-add.  This file must
 * be compiled with -ffp-contract=off (the build script does so); a pinned
 * test detects a build that contracts.
 *
 * Two evaluation strategies, both plain:
 *   - brute force over all |D|^2 ordered pairs (the definition itself);
 *   - the paper's grid (Section IV-B/C) searched as in Algorithm 1: every
 *     point visits the 3^n cells adjacent to its own (its own included),
 *     looks each one up in the sorted array B of non-empty cell ids, and
 *     compares itself with every point of each cell found.  No UNICOMP and no
 *     reduced precision: this is the simple form of the search.
 *
 * Readings where the paper is silent or inexact (each one is listed in the
 * design notes of the repository):
 *   - Section IV-B assumes epsilon divides the index range.  Here the number
 *     of cells in dimension j is floor((g_max_j - g_min_j) / w) + 1 and a
 *     point's cell coordinate is floor((x_j - g_min_j) / w), computed in FP64.
 *   - The cell length is w = eps * (1 + 2^-16) instead of eps: the few-ulp
 *     rounding of the cell computation can then never put two points within
 *     eps of each other more than one cell apart (needs fewer than 2^32
 *     cells per dimension, which the grid functions check).
 *   - The linear id is lexicographic with dimension 1 fastest,
 *     id = c_1 + |g_1| * (c_2 + |g_2| * (c_3 + ...)), as the worked example
 *     of Section IV-D implies (linear id 30 = column 2 + 7 * row 4).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

#define ORACLE_MAX_DIM 16

/* ------------------------------------------------------------------ */
/* Predicate (Section III).                                           */
/* ------------------------------------------------------------------ */

/* fl(eps * eps), the squared threshold every comparison uses. */
double sj_oracle_eps2(double eps) { return eps * eps; }

/* dist(a, b) <= eps, in the squared form fixed above.  Each product and
 * each sum is rounded on its own (the file is built without contraction). */
static int within(const double *a, const double *b, int d, double E2)
{
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        double t = a[j] - b[j];
        double t2 = t * t;
        s = s + t2;
    }
    return s <= E2;
}

int sj_oracle_within(const double *a, const double *b, int d, double eps)
{
    return within(a, b, d, sj_oracle_eps2(eps));
}

/* The squared distance exactly as `within` forms it (for tests that place
 * pairs at the threshold). */
double sj_oracle_sqdist(const double *a, const double *b, int d)
{
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        double t = a[j] - b[j];
        double t2 = t * t;
        s = s + t2;
    }
    return s;
}

/* ------------------------------------------------------------------ */
/* Brute force: the definition, O(|D|^2).                             */
/* ------------------------------------------------------------------ */

/* Writes the keys (i << 32 | j) of all members in ascending order into
 * out[0 .. min(count, cap)), returns the member count.  The loops run over
 * i then j, so the keys come out sorted. */
int64_t sj_oracle_bruteforce(const double *pts, uint64_t n, int d, double eps,
                             uint64_t *out, uint64_t cap)
{
    const double E2 = sj_oracle_eps2(eps);
    uint64_t count = 0;
    for (uint64_t i = 0; i < n; ++i)
        for (uint64_t j = 0; j < n; ++j)
            if (within(pts + i * d, pts + j * d, d, E2)) {
                if (out && count < cap)
                    out[count] = (i << 32) | j;
                ++count;
            }
    return (int64_t)count;
}

/* The two-set join R ⋈ S by the same definition: every (i, j) with point
 * i of R and point j of S within eps, keys (i << 32) | j in the order of the
 * loops (i outer), the first cap of them written to out; returns the count.
 * The self-join is the case S = R. */
int64_t sj_oracle_bruteforce2(const double *R, uint64_t nR, const double *S, uint64_t nS, int d,
                              double eps, uint64_t *out, uint64_t cap)
{
    const double E2 = sj_oracle_eps2(eps);
    uint64_t count = 0;
    for (uint64_t i = 0; i < nR; ++i)
        for (uint64_t j = 0; j < nS; ++j)
            if (within(R + i * d, S + j * d, d, E2)) {
                if (out && count < cap)
                    out[count] = (i << 32) | j;
                ++count;
            }
    return (int64_t)count;
}

/* ------------------------------------------------------------------ */
/* Grid index (Section IV-B, IV-C).                                   */
/* ------------------------------------------------------------------ */

typedef struct {
    int d;
    uint64_t n;
    double eps, E2, w;
    double gmin[ORACLE_MAX_DIM], gmax[ORACLE_MAX_DIM];
    int64_t ng[ORACLE_MAX_DIM];       /* |g_j| */
    uint64_t *cell;                   /* linear cell id of every point */
    uint32_t *A;                      /* point ids ordered by cell id */
    uint64_t *B;                      /* sorted ids of the non-empty cells */
    uint64_t *Gmin, *Gmax;            /* cell h holds A[Gmin[h] .. Gmax[h]) */
    uint64_t nG;                      /* |G| = |B| */
} grid_t;

typedef struct { uint64_t id; uint32_t pt; } cell_entry;

static int cmp_entry(const void *pa, const void *pb)
{
    const cell_entry *a = pa, *b = pb;
    if (a->id != b->id) return a->id < b->id ? -1 : 1;
    if (a->pt != b->pt) return a->pt < b->pt ? -1 : 1;
    return 0;
}

static void grid_free(grid_t *g)
{
    free(g->cell); free(g->A); free(g->B); free(g->Gmin); free(g->Gmax);
    memset(g, 0, sizeof(*g));
}

/* Cell coordinate of value x in dimension j. */
static int64_t cell_coord(const grid_t *g, int j, double x)
{
    double q = (x - g->gmin[j]) / g->w;
    int64_t c = (int64_t)floor(q);
    if (c < 0) c = 0;                       /* defensive; x >= g_min always */
    if (c > g->ng[j] - 1) c = g->ng[j] - 1;
    return c;
}

/* Builds bounds, cell counts, the linear id of every point, A, B and G.
 * Returns 0, or -1 for invalid input (non-finite value, eps <= 0, too many
 * cells), or -2 when out of memory. */
static int grid_build(grid_t *g, const double *pts, uint64_t n, int d, double eps)
{
    memset(g, 0, sizeof(*g));
    if (n == 0 || d < 1 || d > ORACLE_MAX_DIM || !(eps > 0.0) || !isfinite(eps))
        return -1;
    if (n >= ((uint64_t)1 << 32)) return -1;
    g->d = d; g->n = n; g->eps = eps; g->E2 = sj_oracle_eps2(eps);
    g->w = eps * (1.0 + ldexp(1.0, -16));
    for (int j = 0; j < d; ++j) { g->gmin[j] = INFINITY; g->gmax[j] = -INFINITY; }
    for (uint64_t i = 0; i < n; ++i)
        for (int j = 0; j < d; ++j) {
            double x = pts[i * d + j];
            if (!isfinite(x)) return -1;
            if (x < g->gmin[j]) g->gmin[j] = x;
            if (x > g->gmax[j]) g->gmax[j] = x;
        }
    /* Section IV-B: the index range is [min - eps, max + eps]. */
    double total = 1.0;
    for (int j = 0; j < d; ++j) {
        g->gmin[j] = g->gmin[j] - eps;
        g->gmax[j] = g->gmax[j] + eps;
        double cells = floor((g->gmax[j] - g->gmin[j]) / g->w) + 1.0;
        if (!(cells < 4294967296.0)) return -1;
        g->ng[j] = (int64_t)cells;
        total *= cells;
    }
    if (!(total < 9.2e18)) return -1;       /* linear ids must fit in 63 bits */

    g->cell = malloc(n * sizeof(uint64_t));
    g->A = malloc(n * sizeof(uint32_t));
    cell_entry *e = malloc(n * sizeof(cell_entry));
    if (!g->cell || !g->A || !e) { free(e); grid_free(g); return -2; }
    for (uint64_t i = 0; i < n; ++i) {
        /* linear id, dimension 1 fastest */
        uint64_t id = 0;
        for (int j = d - 1; j >= 0; --j)
            id = id * (uint64_t)g->ng[j] + (uint64_t)cell_coord(g, j, pts[i * d + j]);
        g->cell[i] = id;
        e[i].id = id; e[i].pt = (uint32_t)i;
    }
    qsort(e, n, sizeof(cell_entry), cmp_entry);
    uint64_t nG = 0;
    for (uint64_t i = 0; i < n; ++i)
        if (i == 0 || e[i].id != e[i - 1].id) ++nG;
    g->B = malloc(nG * sizeof(uint64_t));
    g->Gmin = malloc(nG * sizeof(uint64_t));
    g->Gmax = malloc(nG * sizeof(uint64_t));
    if (!g->B || !g->Gmin || !g->Gmax) { free(e); grid_free(g); return -2; }
    uint64_t h = 0;
    for (uint64_t i = 0; i < n; ++i) {
        g->A[i] = e[i].pt;
        if (i == 0 || e[i].id != e[i - 1].id) {
            g->B[h] = e[i].id; g->Gmin[h] = i;
            if (h > 0) g->Gmax[h - 1] = i;
            ++h;
        }
    }
    g->Gmax[nG - 1] = n;
    g->nG = nG;
    free(e);
    return 0;
}

/* Position of linear id `id` in B, or -1 when that cell is empty. */
static int64_t find_cell(const grid_t *g, uint64_t id)
{
    uint64_t lo = 0, hi = g->nG;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (g->B[mid] < id) lo = mid + 1; else hi = mid;
    }
    return (lo < g->nG && g->B[lo] == id) ? (int64_t)lo : -1;
}

/* Exposes the grid of Section IV-B for tests: |g_j| for each dimension and
 * the linear cell id of each point.  Returns 0 or a negative error. */
int sj_oracle_grid_cells(const double *pts, uint64_t n, int d, double eps,
                         int64_t *ng_out, uint64_t *cell_out)
{
    grid_t g;
    int rc = grid_build(&g, pts, n, d, eps);
    if (rc) return rc;
    for (int j = 0; j < d; ++j) ng_out[j] = g.ng[j];
    if (cell_out) memcpy(cell_out, g.cell, n * sizeof(uint64_t));
    grid_free(&g);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Algorithm 1 on the CPU: each query point searches its 3^n adjacent */
/* cells (own cell included) and refines every candidate.             */
/* ------------------------------------------------------------------ */

typedef struct { uint32_t *v; uint64_t len, cap; } vec32;

static int vec_push(vec32 *a, uint32_t x)
{
    if (a->len == a->cap) {
        uint64_t nc = a->cap ? 2 * a->cap : 64;
        uint32_t *nv = realloc(a->v, nc * sizeof(uint32_t));
        if (!nv) return -1;
        a->v = nv; a->cap = nc;
    }
    a->v[a->len++] = x;
    return 0;
}

static int cmp_u32(const void *pa, const void *pb)
{
    uint32_t a = *(const uint32_t *)pa, b = *(const uint32_t *)pb;
    return (a > b) - (a < b);
}

/* Appends to `out` the ids j of all members (q, j), ascending. */
static int neighbors_of(const grid_t *g, const double *pts, uint32_t q, vec32 *out)
{
    const int d = g->d;
    const double *p = pts + (uint64_t)q * d;
    int64_t c[ORACLE_MAX_DIM], off[ORACLE_MAX_DIM];
    for (int j = 0; j < d; ++j) { c[j] = cell_coord(g, j, p[j]); off[j] = -1; }
    uint64_t start = out->len;
    for (;;) {
        /* adjacent cell c + off, skipped when outside the grid */
        int inside = 1;
        uint64_t id = 0;
        for (int j = d - 1; j >= 0; --j) {
            int64_t b = c[j] + off[j];
            if (b < 0 || b >= g->ng[j]) { inside = 0; break; }
            id = id * (uint64_t)g->ng[j] + (uint64_t)b;
        }
        if (inside) {
            int64_t h = find_cell(g, id);
            if (h >= 0)
                for (uint64_t k = g->Gmin[h]; k < g->Gmax[h]; ++k) {
                    uint32_t cand = g->A[k];
                    if (within(p, pts + (uint64_t)cand * d, d, g->E2))
                        if (vec_push(out, cand)) return -2;
                }
        }
        /* next offset vector in {-1, 0, 1}^n */
        int j = 0;
        while (j < d && off[j] == 1) { off[j] = -1; ++j; }
        if (j == d) break;
        ++off[j];
    }
    qsort(out->v + start, out->len - start, sizeof(uint32_t), cmp_u32);
    return 0;
}

/* Work shared by the threads of one oracle call. */
typedef struct {
    const grid_t *g;
    const double *pts;
    const uint32_t *queries;   /* NULL: all points in order */
    uint64_t q0, q1;           /* this thread's slice of the query list */
    int mode;                  /* 0 keys, 1 digest, 2 neighbour lists */
    vec32 nb;                  /* mode 0/2: neighbour ids, query order */
    uint64_t *lens;            /* mode 0/2: neighbours per query of the slice */
    uint32_t *degree;          /* mode 1: optional, indexed by point id */
    uint64_t count, hash;      /* mode 1 */
    int rc;
} job_t;

/* splitmix64 finaliser, used for the order-independent pair hash. */
static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

uint64_t sj_oracle_mix64(uint64_t z) { return mix64(z); }

static void *run_job(void *arg)
{
    job_t *jb = arg;
    vec32 tmp = {0};
    for (uint64_t k = jb->q0; k < jb->q1; ++k) {
        uint32_t q = jb->queries ? jb->queries[k] : (uint32_t)k;
        vec32 *dst = (jb->mode == 1) ? &tmp : &jb->nb;
        uint64_t before = dst->len;
        if (neighbors_of(jb->g, jb->pts, q, dst)) { jb->rc = -2; break; }
        uint64_t m = dst->len - before;
        if (jb->mode == 1) {
            for (uint64_t t = 0; t < m; ++t)
                jb->hash += mix64(((uint64_t)q << 32) | tmp.v[t]);
            jb->count += m;
            if (jb->degree) jb->degree[q] = (uint32_t)m;
            tmp.len = 0;
        } else {
            jb->lens[k - jb->q0] = m;
        }
    }
    free(tmp.v);
    return NULL;
}

/* Runs the grid search for a list of queries on `nthreads` threads, each
 * taking a contiguous slice of the list. */
static int run_queries(const grid_t *g, const double *pts, const uint32_t *queries,
                       uint64_t nq, int nthreads, int mode, uint32_t *degree,
                       job_t **jobs_out)
{
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > nq) nthreads = nq ? (int)nq : 1;
    job_t *jobs = calloc((size_t)nthreads, sizeof(job_t));
    pthread_t *th = calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -2; }
    for (int t = 0; t < nthreads; ++t) {
        job_t *jb = &jobs[t];
        jb->g = g; jb->pts = pts; jb->queries = queries; jb->mode = mode;
        jb->degree = degree;
        jb->q0 = nq * (uint64_t)t / nthreads;
        jb->q1 = nq * (uint64_t)(t + 1) / nthreads;
        if (mode != 1) {
            jb->lens = calloc(jb->q1 - jb->q0 + 1, sizeof(uint64_t));
            if (!jb->lens) { jb->rc = -2; }
        }
    }
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        if (jobs[t].rc) break;
        if (pthread_create(&th[t], NULL, run_job, &jobs[t])) { jobs[t].rc = -2; break; }
        ++started;
    }
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    free(th);
    int rc = 0;
    for (int t = 0; t < nthreads; ++t) if (jobs[t].rc) rc = jobs[t].rc;
    if (started < nthreads && !rc) rc = -2;
    *jobs_out = jobs;
    return rc ? rc : nthreads;
}

static void free_jobs(job_t *jobs, int nj)
{
    for (int t = 0; t < nj; ++t) { free(jobs[t].nb.v); free(jobs[t].lens); }
    free(jobs);
}

/* All members as ascending keys (i << 32 | j) via the grid search.
 * Writes min(count, cap) keys, returns the count or a negative error. */
int64_t sj_oracle_grid_join(const double *pts, uint64_t n, int d, double eps,
                            int nthreads, uint64_t *out, uint64_t cap)
{
    grid_t g;
    int rc = grid_build(&g, pts, n, d, eps);
    if (rc) return rc;
    job_t *jobs = NULL;
    int nj = run_queries(&g, pts, NULL, n, nthreads, 0, NULL, &jobs);
    if (nj < 0) { if (jobs) free_jobs(jobs, nthreads < 1 ? 1 : nthreads); grid_free(&g); return nj; }
    uint64_t count = 0;
    for (int t = 0; t < nj; ++t) {
        job_t *jb = &jobs[t];
        uint64_t pos = 0;
        for (uint64_t k = jb->q0; k < jb->q1; ++k) {
            uint64_t m = jb->lens[k - jb->q0];
            for (uint64_t r = 0; r < m; ++r) {
                if (out && count < cap) out[count] = (k << 32) | jb->nb.v[pos + r];
                ++count;
            }
            pos += m;
        }
    }
    free_jobs(jobs, nj);
    grid_free(&g);
    return (int64_t)count;
}

/* Count, per-point degree (may be NULL) and order-independent hash
 * H = sum over members of mix64(i << 32 | j) mod 2^64, via the grid search,
 * without materialising the pairs.  Returns 0 or a negative error. */
int sj_oracle_grid_digest(const double *pts, uint64_t n, int d, double eps,
                          int nthreads, uint32_t *degree, uint64_t *count,
                          uint64_t *hash)
{
    grid_t g;
    int rc = grid_build(&g, pts, n, d, eps);
    if (rc) return rc;
    job_t *jobs = NULL;
    int nj = run_queries(&g, pts, NULL, n, nthreads, 1, degree, &jobs);
    if (nj < 0) { if (jobs) free_jobs(jobs, nthreads < 1 ? 1 : nthreads); grid_free(&g); return nj; }
    uint64_t c = 0, h = 0;
    for (int t = 0; t < nj; ++t) { c += jobs[t].count; h += jobs[t].hash; }
    free_jobs(jobs, nj);
    grid_free(&g);
    *count = c; *hash = h;
    return 0;
}

/* Neighbour lists of the listed query points only: for query k,
 * nbrs[offsets[k] .. offsets[k+1]) are the ids j of the members
 * (queries[k], j), ascending.  offsets has nq + 1 entries.  Writes at most
 * cap ids; returns the total number of ids or a negative error. */
int64_t sj_oracle_grid_neighbors(const double *pts, uint64_t n, int d, double eps,
                                 int nthreads, const uint32_t *queries, uint64_t nq,
                                 uint64_t *offsets, uint32_t *nbrs, uint64_t cap)
{
    for (uint64_t k = 0; k < nq; ++k) if (queries[k] >= n) return -1;
    grid_t g;
    int rc = grid_build(&g, pts, n, d, eps);
    if (rc) return rc;
    job_t *jobs = NULL;
    int nj = run_queries(&g, pts, queries, nq, nthreads, 2, NULL, &jobs);
    if (nj < 0) { if (jobs) free_jobs(jobs, nthreads < 1 ? 1 : nthreads); grid_free(&g); return nj; }
    uint64_t total = 0;
    offsets[0] = 0;
    for (int t = 0; t < nj; ++t) {
        job_t *jb = &jobs[t];
        uint64_t pos = 0;
        for (uint64_t k = jb->q0; k < jb->q1; ++k) {
            uint64_t m = jb->lens[k - jb->q0];
            for (uint64_t r = 0; r < m; ++r) {
                if (nbrs && total + r < cap) nbrs[total + r] = jb->nb.v[pos + r];
            }
            pos += m;
            total += m;
            offsets[k + 1] = total;
        }
    }
    free_jobs(jobs, nj);
    grid_free(&g);
    return (int64_t)total;
}
