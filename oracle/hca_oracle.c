/*
 * CPU oracle for HCA-DBSCAN (Mathur, Mehta, Singh; arXiv 1912.00323).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent, plain, slow reference that the
 * CUDA path is checked against.  Only the test-suite, the smoke check of the repository
 * entry file and the CPU-baseline leg of the benchmark load it.  It shares no code, header,
 * table or constant with the CUDA library, and the CUDA library never calls it.
 *
 * Arithmetic.  Every floating-point quantity is an IEEE double and the file is compiled
 * with -ffp-contract=off, so each expression rounds exactly as written (no fused
 * multiply-add).  The neighbourhood predicate of the whole oracle is
 *
 *     le(p, q)  :=  ( s = 0;  for i = 0..d-1: t = x_p[i] - x_q[i];  s = s + t*t )  <=  eps*eps
 *
 * with every operation rounded to double in that order, and eps*eps rounded once.  This is
 * the squared form of dist(p, q) <= eps of Definition 1 (supplement, "The DBSCAN
 * Algorithm"); for coordinates on a binary lattice the sums near eps^2 are exact and the
 * two forms agree.
 *
 * Canonical labels (the paper numbers clusters in traversal order, Algorithm 4; a fixed
 * rule is needed to compare two implementations element by element):
 *   - a core point's label is the smallest input index of a core point in its cluster;
 *   - a non-core point that lies within eps of a core point takes the smallest label among
 *     the clusters of its core neighbours (Definition 5 allows several; we fix the minimum);
 *   - every other point is noise, label -1.
 *
 * Entry points (all return 0 on success, a negative value on bad arguments or no memory):
 *   hca_oracle_bruteforce   DBSCAN straight from Definitions 1-5, O(n^2).
 *   hca_oracle_grid         HCA-DBSCAN with DBSCAN semantics: Algorithm 1 (hypercubes of
 *                           side eps/sqrt(d)), Algorithm 2 (representative points),
 *                           Algorithm 3 / 4 (merging neighbouring hypercubes), with MINPTS
 *                           handled by dense hypercubes and exact counts.
 *   hca_oracle_grid_mt      the same on several host threads (same result).
 *   hca_oracle_literal      Algorithms 2-4 as printed: representative points only, strict
 *                           "<", no MINPTS.  An ablation, not an authority.
 *   hca_oracle_stencil_count  number of neighbour hypercubes under three rules (Sec. 2).
 *   hca_oracle_grid_cells   hypercube coordinates of each point (Algorithm 1).
 *   hca_oracle_rep_dirs     the 3^d - 1 representative directions (Sec. 2).
 */
#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)
#define ORACLE_ERANGE (-4)

/* ------------------------------------------------------------------------------------- */
/* The predicate of Definition 1, squared, in double precision.                           */
/* ------------------------------------------------------------------------------------- */

static int le_eps(const double *p, const double *q, int d, double eps2)
{
    double s = 0.0;
    for (int i = 0; i < d; ++i) {
        double t = p[i] - q[i];
        s = s + t * t;
        /* every term is >= 0 and rounding is monotone, so the partial sum never decreases:
           once above eps^2 the full sum is too */
        if (s > eps2) return 0;
    }
    return s <= eps2;
}

static int check_args(const double *X, int64_t n, int d, double eps, int min_pts,
                      const int32_t *labels)
{
    if (n < 0 || d < 1 || d > 64 || min_pts < 1) return ORACLE_EINVAL;
    if (!(eps > 0.0) || !isfinite(eps)) return ORACLE_EINVAL;
    if (n > 0 && (X == NULL || labels == NULL)) return ORACLE_EINVAL;
    if (n >= ((int64_t)1 << 31)) return ORACLE_EINVAL;
    for (int64_t k = 0; k < n * (int64_t)d; ++k)
        if (!isfinite(X[k])) return ORACLE_EINVAL;
    return 0;
}

/* ------------------------------------------------------------------------------------- */
/* Brute force: Definitions 1-5.                                                          */
/* ------------------------------------------------------------------------------------- */

typedef struct {
    const double *X;
    int64_t n;
    int d;
    double eps2;
    int64_t lo, hi;
    int32_t *count;        /* |N_eps(p)|, Definition 1 (p itself included) */
    const uint8_t *core;   /* border pass input */
    int32_t *labels;       /* border pass output */
} bf_job;

static void *bf_count_worker(void *arg)
{
    bf_job *j = (bf_job *)arg;
    for (int64_t p = j->lo; p < j->hi; ++p) {
        int32_t c = 0;
        for (int64_t q = 0; q < j->n; ++q)
            c += le_eps(j->X + p * j->d, j->X + q * j->d, j->d, j->eps2);
        j->count[p] = c;
    }
    return NULL;
}

static void *bf_border_worker(void *arg)
{
    bf_job *j = (bf_job *)arg;
    for (int64_t p = j->lo; p < j->hi; ++p) {
        if (j->core[p]) continue;
        int32_t best = -1;
        for (int64_t q = 0; q < j->n; ++q) {
            if (!j->core[q]) continue;
            if (!le_eps(j->X + p * j->d, j->X + q * j->d, j->d, j->eps2)) continue;
            int32_t l = j->labels[q];
            if (best < 0 || l < best) best = l;
        }
        j->labels[p] = best;
    }
    return NULL;
}

static void run_parallel(void *(*fn)(void *), bf_job *proto, int threads)
{
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if ((int64_t)threads > proto->n) threads = proto->n > 0 ? (int)proto->n : 1;
    bf_job jobs[256];
    pthread_t tid[256];
    int started[256];
    for (int t = 0; t < threads; ++t) {
        jobs[t] = *proto;
        jobs[t].lo = proto->n * t / threads;
        jobs[t].hi = proto->n * (t + 1) / threads;
        started[t] = threads > 1 && pthread_create(&tid[t], NULL, fn, &jobs[t]) == 0;
        if (!started[t]) fn(&jobs[t]);
    }
    for (int t = 0; t < threads; ++t)
        if (started[t]) pthread_join(tid[t], NULL);
}

/*
 * DBSCAN from Definitions 1-5 of the supplement:
 *   1. |N_eps(p)| over every q, p included (Definition 1);
 *   2. core(p) iff |N_eps(p)| >= MINPTS (Definition 2, condition 2);
 *   3. clusters are the connected components of core points under le (Definitions 3-5):
 *      a breadth-first search started from each not yet labelled core point in increasing
 *      index order, so the start point is the smallest index of its component;
 *   4. a non-core point takes the smallest label among its core neighbours, else -1.
 * core_out (nullable) receives the core flags.
 */
int hca_oracle_bruteforce(const double *X, int64_t n, int32_t d, double eps, int32_t min_pts,
                          int32_t threads, int32_t *labels, uint8_t *core_out)
{
    int rc = check_args(X, n, d, eps, min_pts, labels);
    if (rc) return rc;
    if (n == 0) return 0;
    const double eps2 = eps * eps;
    int32_t *count = (int32_t *)malloc(sizeof(int32_t) * n);
    uint8_t *core = (uint8_t *)malloc(n);
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * n);
    if (!count || !core || !queue) {
        free(count); free(core); free(queue);
        return ORACLE_ENOMEM;
    }
    bf_job job = {X, n, d, eps2, 0, n, count, core, labels};
    run_parallel(bf_count_worker, &job, threads);
    for (int64_t p = 0; p < n; ++p) {
        core[p] = count[p] >= min_pts;
        labels[p] = -1;
    }
    for (int64_t p = 0; p < n; ++p) {
        if (!core[p] || labels[p] >= 0) continue;
        int64_t head = 0, tail = 0;
        labels[p] = (int32_t)p;
        queue[tail++] = p;
        while (head < tail) {
            int64_t u = queue[head++];
            for (int64_t q = 0; q < n; ++q) {
                if (!core[q] || labels[q] >= 0) continue;
                if (le_eps(X + u * d, X + q * d, d, eps2)) {
                    labels[q] = (int32_t)p;
                    queue[tail++] = q;
                }
            }
        }
    }
    run_parallel(bf_border_worker, &job, threads);
    if (core_out) memcpy(core_out, core, n);
    free(count); free(core); free(queue);
    return 0;
}

/* ------------------------------------------------------------------------------------- */
/* Shared pieces of the hypercube oracles.                                                 */
/* ------------------------------------------------------------------------------------- */

/* Lexicographic order of integer coordinate rows, ties broken by point index: the
 * pre-sort of Sec. 2 (leading dimension first, secondary dimensions break ties), applied
 * to hypercube coordinates. */
typedef struct {
    const int64_t *cc; /* n x d cell coordinates */
    int d;
} sort_ctx;

static int cmp_rows(const sort_ctx *c, int64_t a, int64_t b)
{
    const int64_t *ra = c->cc + a * c->d, *rb = c->cc + b * c->d;
    for (int i = 0; i < c->d; ++i) {
        if (ra[i] < rb[i]) return -1;
        if (ra[i] > rb[i]) return 1;
    }
    return (a < b) ? -1 : (a > b);
}

static void merge_sort_idx(const sort_ctx *c, int64_t *a, int64_t *tmp, int64_t n)
{
    if (n < 2) return;
    int64_t h = n / 2;
    merge_sort_idx(c, a, tmp, h);
    merge_sort_idx(c, a + h, tmp, n - h);
    int64_t i = 0, j = h, k = 0;
    while (i < h && j < n) tmp[k++] = (cmp_rows(c, a[i], a[j]) <= 0) ? a[i++] : a[j++];
    while (i < h) tmp[k++] = a[i++];
    while (j < n) tmp[k++] = a[j++];
    memcpy(a, tmp, sizeof(int64_t) * n);
}

/* Union-find over hypercube ids, root = smallest id. */
static int64_t uf_find(int64_t *parent, int64_t x)
{
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

static void uf_union(int64_t *parent, int64_t a, int64_t b)
{
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a == b) return;
    if (a < b) parent[b] = a; else parent[a] = b;
}

/* Hypercube grid of Algorithm 1: origin shifted to the per-dimension minimum (Sec. 2,
 * origin shift), bands of width `side` from there, cell coordinate = band index. */
typedef struct {
    int64_t n;
    int d;
    double side;
    double *origin;     /* d */
    int64_t *cc;        /* n x d cell coordinates of each point */
    int64_t *order;     /* points sorted by (cell, index) */
    int64_t ncell;
    int64_t *cell_first;  /* ncell + 1 offsets into order */
    int64_t *cell_of;     /* n: cell id of each point */
} grid_t;

static void grid_free(grid_t *g)
{
    free(g->origin); free(g->cc); free(g->order); free(g->cell_first); free(g->cell_of);
    memset(g, 0, sizeof(*g));
}

static int grid_build(grid_t *g, const double *X, int64_t n, int d, double side)
{
    memset(g, 0, sizeof(*g));
    g->n = n; g->d = d; g->side = side;
    g->origin = (double *)malloc(sizeof(double) * d);
    g->cc = (int64_t *)malloc(sizeof(int64_t) * n * d);
    g->order = (int64_t *)malloc(sizeof(int64_t) * n);
    g->cell_first = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
    g->cell_of = (int64_t *)malloc(sizeof(int64_t) * n);
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * n);
    if (!g->origin || !g->cc || !g->order || !g->cell_first || !g->cell_of || !tmp) {
        free(tmp); grid_free(g);
        return ORACLE_ENOMEM;
    }
    for (int i = 0; i < d; ++i) {
        double m = X[i];
        for (int64_t p = 1; p < n; ++p) if (X[p * d + i] < m) m = X[p * d + i];
        g->origin[i] = m;
    }
    for (int64_t p = 0; p < n; ++p) {
        for (int i = 0; i < d; ++i) {
            double t = floor((X[p * d + i] - g->origin[i]) / side);
            if (!(t < 9.0e15)) { free(tmp); grid_free(g); return ORACLE_ERANGE; }
            g->cc[p * d + i] = (int64_t)t;
        }
        g->order[p] = p;
    }
    sort_ctx c = {g->cc, d};
    merge_sort_idx(&c, g->order, tmp, n);
    free(tmp);
    g->ncell = 0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = g->order[k];
        if (k == 0 || memcmp(g->cc + p * d, g->cc + g->order[k - 1] * d, sizeof(int64_t) * d) != 0)
            g->cell_first[g->ncell++] = k;
        g->cell_of[p] = g->ncell - 1;
    }
    g->cell_first[g->ncell] = n;
    return 0;
}

/* Cell id with the given coordinates, or -1: binary search over the sorted cells
 * (the O(log n) neighbour lookup of the complexity analysis). */
static int64_t grid_lookup(const grid_t *g, const int64_t *coord)
{
    int64_t lo = 0, hi = g->ncell - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        const int64_t *r = g->cc + g->order[g->cell_first[mid]] * g->d;
        int c = 0;
        for (int i = 0; i < g->d && c == 0; ++i) c = (r[i] < coord[i]) ? -1 : (r[i] > coord[i]);
        if (c == 0) return mid;
        if (c < 0) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

static const int64_t *grid_cell_coord(const grid_t *g, int64_t cell)
{
    return g->cc + g->order[g->cell_first[cell]] * g->d;
}

/* Enumerate offsets delta in [-R, R]^d, delta != 0, into `out` (rows of d int64).
 * rule 0: the paper's count (2*ceil(sqrt(d))+1)^d - (C+1), C = corner cubes whose every
 *         |delta_i| equals ceil(sqrt(d))                    (Sec. 2, "Depth First Search")
 * rule 1: the exact geometric rule for side eps/sqrt(d) with strict "<":
 *         sum_i max(|delta_i|-1, 0)^2 < d                   (Sec. 2 "Layering": a cube can
 *         hold a point within eps only if the gap between the cubes is below eps)
 * rule 2: the conservative rule the oracle uses, for side `side` and reach eps:
 *         sum_i (max(|delta_i|-1, 0) * side)^2 <= eps^2 * (1 + 1e-6)
 * Returns the count; writes rows only when out != NULL. */
static int64_t enum_offsets(int d, int rule, double side, double eps, int64_t *out)
{
    int R;
    if (rule == 0) {
        R = (int)ceil(sqrt((double)d));
    } else if (rule == 1) {
        R = 1;
        while ((double)(R * R) < (double)d) ++R; /* (R-1)^2 < d */
    } else {
        R = 1;
        while ((double)R * side * (double)R * side <= eps * eps * (1.0 + 1e-6)) ++R;
    }
    int64_t count = 0;
    int64_t *delta = (int64_t *)calloc(d, sizeof(int64_t));
    if (!delta) return -1;
    for (int i = 0; i < d; ++i) delta[i] = -R;
    for (;;) {
        int zero = 1, corner = 1;
        double gap2 = 0.0;
        int64_t gapi = 0;
        for (int i = 0; i < d; ++i) {
            int64_t a = delta[i] < 0 ? -delta[i] : delta[i];
            if (a != 0) zero = 0;
            if (a != R) corner = 0;
            int64_t g = a > 1 ? a - 1 : 0;
            gapi += g * g;
            gap2 += ((double)g * side) * ((double)g * side);
        }
        int keep;
        if (zero) keep = 0;
        else if (rule == 0) keep = !corner;
        else if (rule == 1) keep = gapi < d;
        else keep = gap2 <= eps * eps * (1.0 + 1e-6);
        if (keep) {
            if (out) memcpy(out + count * d, delta, sizeof(int64_t) * d);
            ++count;
        }
        int i = 0;
        while (i < d && delta[i] == R) delta[i++] = -R;
        if (i == d) break;
        ++delta[i];
    }
    free(delta);
    return count;
}

int64_t hca_oracle_stencil_count(int32_t d, int32_t rule, double side, double eps)
{
    if (d < 1 || d > 12 || rule < 0 || rule > 2) return -1;
    return enum_offsets(d, rule, side, eps, NULL);
}

/* The 3^d - 1 representative directions of Sec. 2: every delta in {-1,0,1}^d except 0,
 * in the order delta_0 fastest.  Returns the count; rows written when out != NULL. */
int64_t hca_oracle_rep_dirs(int32_t d, int8_t *out)
{
    if (d < 1 || d > 12) return -1;
    int64_t total = 1;
    for (int i = 0; i < d; ++i) total *= 3;
    int64_t k = 0;
    for (int64_t code = 0; code < total; ++code) {
        int64_t c = code;
        int zero = 1;
        int8_t row[12];
        for (int i = 0; i < d; ++i) {
            row[i] = (int8_t)(c % 3) - 1;
            if (row[i]) zero = 0;
            c /= 3;
        }
        if (zero) continue;
        if (out) memcpy(out + k * d, row, d);
        ++k;
    }
    return k;
}

/* Hypercube side of Algorithm 1: space diagonal eps (Sec. 2, "Overlaying Hypercubes"),
 * i.e. eps/sqrt(d), shrunk by a relative 2^-20 so that rounding in the band computation
 * can never give a hypercube a diagonal above eps. */
static double oracle_side(double eps, int d)
{
    return eps / sqrt((double)d) * (1.0 - 1.0 / 1048576.0);
}

int hca_oracle_grid_cells(const double *X, int64_t n, int32_t d, double eps, int64_t *cells_out)
{
    if (n < 0 || d < 1 || d > 64 || !(eps > 0.0) || (n > 0 && (!X || !cells_out)))
        return ORACLE_EINVAL;
    if (n == 0) return 0;
    grid_t g;
    int rc = grid_build(&g, X, n, d, oracle_side(eps, d));
    if (rc) return rc;
    memcpy(cells_out, g.cc, sizeof(int64_t) * n * d);
    grid_free(&g);
    return 0;
}

/* ------------------------------------------------------------------------------------- */
/* Representative points, Algorithm 2.                                                      */
/* ------------------------------------------------------------------------------------- */

/* Squared distance from point x (in cell c) to the ideal position of direction delta: the
 * face, edge or corner of the cube in that direction (Sec. 2, "ideal position ... on the
 * edge").  Only the dimensions with delta_i != 0 constrain the ideal position. */
static double ideal_dist2(const double *x, const int64_t *c, const int8_t *delta,
                          const double *origin, double side, int d)
{
    double s = 0.0;
    for (int i = 0; i < d; ++i) {
        if (delta[i] == 0) continue;
        double b = origin[i] + (double)(c[i] + (delta[i] > 0 ? 1 : 0)) * side;
        double t = b - x[i];
        s = s + t * t;
    }
    return s;
}

/* For every cell and direction, the representative point (an input index or -1) chosen by
 * Algorithm 2: the first eligible point initialises every direction, a later point replaces
 * the representative only if strictly closer to the ideal position.  Eligible points are
 * taken in increasing input index; `eligible` == NULL means every point. */
static int64_t *compute_reps(const grid_t *g, const double *X, const uint8_t *eligible,
                             const int8_t *dirs, int64_t ndir)
{
    int d = g->d;
    int64_t *rep = (int64_t *)malloc(sizeof(int64_t) * (g->ncell * ndir + 1));
    if (!rep) return NULL;
    for (int64_t k = 0; k < g->ncell * ndir; ++k) rep[k] = -1;
    for (int64_t cell = 0; cell < g->ncell; ++cell) {
        /* order[] lists a cell's points in increasing input index (ties of the sort) */
        for (int64_t k = g->cell_first[cell]; k < g->cell_first[cell + 1]; ++k) {
            int64_t p = g->order[k];
            if (eligible && !eligible[p]) continue;
            const int64_t *c = g->cc + p * d;
            for (int64_t r = 0; r < ndir; ++r) {
                int64_t *slot = &rep[cell * ndir + r];
                if (*slot < 0) { *slot = p; continue; }
                double a = ideal_dist2(X + p * d, c, dirs + r * d, g->origin, g->side, d);
                double b = ideal_dist2(X + *slot * d, c, dirs + r * d, g->origin, g->side, d);
                if (a < b) *slot = p;
            }
        }
    }
    return rep;
}

/* Index of direction sign(delta) in the table of hca_oracle_rep_dirs (delta_0 fastest). */
static int64_t dir_index(const int64_t *delta, int d)
{
    int64_t code = 0, mul = 1;
    for (int i = 0; i < d; ++i) {
        int s = delta[i] > 0 ? 1 : (delta[i] < 0 ? -1 : 0);
        code += (int64_t)(s + 1) * mul;
        mul *= 3;
    }
    int64_t zero = (mul - 1) / 2; /* the all-zero code is skipped in the table */
    return code < zero ? code : code - 1;
}

/* ------------------------------------------------------------------------------------- */
/* HCA-DBSCAN with DBSCAN semantics.                                                        */
/* ------------------------------------------------------------------------------------- */

#define STENCIL_MAX_D 4

/* Everything the threads of one hca_oracle_grid call share.  Each phase hands out its items
 * (cells or points) in chunks from the counter `next`; a thread writes only the slots of the
 * items it took (core flags in the count phase, labels in the border phase), so the threads
 * never write the same memory. */
typedef struct {
    const double *X;
    int64_t n;
    int d;
    double eps2;
    int min_pts;
    const grid_t *g;
    int use_stencil;
    const int64_t *offs;        /* stencil offsets, noff rows of d (d <= 4) */
    int64_t noff;
    const int64_t *xorder;      /* points sorted by x_0, ties by index (d > 4) */
    const int64_t *pos;         /* position of each point in xorder */
    double win;                 /* window of the leading-dimension sweep */
    const double *x0s;          /* x_0 of the point at each position of xorder */
    const double *x1s;          /* x_1 of the point at each position of xorder (NULL if d = 1) */
    const int64_t *cell_s;      /* cube of the point at each position of xorder */
    uint8_t *core_s;            /* core flag of the point at each position (after the counts) */
    uint8_t *core;              /* count phase output */
    const uint8_t *cell_core;   /* cells holding a core point */
    const int64_t *rep;         /* representative points, ndir per cell (stencil path) */
    int64_t ndir;
    const int64_t *cell_label;  /* border phase: canonical id of each cell's cluster, or INT64_MAX */
    int32_t *labels;            /* border phase output */
    int64_t items, chunk;       /* the current phase's items and chunk size */
    _Atomic int64_t next;       /* next unclaimed item of the current phase */
} grid_ctx;

typedef struct {
    grid_ctx *c;
    int rc;
    int64_t *edges;             /* merge phase: cell pairs joined by this thread's union-find */
    int64_t nedge, cap;
} grid_job;

static int claim(grid_ctx *c, int64_t *lo, int64_t *hi)
{
    int64_t a = atomic_fetch_add(&c->next, c->chunk);
    if (a >= c->items) return 0;
    *lo = a;
    *hi = a + c->chunk < c->items ? a + c->chunk : c->items;
    return 1;
}

/* Run fn on `threads` threads (the calling thread included) over c->items items. */
static void run_phase(void *(*fn)(void *), grid_ctx *c, grid_job *jobs, int threads, int64_t items,
                      int64_t chunk)
{
    c->items = items;
    c->chunk = chunk < 1 ? 1 : chunk;
    atomic_store(&c->next, 0);
    pthread_t tid[256];
    int started[256];
    for (int t = 1; t < threads; ++t) started[t] = pthread_create(&tid[t], NULL, fn, &jobs[t]) == 0;
    fn(&jobs[0]);
    for (int t = 1; t < threads; ++t) {
        if (started[t]) pthread_join(tid[t], NULL);
        else fn(&jobs[t]); /* the counter is shared, so a thread that failed to start just runs late */
    }
}

/* MINPTS (Definition 2): a cube with at least MINPTS points is dense, and every point in it
 * is core; a point of another cube is counted exactly over its own cube (all within eps, the
 * diagonal is at most eps) and the neighbour cubes.  The count stops once it reaches MINPTS:
 * core(p) needs only |N_eps(p)| >= MINPTS. */
static void *grid_count_worker(void *arg)
{
    grid_job *j = (grid_job *)arg;
    grid_ctx *c = j->c;
    const grid_t *g = c->g;
    const int d = c->d;
    const double *X = c->X;
    int64_t coord[STENCIL_MAX_D];
    int64_t lo, hi;
    while (claim(c, &lo, &hi)) {
        for (int64_t cell = lo; cell < hi; ++cell) {
            int64_t f = g->cell_first[cell], l = g->cell_first[cell + 1];
            int dense = (l - f) >= c->min_pts;
            for (int64_t k = f; k < l; ++k) {
                int64_t p = g->order[k];
                if (dense) { c->core[p] = 1; continue; }
                int64_t cnt = l - f; /* own cube: every point within eps (diagonal <= eps) */
                if (c->use_stencil) {
                    const int64_t *cp = g->cc + p * d;
                    for (int64_t o = 0; o < c->noff && cnt < c->min_pts; ++o) {
                        for (int i = 0; i < d; ++i) coord[i] = cp[i] + c->offs[o * d + i];
                        int64_t nb = grid_lookup(g, coord);
                        if (nb < 0) continue;
                        for (int64_t kk = g->cell_first[nb]; kk < g->cell_first[nb + 1]; ++kk)
                            cnt += le_eps(X + p * d, X + g->order[kk] * d, d, c->eps2);
                    }
                } else {
                    int64_t pos = c->pos[p];
                    for (int dir = -1; dir <= 1 && cnt < c->min_pts; dir += 2) {
                        for (int64_t k2 = pos + dir; k2 >= 0 && k2 < c->n && cnt < c->min_pts; k2 += dir) {
                            if (fabs(c->x0s[k2] - X[p * d]) > c->win) break;
                            if (c->cell_s[k2] == cell) continue; /* counted above */
                            if (c->x1s && fabs(c->x1s[k2] - X[p * d + 1]) > c->win) continue;
                            cnt += le_eps(X + p * d, X + c->xorder[k2] * d, d, c->eps2);
                        }
                    }
                }
                c->core[p] = cnt >= c->min_pts;
            }
        }
    }
    return NULL;
}

static int push_edge(grid_job *j, int64_t a, int64_t b)
{
    if (j->nedge == j->cap) {
        int64_t cap = j->cap ? 2 * j->cap : 1024;
        int64_t *e = (int64_t *)realloc(j->edges, sizeof(int64_t) * 2 * cap);
        if (!e) return ORACLE_ENOMEM;
        j->edges = e;
        j->cap = cap;
    }
    j->edges[2 * j->nedge] = a;
    j->edges[2 * j->nedge + 1] = b;
    ++j->nedge;
    return 0;
}

/* Algorithm 3 over the items this thread takes: two neighbouring cubes that both hold core
 * points are joined iff some core point of one lies within eps of some core point of the
 * other.  Each thread keeps its own union-find over the cubes and records every pair it
 * joins; a pair whose cubes its union-find already connects adds nothing to the components
 * and is skipped.  The recorded pairs of all threads span the same components as all pairs,
 * and are joined into one union-find afterwards. */
static void *grid_merge_worker(void *arg)
{
    grid_job *j = (grid_job *)arg;
    grid_ctx *c = j->c;
    const grid_t *g = c->g;
    const int d = c->d;
    const double *X = c->X;
    int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * g->ncell);
    if (!parent) { j->rc = ORACLE_ENOMEM; return NULL; }
    for (int64_t cell = 0; cell < g->ncell; ++cell) parent[cell] = cell;
    int64_t coord[STENCIL_MAX_D];
    int64_t lo, hi;
    while (claim(c, &lo, &hi) && j->rc == 0) {
        if (c->use_stencil) {
            for (int64_t a = lo; a < hi; ++a) {
                if (!c->cell_core[a]) continue;
                const int64_t *ca = grid_cell_coord(g, a);
                for (int64_t o = 0; o < c->noff; ++o) {
                    for (int i = 0; i < d; ++i) coord[i] = ca[i] + c->offs[o * d + i];
                    int64_t b = grid_lookup(g, coord);
                    if (b <= a || !c->cell_core[b]) continue; /* each unordered pair once */
                    if (uf_find(parent, a) == uf_find(parent, b)) continue;
                    int64_t di = dir_index(c->offs + o * d, d);
                    int64_t ra = c->rep[a * c->ndir + di], rb = c->rep[b * c->ndir + (c->ndir - 1 - di)];
                    int found = le_eps(X + ra * d, X + rb * d, d, c->eps2);
                    for (int64_t i = g->cell_first[a]; i < g->cell_first[a + 1] && !found; ++i) {
                        int64_t p = g->order[i];
                        if (!c->core[p]) continue;
                        for (int64_t k = g->cell_first[b]; k < g->cell_first[b + 1] && !found; ++k) {
                            int64_t q = g->order[k];
                            if (c->core[q] && le_eps(X + p * d, X + q * d, d, c->eps2)) found = 1;
                        }
                    }
                    if (found) {
                        uf_union(parent, a, b);
                        if (push_edge(j, a, b)) { j->rc = ORACLE_ENOMEM; break; }
                    }
                }
            }
        } else {
            /* leading-dimension sweep: every pair within the window is met from the point
             * that comes first in xorder, so scanning forward sees each pair once */
            for (int64_t p = lo; p < hi; ++p) {
                if (!c->core[p]) continue;
                int64_t cp = g->cell_of[p];
                for (int64_t k2 = c->pos[p] + 1; k2 < c->n; ++k2) {
                    if (fabs(c->x0s[k2] - X[p * d]) > c->win) break;
                    int64_t cq = c->cell_s[k2];
                    if (!c->core_s[k2] || cq == cp) continue;
                    if (c->x1s && fabs(c->x1s[k2] - X[p * d + 1]) > c->win) continue;
                    if (uf_find(parent, cp) == uf_find(parent, cq)) continue;
                    if (le_eps(X + p * d, X + c->xorder[k2] * d, d, c->eps2)) {
                        uf_union(parent, cp, cq);
                        if (push_edge(j, cp, cq)) { j->rc = ORACLE_ENOMEM; break; }
                    }
                }
            }
        }
    }
    free(parent);
    return NULL;
}

/* Algorithm 4, non-core points: the smallest id among the clusters of the core points
 * within eps (own cube first: all of its points are within eps), else noise. */
static void *grid_border_worker(void *arg)
{
    grid_job *j = (grid_job *)arg;
    grid_ctx *c = j->c;
    const grid_t *g = c->g;
    const int d = c->d;
    const double *X = c->X;
    int64_t coord[STENCIL_MAX_D];
    int64_t lo, hi;
    while (claim(c, &lo, &hi)) {
        for (int64_t p = lo; p < hi; ++p) {
            if (c->core[p]) continue;
            int64_t own = g->cell_of[p];
            int64_t best = c->cell_label[own];
            if (c->use_stencil) {
                const int64_t *cp = g->cc + p * d;
                for (int64_t o = 0; o < c->noff; ++o) {
                    for (int i = 0; i < d; ++i) coord[i] = cp[i] + c->offs[o * d + i];
                    int64_t nb = grid_lookup(g, coord);
                    if (nb < 0 || !c->cell_core[nb]) continue;
                    int64_t lab = c->cell_label[nb];
                    if (lab >= best) continue;
                    for (int64_t kk = g->cell_first[nb]; kk < g->cell_first[nb + 1]; ++kk) {
                        int64_t q = g->order[kk];
                        if (c->core[q] && le_eps(X + p * d, X + q * d, d, c->eps2)) { best = lab; break; }
                    }
                }
            } else {
                int64_t pos = c->pos[p];
                for (int dir = -1; dir <= 1; dir += 2) {
                    for (int64_t k2 = pos + dir; k2 >= 0 && k2 < c->n; k2 += dir) {
                        if (fabs(c->x0s[k2] - X[p * d]) > c->win) break;
                        if (!c->core_s[k2]) continue;
                        if (c->x1s && fabs(c->x1s[k2] - X[p * d + 1]) > c->win) continue;
                        int64_t lab = c->cell_label[c->cell_s[k2]];
                        if (lab < best && le_eps(X + p * d, X + c->xorder[k2] * d, d, c->eps2)) best = lab;
                    }
                }
            }
            c->labels[p] = best == INT64_MAX ? -1 : (int32_t)best;
        }
    }
    return NULL;
}

/*
 * Steps, in the paper's order:
 *  Alg. 1   hypercubes of side eps/sqrt(d) (shrunk, see oracle_side) from the shifted
 *           origin; the non-empty cubes are found by the lexicographic pre-sort (Sec. 2).
 *  MINPTS   a cube with at least MINPTS points is dense: its diagonal is at most eps
 *           (Sec. 2 and Conclusion: all points of a cube are within eps of each other), so
 *           each of its points has at least MINPTS points within eps and is core
 *           (Definition 2).  Points of the other cubes are counted exactly over their own
 *           cube and the neighbour cubes.
 *  Alg. 2   representative points of every cube with a core point, over its core points.
 *  Alg. 3   two neighbouring cubes that both hold core points belong to one cluster iff some
 *           core point of one lies within eps of some core point of the other; the pair of
 *           complementary representative points is tried first (a pair within eps settles
 *           it), then every pair of core points.
 *  Alg. 4   clusters = connected components of the cubes (union-find replaces the
 *           recursive traversal; the components are the same), canonical labels as above.
 * Neighbour cubes: for d <= 4 the offsets of enum_offsets(rule 2) looked up by binary search;
 * for d > 4, or when a band index would exceed 1e7 (where the rounding bound of the band
 * computation no longer holds), the neighbours of a point are found with the leading-
 * dimension pre-sort of Sec. 2: points sorted by coordinate 0, window |x_0 - y_0| <= eps.
 * `threads` host threads share the counts, the merging and the border points; the result
 * does not depend on their number (the representative points and the joining of the
 * threads' merged pairs run on one thread).
 */
int hca_oracle_grid_mt(const double *X, int64_t n, int32_t d, double eps, int32_t min_pts,
                       int32_t threads, int32_t *labels, uint8_t *core_out)
{
    int rc = check_args(X, n, d, eps, min_pts, labels);
    if (rc) return rc;
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if (n == 0) return 0;
    const double eps2 = eps * eps;
    const double side = oracle_side(eps, d);

    grid_t g;
    rc = grid_build(&g, X, n, d, side);
    if (rc) return rc;
    int use_stencil = d <= STENCIL_MAX_D;
    for (int64_t k = 0; k < n * (int64_t)d && use_stencil; ++k)
        if (g.cc[k] > 10000000) use_stencil = 0;

    uint8_t *core = (uint8_t *)calloc(n, 1);
    uint8_t *cell_core = (uint8_t *)calloc(g.ncell, 1);
    int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * g.ncell);
    int64_t *comp_min = (int64_t *)malloc(sizeof(int64_t) * g.ncell);
    int64_t *cell_label = (int64_t *)malloc(sizeof(int64_t) * g.ncell);
    grid_job *jobs = (grid_job *)calloc(threads, sizeof(grid_job));
    grid_ctx *ctx = (grid_ctx *)calloc(1, sizeof(grid_ctx));
    int64_t *offs = NULL, noff = 0;
    int64_t *xorder = NULL, *tmp = NULL, *cell_s = NULL;
    double *x0s = NULL, *x1s = NULL;
    uint8_t *core_s = NULL;
    int8_t *dirs = NULL;
    int64_t *rep = NULL;
    rc = ORACLE_ENOMEM;
    if (!core || !cell_core || !parent || !comp_min || !cell_label || !jobs || !ctx) goto done;

    if (use_stencil) {
        noff = enum_offsets(d, 2, side, eps, NULL);
        offs = (int64_t *)malloc(sizeof(int64_t) * (noff * d + 1));
        if (!offs) goto done;
        enum_offsets(d, 2, side, eps, offs);
    } else {
        /* leading-dimension pre-sort: order by x_0, ties by index */
        xorder = (int64_t *)malloc(sizeof(int64_t) * n);
        tmp = (int64_t *)malloc(sizeof(int64_t) * n);
        int64_t *key = (int64_t *)malloc(sizeof(int64_t) * n);
        if (!xorder || !tmp || !key) { free(key); goto done; }
        for (int64_t p = 0; p < n; ++p) xorder[p] = p;
        /* simple merge sort on x_0 with an explicit comparator */
        {
            int64_t w;
            for (w = 1; w < n; w *= 2) {
                for (int64_t lo = 0; lo < n; lo += 2 * w) {
                    int64_t mid = lo + w < n ? lo + w : n, hi = lo + 2 * w < n ? lo + 2 * w : n;
                    int64_t i = lo, j = mid, k = lo;
                    while (i < mid && j < hi) {
                        double a = X[xorder[i] * d], b = X[xorder[j] * d];
                        tmp[k++] = (a < b || (a == b && xorder[i] < xorder[j])) ? xorder[i++] : xorder[j++];
                    }
                    while (i < mid) tmp[k++] = xorder[i++];
                    while (j < hi) tmp[k++] = xorder[j++];
                }
                memcpy(xorder, tmp, sizeof(int64_t) * n);
            }
        }
        for (int64_t k = 0; k < n; ++k) key[xorder[k]] = k; /* position of each point */
        free(tmp);
        tmp = key; /* tmp now holds the position of each point in xorder */
        /* the sweep reads x_0, x_1, the cube and the core flag of the points in xorder order;
           a pair with |x_0 - y_0| or |x_1 - y_1| above eps (1 + 1e-9) is farther than eps
           (its first or second term alone exceeds eps^2), so those comparisons are skipped */
        x0s = (double *)malloc(sizeof(double) * n);
        x1s = d >= 2 ? (double *)malloc(sizeof(double) * n) : NULL;
        cell_s = (int64_t *)malloc(sizeof(int64_t) * n);
        core_s = (uint8_t *)malloc(n);
        if (!x0s || (d >= 2 && !x1s) || !cell_s || !core_s) goto done;
        for (int64_t k = 0; k < n; ++k) {
            x0s[k] = X[xorder[k] * d];
            if (x1s) x1s[k] = X[xorder[k] * d + 1];
            cell_s[k] = g.cell_of[xorder[k]];
        }
    }

    ctx->X = X; ctx->n = n; ctx->d = d; ctx->eps2 = eps2; ctx->min_pts = min_pts;
    ctx->g = &g; ctx->use_stencil = use_stencil; ctx->offs = offs; ctx->noff = noff;
    ctx->xorder = xorder; ctx->pos = tmp; ctx->win = eps * (1.0 + 1e-9);
    ctx->x0s = x0s; ctx->x1s = x1s; ctx->cell_s = cell_s; ctx->core_s = core_s;
    ctx->core = core; ctx->cell_core = cell_core; ctx->cell_label = cell_label; ctx->labels = labels;
    for (int t = 0; t < threads; ++t) jobs[t].c = ctx;

    /* ---- MINPTS: dense cubes, then exact counts for the other cubes' points ---- */
    run_phase(grid_count_worker, ctx, jobs, threads, g.ncell, 64);
    for (int64_t p = 0; p < n; ++p)
        if (core[p]) cell_core[g.cell_of[p]] = 1;
    if (core_s)
        for (int64_t k = 0; k < n; ++k) core_s[k] = core[xorder[k]];

    /* ---- Alg. 2: representative points over core points (stencil path) ---- */
    int64_t ndir = 0;
    if (use_stencil) {
        ndir = hca_oracle_rep_dirs(d, NULL);
        dirs = (int8_t *)malloc(ndir * d);
        if (!dirs) goto done;
        hca_oracle_rep_dirs(d, dirs);
        rep = compute_reps(&g, X, core, dirs, ndir);
        if (!rep) goto done;
    }
    ctx->rep = rep;
    ctx->ndir = ndir;

    /* ---- Alg. 3: merge neighbouring cubes that hold core points ---- */
    run_phase(grid_merge_worker, ctx, jobs, threads, use_stencil ? g.ncell : n, use_stencil ? 64 : 256);
    for (int64_t cell = 0; cell < g.ncell; ++cell) parent[cell] = cell;
    for (int t = 0; t < threads; ++t) {
        if (jobs[t].rc) goto done;
        for (int64_t e = 0; e < jobs[t].nedge; ++e)
            uf_union(parent, jobs[t].edges[2 * e], jobs[t].edges[2 * e + 1]);
    }

    /* ---- Alg. 4: canonical cluster ids, then border and noise points ---- */
    for (int64_t cell = 0; cell < g.ncell; ++cell) comp_min[cell] = INT64_MAX;
    for (int64_t p = 0; p < n; ++p) {
        if (!core[p]) continue;
        int64_t r = uf_find(parent, g.cell_of[p]);
        if (p < comp_min[r]) comp_min[r] = p;
    }
    for (int64_t cell = 0; cell < g.ncell; ++cell)
        cell_label[cell] = cell_core[cell] ? comp_min[uf_find(parent, cell)] : INT64_MAX;
    for (int64_t p = 0; p < n; ++p)
        labels[p] = core[p] ? (int32_t)cell_label[g.cell_of[p]] : -1;
    run_phase(grid_border_worker, ctx, jobs, threads, n, 256);
    if (core_out) memcpy(core_out, core, n);
    rc = 0;
done:
    if (jobs)
        for (int t = 0; t < threads; ++t) free(jobs[t].edges);
    free(core); free(cell_core); free(parent); free(comp_min); free(cell_label); free(jobs); free(ctx);
    free(offs); free(xorder); free(tmp); free(dirs); free(rep); free(x0s); free(x1s); free(cell_s); free(core_s);
    grid_free(&g);
    return rc;
}

/* hca_oracle_grid_mt on the calling thread alone. */
int hca_oracle_grid(const double *X, int64_t n, int32_t d, double eps, int32_t min_pts,
                    int32_t *labels, uint8_t *core_out)
{
    return hca_oracle_grid_mt(X, n, d, eps, min_pts, 1, labels, core_out);
}

/* ------------------------------------------------------------------------------------- */
/* Algorithms 2-4 as printed (ablation).                                                    */
/* ------------------------------------------------------------------------------------- */

/*
 * Reading of the printed algorithm: cubes of side exactly eps/sqrt(d); representative
 * points over all points of a cube (Algorithm 2); two cubes are merged iff the complementary
 * representative points are at distance strictly below eps (Algorithm 3, "< eps"); the
 * neighbour cubes are the (2*ceil(sqrt(d))+1)^d block without its corner cubes and the cube
 * itself (Sec. 2, "Depth First Search"); every non-empty cube belongs to a cluster, so there
 * is no noise and MINPTS plays no part (Algorithm 4).  Labels use the canonical rule.
 * Only d <= 4 is accepted.
 */
int hca_oracle_literal(const double *X, int64_t n, int32_t d, double eps, int32_t *labels)
{
    int rc = check_args(X, n, d, eps, 1, labels);
    if (rc) return rc;
    if (d > STENCIL_MAX_D) return ORACLE_EINVAL;
    if (n == 0) return 0;
    const double eps2 = eps * eps;
    const double side = eps / sqrt((double)d);
    grid_t g;
    rc = grid_build(&g, X, n, d, side);
    if (rc) return rc;
    int64_t noff = enum_offsets(d, 0, side, eps, NULL);
    int64_t ndir = hca_oracle_rep_dirs(d, NULL);
    int64_t *offs = (int64_t *)malloc(sizeof(int64_t) * (noff * d + 1));
    int8_t *dirs = (int8_t *)malloc(ndir * d);
    int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * g.ncell);
    int64_t *comp_min = (int64_t *)malloc(sizeof(int64_t) * g.ncell);
    int64_t *coord = (int64_t *)malloc(sizeof(int64_t) * d);
    int64_t *rep = NULL;
    rc = ORACLE_ENOMEM;
    if (!offs || !dirs || !parent || !comp_min || !coord) goto done;
    enum_offsets(d, 0, side, eps, offs);
    hca_oracle_rep_dirs(d, dirs);
    rep = compute_reps(&g, X, NULL, dirs, ndir);
    if (!rep) goto done;
    for (int64_t c = 0; c < g.ncell; ++c) parent[c] = c;
    for (int64_t a = 0; a < g.ncell; ++a) {
        const int64_t *ca = grid_cell_coord(&g, a);
        for (int64_t o = 0; o < noff; ++o) {
            for (int i = 0; i < d; ++i) coord[i] = ca[i] + offs[o * d + i];
            int64_t b = grid_lookup(&g, coord);
            if (b <= a) continue;
            int64_t di = dir_index(offs + o * d, d);
            int64_t ra = rep[a * ndir + di], rb = rep[b * ndir + (ndir - 1 - di)];
            double s = 0.0;
            for (int i = 0; i < d; ++i) {
                double t = X[ra * d + i] - X[rb * d + i];
                s = s + t * t;
            }
            if (s < eps2) uf_union(parent, a, b);
        }
    }
    for (int64_t c = 0; c < g.ncell; ++c) comp_min[c] = INT64_MAX;
    for (int64_t p = 0; p < n; ++p) {
        int64_t r = uf_find(parent, g.cell_of[p]);
        if (p < comp_min[r]) comp_min[r] = p;
    }
    for (int64_t p = 0; p < n; ++p) labels[p] = (int32_t)comp_min[uf_find(parent, g.cell_of[p])];
    rc = 0;
done:
    free(offs); free(dirs); free(parent); free(comp_min); free(coord); free(rep);
    grid_free(&g);
    return rc;
}
