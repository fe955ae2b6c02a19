/*
 * gj_oracle.c -- CPU oracle for the epsilon-distance similarity self-join.
 *
 * TEST INFRASTRUCTURE ONLY.  The CUDA library never links, loads or calls this
 * file; only the tests, the smoke check and the benchmark's CPU-baseline leg
 * do.  It shares no code, header, table or constant with the library.
 *
 * Build:  gcc -O2 -ffp-contract=off -fPIC -shared -pthread
 * (-ffp-contract=off matters: the definition below forbids fused multiply-add,
 * and gcc contracts by default on some targets.)
 *
 * The definition (Sec. 3.1, problem statement):
 *   e2      = fl(eps * eps)
 *   s(i,j)  = (((0 + fl(x_i0 - x_j0)^2) + fl(x_i1 - x_j1)^2) + ...) summed in the
 *             ORIGINAL dimension order, every square and add rounded to nearest
 *   R       = { (i,j) in [0,n)^2 : s(i,j) <= e2 }   -- inclusive (Sec. 3.1),
 *             both orientations and the n self-pairs (Sec. 5.2, selectivity S_D).
 * s is bitwise symmetric because fl(a-b) = -fl(b-a).
 *
 * Two routes to R live here:
 *   gjo_brute      -- the nested-loop join of Sec. 3.1 (O(n^2)), the definition.
 *   gjo_brute_qe   -- the same definition for two sets, Q join_eps E (Sec. 3.1).
 *   gjo_grid_join  -- the paper's method, steps in the paper's order:
 *                     REORDER (Sec. 4.2), grid index on the first k reordered
 *                     dimensions (Sec. 3.2.1, 4.1), 3^k adjacent-cell search
 *                     (Sec. 3.2.1, Fig. 1), SORTIDU window on one un-indexed
 *                     dimension (Sec. 4.3), SHORTC early exit (Sec. 4.4).
 * The grid, REORDER, SORTIDU and SHORTC only skip work, so both routes must
 * return the same set; the tests hold them to that.
 *
 * Readings of the paper taken here (every one is a filter that may only skip
 * pairs outside R):
 *   - grid origin is the per-dimension minimum (Sec. 3.2.1 assumes 0 "without
 *     loss of generality"); cell width w_j = max(eps*(1+2^-30), range_j*2^-19)
 *     so that rounding in floor((y-m)/w) never separates a pair of R by more
 *     than one cell (the argument needs fewer than 2^20 cells per dimension);
 *   - SORTIDU keeps q when |fl(q_u - p_u)| <= fl(eps*(1+2^-40)): a pair of R has
 *     fl(fl(dq)^2) <= e2, hence |fl(dq)| <= eps*(1+2^-52);
 *   - SHORTC stops once the running sum in original order exceeds e2 (squared
 *     threshold; RN addition of non-negative terms is monotone, so a partial sum
 *     above e2 implies the full sum is above e2).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GJO_REORDER 1
#define GJO_SORTIDU 2
#define GJO_SHORTC  4

/* ------------------------------------------------------------------------- */
/* The distance of the definition.                                            */
/* ------------------------------------------------------------------------- */

double gjo_sqdist(const double *a, const double *b, int d)
{
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        double t = a[j] - b[j];
        s = s + t * t;
    }
    return s;
}

/* Same sum with the SHORTC exit; returns a value > e2 as soon as one is seen. */
static double sqdist_shortc(const double *a, const double *b, int d, double e2)
{
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        double t = a[j] - b[j];
        s = s + t * t;
        if (s > e2)
            return s;
    }
    return s;
}

/* ------------------------------------------------------------------------- */
/* Growable per-thread pair lists.                                            */
/* ------------------------------------------------------------------------- */

typedef struct {
    uint64_t *v;
    int64_t n, cap;
    int oom;
} keyvec;

static void kv_push(keyvec *k, uint64_t x)
{
    if (k->oom)
        return;
    if (k->n == k->cap) {
        int64_t nc = k->cap ? 2 * k->cap : 1024;
        uint64_t *nv = (uint64_t *)realloc(k->v, (size_t)nc * sizeof(uint64_t));
        if (!nv) {
            k->oom = 1;
            return;
        }
        k->v = nv;
        k->cap = nc;
    }
    k->v[k->n++] = x;
}

static int cmp_u32(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* Concatenate thread lists (already in ascending key order across threads). */
static int64_t gather(keyvec *lists, int nt, uint64_t *out, int64_t cap, int *oom)
{
    int64_t total = 0;
    for (int t = 0; t < nt; ++t) {
        if (lists[t].oom)
            *oom = 1;
        for (int64_t i = 0; i < lists[t].n; ++i) {
            if (out && total < cap)
                out[total] = lists[t].v[i];
            ++total;
        }
        free(lists[t].v);
    }
    return total;
}

/* ------------------------------------------------------------------------- */
/* Nested-loop join (Sec. 3.1).                                               */
/* ------------------------------------------------------------------------- */

typedef struct {
    const double *X;
    int64_t n, lo, hi;
    int d;
    double e2;
    keyvec out;
} brute_arg;

static void *brute_worker(void *p)
{
    brute_arg *a = (brute_arg *)p;
    for (int64_t i = a->lo; i < a->hi; ++i)
        for (int64_t j = 0; j < a->n; ++j)
            if (gjo_sqdist(a->X + i * a->d, a->X + j * a->d, a->d) <= a->e2)
                kv_push(&a->out, ((uint64_t)i << 32) | (uint64_t)j);
    return NULL;
}

/* All ordered pairs of R as keys (i<<32 | j), ascending.  Returns |R| (writes at
 * most cap keys), or -1 when memory ran out. */
int64_t gjo_brute(const double *X, int64_t n, int d, double eps, uint64_t *out,
                  int64_t cap, int nthreads)
{
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > n && n > 0)
        nthreads = (int)n;
    double e2 = eps * eps;
    brute_arg *args = (brute_arg *)calloc((size_t)nthreads, sizeof(brute_arg));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    keyvec *lists = (keyvec *)calloc((size_t)nthreads, sizeof(keyvec));
    for (int t = 0; t < nthreads; ++t) {
        args[t].X = X;
        args[t].n = n;
        args[t].d = d;
        args[t].e2 = e2;
        args[t].lo = n * t / nthreads;
        args[t].hi = n * (t + 1) / nthreads;
        pthread_create(&th[t], NULL, brute_worker, &args[t]);
    }
    for (int t = 0; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        lists[t] = args[t].out;
    }
    int oom = 0;
    int64_t total = gather(lists, nthreads, out, cap, &oom);
    free(args);
    free(th);
    free(lists);
    return oom ? -1 : total;
}

/* ------------------------------------------------------------------------- */
/* Similarity join Q join_eps E (Sec. 3.1: the self-join is the case Q = E).   */
/* ------------------------------------------------------------------------- */

typedef struct {
    const double *Q, *E;
    int64_t ne, lo, hi;
    int d;
    double e2;
    keyvec out;
} qe_arg;

static void *qe_worker(void *p)
{
    qe_arg *a = (qe_arg *)p;
    for (int64_t i = a->lo; i < a->hi; ++i)
        for (int64_t j = 0; j < a->ne; ++j)
            if (gjo_sqdist(a->Q + i * a->d, a->E + j * a->d, a->d) <= a->e2)
                kv_push(&a->out, ((uint64_t)i << 32) | (uint64_t)j);
    return NULL;
}

/* Every pair (q, e) of a row q of Q and a row e of E with s(q, e) <= fl(eps^2),
 * as keys (q<<32 | e), ascending: the nested loop over Q x E.  Returns the
 * count (writes at most cap keys), or -1 when memory ran out. */
int64_t gjo_brute_qe(const double *Q, int64_t nq, const double *E, int64_t ne, int d, double eps,
                     uint64_t *out, int64_t cap, int nthreads)
{
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > nq && nq > 0)
        nthreads = (int)nq;
    double e2 = eps * eps;
    qe_arg *args = (qe_arg *)calloc((size_t)nthreads, sizeof(qe_arg));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    keyvec *lists = (keyvec *)calloc((size_t)nthreads, sizeof(keyvec));
    for (int t = 0; t < nthreads; ++t) {
        args[t].Q = Q;
        args[t].E = E;
        args[t].ne = ne;
        args[t].d = d;
        args[t].e2 = e2;
        args[t].lo = nq * t / nthreads;
        args[t].hi = nq * (t + 1) / nthreads;
        pthread_create(&th[t], NULL, qe_worker, &args[t]);
    }
    for (int t = 0; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        lists[t] = args[t].out;
    }
    int oom = 0;
    int64_t total = gather(lists, nthreads, out, cap, &oom);
    free(args);
    free(th);
    free(lists);
    return oom ? -1 : total;
}

/* Neighbours of one query by the definition (j ascending).  Returns the count
 * (writes at most cap). */
int64_t gjo_query_neighbors(const double *X, int64_t n, int d, double eps, int64_t q,
                            uint32_t *out, int64_t cap)
{
    double e2 = eps * eps;
    int64_t c = 0;
    for (int64_t j = 0; j < n; ++j)
        if (gjo_sqdist(X + q * d, X + j * d, d) <= e2) {
            if (out && c < cap)
                out[c] = (uint32_t)j;
            ++c;
        }
    return c;
}

/* ------------------------------------------------------------------------- */
/* REORDER (Sec. 4.2): variance per dimension, dimensions by descending       */
/* variance.  The paper estimates the variance on a 1% sample; the oracle     */
/* takes the population variance over all points (two passes), ties broken   */
/* toward the lower dimension index.                                          */
/* ------------------------------------------------------------------------- */

void gjo_variance(const double *X, int64_t n, int d, double *mean, double *var)
{
    for (int j = 0; j < d; ++j) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i)
            s += X[i * d + j];
        double m = n ? s / (double)n : 0.0;
        double q = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double t = X[i * d + j] - m;
            q += t * t;
        }
        if (mean)
            mean[j] = m;
        var[j] = n ? q / (double)n : 0.0;
    }
}

void gjo_reorder_perm(const double *var, int d, int32_t *perm)
{
    for (int j = 0; j < d; ++j)
        perm[j] = j;
    /* insertion sort: stable, so equal variances keep ascending index */
    for (int a = 1; a < d; ++a) {
        int32_t p = perm[a];
        int b = a - 1;
        while (b >= 0 && var[perm[b]] < var[p]) {
            perm[b + 1] = perm[b];
            --b;
        }
        perm[b + 1] = p;
    }
}

/* Fraction of adjacent cells no longer searched when k of n dimensions are
 * indexed (Sec. 4.1): l(n,k) = (3^n - 3^k) / 3^n. */
double gjo_index_loss(int n, int k)
{
    double a = pow(3.0, (double)n), b = pow(3.0, (double)k);
    return (a - b) / a;
}

/* ------------------------------------------------------------------------- */
/* Grid pieces (Sec. 3.2.1, Fig. 1), exposed for the worked-example checks.   */
/* ------------------------------------------------------------------------- */

/* Cell coordinate floor((y_j - origin_j) / w_j) of every point in the first k
 * dimensions (rows of Y have stride ld). */
void gjo_cell_coords(const double *Y, int64_t n, int ld, int k, const double *origin,
                     const double *w, int64_t *coords)
{
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < k; ++j)
            coords[i * k + j] = (int64_t)floor((Y[i * ld + j] - origin[j]) / w[j]);
}

/* Row-major linear id, dimension 0 most significant (the numbering of Fig. 1).
 * Returns -1 if a coordinate lies outside [0, ncells_j). */
int64_t gjo_linearise(const int64_t *c, const int64_t *ncells, int k)
{
    int64_t id = 0;
    for (int j = 0; j < k; ++j) {
        if (c[j] < 0 || c[j] >= ncells[j])
            return -1;
        id = id * ncells[j] + c[j];
    }
    return id;
}

static int64_t lower_bound_i64(const int64_t *a, int64_t n, int64_t x)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

/* Non-empty cells among the 3^k cells around `coord` (origin cell included),
 * found by binary search in the sorted non-empty linear ids (Sec. 3.2.1).
 * Writes their ids in ascending order; returns how many. */
int gjo_adjacent_nonempty(const int64_t *ids_sorted, int64_t G, const int64_t *coord,
                          const int64_t *ncells, int k, int64_t *out)
{
    int64_t total = 1;
    for (int j = 0; j < k; ++j)
        total *= 3;
    int64_t nb[64];
    int found = 0;
    for (int64_t t = 0; t < total; ++t) {
        int64_t r = t;
        for (int j = k - 1; j >= 0; --j) {
            nb[j] = coord[j] + (r % 3) - 1;
            r /= 3;
        }
        int64_t id = gjo_linearise(nb, ncells, k);
        if (id < 0)
            continue;
        int64_t pos = lower_bound_i64(ids_sorted, G, id);
        if (pos < G && ids_sorted[pos] == id)
            out[found++] = id;
    }
    return found;
}

/* ------------------------------------------------------------------------- */
/* The paper's method on the CPU.                                             */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t candidates;        /* unordered pairs i<j in adjacent cells (no SORTIDU) */
    int64_t window_candidates; /* unordered pairs i<j that survive the SORTIDU window */
    int64_t nonempty_cells;
    int32_t k_used;
    int32_t perm[128];         /* REORDER permutation (first min(d,128) entries) */
} gjo_stats;

typedef struct {
    /* shared, read-only */
    const double *X;   /* original points, n x d */
    const double *Y;   /* reordered points, n x d */
    int64_t n;
    int d, k, u, flags;
    double e2, ew;
    const int64_t *coords;      /* n x k cell coordinates (by original index) */
    const int64_t *cell_coord;  /* G x k, lexicographically ascending */
    const int64_t *cell_start;  /* G+1 offsets into order[] */
    const int64_t *order;       /* point indices grouped by cell (SORTIDU: by u inside) */
    int64_t G;
    int64_t lo, hi;             /* query range (original indices) */
    /* outputs */
    keyvec out;
    int64_t cand2, wcand2;
} grid_arg;

static int cmp_tuple(const int64_t *a, const int64_t *b, int k)
{
    for (int j = 0; j < k; ++j) {
        if (a[j] < b[j])
            return -1;
        if (a[j] > b[j])
            return 1;
    }
    return 0;
}

/* qsort context (single-threaded sort phase) */
static const int64_t *g_sort_coords;
static const double *g_sort_Y;
static int g_sort_k, g_sort_d, g_sort_u, g_sort_byu;

static int cmp_point(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    int c = cmp_tuple(g_sort_coords + a * g_sort_k, g_sort_coords + b * g_sort_k, g_sort_k);
    if (c)
        return c;
    if (g_sort_byu) {
        double ua = g_sort_Y[a * g_sort_d + g_sort_u], ub = g_sort_Y[b * g_sort_d + g_sort_u];
        if (ua < ub)
            return -1;
        if (ua > ub)
            return 1;
    }
    return (a > b) - (a < b);
}

static int64_t find_cell(const int64_t *cell_coord, int64_t G, int k, const int64_t *t)
{
    int64_t lo = 0, hi = G;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (cmp_tuple(cell_coord + mid * k, t, k) < 0)
            lo = mid + 1;
        else
            hi = mid;
    }
    if (lo < G && cmp_tuple(cell_coord + lo * k, t, k) == 0)
        return lo;
    return -1;
}

static void *grid_worker(void *p)
{
    grid_arg *a = (grid_arg *)p;
    const int k = a->k, d = a->d;
    int64_t total = 1;
    for (int j = 0; j < k; ++j)
        total *= 3;
    int64_t nb[64];
    uint32_t *hits = NULL;
    int64_t hcap = 0;
    for (int64_t i = a->lo; i < a->hi; ++i) {
        const int64_t *ci = a->coords + i * k;
        const double *xi = a->X + (size_t)i * d;
        double ui = a->Y[(size_t)i * d + a->u];
        int64_t nh = 0;
        for (int64_t t = 0; t < total; ++t) {
            int64_t r = t;
            for (int j = k - 1; j >= 0; --j) {
                nb[j] = ci[j] + (r % 3) - 1;
                r /= 3;
            }
            int64_t c = find_cell(a->cell_coord, a->G, k, nb);
            if (c < 0)
                continue;
            int64_t s = a->cell_start[c], e = a->cell_start[c + 1];
            a->cand2 += e - s;
            if (a->flags & GJO_SORTIDU) {
                /* first q with fl(q_u - p_u) >= -ew, then scan while <= ew */
                int64_t lo = s, hi = e;
                while (lo < hi) {
                    int64_t mid = lo + (hi - lo) / 2;
                    double qu = a->Y[(size_t)a->order[mid] * d + a->u];
                    if (qu - ui < -a->ew)
                        lo = mid + 1;
                    else
                        hi = mid;
                }
                s = lo;
                int64_t stop = s;
                while (stop < e && a->Y[(size_t)a->order[stop] * d + a->u] - ui <= a->ew)
                    ++stop;
                e = stop;
            }
            a->wcand2 += e - s;
            for (int64_t q = s; q < e; ++q) {
                int64_t j = a->order[q];
                const double *xj = a->X + (size_t)j * d;
                double sd = (a->flags & GJO_SHORTC) ? sqdist_shortc(xi, xj, d, a->e2)
                                                    : gjo_sqdist(xi, xj, d);
                if (sd <= a->e2) {
                    if (nh == hcap) {
                        hcap = hcap ? 2 * hcap : 256;
                        uint32_t *nhp = (uint32_t *)realloc(hits, (size_t)hcap * 4);
                        if (!nhp) {
                            a->out.oom = 1;
                            free(hits);
                            return NULL;
                        }
                        hits = nhp;
                    }
                    hits[nh++] = (uint32_t)j;
                }
            }
        }
        /* sort this query's neighbours so the global list comes out ascending */
        qsort(hits, (size_t)nh, sizeof(uint32_t), cmp_u32);
        for (int64_t x = 0; x < nh; ++x)
            kv_push(&a->out, ((uint64_t)i << 32) | hits[x]);
    }
    free(hits);
    return NULL;
}

/* The self-join by the paper's method.  k = number of indexed (reordered)
 * dimensions, 0 <= k <= d (k = 0: one cell, i.e. the nested loop).  flags:
 * GJO_REORDER | GJO_SORTIDU | GJO_SHORTC.  Writes at most cap keys
 * (i<<32 | j, ascending); returns |R|, -1 on out-of-memory, -2 on bad input. */
int64_t gjo_grid_join(const double *X, int64_t n, int d, double eps, int k, int flags,
                      int nthreads, uint64_t *out, int64_t cap, gjo_stats *st)
{
    if (n < 0 || d < 1 || k < 0 || k > d || k > 63 || !(eps > 0.0))
        return -2;
    if (nthreads < 1)
        nthreads = 1;
    if (n > 0 && nthreads > n)
        nthreads = (int)n;
    const double e2 = eps * eps;
    const double ew = eps * (1.0 + ldexp(1.0, -40));

    /* REORDER */
    int32_t *perm = (int32_t *)malloc((size_t)d * sizeof(int32_t));
    double *var = (double *)malloc((size_t)d * sizeof(double));
    if (flags & GJO_REORDER) {
        gjo_variance(X, n, d, NULL, var);
        gjo_reorder_perm(var, d, perm);
    } else {
        for (int j = 0; j < d; ++j)
            perm[j] = j;
    }
    double *Y = (double *)malloc((size_t)n * d * sizeof(double) + 8);
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < d; ++j)
            Y[i * d + j] = X[i * d + perm[j]];

    /* grid over the first k reordered dimensions */
    double origin[64], w[64];
    for (int j = 0; j < k; ++j) {
        double mn = INFINITY, mx = -INFINITY;
        for (int64_t i = 0; i < n; ++i) {
            double v = Y[i * d + j];
            if (v < mn)
                mn = v;
            if (v > mx)
                mx = v;
        }
        origin[j] = mn;
        double wj = eps * (1.0 + ldexp(1.0, -30));
        double wr = (mx - mn) * ldexp(1.0, -19);
        w[j] = wr > wj ? wr : wj;
    }
    int64_t *coords = (int64_t *)malloc((size_t)n * (k ? k : 1) * sizeof(int64_t));
    gjo_cell_coords(Y, n, d, k, origin, w, coords);

    int u = (k < d) ? k : 0;  /* SORTIDU dimension (reordered index) */
    int64_t *order = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i)
        order[i] = i;
    g_sort_coords = coords;
    g_sort_Y = Y;
    g_sort_k = k;
    g_sort_d = d;
    g_sort_u = u;
    g_sort_byu = (flags & GJO_SORTIDU) ? 1 : 0;
    qsort(order, (size_t)n, sizeof(int64_t), cmp_point);

    int64_t G = 0;
    int64_t *cell_start = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    int64_t *cell_coord = (int64_t *)malloc((size_t)(n ? n : 1) * (k ? k : 1) * sizeof(int64_t));
    for (int64_t q = 0; q < n; ++q) {
        if (q == 0 || cmp_tuple(coords + order[q] * k, coords + order[q - 1] * k, k) != 0) {
            cell_start[G] = q;
            memcpy(cell_coord + G * k, coords + order[q] * k, (size_t)k * sizeof(int64_t));
            ++G;
        }
    }
    cell_start[G] = n;

    grid_arg *args = (grid_arg *)calloc((size_t)nthreads, sizeof(grid_arg));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    keyvec *lists = (keyvec *)calloc((size_t)nthreads, sizeof(keyvec));
    int64_t cand2 = 0, wcand2 = 0;
    for (int t = 0; t < nthreads; ++t) {
        grid_arg *a = &args[t];
        a->X = X;
        a->Y = Y;
        a->n = n;
        a->d = d;
        a->k = k;
        a->u = u;
        a->flags = flags;
        a->e2 = e2;
        a->ew = ew;
        a->coords = coords;
        a->cell_coord = cell_coord;
        a->cell_start = cell_start;
        a->order = order;
        a->G = G;
        a->lo = n * t / nthreads;
        a->hi = n * (t + 1) / nthreads;
        pthread_create(&th[t], NULL, grid_worker, a);
    }
    for (int t = 0; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        lists[t] = args[t].out;
        cand2 += args[t].cand2;
        wcand2 += args[t].wcand2;
    }
    int oom = 0;
    int64_t total = gather(lists, nthreads, out, cap, &oom);
    if (st) {
        st->candidates = (cand2 - n) / 2;
        st->window_candidates = (wcand2 - n) / 2;
        st->nonempty_cells = G;
        st->k_used = k;
        for (int j = 0; j < d && j < 128; ++j)
            st->perm[j] = perm[j];
    }
    free(args);
    free(th);
    free(lists);
    free(cell_coord);
    free(cell_start);
    free(order);
    free(coords);
    free(Y);
    free(var);
    free(perm);
    return oom ? -1 : total;
}

/* ------------------------------------------------------------------------- */
/* SHORTC depth statistics (Sec. 4.4).  For each listed query q and every     */
/* other point j, the number of dimensions evaluated, in the order `perm`,    */
/* until the running sum first exceeds e2 (d if it never does).  Sums go to   */
/* depth_sum / pair_count.  This is the per-candidate-pair work figure that   */
/* the throughput numbers are measured against.                               */
/* ------------------------------------------------------------------------- */

typedef struct {
    const double *X;
    int64_t n;
    int d;
    const int32_t *perm;
    double e2;
    const int64_t *q;
    int64_t lo, hi;
    int64_t depth, pairs;
} depth_arg;

static void *depth_worker(void *p)
{
    depth_arg *a = (depth_arg *)p;
    for (int64_t t = a->lo; t < a->hi; ++t) {
        int64_t i = a->q[t];
        const double *xi = a->X + (size_t)i * a->d;
        for (int64_t j = 0; j < a->n; ++j) {
            if (j == i)
                continue;
            const double *xj = a->X + (size_t)j * a->d;
            double s = 0.0;
            int dep = a->d;
            for (int c = 0; c < a->d; ++c) {
                double v = xi[a->perm[c]] - xj[a->perm[c]];
                s = s + v * v;
                if (s > a->e2) {
                    dep = c + 1;
                    break;
                }
            }
            a->depth += dep;
            a->pairs += 1;
        }
    }
    return NULL;
}

void gjo_depth_stats(const double *X, int64_t n, int d, double eps, const int32_t *perm,
                     const int64_t *queries, int64_t nq, int nthreads, int64_t *depth_sum,
                     int64_t *pair_count)
{
    if (nthreads < 1)
        nthreads = 1;
    if (nq > 0 && nthreads > nq)
        nthreads = (int)nq;
    depth_arg *args = (depth_arg *)calloc((size_t)nthreads, sizeof(depth_arg));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) {
        args[t].X = X;
        args[t].n = n;
        args[t].d = d;
        args[t].perm = perm;
        args[t].e2 = eps * eps;
        args[t].q = queries;
        args[t].lo = nq * t / nthreads;
        args[t].hi = nq * (t + 1) / nthreads;
        pthread_create(&th[t], NULL, depth_worker, &args[t]);
    }
    int64_t ds = 0, pc = 0;
    for (int t = 0; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        ds += args[t].depth;
        pc += args[t].pairs;
    }
    *depth_sum = ds;
    *pair_count = pc;
    free(args);
    free(th);
}

/* keep the comparator referenced for builds that strip unused statics */
void gjo_sort_keys(uint64_t *keys, int64_t n) { qsort(keys, (size_t)n, sizeof(uint64_t), cmp_u64); }
