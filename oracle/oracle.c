/*
 * Plain CPU oracle for the vector-geometric ray-casting point-in-polygon method.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this file:
 * only the test suite, the smoke check and the benchmark's CPU-baseline arm load
 * it.  It shares no code, header or helper with the CUDA path.
 *
 * What it computes (Method section, the seven-step algorithm; Constraint 1):
 * for an integer point p = (p_x, p_y) and a closed polygon R_0 .. R_{m-1} (the
 * edge from R_{m-1} back to R_0 is implicit, and a repeated closing vertex
 * R_n = R_0 as in the paper's convention only adds a zero-length edge), cast the
 * ray d = (1, 0) from p, so the ray's normal is (0, 1) and f(r) = r_y - p_y.
 *
 *   step 2   f_i = y_i - p_y for every vertex
 *   step 3-4 edge i -> i+1 is a candidate crossing when f_i and f_{i+1} lie on
 *            opposite sides of the ray.  Reading (half-open): a vertex with
 *            f = 0 is taken to lie below the ray, so the test is
 *            (f_i > 0) != (f_{i+1} > 0); a horizontal edge never qualifies.
 *   Constraint 1: with d = r_{i+1} - r_i and the edge normal n = (d_y, -d_x),
 *            flipped so that n_x >= 0 (acute with (1, 0)), the crossing lies to
 *            the right of p when line_pos = (p - r_i) . n is negative.
 *            Reading: strictly negative (a crossing exactly at p does not count).
 *   step 7   p is inside when the number of counted edges is odd.
 *
 * The two readings are the unique rule that classifies p exactly as the point
 * p + (eps, delta), 0 < delta << eps infinitesimal, would be classified by the
 * even-odd rule, so every point (including boundary points) has one answer.
 *
 * Arithmetic: coordinates are int32; f, d and p - r_i are formed in int64 and
 * line_pos in 128-bit integers, so no step rounds or overflows for any int32
 * input.  Work is split over points with POSIX threads (the paper parallelises
 * over points with Numba prange, Algorithm 4).
 *
 * oracle_classify_rule also evaluates the paper's printed algorithms literally,
 * to measure how often their rule differs from the one above:
 *   rule 1 (Algorithm 1, Constraint 1): an edge is a candidate when
 *          f_i * f_{i+1} <= 0 (both vertices on or across the ray, horizontal
 *          edges on the ray included), n = (d_y, -d_x) flipped when n_x < 0,
 *          and it counts when (p - r_i) . n <= 0 -- exact integers;
 *   rule 2 (Algorithm 2, Constraint 2): the same candidates, the crossing
 *          abscissa x_new = x_i + ((p_y - y_i) / d_y) d_x in IEEE float64 (a
 *          division 0/0 gives NaN), and it counts when x_new > p_x.  The
 *          float64 operations are the three the algorithm writes, each rounded
 *          once (the file is compiled without floating-point contraction).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef __int128 i128;

/* One point against one polygon: Method, steps 2-7 with Constraint 1. */
static int oracle_point_in_polygon(int64_t px, int64_t py, const int32_t *v, int64_t m)
{
    int64_t count = 0;
    for (int64_t i = 0; i < m; ++i) {
        int64_t j = (i + 1 == m) ? 0 : i + 1;
        int64_t x_i = v[2 * i], y_i = v[2 * i + 1];
        int64_t x_j = v[2 * j], y_j = v[2 * j + 1];
        int64_t f_i = y_i - py;                 /* step 2 */
        int64_t f_j = y_j - py;
        if ((f_i > 0) == (f_j > 0))             /* steps 3-4, half-open */
            continue;
        int64_t d_x = x_j - x_i, d_y = y_j - y_i;   /* d_y != 0 here */
        int64_t n_x = d_y, n_y = -d_x;              /* normal to the edge */
        if (n_x < 0) { n_x = -n_x; n_y = -n_y; }    /* acute with (1, 0) */
        i128 line_pos = (i128)(px - x_i) * n_x + (i128)(py - y_i) * n_y;
        if (line_pos < 0)                       /* crossing right of p */
            ++count;
    }
    return (int)(count & 1);                    /* step 7 */
}

/* Algorithm 1 as printed (Constraint 1, inclusive tests). */
static int paper_alg1(int64_t px, int64_t py, const int32_t *v, int64_t m)
{
    int64_t counted = 0;
    for (int64_t e = 0; e < m; ++e) {
        const int32_t *r = v + 2 * e, *s = v + 2 * ((e + 1 < m) ? e + 1 : 0);
        int64_t fa = (int64_t)r[1] - py, fb = (int64_t)s[1] - py;
        if ((i128)fa * fb > 0)                  /* not a candidate */
            continue;
        int64_t nx = (int64_t)s[1] - r[1], ny = (int64_t)r[0] - s[0];
        if (nx < 0) { nx = -nx; ny = -ny; }
        i128 lp = (i128)(px - r[0]) * nx + (i128)(py - r[1]) * ny;
        if (lp <= 0)
            ++counted;
    }
    return (int)(counted & 1);
}

/* Algorithm 2 as printed (Constraint 2, float64 crossing abscissa). */
static int paper_alg2(int64_t px, int64_t py, const int32_t *v, int64_t m)
{
    int64_t counted = 0;
    for (int64_t e = 0; e < m; ++e) {
        const int32_t *r = v + 2 * e, *s = v + 2 * ((e + 1 < m) ? e + 1 : 0);
        int64_t fa = (int64_t)r[1] - py, fb = (int64_t)s[1] - py;
        if ((i128)fa * fb > 0)
            continue;
        double dxe = (double)((int64_t)s[0] - r[0]), dye = (double)((int64_t)s[1] - r[1]);
        double lam = (double)(py - r[1]) / dye;      /* NaN when 0 / 0 */
        double x_new = (double)r[0] + lam * dxe;
        if (x_new > (double)px)
            ++counted;
    }
    return (int)(counted & 1);
}

static int classify_point(int rule, int64_t px, int64_t py, const int32_t *v, int64_t m)
{
    if (rule == 1) return paper_alg1(px, py, v, m);
    if (rule == 2) return paper_alg2(px, py, v, m);
    return oracle_point_in_polygon(px, py, v, m);
}

int oracle_pip_single(int32_t px, int32_t py, const int32_t *verts, int64_t m)
{
    if (m < 0 || (m > 0 && !verts)) return -1;
    return oracle_point_in_polygon(px, py, verts, m);
}

/* Shared description of one classify job (CSR or dense). */
typedef struct {
    const int32_t *points;
    int64_t n_points;
    const int32_t *poly_offsets;
    const int32_t *verts;
    int32_t n_polys;
    const int32_t *cand_offsets;
    const int32_t *cand_ids;
    uint32_t *out_bits;
    int64_t n_bits;          /* candidates (CSR) or n_polys * 32 * W (dense) */
    int64_t words_per_poly;  /* dense only: W = ceil(n_points / 32) */
    int64_t word_lo, word_hi;
    int rule;                /* 0 half-open (the method), 1 Algorithm 1, 2 Algorithm 2 */
} job_t;

/* Largest k with cand_offsets[k] <= c (the polygon owning candidate c). */
static int64_t owner_of(const job_t *J, int64_t c)
{
    int64_t lo = 0, hi = J->n_polys; /* answer in [lo, hi) ; -1 if none */
    if (J->n_polys == 0 || (int64_t)J->cand_offsets[0] > c) return -1;
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if ((int64_t)J->cand_offsets[mid] <= c) lo = mid; else hi = mid;
    }
    return lo;
}

static void *run_words(void *arg)
{
    job_t *J = (job_t *)arg;
    for (int64_t w = J->word_lo; w < J->word_hi; ++w) {
        uint32_t word = 0;
        for (int b = 0; b < 32; ++b) {
            int64_t c = w * 32 + b;
            if (c >= J->n_bits) break;
            int64_t k, pid;
            if (J->cand_offsets) {
                k = owner_of(J, c);
                if (k < 0 || (int64_t)J->cand_offsets[k + 1] <= c) continue;
                pid = J->cand_ids[c];
            } else {
                k = c / (32 * J->words_per_poly);
                pid = c - k * 32 * J->words_per_poly;
                if (pid >= J->n_points) continue;
            }
            int64_t v0 = J->poly_offsets[k], v1 = J->poly_offsets[k + 1];
            int bit = classify_point(J->rule, J->points[2 * pid], J->points[2 * pid + 1],
                                     J->verts + 2 * v0, v1 - v0);
            word |= (uint32_t)bit << b;
        }
        J->out_bits[w] = word;
    }
    return NULL;
}

/*
 * Classify with the same argument layout as the GPU library, host pointers.
 *   points       int32 [n_points][2]  (x, y)
 *   poly_offsets int32 [n_polys + 1]  polygon k owns verts[poly_offsets[k] .. poly_offsets[k+1])
 *   verts        int32 [V][2]
 *   cand_offsets int32 [n_polys + 1], cand_ids int32 [C]: CSR candidate lists; both NULL
 *                selects dense mode (every point against every polygon).
 *   out_bits     uint32: CSR -> ceil(C / 32) words, bit c = candidate c;
 *                dense -> n_polys * W words, W = ceil(n_points / 32), bit k*32*W + j.
 *   n_threads    <= 0 means one thread.
 * Returns 0, or -1 on a NULL or size error.
 */
int oracle_classify_rule(const int32_t *points, int64_t n_points,
                         const int32_t *poly_offsets, const int32_t *verts, int32_t n_polys,
                         const int32_t *cand_offsets, const int32_t *cand_ids,
                         int rule, uint32_t *out_bits, int n_threads)
{
    if (n_points < 0 || n_polys < 0 || rule < 0 || rule > 2) return -1;
    if ((cand_offsets == NULL) != (cand_ids == NULL)) return -1;
    if (n_polys > 0 && !poly_offsets) return -1;
    job_t base;
    memset(&base, 0, sizeof base);
    base.points = points; base.n_points = n_points;
    base.poly_offsets = poly_offsets; base.verts = verts; base.n_polys = n_polys;
    base.cand_offsets = cand_offsets; base.cand_ids = cand_ids; base.out_bits = out_bits;
    base.rule = rule;
    if (cand_offsets) {
        base.n_bits = n_polys > 0 ? cand_offsets[n_polys] : 0;
    } else {
        base.words_per_poly = (n_points + 31) / 32;
        base.n_bits = (int64_t)n_polys * 32 * base.words_per_poly;
    }
    int64_t n_words = (base.n_bits + 31) / 32;
    if (n_words == 0) return 0;
    if (!out_bits) return -1;
    if (n_threads <= 0) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    if (n_threads > n_words) n_threads = (int)n_words;
    job_t jobs[256];
    pthread_t tid[256];
    for (int t = 0; t < n_threads; ++t) {
        jobs[t] = base;
        jobs[t].word_lo = n_words * t / n_threads;
        jobs[t].word_hi = n_words * (t + 1) / n_threads;
    }
    for (int t = 1; t < n_threads; ++t)
        pthread_create(&tid[t], NULL, run_words, &jobs[t]);
    run_words(&jobs[0]);
    for (int t = 1; t < n_threads; ++t)
        pthread_join(tid[t], NULL);
    return 0;
}

int oracle_classify(const int32_t *points, int64_t n_points,
                    const int32_t *poly_offsets, const int32_t *verts, int32_t n_polys,
                    const int32_t *cand_offsets, const int32_t *cand_ids,
                    uint32_t *out_bits, int n_threads)
{
    return oracle_classify_rule(points, n_points, poly_offsets, verts, n_polys, cand_offsets,
                                cand_ids, 0, out_bits, n_threads);
}

/*
 * Sampled classify: bit for each listed candidate index (CSR) or listed
 * (polygon, point) pair in dense mode (index k*32*W + j).  out[s] = 0/1.
 */
int oracle_classify_sample(const int32_t *points, int64_t n_points,
                           const int32_t *poly_offsets, const int32_t *verts, int32_t n_polys,
                           const int32_t *cand_offsets, const int32_t *cand_ids,
                           const int64_t *sample, int64_t n_sample, uint8_t *out)
{
    job_t J;
    memset(&J, 0, sizeof J);
    J.points = points; J.n_points = n_points; J.poly_offsets = poly_offsets;
    J.verts = verts; J.n_polys = n_polys; J.cand_offsets = cand_offsets; J.cand_ids = cand_ids;
    if (cand_offsets) J.n_bits = n_polys > 0 ? cand_offsets[n_polys] : 0;
    else { J.words_per_poly = (n_points + 31) / 32; J.n_bits = (int64_t)n_polys * 32 * J.words_per_poly; }
    for (int64_t s = 0; s < n_sample; ++s) {
        int64_t c = sample[s], k, pid;
        out[s] = 0;
        if (c < 0 || c >= J.n_bits) return -1;
        if (cand_offsets) {
            k = owner_of(&J, c);
            if (k < 0 || (int64_t)cand_offsets[k + 1] <= c) continue;
            pid = cand_ids[c];
        } else {
            k = c / (32 * J.words_per_poly);
            pid = c - k * 32 * J.words_per_poly;
            if (pid >= n_points) continue;
        }
        int64_t v0 = poly_offsets[k], v1 = poly_offsets[k + 1];
        out[s] = (uint8_t)oracle_point_in_polygon(points[2 * pid], points[2 * pid + 1],
                                                  verts + 2 * v0, v1 - v0);
    }
    return 0;
}

/*
 * Closed-bounding-box join for a list of polygons, by brute force over all
 * points: counts[s] = #{ j : x_min <= x_j <= x_max and y_min <= y_j <= y_max }
 * for polygon polys[s], and (if ids != NULL) the matching point ids in
 * ascending order, polygon after polygon, in ids[] (capacity ids_cap).
 * This is the candidate set that a uniform-grid binning pass must produce.
 * Returns the total number of ids, or -1 if ids_cap is too small.
 */
int64_t oracle_bbox_join(const int32_t *points, int64_t n_points,
                         const int32_t *poly_offsets, const int32_t *verts,
                         const int32_t *polys, int64_t n_list,
                         int64_t *counts, int32_t *ids, int64_t ids_cap)
{
    int64_t total = 0;
    for (int64_t s = 0; s < n_list; ++s) {
        int64_t k = polys[s];
        int64_t v0 = poly_offsets[k], v1 = poly_offsets[k + 1];
        int64_t cnt = 0;
        if (v1 > v0) {
            int32_t x0 = verts[2 * v0], x1 = x0, y0 = verts[2 * v0 + 1], y1 = y0;
            for (int64_t v = v0 + 1; v < v1; ++v) {
                int32_t x = verts[2 * v], y = verts[2 * v + 1];
                if (x < x0) x0 = x;
                if (x > x1) x1 = x;
                if (y < y0) y0 = y;
                if (y > y1) y1 = y;
            }
            for (int64_t j = 0; j < n_points; ++j) {
                int32_t x = points[2 * j], y = points[2 * j + 1];
                if (x >= x0 && x <= x1 && y >= y0 && y <= y1) {
                    if (ids) {
                        if (total + cnt >= ids_cap) return -1;
                        ids[total + cnt] = (int32_t)j;
                    }
                    ++cnt;
                }
            }
        }
        counts[s] = cnt;
        total += cnt;
    }
    return total;
}
