/*
 * oracle.c -- plain, slow CPU oracle for grid resistance (gres).
 *
 * TEST INFRASTRUCTURE ONLY. The product path never calls this file: only the
 * tests, the package's smoke check and the CPU-baseline leg of the benchmark
 * load it. It shares no code, header, table or helper with the CUDA library.
 *
 * Everything here follows the paper's definitions literally and favours
 * obviousness over speed:
 *   - dominance and skyline:       Def. 1 (Sec. 2)
 *   - grid projection gproj(t, g): Sec. 2, the lowest corner of t's cell
 *   - grid resistance gres(t; r):  Def. 2 (Sec. 2), Algorithm 1 (Sec. 3.2)
 *   - stability of gres:           Sec. 3.2 (gres ignores dominated tuples)
 *   - the bound g_bar = floor(1/l): Sec. 3.2, l the smallest non-zero
 *                                   same-attribute difference
 *   - Grid / Angular / Sliced partition numbers: Sec. 3.1
 *
 * Fixed-point reading (values are integers, no floating point decides a
 * result): a value v stands for the real v / 2^B. A grid of cell width delta
 * (an integer) projects v to floor(v / delta); with delta = 2^B / g this is the
 * paper's floor(t[i] * g) exactly. Step lists are ascending widths, so the
 * paper's scan g = g_bar, ..., 2 (coarser and coarser grids) is a scan over
 * ascending widths, and "the first g at which t leaves the skyline" is the
 * first index k in the step list. The result is that index, or K when t never
 * leaves (the paper's gres = 1).
 *
 * Direction: dir = 0 means smaller is better (the paper's convention,
 * Sec. 2); dir = 1 means larger is better (the opposite convention the paper
 * allows). With dir = 1 the projection is still the lowest corner
 * floor(v / delta) and only the comparisons flip.
 *
 * Parity of every function here is pinned by the "not gpu" tests (hand cases,
 * brute force on tiny inputs, invariants, the paper's Grid example).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- Def. 1: dominance ------------------------------------------------ */

/* 1 iff s dominates t: s is at least as good in every attribute and strictly
 * better in one. Equal tuples do not dominate each other. */
int oracle_dominates(const uint32_t *s, const uint32_t *t, int d, int dir)
{
    int strictly_better_somewhere = 0;
    for (int i = 0; i < d; i++) {
        if (dir == 0) {
            if (s[i] > t[i]) return 0;
            if (s[i] < t[i]) strictly_better_somewhere = 1;
        } else {
            if (s[i] < t[i]) return 0;
            if (s[i] > t[i]) strictly_better_somewhere = 1;
        }
    }
    return strictly_better_somewhere;
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* ---- Def. 1: skyline, block-nested-loops (Borzsonyi et al., cited in Sec. 2)
 * Window kept in memory without limit. Each tuple, in input order, is dropped
 * if a window tuple dominates it; otherwise it evicts the window tuples it
 * dominates and joins the window. The final window is the skyline. Output:
 * row indices in ascending order. Returns the skyline size. */
int64_t oracle_skyline_bnl(const uint32_t *data, int64_t n, int d, int dir,
                           int64_t *out)
{
    int64_t *win = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t w = 0;
    for (int64_t x = 0; x < n; x++) {
        const uint32_t *tx = data + x * d;
        int dominated = 0;
        for (int64_t j = 0; j < w; j++) {
            if (oracle_dominates(data + win[j] * d, tx, d, dir)) { dominated = 1; break; }
        }
        if (dominated) continue;
        int64_t keep = 0;
        for (int64_t j = 0; j < w; j++) {
            if (!oracle_dominates(tx, data + win[j] * d, d, dir)) win[keep++] = win[j];
        }
        w = keep;
        win[w++] = x;
    }
    qsort(win, (size_t)w, sizeof(int64_t), cmp_i64);
    memcpy(out, win, sizeof(int64_t) * (size_t)w);
    free(win);
    return w;
}

/* Def. 1 read directly: t is in the skyline iff no tuple of r dominates it.
 * Quadratic; for small inputs. Output ascending. */
int64_t oracle_skyline_allpairs(const uint32_t *data, int64_t n, int d, int dir,
                                int64_t *out)
{
    int64_t c = 0;
    for (int64_t x = 0; x < n; x++) {
        int dominated = 0;
        for (int64_t y = 0; y < n && !dominated; y++)
            if (oracle_dominates(data + y * d, data + x * d, d, dir)) dominated = 1;
        if (!dominated) out[c++] = x;
    }
    return c;
}

/* Def. 1 read directly for chosen rows: flag[j] = 1 iff no tuple of r
 * dominates row rows[j] (so flag[j] = 1 iff rows[j] is in Sky(r)). The same
 * test as the all-pairs skyline, asked row by row, so that a large input can
 * be checked on a sample of rows, or on every row with nthreads > 1 (OpenMP
 * over the rows asked about; each answer is independent of the others). */
void oracle_skyline_member(const uint32_t *data, int64_t n, int d, int dir,
                           const int64_t *rows, int64_t nrows, int32_t *flag, int nthreads)
{
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
    #pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
#else
    (void)nthreads;
#endif
    for (int64_t j = 0; j < nrows; j++) {
        const uint32_t *t = data + rows[j] * d;
        int dominated = 0;
        for (int64_t y = 0; y < n && !dominated; y++)
            if (oracle_dominates(data + y * d, t, d, dir)) dominated = 1;
        flag[j] = !dominated;
    }
}

/* ---- Sec. 2: grid projection, width form: floor(v / delta) -------------- */
void oracle_gproj(const uint32_t *v, int64_t count, uint32_t delta, uint32_t *out)
{
    for (int64_t i = 0; i < count; i++) out[i] = v[i] / delta;
}

/* Cell corner of a whole tuple: q[i] = floor(t[i] / delta). */
static void project(const uint32_t *t, int d, uint32_t delta, uint32_t *q)
{
    for (int i = 0; i < d; i++) q[i] = t[i] / delta;
}

/* ---- Def. 2 / Algorithm 1: gres, pairwise form ---------------------------
 * For each target row t (targets[]), scan the steps in ascending width
 * order; t leaves the skyline of the projected relation at step k iff some
 * candidate row s has gproj(s) dominating gproj(t) (Def. 1 on projections).
 * out[j] = first such k, or K if none.
 * Candidates: any row set; by stability (Sec. 3.2) the full relation r and
 * its skyline Sky(r) give the same answer. nthreads > 1 splits the targets
 * over OpenMP threads (each target is independent). */
void oracle_gres(const uint32_t *data, int64_t n, int d, int dir,
                 const int64_t *cand, int64_t ncand,
                 const int64_t *targets, int64_t ntargets,
                 const uint32_t *steps, int32_t K, int32_t *out, int nthreads)
{
    (void)n;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
    #pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#else
    (void)nthreads;
#endif
    for (int64_t j = 0; j < ntargets; j++) {
        const uint32_t *t = data + targets[j] * d;
        uint32_t qt[64], qs[64];
        int32_t result = K;
        for (int32_t k = 0; k < K && result == K; k++) {
            project(t, d, steps[k], qt);
            for (int64_t c = 0; c < ncand; c++) {
                project(data + cand[c] * d, d, steps[k], qs);
                if (oracle_dominates(qs, qt, d, dir)) { result = k; break; }
            }
        }
        out[j] = result;
    }
}

/* ---- Algorithm 1, literal set form (tiny inputs) -------------------------
 * For each step (ascending widths = the paper's g from g_bar down to 2):
 * build the SET gproj(r, delta_k) (duplicates removed), compute its skyline
 * with Def. 1, and mark every target whose projection is not a member and
 * has no value yet. Unmarked targets get K (the paper's gres = 1).
 * Returns 0, or -1 on allocation failure. */
static int g_d_for_sort;
static int cmp_row(const void *a, const void *b)
{
    const uint32_t *x = (const uint32_t *)a, *y = (const uint32_t *)b;
    for (int i = 0; i < g_d_for_sort; i++) {
        if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
    }
    return 0;
}

int oracle_gres_literal(const uint32_t *data, int64_t n, int d, int dir,
                        const int64_t *targets, int64_t ntargets,
                        const uint32_t *steps, int32_t K, int32_t *out)
{
    uint32_t *set = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n * d + 1));
    uint32_t *sky = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n * d + 1));
    if (!set || !sky) { free(set); free(sky); return -1; }
    for (int64_t j = 0; j < ntargets; j++) out[j] = -1;           /* nil */
    for (int32_t k = 0; k < K; k++) {
        /* gproj(r, delta_k) as a set */
        for (int64_t x = 0; x < n; x++) project(data + x * d, d, steps[k], set + x * d);
        g_d_for_sort = d;
        qsort(set, (size_t)n, sizeof(uint32_t) * (size_t)d, cmp_row);
        int64_t m = 0;
        for (int64_t x = 0; x < n; x++) {
            if (m == 0 || cmp_row(set + (m - 1) * d, set + x * d) != 0) {
                memmove(set + m * d, set + x * d, sizeof(uint32_t) * (size_t)d);
                m++;
            }
        }
        /* s' = Sky(gproj(r, delta_k)) */
        int64_t ns = 0;
        for (int64_t x = 0; x < m; x++) {
            int dominated = 0;
            for (int64_t y = 0; y < m && !dominated; y++)
                if (oracle_dominates(set + y * d, set + x * d, d, dir)) dominated = 1;
            if (!dominated) { memcpy(sky + ns * d, set + x * d, sizeof(uint32_t) * (size_t)d); ns++; }
        }
        /* membership of gproj(t, delta_k) in s' */
        for (int64_t j = 0; j < ntargets; j++) {
            if (out[j] != -1) continue;
            uint32_t qt[64];
            project(data + targets[j] * d, d, steps[k], qt);
            int member = 0;
            for (int64_t y = 0; y < ns && !member; y++)
                if (memcmp(sky + y * d, qt, sizeof(uint32_t) * (size_t)d) == 0) member = 1;
            if (!member) out[j] = k;
        }
    }
    for (int64_t j = 0; j < ntargets; j++) if (out[j] == -1) out[j] = K;
    free(set); free(sky);
    return 0;
}

/* ---- Sec. 2 with the paper's own grid parameter g ------------------------
 * Values v stand for v / 2^bits in [0, 1). gproj(t, g)[i] = floor(t[i] * g)
 * (the numerator of the paper's floor(t[i] g) / g). The g values are scanned
 * in the order given; Algorithm 1 scans g = g_bar, g_bar - 1, ..., 2.
 * out[j] is the first g at which t leaves the skyline, or 1 if it never does
 * (gres = 1/out[j]). */
void oracle_gres_glist(const uint32_t *data, int64_t n, int d, int dir, int bits,
                       const int64_t *cand, int64_t ncand,
                       const int64_t *targets, int64_t ntargets,
                       const uint32_t *glist, int32_t ng, int32_t *out)
{
    (void)n;
    for (int64_t j = 0; j < ntargets; j++) {
        const uint32_t *t = data + targets[j] * d;
        int32_t result = 1;
        for (int32_t gi = 0; gi < ng && result == 1; gi++) {
            uint64_t g = glist[gi];
            uint32_t qt[64], qs[64];
            for (int i = 0; i < d; i++) qt[i] = (uint32_t)(((uint64_t)t[i] * g) >> bits);
            for (int64_t c = 0; c < ncand; c++) {
                const uint32_t *s = data + cand[c] * d;
                for (int i = 0; i < d; i++) qs[i] = (uint32_t)(((uint64_t)s[i] * g) >> bits);
                if (oracle_dominates(qs, qt, d, dir)) { result = (int32_t)g; break; }
            }
        }
        out[j] = result;
    }
}

/* ---- Sec. 3.2: l, the smallest non-zero difference between two values of
 * the same attribute (0 if every attribute is constant). In fixed point the
 * bound g_bar = floor(1 / l) reads floor(2^bits / l). */
uint32_t oracle_min_gap(const uint32_t *data, int64_t n, int d)
{
    uint32_t best = 0;
    for (int i = 0; i < d; i++)
        for (int64_t x = 0; x < n; x++)
            for (int64_t y = 0; y < n; y++) {
                uint32_t a = data[x * d + i], b = data[y * d + i];
                uint32_t diff = a > b ? a - b : b - a;
                if (diff != 0 && (best == 0 || diff < best)) best = diff;
            }
    return best;
}

/* ---- Sec. 3.1: partitioning strategies ----------------------------------
 * All three work on the "better-is-smaller" view of the rows: with dir = 1
 * a value v is read as 0xFFFFFFFF - v. Coordinates are taken relative to the
 * per-attribute range [lo_i, hi_i] of the rows given, so a partition number
 * never depends on values outside the input. */
static uint32_t view(uint32_t v, int dir) { return dir == 0 ? v : 0xFFFFFFFFu - v; }

static void ranges(const uint32_t *data, int64_t n, int d, int dir, uint32_t *lo, uint32_t *hi)
{
    for (int i = 0; i < d; i++) { lo[i] = 0xFFFFFFFFu; hi[i] = 0; }
    for (int64_t x = 0; x < n; x++)
        for (int i = 0; i < d; i++) {
            uint32_t v = view(data[x * d + i], dir);
            if (v < lo[i]) lo[i] = v;
            if (v > hi[i]) hi[i] = v;
        }
}

/* Grid: cell coordinate c_i = floor((v_i - lo_i) * m / (hi_i - lo_i + 1)),
 * in [0, m-1]; partition number p = sum_i c_i * m^i (0-based attributes). */
void oracle_grid_pid(const uint32_t *data, int64_t n, int d, int dir, int m, int64_t *out)
{
    uint32_t lo[64], hi[64];
    ranges(data, n, d, dir, lo, hi);
    for (int64_t x = 0; x < n; x++) {
        int64_t p = 0, w = 1;
        for (int i = 0; i < d; i++) {
            uint64_t span = (uint64_t)hi[i] - lo[i] + 1;
            uint64_t c = ((uint64_t)(view(data[x * d + i], dir) - lo[i]) * (uint64_t)m) / span;
            p += (int64_t)c * w;
            w *= m;
        }
        out[x] = p;
    }
}

/* Grid dominance between cells (Sec. 3.1): cell a grid-dominates cell b iff
 * a's coordinate is strictly smaller in every dimension. Cells are given by
 * their partition numbers p = sum_i c_i m^i. */
int oracle_cell_grid_dominates(int64_t a, int64_t b, int d, int m)
{
    for (int i = 0; i < d; i++) {
        if (a % m >= b % m) return 0;
        a /= m; b /= m;
    }
    return 1;
}

/* Angular: hyperspherical angles of x = v - lo,
 * phi_i = atan2(sqrt(x_{i+1}^2 + ... + x_{d-1}^2), x_i), i = 0 .. d-2 (in
 * [0, pi/2]), bin_i = floor(2 phi_i m / pi) clamped to m - 1 (Eq. 1), and
 * p = sum_i bin_i m^i. The bin is the number of thresholds j pi / (2m),
 * j = 1 .. m-1, that phi_i reaches. phi_i >= theta is decided exactly as
 * Y >= X tan^2(theta) with Y = sum_{j>i} x_j^2, X = x_i^2, in 128-bit
 * integers against tan^2(theta) rounded to 32 fractional bits; phi = 0 when
 * X = Y = 0. */
void oracle_angular_pid(const uint32_t *data, int64_t n, int d, int dir, int m, int64_t *out)
{
    uint32_t lo[64], hi[64];
    unsigned __int128 thr[64];
    const double pi = 3.14159265358979323846;
    ranges(data, n, d, dir, lo, hi);
    for (int j = 1; j < m; j++) {
        double t = tan((double)j * pi / (2.0 * (double)m));
        thr[j] = (unsigned __int128)llround(t * t * 4294967296.0);
    }
    for (int64_t x = 0; x < n; x++) {
        int64_t p = 0, w = 1;
        for (int i = 0; i + 1 < d; i++) {
            unsigned __int128 X, Y = 0;
            uint64_t xi = view(data[x * d + i], dir) - lo[i];
            X = (unsigned __int128)xi * xi;
            for (int j = i + 1; j < d; j++) {
                uint64_t xj = view(data[x * d + j], dir) - lo[j];
                Y += (unsigned __int128)xj * xj;
            }
            int bin = 0;
            if (!(X == 0 && Y == 0)) {
                for (int j = 1; j < m; j++)
                    if ((Y << 32) >= X * thr[j]) bin = j;
            }
            p += (int64_t)bin * w;
            w *= m;
        }
        out[x] = p;
    }
}

/* Sliced: order the rows by one chosen attribute (ties: lower row first);
 * the i-th row (0-based) of that order gets p = floor(i * p / n). */
static const uint32_t *g_sl_data; static int g_sl_d, g_sl_dim, g_sl_dir;
static int cmp_sliced(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    uint32_t vx = view(g_sl_data[x * g_sl_d + g_sl_dim], g_sl_dir);
    uint32_t vy = view(g_sl_data[y * g_sl_d + g_sl_dim], g_sl_dir);
    if (vx != vy) return vx < vy ? -1 : 1;
    return (x > y) - (x < y);
}

void oracle_sliced_pid(const uint32_t *data, int64_t n, int d, int dir, int dim, int p,
                       int64_t *out)
{
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t x = 0; x < n; x++) order[x] = x;
    g_sl_data = data; g_sl_d = d; g_sl_dim = dim; g_sl_dir = dir;
    qsort(order, (size_t)n, sizeof(int64_t), cmp_sliced);
    for (int64_t i = 0; i < n; i++) out[order[i]] = (i * (int64_t)p) / n;
    free(order);
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
