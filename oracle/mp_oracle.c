/*
 * CPU reference ("oracle") for the dictionary AB-join -- TEST INFRASTRUCTURE.
 *
 * Only the test suite, the package smoke check and the benchmark's CPU
 * baseline use this file. The GPU library never links, loads or calls it, and
 * it shares no code, header or table with the GPU library.
 *
 * What it computes, in float64, by the plain definitions of the paper:
 *
 *   * Def. 2 / Def. 3 (Sec. 2.1): the length-m subsequences (windows) of a
 *     series, indexed from 0 here (the paper indexes from 1).
 *   * Sec. 2.1, z-normalised Euclidean distance: each window is z-normalised,
 *     z(x) = (x - mean(x)) / std(x) with the population standard deviation,
 *     and the distance is the Euclidean norm of the difference. The paper names
 *     the distance without printing a formula; this is the textbook one.
 *     A window whose m samples all compare equal is "constant"; its
 *     z-normalisation is taken to be the zero vector (the paper is silent on
 *     this case), so d(constant, non-constant) = sqrt(m) and
 *     d(constant, constant) = 0.
 *   * Def. 8 (Sec. 3.3): the windows of a dictionary slide inside each
 *     dictionary element (segment); no window crosses a segment boundary.
 *   * Algorithm 2 (Sec. 3.2): the approximate matrix profile starts at +inf,
 *     and for each segment the 1NN join of the query with that segment is
 *     merged in by an element-wise minimum. The nearest-neighbour index
 *     (Def. 5 / Def. 6: the partner in the similarity join set) is returned as
 *     the global window index g, i.e. the window's start offset in the
 *     concatenated segment buffer. On exactly equal distances the lowest g
 *     wins (the paper does not say how ties are broken).
 *
 * Parity is pinned outside this file (brute-force cross-checks, closed forms,
 * invariants and the paper's Lemma 1 / Lemma 2 guarantees).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MPO_OK 0
#define MPO_EARG -1
#define MPO_ENOMEM -2

/* 1 if all m samples of x compare equal (the window is constant). */
int mpo_window_is_constant(const double *x, int32_t m)
{
    for (int32_t k = 1; k < m; ++k)
        if (!(x[k] == x[0]))
            return 0;
    return 1;
}

/* Mean and population standard deviation of one window, two passes. */
void mpo_window_mean_std(const double *x, int32_t m, double *mean, double *std)
{
    double s = 0.0;
    for (int32_t k = 0; k < m; ++k)
        s += x[k];
    const double mu = s / (double)m;
    double v = 0.0;
    for (int32_t k = 0; k < m; ++k) {
        const double d = x[k] - mu;
        v += d * d;
    }
    *mean = mu;
    *std = sqrt(v / (double)m);
}

/* Statistics of every window of a series of length n (n - m + 1 windows). */
int mpo_window_stats(const double *x, int64_t n, int32_t m, double *mean, double *std, uint8_t *is_const)
{
    if (!x || !mean || !std || !is_const || m < 1 || n < m)
        return MPO_EARG;
    const int64_t nw = n - m + 1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nw; ++i) {
        is_const[i] = (uint8_t)mpo_window_is_constant(x + i, m);
        mpo_window_mean_std(x + i, m, &mean[i], &std[i]);
    }
    return MPO_OK;
}

/*
 * z-normalised Euclidean distance of two windows given their statistics.
 * A constant window normalises to the zero vector and a non-constant one to a
 * vector of squared norm exactly m (population std), so the mixed case is
 * sqrt(m) and the all-constant case 0; both are returned exactly, which keeps
 * the lowest-index rule meaningful among the equal distances they produce.
 */
static double znorm_distance(const double *x, double mx, double sx, int cx,
                             const double *y, double my, double sy, int cy, int32_t m)
{
    if (cx && cy)
        return 0.0;
    if (cx || cy)
        return sqrt((double)m);
    double acc = 0.0;
    for (int32_t k = 0; k < m; ++k) {
        const double zx = (x[k] - mx) / sx;
        const double zy = (y[k] - my) / sy;
        const double d = zx - zy;
        acc += d * d;
    }
    return sqrt(acc);
}

/* Distance of two length-m windows, computing their statistics first. */
double mpo_pair_distance(const double *x, const double *y, int32_t m)
{
    double mx, sx, my, sy;
    mpo_window_mean_std(x, m, &mx, &sx);
    mpo_window_mean_std(y, m, &my, &sy);
    return znorm_distance(x, mx, sx, mpo_window_is_constant(x, m), y, my, sy, mpo_window_is_constant(y, m), m);
}

/*
 * The dictionary AB-join (Algorithm 2).
 *
 *   a, na          query series T_A (na samples)
 *   b, offs, nseg  dictionary D_B: segment s is b[offs[s] .. offs[s+1])
 *   m              window length
 *   rows, nrows    which query windows to evaluate (rows == NULL: all of
 *                  0 .. na-m, and nrows must then be na-m+1)
 *   dist, idx      out, per evaluated row: nearest-neighbour distance and the
 *                  global window index g of the neighbour (+inf / -1 when the
 *                  dictionary has no window of length m)
 *   dist2          out (may be NULL): smallest distance over all windows other
 *                  than idx (+inf if there is none); the gap dist2 - dist says
 *                  whether the nearest neighbour is unique to a tolerance
 *   nthreads       OpenMP threads (<= 0: the runtime's default)
 */
int mpo_ab_join(const double *a, int64_t na, const double *b, const int64_t *offs, int32_t nseg, int32_t m,
                const int64_t *rows, int64_t nrows, double *dist, int64_t *idx, double *dist2, int nthreads)
{
    if (!a || !b || !offs || !dist || !idx || m < 1 || na < m || nseg < 0 || nrows < 0)
        return MPO_EARG;
    const int64_t nq = na - m + 1;
    if (!rows && nrows != nq)
        return MPO_EARG;
    for (int32_t s = 0; s < nseg; ++s)
        if (offs[s + 1] < offs[s])
            return MPO_EARG;
    for (int64_t r = 0; rows && r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= nq)
            return MPO_EARG;

    /* Statistics of every dictionary window that lies inside one segment. */
    const int64_t total = offs[nseg] - offs[0];
    double *bm = NULL, *bs = NULL;
    uint8_t *bc = NULL;
    if (total > 0) {
        bm = (double *)malloc(sizeof(double) * (size_t)total);
        bs = (double *)malloc(sizeof(double) * (size_t)total);
        bc = (uint8_t *)malloc((size_t)total);
        if (!bm || !bs || !bc) {
            free(bm); free(bs); free(bc);
            return MPO_ENOMEM;
        }
        for (int32_t s = 0; s < nseg; ++s) {
            const int64_t L = offs[s + 1] - offs[s];
            for (int64_t o = 0; o + m <= L; ++o) {
                const int64_t g = offs[s] + o - offs[0];
                bc[g] = (uint8_t)mpo_window_is_constant(b + offs[s] + o, m);
                mpo_window_mean_std(b + offs[s] + o, m, &bm[g], &bs[g]);
            }
        }
    }

#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif

#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t i = rows ? rows[r] : r;
        const double *x = a + i;
        double mx, sx;
        mpo_window_mean_std(x, m, &mx, &sx);
        const int cx = mpo_window_is_constant(x, m);

        double best = INFINITY, second = INFINITY;
        int64_t best_g = -1;
        for (int32_t s = 0; s < nseg; ++s) {
            /* P_AD: the 1NN join of this query window with segment s. */
            const int64_t L = offs[s + 1] - offs[s];
            double seg_best = INFINITY;
            int64_t seg_g = -1;
            for (int64_t o = 0; o + m <= L; ++o) {
                const int64_t g = offs[s] + o;
                const int64_t gl = g - offs[0];
                const double d = znorm_distance(x, mx, sx, cx, b + g, bm[gl], bs[gl], bc[gl], m);
                if (d < seg_best) {
                    if (seg_best < second) second = seg_best;
                    seg_best = d;
                    seg_g = g;
                } else if (d < second) {
                    second = d;
                }
            }
            /* ElementwiseMin of the running profile with P_AD. */
            if (seg_g >= 0) {
                if (seg_best < best) {
                    if (best < second) second = best;
                    best = seg_best;
                    best_g = seg_g;
                } else if (seg_best < second) {
                    second = seg_best;
                }
            }
        }
        dist[r] = best;
        idx[r] = best_g;
        if (dist2)
            dist2[r] = second;
    }
    free(bm);
    free(bs);
    free(bc);
    return MPO_OK;
}

/*
 * The self-join matrix profile of one series (the P_B of Algorithm 1,
 * Sec. 3.1): for every window i, the nearest window g of the same series with
 * |g - i| >= excl (closer windows overlap i and are its trivial matches),
 * lowest g on ties; +inf / -1 if no window lies outside the zone.
 */
int mpo_self_join(const double *a, int64_t na, int32_t m, int32_t excl, double *dist, int64_t *idx, int nthreads)
{
    if (!a || !dist || !idx || m < 1 || na < m || excl < 1)
        return MPO_EARG;
    const int64_t nq = na - m + 1;
    double *mu = (double *)malloc(sizeof(double) * (size_t)nq);
    double *sd = (double *)malloc(sizeof(double) * (size_t)nq);
    uint8_t *cs = (uint8_t *)malloc((size_t)nq);
    if (!mu || !sd || !cs) {
        free(mu); free(sd); free(cs);
        return MPO_ENOMEM;
    }
    for (int64_t g = 0; g < nq; ++g) {
        cs[g] = (uint8_t)mpo_window_is_constant(a + g, m);
        mpo_window_mean_std(a + g, m, &mu[g], &sd[g]);
    }
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < nq; ++i) {
        double best = INFINITY;
        int64_t best_g = -1;
        for (int64_t g = 0; g < nq; ++g) {
            if (g > i - excl && g < i + excl)
                continue; /* trivial match */
            const double d = znorm_distance(a + i, mu[i], sd[i], cs[i], a + g, mu[g], sd[g], cs[g], m);
            if (d < best) {
                best = d;
                best_g = g;
            }
        }
        dist[i] = best;
        idx[i] = best_g;
    }
    free(mu);
    free(sd);
    free(cs);
    return MPO_OK;
}
