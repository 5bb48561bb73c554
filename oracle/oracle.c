/*
 * FP64 CPU oracle for point-to-point correlation measures between ensemble
 * member vectors (arxiv 2309.03308, Section 3 and 3.2).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the
 * CUDA library is checked against. It shares no code with the library and the
 * library never calls it. Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load it.
 *
 * Conventions
 *   field F : fp32, member-major [n][P] (P grid points, x fastest), read-only.
 *   point ids are linear x + X*(y + Y*z).
 *   every floating-point result is FP64 unless a step is defined in fp32
 *   (bin index formula, KSG distances), where fp32 is emulated exactly by
 *   float arithmetic (the file is built with -ffp-contract=off, no fast-math).
 *
 * Readings of the paper where it is silent or garbled are marked READING.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_PEARSON = 0, OR_SPEARMAN = 1, OR_MI_BINNED = 2, OR_MI_KSG = 3 };

static void gather(const float* F, int64_t P, int n, int64_t p, float* out) {
    for (int m = 0; m < n; ++m) out[m] = F[(int64_t)m * P + p];
}

int or_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------
 * Pearson product-moment correlation (PPMCC), Section 3.2: means and
 * variances, then the normalised covariance. Two-pass FP64.
 * READING: a constant vector (zero variance) has correlation 0 by convention.
 */
double or_pearson_vec(const double* x, const double* y, int n) {
    double mx = 0.0, my = 0.0;
    for (int i = 0; i < n; ++i) {
        mx += x[i];
        my += y[i];
    }
    mx /= n;
    my /= n;
    double sxx = 0.0, syy = 0.0, sxy = 0.0;
    for (int i = 0; i < n; ++i) {
#ifdef PLANT_PEARSON_MEAN /* planted mistake, used only by the pin tests */
        double dx = x[i] - mx, dy = y[i];
#else
        double dx = x[i] - mx, dy = y[i] - my;
#endif
        sxx += dx * dx;
        syy += dy * dy;
        sxy += dx * dy;
    }
    if (sxx == 0.0 || syy == 0.0) return 0.0;
    return sxy / sqrt(sxx * syy);
}

/* ---------------------------------------------------------------------------
 * Average ranks (Spearman; not in the paper, a project measure). For member i,
 * with L = #{j : x_j < x_i} and E = #{j : x_j == x_i} (E counts i itself), the
 * tied group occupies 1-based ranks L+1 .. L+E, whose average is L + (E+1)/2.
 * Returned doubled so it is an integer: rank2_i = 2L + E + 1.
 * Comparisons are IEEE fp32 comparisons, so -0.0 and +0.0 tie.
 */
void or_rank2(const float* x, int n, int32_t* rank2) {
    for (int i = 0; i < n; ++i) {
        int L = 0, E = 0;
        for (int j = 0; j < n; ++j) {
            if (x[j] < x[i]) ++L;
            else if (x[j] == x[i]) ++E;
        }
#ifdef PLANT_RANK_TIES /* planted mistake: ties get the lowest rank */
        rank2[i] = 2 * L + 2;
#else
        rank2[i] = 2 * L + E + 1;
#endif
    }
}

/* Spearman correlation: Pearson correlation of the average ranks. */
double or_spearman_vec(const float* x, const float* y, int n, double* wx, double* wy,
                       int32_t* rk) {
    or_rank2(x, n, rk);
    for (int i = 0; i < n; ++i) wx[i] = (double)rk[i];
    or_rank2(y, n, rk);
    for (int i = 0; i < n; ++i) wy[i] = (double)rk[i];
    return or_pearson_vec(wx, wy, n);
}

/* ---------------------------------------------------------------------------
 * Equal-width binning for the joint-histogram MI estimator (Section 3.2,
 * binning of the two continuous variables).
 * READING: each point is binned over its own member range [lo, hi]; bin
 *   b = floor(((v - lo) / (hi - lo)) * B), clamped to [0, B-1], every step an
 *   IEEE fp32 operation; hi == lo puts every member in bin 0.
 */
void or_bins(const float* x, int n, int B, uint8_t* out) {
    float lo = x[0], hi = x[0];
    for (int i = 1; i < n; ++i) {
        if (x[i] < lo) lo = x[i];
        if (x[i] > hi) hi = x[i];
    }
    if (!(hi > lo)) {
        for (int i = 0; i < n; ++i) out[i] = 0;
        return;
    }
    const float w = hi - lo;
    for (int i = 0; i < n; ++i) {
#ifdef PLANT_BINS_FLIP /* planted mistake: measured from the top */
        float t = hi - x[i];
#else
        float t = x[i] - lo;
#endif
        float r = t / w;
        float s = r * (float)B;
        int b = (int)floorf(s);
        if (b < 0) b = 0;
        if (b > B - 1) b = B - 1;
        out[i] = (uint8_t)b;
    }
}

/*
 * Mutual information from the joint histogram of two binned variables,
 * Eq. (1) evaluated on the empirical distribution: sum over non-empty cells of
 * p_xy * ln(p_xy / (p_x p_y)), in nats (READING: natural log, as for KSG).
 */
double or_hist_mi_bins(const uint8_t* bx, const uint8_t* by, int n, int B) {
    int64_t* c = (int64_t*)calloc((size_t)B * B + 2 * B, sizeof(int64_t));
    int64_t* cx = c + (size_t)B * B;
    int64_t* cy = cx + B;
    for (int i = 0; i < n; ++i) {
        c[bx[i] * B + by[i]]++;
        cx[bx[i]]++;
        cy[by[i]]++;
    }
    double mi = 0.0;
    for (int a = 0; a < B; ++a)
        for (int b = 0; b < B; ++b) {
            int64_t cab = c[a * B + b];
            if (cab == 0) continue;
            double pxy = (double)cab / n;
#ifdef PLANT_HIST_LOG2 /* planted mistake: bits instead of nats */
            mi += pxy * log2((double)n * (double)cab / ((double)cx[a] * (double)cy[b]));
#else
            mi += pxy * log((double)n * (double)cab / ((double)cx[a] * (double)cy[b]));
#endif
        }
    free(c);
    return mi;
}

/* ---------------------------------------------------------------------------
 * Digamma at a positive integer, Eq. (2): psi(1) = -gamma and
 * psi(m+1) = psi(m) + 1/m, so psi(m) = -gamma + sum_{j=1}^{m-1} 1/j.
 * READING: every KSG argument is an integer in [1, n], so this exact harmonic
 * form replaces the paper's Lanczos approximation.
 */
double or_digamma_int(int m) {
    long double s = -0.577215664901532860606512090082402431L;
    for (int j = 1; j < m; ++j) s += 1.0L / (long double)j;
    return (double)s;
}

static int cmp_float(const void* a, const void* b) {
    float x = *(const float*)a, y = *(const float*)b;
    return (x > y) - (x < y);
}

/*
 * Kraskov (KSG) estimator, Section 3.2. Joint samples z_i = (x_i, y_i).
 *   d_ij   = max(|x_i - x_j|, |y_i - y_j|) (Chebyshev), each difference the
 *            correctly rounded fp32 difference (READING: bit-exact from the
 *            same fp32 inputs).
 *   eps_i  = k-th smallest d_ij over j != i, ties counted with multiplicity.
 *   n_x,i  = 1 + #{j != i : |x_i - x_j| < eps_i}; n_y,i likewise
 *            (READING: the paper's psi(n_x,i) is Kraskov's psi(n_x + 1); the
 *            comparison is strict, as the paper states).
 *   MI     = psi(n) + psi(k) - (1/n) sum_i [psi(n_x,i) + psi(n_y,i)]
 *            (READING: the garbled sum covers both digamma terms).
 * Brute force: all distances of i are sorted and the k-th is taken.
 * nx, ny, eps may be NULL; work holds n floats.
 */
double or_ksg_vec(const float* x, const float* y, int n, int k, int32_t* nx, int32_t* ny,
                  float* eps, float* work) {
    /* psi(1..n) by the recurrence of or_digamma_int, accumulated in long double */
    double* psi = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    long double acc = -0.577215664901532860606512090082402431L;
    for (int m = 1; m <= n; ++m) {
        psi[m] = (double)acc;
        acc += 1.0L / (long double)m;
    }
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
        int c = 0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            float dx = fabsf(x[i] - x[j]);
            float dy = fabsf(y[i] - y[j]);
            work[c++] = dx > dy ? dx : dy;
        }
        qsort(work, (size_t)c, sizeof(float), cmp_float);
        const float e = work[k - 1];
        int cx = 1, cy = 1;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
#ifdef PLANT_KSG_LE /* planted mistake: non-strict marginal comparison */
            if (fabsf(x[i] - x[j]) <= e) ++cx;
            if (fabsf(y[i] - y[j]) <= e) ++cy;
#else
            if (fabsf(x[i] - x[j]) < e) ++cx;
            if (fabsf(y[i] - y[j]) < e) ++cy;
#endif
        }
        if (nx) nx[i] = cx;
        if (ny) ny[i] = cy;
        if (eps) eps[i] = e;
#ifdef PLANT_KSG_DROP_Y /* planted mistake: the garbled sum read literally */
        s += psi[cx];
#else
        s += psi[cx] + psi[cy];
#endif
    }
    const double mi = psi[n] + psi[k] - s / n;
    free(psi);
    return mi;
}

/* k rule of Section 3.2: k = ceil(3n / 100). */
int or_k_rule(int n) { return (3 * n + 99) / 100; }

/* ---------------------------------------------------------------------------
 * One measure between grid points p and q of fields Fa, Fb (sizes Pa, Pb).
 */
typedef struct {
    float *x, *y, *work;
    double *wx, *wy;
    int32_t* rk;
    uint8_t *bx, *by;
} scratch_t;

static int scratch_init(scratch_t* s, int n) {
    s->x = (float*)malloc(sizeof(float) * n * 3);
    s->wx = (double*)malloc(sizeof(double) * n * 2);
    s->rk = (int32_t*)malloc(sizeof(int32_t) * n);
    s->bx = (uint8_t*)malloc((size_t)n * 2);
    if (!s->x || !s->wx || !s->rk || !s->bx) return -1;
    s->y = s->x + n;
    s->work = s->y + n;
    s->wy = s->wx + n;
    s->by = s->bx + n;
    return 0;
}

static void scratch_free(scratch_t* s) {
    free(s->x);
    free(s->wx);
    free(s->rk);
    free(s->bx);
}

static double measure(const float* Fa, int64_t Pa, const float* Fb, int64_t Pb, int n,
                      int64_t p, int64_t q, int kind, int k, int B, scratch_t* s,
                      int32_t* nx, int32_t* ny, float* eps) {
    gather(Fa, Pa, n, p, s->x);
    gather(Fb, Pb, n, q, s->y);
    switch (kind) {
        case OR_PEARSON:
            for (int i = 0; i < n; ++i) {
                s->wx[i] = s->x[i];
                s->wy[i] = s->y[i];
            }
            return or_pearson_vec(s->wx, s->wy, n);
        case OR_SPEARMAN:
            return or_spearman_vec(s->x, s->y, n, s->wx, s->wy, s->rk);
        case OR_MI_BINNED:
            or_bins(s->x, n, B, s->bx);
            or_bins(s->y, n, B, s->by);
            return or_hist_mi_bins(s->bx, s->by, n, B);
        case OR_MI_KSG:
            return or_ksg_vec(s->x, s->y, n, k, nx, ny, eps, s->work);
    }
    return NAN;
}

/*
 * Measure on a batch of point pairs (pa[t], pb[t]). Optional KSG outputs
 * nx, ny, eps are [N][n] in the original member order.
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int or_eval_pairs(const float* Fa, int64_t Pa, const float* Fb, int64_t Pb, int n, int kind,
                  int k, int B, const uint32_t* pa, const uint32_t* pb, int64_t N, double* out,
                  int32_t* nx, int32_t* ny, float* eps) {
    if (n < 2 || kind < 0 || kind > 3) return -1;
    if (kind == OR_MI_KSG) {
        if (k < 0) k = or_k_rule(n);
        if (k < 1 || k > n - 1) return -1;
    }
    if (kind == OR_MI_BINNED && (B < 1 || B > 256)) return -1;
    int err = 0;
#pragma omp parallel
    {
        scratch_t s;
        int ok = scratch_init(&s, n) == 0;
        if (!ok) {
#pragma omp atomic write
            err = -1;
        }
#pragma omp for schedule(dynamic, 64)
        for (int64_t t = 0; t < N; ++t) {
            if (!ok) continue;
            if (pa[t] >= (uint64_t)Pa || pb[t] >= (uint64_t)Pb) {
                out[t] = NAN;
                continue;
            }
            out[t] = measure(Fa, Pa, Fb, Pb, n, pa[t], pb[t], kind, k, B, &s,
                             nx ? nx + t * n : NULL, ny ? ny + t * n : NULL,
                             eps ? eps + t * n : NULL);
        }
        if (ok) scratch_free(&s);
    }
    return err;
}

/* Per-point ranks (doubled) and bins, for bit-exact checks: out is [count][n]. */
void or_rank2_points(const float* F, int64_t P, int n, const uint32_t* pts, int64_t count,
                     int32_t* out) {
#pragma omp parallel
    {
        float* x = (float*)malloc(sizeof(float) * n);
#pragma omp for schedule(static)
        for (int64_t t = 0; t < count; ++t) {
            gather(F, P, n, pts[t], x);
            or_rank2(x, n, out + t * n);
        }
        free(x);
    }
}

void or_bins_points(const float* F, int64_t P, int n, int B, const uint32_t* pts, int64_t count,
                    uint8_t* out) {
#pragma omp parallel
    {
        float* x = (float*)malloc(sizeof(float) * n);
#pragma omp for schedule(static)
        for (int64_t t = 0; t < count; ++t) {
            gather(F, P, n, pts[t], x);
            or_bins(x, n, B, out + t * n);
        }
        free(x);
    }
}

/* ---------------------------------------------------------------------------
 * Region-pair extremes (Section 3: the brick-pair indicator is the maximum of
 * the point-to-point correlations; Section 5.3 normalises by the exact min and
 * max). Exhaustive over a in A, b in B with linear pair index a*|B| + b.
 * READING: for A == B (self pair) only a < b is used, each unordered pair once;
 * ties resolve to the smallest pair index. res = {max, min, argmax, argmin,
 * count}; values (optional) receives every pair value at its linear index.
 */
int or_region_extremes(const float* F, int64_t P, int n, const uint32_t* A, int64_t na,
                       const uint32_t* Bp, int64_t nb, int self, int kind, int k, int B,
                       double* res, double* values) {
    if (kind == OR_MI_KSG && k < 0) k = or_k_rule(n);
    double gmax = -INFINITY, gmin = INFINITY;
    int64_t gamax = -1, gamin = -1, gcount = 0;
    int err = 0;
#pragma omp parallel
    {
        scratch_t s;
        int ok = scratch_init(&s, n) == 0;
        if (!ok) {
#pragma omp atomic write
            err = -1;
        }
        double lmax = -INFINITY, lmin = INFINITY;
        int64_t lamax = -1, lamin = -1, lcount = 0;
#pragma omp for schedule(dynamic, 4)
        for (int64_t a = 0; a < na; ++a) {
            if (!ok) continue;
            for (int64_t b = self ? a + 1 : 0; b < nb; ++b) {
                double v = measure(F, P, F, P, n, A[a], Bp[b], kind, k, B, &s, NULL, NULL, NULL);
                int64_t idx = a * nb + b;
                if (values) values[idx] = v;
                ++lcount;
                if (v > lmax || (v == lmax && idx < lamax)) {
                    lmax = v;
                    lamax = idx;
                }
                if (v < lmin || (v == lmin && idx < lamin)) {
                    lmin = v;
                    lamin = idx;
                }
            }
        }
#pragma omp critical
        {
            if (lamax >= 0 && (lmax > gmax || (lmax == gmax && lamax < gamax) || gamax < 0)) {
                gmax = lmax;
                gamax = lamax;
            }
            if (lamin >= 0 && (lmin < gmin || (lmin == gmin && lamin < gamin) || gamin < 0)) {
                gmin = lmin;
                gamin = lamin;
            }
            gcount += lcount;
        }
        if (ok) scratch_free(&s);
    }
    res[0] = gmax;
    res[1] = gmin;
    res[2] = (double)gamax;
    res[3] = (double)gamin;
    res[4] = (double)gcount;
    return err;
}

/* ---------------------------------------------------------------------------
 * Uniform random point-pair sampling (Section 3.1: sample positions in the 6D
 * space of two bricks). Random numbers come from Philox4x64-10 (Salmon, Moraes,
 * Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011),
 * implemented here from that definition.
 */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
    unsigned __int128 p = (unsigned __int128)a * b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void or_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
#ifdef PLANT_PHILOX_9 /* planted mistake: one round short */
    for (int r = 0; r < 9; ++r) {
#else
    for (int r = 0; r < 10; ++r) {
#endif
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(0xD2E7470EE14C6C93ull, c0, &hi0, &lo0);
        mulhilo64(0xCA5A826395121157ull, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

static uint64_t scale_u64(uint64_t u, uint64_t m) {
    unsigned __int128 p = (unsigned __int128)u * m;
    return (uint64_t)(p >> 64);
}

/*
 * Pair t of a batch uses block Philox(ctr = {first + t, 0, 0, 0},
 * key = {seed, stream}) with outputs w0, w1:
 *   cross pair (self = 0): a = floor(w0 * na / 2^64), b = floor(w1 * nb / 2^64)
 *   self pair  (self = 1): a = floor(w0 * na / 2^64),
 *                          b' = floor(w1 * (na - 1) / 2^64), b = b' + (b' >= a),
 *                          then the pair is ordered (min, max).
 * Outputs are region-local indices.
 */
int or_sample_pairs(uint64_t seed, uint64_t stream, uint64_t first, int64_t na, int64_t nb,
                    int self, int64_t N, uint32_t* ia, uint32_t* ib) {
    if (na < 1 || nb < 1 || (self && na < 2)) return -1;
    for (int64_t t = 0; t < N; ++t) {
        uint64_t ctr[4] = {first + (uint64_t)t, 0, 0, 0}, key[2] = {seed, stream}, w[4];
        or_philox4x64_10(ctr, key, w);
        uint64_t a = scale_u64(w[0], (uint64_t)na), b;
        if (self) {
            b = scale_u64(w[1], (uint64_t)na - 1);
            b += (b >= a);
            if (b < a) {
                uint64_t tmp = a;
                a = b;
                b = tmp;
            }
        } else {
            b = scale_u64(w[1], (uint64_t)nb);
        }
        ia[t] = (uint32_t)a;
        ib[t] = (uint32_t)b;
    }
    return 0;
}

void or_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
