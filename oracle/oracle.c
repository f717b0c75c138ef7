/*
 * FP64 CPU oracle for PPS silhouette approximation -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the plain, slow, obviously-correct statement of what the GPU
 * library computes.  Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it; the library never does, and the two share
 * no code.  Every floating-point step is IEEE double, evaluated in the order
 * written (build with -ffp-contract=off so no multiply-add is fused).
 *
 * Sources (Altieri, Pietracaprina, Pucci, Vandin, "Scalable and Distributed
 * Silhouette Approximation"):
 *   - silhouette of an element, a(e), b(e):            Eq. 1, Eq. 2
 *   - silhouette of a clustering:                        Eq. 3
 *   - cluster weight W_Cj(e):                            Eq. 4
 *   - silh-pps-all (Phase 1 PPS sampling, Phase 2):      Algorithm 1
 *   - estimates a_hat, b_hat, s_hat:                     Eq. 8 (Sec. 4.1.1)
 *   - uniform-sampling variant (constant p = t/|Cj|):    Sec. 4.1.3
 *   - distances d_eucl, d_cos, d_manh, d_can:            Sec. 5.1.1
 *   - counter-based generator: Philox4x64-10 of Salmon, Moraes, Dror, Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3" (SC'11), written from the
 *     published round function and constants.
 *
 * Readings where the paper is silent or inconsistent:
 *   - d_cos: the printed formula subtracts coordinates in the numerator; the
 *     cosine distance is 1 - sum x_i y_i / (|x| |y|).  A zero-norm operand gives
 *     distance 1; the result is clamped to [0, 2].
 *   - Canberra 0/0 term (both coordinates zero) contributes 0.
 *   - An empty initial sample F0_j: the inner maximum over F0_j is taken as 0,
 *     so gamma_e = 1/|Cj| (the first term of the maximum alone).
 *   - W(e_bar) = 0 (all points of Cj coincide): the term d/W is taken as 0.
 *   - max(a_hat, b_hat) = 0 (duplicate points): s_hat = 0.
 *   - the initial-sample probability is min(1, m0/|Cj|) with
 *     m0 = 2 ln(5k/delta) as in Algorithm 1 (callers may fix m0 directly).
 *
 * Uniform draw U(seed, stream, cid, e): Philox4x64-10 with key (seed, 0) and
 * counter (e, stream, cid, 0); u = (first output word >> 11) * 2^-53.
 * stream 0 draws F0, stream 1 draws F.
 *
 * Status codes: 0 ok, -1 invalid argument.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_EUCLIDEAN = 0, ORC_COSINE = 1, ORC_MANHATTAN = 2, ORC_CANBERRA = 3 };

/* ---------------------------------------------------------------- Philox */

static void orc_mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

/* Philox4x64 with 10 rounds: each round multiplies words 0 and 2 by the two
 * round multipliers, permutes, and xors the high halves with the round key;
 * the key advances by the two Weyl constants between rounds. */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B97F4A7C15ULL;
            k1 += 0xBB67AE8584CAA73BULL;
        }
        uint64_t hi0, lo0, hi1, lo1;
        orc_mulhilo64(0xD2E7470EE14C6C93ULL, x0, &hi0, &lo0);
        orc_mulhilo64(0xCA5A826395121157ULL, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0;
        uint64_t y1 = lo1;
        uint64_t y2 = hi0 ^ x3 ^ k1;
        uint64_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

double orc_uniform(uint64_t seed, uint64_t stream, uint64_t cid, uint64_t e)
{
    uint64_t ctr[4] = {e, stream, cid, 0};
    uint64_t key[2] = {seed, 0};
    uint64_t out[4];
    orc_philox4x64_10(ctr, key, out);
    return (double)(out[0] >> 11) * 0x1.0p-53;
}

/* ------------------------------------------------------------- distances */

double orc_dist(int metric, const double *x, const double *y, int d)
{
    double s = 0.0;
    if (metric == ORC_EUCLIDEAN) {
        for (int i = 0; i < d; ++i) {
            double t = x[i] - y[i];
            s = s + t * t;
        }
        return sqrt(s);
    }
    if (metric == ORC_MANHATTAN) {
        for (int i = 0; i < d; ++i) s = s + fabs(x[i] - y[i]);
        return s;
    }
    if (metric == ORC_CANBERRA) {
        for (int i = 0; i < d; ++i) {
            double num = fabs(x[i] - y[i]);
            double den = fabs(x[i]) + fabs(y[i]);
            if (den > 0.0) s = s + num / den;
        }
        return s;
    }
    /* cosine */
    double dot = 0.0, nx = 0.0, ny = 0.0;
    for (int i = 0; i < d; ++i) {
        dot = dot + x[i] * y[i];
        nx = nx + x[i] * x[i];
        ny = ny + y[i] * y[i];
    }
    if (nx == 0.0 || ny == 0.0) return 1.0;
    double c = 1.0 - dot / (sqrt(nx) * sqrt(ny));
    if (c < 0.0) c = 0.0;
    if (c > 2.0) c = 2.0;
    return c;
}

/* out[i*ny + j] = d(X_i, Y_j) */
void orc_pairwise(int metric, const double *X, int64_t nx, const double *Y, int64_t ny, int d,
                  double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nx; ++i)
        for (int64_t j = 0; j < ny; ++j)
            out[i * ny + j] = orc_dist(metric, X + i * d, Y + j * d, d);
}

/* --------------------------------------------------------- bookkeeping */

/* |Cj| for every j; -1 if a label is outside [0,k), a cluster is empty, k < 2
 * or n < 2 (a clustering is a partition of V into k non-empty sets, Sec. 2). */
int orc_cluster_sizes(const int32_t *labels, int64_t n, int k, int64_t *sizes)
{
    if (k < 2 || n < 2) return -1;
    for (int j = 0; j < k; ++j) sizes[j] = 0;
    for (int64_t e = 0; e < n; ++e) {
        if (labels[e] < 0 || labels[e] >= k) return -1;
        sizes[labels[e]] += 1;
    }
    for (int j = 0; j < k; ++j)
        if (sizes[j] == 0) return -1;
    return 0;
}

/* s(e) from the k cluster weights W_j(e) of an element in cluster c (Eq. 1-2
 * with Eq. 4): a = W_c/(|C|-1), b = min_{j != c} W_j/|Cj|; singleton -> 0.
 * nb: the neighbouring cluster, the j != c attaining b (Example 1 names it
 * for e14), the lowest such j among equal ratios. */
static void orc_silhouette_from_weights(const double *W, const int64_t *sizes, int k, int c,
                                        double *s, double *a, double *b, int *nb)
{
    double bv = INFINITY;
    int arg = -1;
    for (int j = 0; j < k; ++j) {
        if (j == c) continue;
        double v = W[j] / (double)sizes[j];
        if (v < bv) { bv = v; arg = j; }
    }
    *b = bv;
    *nb = arg;
    if (sizes[c] == 1) {
        *s = 0.0; *a = 0.0;
        return;
    }
    double av = W[c] / (double)(sizes[c] - 1);
    double m = av > bv ? av : bv;
    *a = av;
    *s = (m > 0.0) ? (bv - av) / m : 0.0;
}

/* ------------------------------------------------------------ exact */

/* Exact silhouette (Eq. 1-2) of the listed rows (rows == NULL: all n).
 * W_j(e) = sum over every e' with label j of d(e, e'), e' ascending. */
int orc_exact(const double *X, int64_t n, int d, const int32_t *labels, int k, int metric,
              const int64_t *rows, int64_t nrows, double *s, double *a, double *b, int32_t *nb)
{
    int64_t *sizes = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    if (orc_cluster_sizes(labels, n, k, sizes) != 0 || d < 1) { free(sizes); return -1; }
    if (rows == NULL) nrows = n;
    for (int64_t r = 0; rows != NULL && r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= n) { free(sizes); return -1; }
#pragma omp parallel
    {
        double *W = (double *)malloc(sizeof(double) * (size_t)k);
#pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < nrows; ++r) {
            int64_t e = rows ? rows[r] : r;
            for (int j = 0; j < k; ++j) W[j] = 0.0;
            for (int64_t f = 0; f < n; ++f)
                W[labels[f]] = W[labels[f]] + orc_dist(metric, X + e * d, X + f * d, d);
            double sv, av, bv;
            int nv;
            orc_silhouette_from_weights(W, sizes, k, labels[e], &sv, &av, &bv, &nv);
            s[r] = sv;
            if (a) a[r] = av;
            if (b) b[r] = bv;
            if (nb) nb[r] = nv;
        }
        free(W);
    }
    free(sizes);
    return 0;
}

/* ------------------------------------------------------------ Phase 1 */

/* Poisson sampling: flag[e] = U(seed, stream, cid, e) < prob[e]. */
void orc_poisson_draw(uint64_t seed, uint64_t stream, uint64_t cid, int64_t n,
                      const double *prob, uint8_t *flag)
{
    for (int64_t e = 0; e < n; ++e)
        flag[e] = (orc_uniform(seed, stream, cid, (uint64_t)e) < prob[e]) ? 1 : 0;
}

/* Algorithm 1, Phase 1 (PPS sampling), per cluster in turn.
 *   in_f0[e]  1 if e was drawn into F0 of its cluster
 *   w0[e]     W_{Cj}(e) for e in F0 (else 0)
 *   gamma[e]  gamma_e (1 for elements of clusters with |Cj| <= t)
 *   p[e]      inclusion probability p_e (1 when |Cj| <= t)
 *   in_f[e]   1 if e is in F_{Cj}
 * uniform != 0 selects the uniform variant: p_e = min(1, t/|Cj|) and no F0.
 */
int orc_sample_pps(const double *X, int64_t n, int d, const int32_t *labels, int k, int metric,
                   double t, double m0, uint64_t seed, uint64_t cid, int uniform,
                   uint8_t *in_f0, double *w0, double *gamma, double *p, uint8_t *in_f)
{
    if (!(t > 0.0) || d < 1) return -1;
    int64_t *sizes = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    if (orc_cluster_sizes(labels, n, k, sizes) != 0) { free(sizes); return -1; }
    /* members of every cluster, ascending element index */
    int64_t *start = (int64_t *)calloc((size_t)k + 1, sizeof(int64_t));
    int64_t *fill = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    int64_t *members = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int j = 0; j < k; ++j) start[j + 1] = start[j] + sizes[j];
    for (int64_t e = 0; e < n; ++e) {
        int j = labels[e];
        members[start[j] + fill[j]] = e;
        fill[j] += 1;
    }
    for (int64_t e = 0; e < n; ++e) { in_f0[e] = 0; w0[e] = 0.0; }

    for (int j = 0; j < k; ++j) {
        const int64_t *C = members + start[j];
        int64_t nc = sizes[j];
        if ((double)nc <= t) {                        /* F_j = C_j */
            for (int64_t i = 0; i < nc; ++i) { gamma[C[i]] = 1.0; p[C[i]] = 1.0; }
            continue;
        }
        if (uniform) {
            double pu = t / (double)nc;
            if (pu > 1.0) pu = 1.0;
            for (int64_t i = 0; i < nc; ++i) { gamma[C[i]] = 1.0 / (double)nc; p[C[i]] = pu; }
            continue;
        }
        /* initial Poisson sample F0 with probability m0/|Cj| */
        double q = m0 / (double)nc;
        if (q > 1.0) q = 1.0;
        int64_t nf0 = 0;
        int64_t *F0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)nc);
        for (int64_t i = 0; i < nc; ++i)
            if (orc_uniform(seed, 0, cid, (uint64_t)C[i]) < q) { F0[nf0++] = C[i]; in_f0[C[i]] = 1; }
        /* W_{Cj}(e_bar) for e_bar in F0 */
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t f = 0; f < nf0; ++f) {
            double W = 0.0;
            for (int64_t i = 0; i < nc; ++i)
                W = W + orc_dist(metric, X + F0[f] * d, X + C[i] * d, d);
            w0[F0[f]] = W;
        }
        /* gamma_e, p_e */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < nc; ++i) {
            int64_t e = C[i];
            double g2 = 0.0;
            for (int64_t f = 0; f < nf0; ++f) {
                double W = w0[F0[f]];
                double r = (W > 0.0) ? orc_dist(metric, X + e * d, X + F0[f] * d, d) / W : 0.0;
                if (r > g2) g2 = r;
            }
            double g1 = 1.0 / (double)nc;
            double g = g1 > g2 ? g1 : g2;
            gamma[e] = g;
            double pe = t * g;
            p[e] = pe < 1.0 ? pe : 1.0;
        }
        free(F0);
    }
    /* final Poisson sample F with probabilities p_e */
    orc_poisson_draw(seed, 1, cid, n, p, in_f);
    for (int j = 0; j < k; ++j)                       /* |Cj| <= t: every element */
        if ((double)sizes[j] <= t)
            for (int64_t i = 0; i < sizes[j]; ++i) in_f[members[start[j] + i]] = 1;
    free(sizes); free(start); free(fill); free(members);
    return 0;
}

/* Sample set as per-cluster lists: offsets[k+1], idx (ascending within a
 * cluster) and the inclusion probability of each sampled element. */
int64_t orc_build_sample(const int32_t *labels, int64_t n, int k, const uint8_t *in_f,
                         const double *p, int64_t *offsets, int64_t *idx, double *ps)
{
    if (k < 1) return 0;
    for (int j = 0; j <= k; ++j) offsets[j] = 0;
    for (int64_t e = 0; e < n; ++e)
        if (in_f[e]) offsets[labels[e] + 1] += 1;
    for (int j = 0; j < k; ++j) offsets[j + 1] += offsets[j];
    int64_t *fill = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    for (int64_t e = 0; e < n; ++e) {
        if (!in_f[e]) continue;
        int j = labels[e];
        int64_t pos = offsets[j] + fill[j];
        idx[pos] = e;
        ps[pos] = p[e];
        fill[j] += 1;
    }
    free(fill);
    return offsets[k];
}

/* ------------------------------------------------------------ Phase 2 */

/* Algorithm 1, Phase 2 for the listed rows (rows == NULL: all n):
 * W_hat_j(e) = sum_{e' in F_j} d(e, e') / p_{e'}, then a_hat, b_hat, s_hat.
 * w_hat (nullable) receives the nrows x k estimated weights, nb (nullable) the
 * neighbouring cluster of each row. */
int orc_estimate(const double *X, int64_t n, int d, const int32_t *labels, int k, int metric,
                 const int64_t *offsets, const int64_t *idx, const double *ps,
                 const int64_t *rows, int64_t nrows, double *s, double *a, double *b,
                 double *w_hat, int32_t *nb)
{
    int64_t *sizes = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    if (orc_cluster_sizes(labels, n, k, sizes) != 0 || d < 1) { free(sizes); return -1; }
    if (rows == NULL) nrows = n;
    for (int64_t r = 0; rows != NULL && r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= n) { free(sizes); return -1; }
#pragma omp parallel
    {
        double *W = (double *)malloc(sizeof(double) * (size_t)k);
#pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < nrows; ++r) {
            int64_t e = rows ? rows[r] : r;
            for (int j = 0; j < k; ++j) {
                double acc = 0.0;
                for (int64_t i = offsets[j]; i < offsets[j + 1]; ++i)
                    acc = acc + orc_dist(metric, X + e * d, X + idx[i] * d, d) / ps[i];
                W[j] = acc;
                if (w_hat) w_hat[r * k + j] = acc;
            }
            double sv, av, bv;
            int nv;
            orc_silhouette_from_weights(W, sizes, k, labels[e], &sv, &av, &bv, &nv);
            s[r] = sv;
            if (a) a[r] = av;
            if (b) b[r] = bv;
            if (nb) nb[r] = nv;
        }
        free(W);
    }
    free(sizes);
    return 0;
}

/* --------------------------------------------------- cohesion, separation */

/* Cohesion and separation of the clustering (Sec. "Estimating other clustering
 * validation measures") from the per-element cluster weights W (n x k; the
 * exact W of Eq. 4 or the estimates W_hat):
 *   Coh = (1/2) sum_j sum_{e in Cj} W_Cj(e) / sum_j C(|Cj|, 2)
 *   Sep = sum_{j1 < j2} sum_{e in Cj1} W_Cj2(e) / sum_{j1 < j2} |Cj1| |Cj2|
 * (the printed |C_{j-1}| in Sep's denominator is read as |C_{j1}|). */
int orc_cohsep(const double *W, const int32_t *labels, int64_t n, int k, double *coh, double *sep)
{
    int64_t *sizes = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    if (orc_cluster_sizes(labels, n, k, sizes) != 0) { free(sizes); return -1; }
    double num_c = 0.0, num_s = 0.0, den_c = 0.0, den_s = 0.0;
    for (int64_t e = 0; e < n; ++e) {
        int c = labels[e];
        num_c = num_c + W[e * k + c];
        for (int j = c + 1; j < k; ++j) num_s = num_s + W[e * k + j];
    }
    for (int j = 0; j < k; ++j) {
        den_c = den_c + 0.5 * (double)sizes[j] * (double)(sizes[j] - 1);
        for (int j2 = j + 1; j2 < k; ++j2) den_s = den_s + (double)sizes[j] * (double)sizes[j2];
    }
    *coh = den_c > 0.0 ? 0.5 * num_c / den_c : 0.0;
    *sep = den_s > 0.0 ? num_s / den_s : 0.0;
    free(sizes);
    return 0;
}

/* ------------------------------------------------------------- global */

/* Mean of n values (Eq. 3 / Eq. 6), Neumaier-compensated sum. */
double orc_mean(const double *v, int64_t n)
{
    double sum = 0.0, comp = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double t = sum + v[i];
        if (fabs(sum) >= fabs(v[i])) comp += (sum - t) + v[i];
        else comp += (v[i] - t) + sum;
        sum = t;
    }
    return (sum + comp) / (double)n;
}

/* Sample size of Lemma 1: t = ceil((3c / eps^2) ln(5 n k / delta)), c = 18. */
double orc_t_from_eps(double eps, double delta, int64_t n, int k)
{
    return ceil((3.0 * 18.0 / (eps * eps)) * log(5.0 * (double)n * (double)k / delta));
}

int orc_nthreads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
