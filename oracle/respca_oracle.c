/*
 * RES-PCA oracle -- TEST INFRASTRUCTURE ONLY (see respca_oracle.h).
 *
 * Plain FP64, single thread, no blocking, no fusion, no reordering beyond
 * what each equation states.  Each function names the passage it follows in
 * Peng et al., "RES-PCA: A Scalable Approach to Recovering Low-rank
 * Matrices" (arXiv 1904.07497).  Column-major, leading dimension d.
 */
#include "respca_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* splitmix64 (Steele, Lea and Flood, OOPSLA 2014), the published
 * public-domain generator: add the golden-ratio increment, then two
 * xor-shift-multiply rounds and a final xor-shift. */
uint64_t oracle_splitmix64(uint64_t *state)
{
    uint64_t z;
    *state += 0x9E3779B97F4A7C15ULL;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

double oracle_uniform(uint64_t *state)
{
    return (double)(oracle_splitmix64(state) >> 11) * (1.0 / 9007199254740992.0);
}

/* Sec. 5 stopping rule uses Frobenius norms. */
double oracle_fro(const double *A, int64_t count)
{
    double s = 0.0;
    for (int64_t k = 0; k < count; ++k) s += A[k] * A[k];
    return sqrt(s);
}

/* Sec. 6 anomaly score: ||S_j||_2 for each column j. */
void oracle_column_norms(const double *S, int64_t d, int64_t n, double *out)
{
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t r = 0; r < d; ++r) s += S[j * d + r] * S[j * d + r];
        out[j] = sqrt(s);
    }
}

/* Eq. (18): the cluster-mean term 1^T P_i(D) / n_i, n_i = ||p_i|| read as the
 * number of columns in cluster i. */
void oracle_cluster_means(const double *Y, int64_t d, int64_t n,
                          const int32_t *labels, int32_t c,
                          double *mu, int64_t *counts)
{
    double *sum = (double *)calloc((size_t)(d * c), sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)c, sizeof(int64_t));
    for (int64_t j = 0; j < n; ++j) {
        int32_t i = labels[j];
        cnt[i] += 1;
        for (int64_t r = 0; r < d; ++r) sum[i * d + r] += Y[j * d + r];
    }
    for (int32_t i = 0; i < c; ++i) {
        if (cnt[i] > 0)
            for (int64_t r = 0; r < d; ++r) mu[i * d + r] = sum[i * d + r] / (double)cnt[i];
        if (counts) counts[i] = cnt[i];
    }
    free(sum);
    free(cnt);
}

/* Sec. 4.1, L-minimisation.  D = X - S + Theta/rho (defined after Eq. (14));
 * Eq. (18) gives, per cluster i,
 *   P_i(L) = rho/(2 lambda + rho) P_i(D)
 *          + 2 lambda / (n_i (2 lambda + rho)) (sum of the columns of P_i(D)) 1^T,
 * the product taken from the right (Eq. (14) multiplies P_i(L) by M_i from
 * the right). */
void oracle_l_step(const double *X, const double *S, const double *Theta,
                   double rho, double lambda, const int32_t *labels, int32_t c,
                   int64_t d, int64_t n, double *L, double *mu_out,
                   int64_t *counts_out)
{
    const int64_t N = d * n;
    double *D = (double *)malloc((size_t)N * sizeof(double));
    double *colsum = (double *)calloc((size_t)(d * c), sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)c, sizeof(int64_t));

    for (int64_t k = 0; k < N; ++k) D[k] = X[k] - S[k] + Theta[k] / rho;

    for (int64_t j = 0; j < n; ++j) {
        int32_t i = labels[j];
        cnt[i] += 1;
        for (int64_t r = 0; r < d; ++r) colsum[i * d + r] += D[j * d + r];
    }

    const double first = rho / (2.0 * lambda + rho);
    for (int64_t j = 0; j < n; ++j) {
        int32_t i = labels[j];
        const double second = 2.0 * lambda / ((double)cnt[i] * (2.0 * lambda + rho));
        for (int64_t r = 0; r < d; ++r)
            L[j * d + r] = first * D[j * d + r] + second * colsum[i * d + r];
    }

    for (int32_t i = 0; i < c; ++i) {
        if (mu_out && cnt[i] > 0)
            for (int64_t r = 0; r < d; ++r) mu_out[i * d + r] = colsum[i * d + r] / (double)cnt[i];
        if (counts_out) counts_out[i] = cnt[i];
    }
    free(D);
    free(colsum);
    free(cnt);
}

/* Sec. 4.2: Eq. (21) is the K-means problem; one assignment pass of Lloyd's
 * method puts column j in the cluster whose centroid is nearest in squared
 * Euclidean distance (written as the plain sum of squared differences). */
int64_t oracle_assign(const double *Y, int64_t d, int64_t n,
                      const double *mu, const uint8_t *active, int32_t c,
                      int32_t *labels)
{
    int64_t changed = 0;
    for (int64_t j = 0; j < n; ++j) {
        int32_t best = -1;
        double bestd = 0.0;
        for (int32_t i = 0; i < c; ++i) {
            if (!active[i]) continue;
            double dist = 0.0;
            for (int64_t r = 0; r < d; ++r) {
                const double diff = Y[j * d + r] - mu[i * d + r];
                dist += diff * diff;
            }
            if (best < 0 || dist < bestd) {
                best = i;
                bestd = dist;
            }
        }
        if (best != labels[j]) {
            labels[j] = best;
            changed += 1;
        }
    }
    return changed;
}

/* Lloyd's method for Eq. (21)-(22): alternate assignment and centroid
 * update until an assignment changes nothing (or km_max passes). */
int32_t oracle_lloyd(const double *Y, int64_t d, int64_t n, int32_t c,
                     int32_t *labels, double *mu, uint8_t *active,
                     int32_t km_max, int64_t *changed_out)
{
    int32_t *entry = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int64_t *cnt = (int64_t *)malloc((size_t)c * sizeof(int64_t));
    memcpy(entry, labels, (size_t)n * sizeof(int32_t));
    int32_t steps = 0;
    while (steps < km_max) {
        const int64_t changed = oracle_assign(Y, d, n, mu, active, c, labels);
        steps += 1;
        if (changed == 0) break;
        oracle_cluster_means(Y, d, n, labels, c, mu, cnt);
        for (int32_t i = 0; i < c; ++i) active[i] = (uint8_t)(cnt[i] > 0);
    }
    if (changed_out) {
        int64_t ch = 0;
        for (int64_t j = 0; j < n; ++j) ch += (labels[j] != entry[j]);
        *changed_out = ch;
    }
    free(entry);
    free(cnt);
    return steps;
}

static double col_dist2(const double *X, int64_t d, int64_t a, int64_t b)
{
    double s = 0.0;
    for (int64_t r = 0; r < d; ++r) {
        const double diff = X[a * d + r] - X[b * d + r];
        s += diff * diff;
    }
    return s;
}

/* k-means++ (Arthur and Vassilvitskii, 2007): first centre uniform, each next
 * centre drawn with probability proportional to the squared distance to the
 * nearest centre chosen so far.  The draw u in [0,1) picks the first column
 * whose running sum of squared distances exceeds u times their total. */
void oracle_kmeanspp(const double *X, int64_t d, int64_t n, int32_t c,
                     uint64_t seed, int64_t *centers)
{
    uint64_t st = seed;
    double *D2 = (double *)malloc((size_t)n * sizeof(double));
    double u = oracle_uniform(&st);
    int64_t first = (int64_t)(u * (double)n);
    if (first >= n) first = n - 1;
    centers[0] = first;
    for (int64_t j = 0; j < n; ++j) D2[j] = col_dist2(X, d, j, first);

    for (int32_t k = 1; k < c; ++k) {
        u = oracle_uniform(&st);
        double total = 0.0;
        for (int64_t j = 0; j < n; ++j) total += D2[j];
        int64_t pick = -1;
        if (total > 0.0) {
            const double target = u * total;
            double cum = 0.0;
            for (int64_t j = 0; j < n; ++j) {
                cum += D2[j];
                if (cum > target) {
                    pick = j;
                    break;
                }
            }
            if (pick < 0)
                for (int64_t j = n - 1; j >= 0; --j)
                    if (D2[j] > 0.0) {
                        pick = j;
                        break;
                    }
        } else {
            pick = (int64_t)(u * (double)n);
            if (pick >= n) pick = n - 1;
        }
        centers[k] = pick;
        for (int64_t j = 0; j < n; ++j) {
            const double dn = col_dist2(X, d, j, pick);
            if (dn < D2[j]) D2[j] = dn;
        }
    }
    free(D2);
}

int32_t oracle_init_labels(const double *X, int64_t d, int64_t n, int32_t c,
                           uint64_t seed, int32_t km_max, int32_t *labels)
{
    int64_t *centers = (int64_t *)malloc((size_t)c * sizeof(int64_t));
    double *mu = (double *)malloc((size_t)(d * c) * sizeof(double));
    uint8_t *active = (uint8_t *)malloc((size_t)c);
    oracle_kmeanspp(X, d, n, c, seed, centers);
    for (int32_t i = 0; i < c; ++i) {
        memcpy(mu + i * d, X + centers[i] * d, (size_t)d * sizeof(double));
        active[i] = 1;
    }
    for (int64_t j = 0; j < n; ++j) labels[j] = -1;
    const int32_t steps = oracle_lloyd(X, d, n, c, labels, mu, active, km_max, NULL);
    free(centers);
    free(mu);
    free(active);
    return steps;
}

/* Sec. 4.3, Eq. (24): soft-thresholding of B = X - L + Theta/rho at 1/rho;
 * sign(0) = 0. */
void oracle_s_step(const double *X, const double *L, const double *Theta,
                   double rho, int64_t count, double *S)
{
    for (int64_t k = 0; k < count; ++k) {
        const double B = X[k] - L[k] + Theta[k] / rho;
        const double mag = fabs(B) - 1.0 / rho;
        const double sgn = (B > 0.0) ? 1.0 : ((B < 0.0) ? -1.0 : 0.0);
        S[k] = (mag > 0.0 ? mag : 0.0) * sgn;
    }
}

/* Block soft-thresholding: the prox of (1/rho)||.||_{2,1}, column by column. */
void oracle_s_step_l21(const double *X, const double *L, const double *Theta,
                       double rho, int64_t d, int64_t n, double *S)
{
    for (int64_t j = 0; j < n; ++j) {
        double nb2 = 0.0;
        for (int64_t r = 0; r < d; ++r) {
            const int64_t k = j * d + r;
            const double B = X[k] - L[k] + Theta[k] / rho;
            nb2 += B * B;
        }
        const double nb = sqrt(nb2);
        const double f = (nb > 1.0 / rho) ? 1.0 - 1.0 / (rho * nb) : 0.0;
        for (int64_t r = 0; r < d; ++r) {
            const int64_t k = j * d + r;
            S[k] = f * (X[k] - L[k] + Theta[k] / rho);
        }
    }
}

/* Sec. 4.4, Eq. (25): Theta = Theta + rho (X - L - S). */
void oracle_theta_step(const double *X, const double *L, const double *S,
                       double rho, int64_t count, double *Theta)
{
    for (int64_t k = 0; k < count; ++k) Theta[k] = Theta[k] + rho * (X[k] - L[k] - S[k]);
}

int64_t oracle_iteration(const double *X, int64_t d, int64_t n, int32_t c,
                         double lambda, double kappa, int32_t km_max,
                         double *L, double *S, double *Theta, int32_t *labels,
                         double *rho, double norms[3], int32_t *lloyd_out)
{
    return oracle_iteration_ex(X, d, n, c, lambda, kappa, km_max, L, S, Theta, labels, rho, norms,
                               lloyd_out, 0);
}

int64_t oracle_iteration_ex(const double *X, int64_t d, int64_t n, int32_t c,
                            double lambda, double kappa, int32_t km_max,
                            double *L, double *S, double *Theta, int32_t *labels,
                            double *rho, double norms[3], int32_t *lloyd_out, int32_t snorm)
{
    const int64_t N = d * n;
    double *Lprev = (double *)malloc((size_t)N * sizeof(double));
    double *Sprev = (double *)malloc((size_t)N * sizeof(double));
    double *mu = (double *)calloc((size_t)(d * c), sizeof(double));
    int64_t *cnt = (int64_t *)malloc((size_t)c * sizeof(int64_t));
    uint8_t *active = (uint8_t *)malloc((size_t)c);
    memcpy(Lprev, L, (size_t)N * sizeof(double));
    memcpy(Sprev, S, (size_t)N * sizeof(double));

    /* Sec. 4.1: L step (labels of the previous p step). */
    oracle_l_step(X, S, Theta, *rho, lambda, labels, c, d, n, L, mu, cnt);
    /* Sec. 4.2: p step, K-means on the columns of L, warm-started from the
     * current labels; the cluster means of L under them equal those of D. */
    for (int32_t i = 0; i < c; ++i) active[i] = (uint8_t)(cnt[i] > 0);
    int64_t changed = 0;
    const int32_t steps = oracle_lloyd(L, d, n, c, labels, mu, active, km_max, &changed);
    /* Sec. 4.3: S step (l1, Eq. (24); or l2,1). */
    if (snorm == 1) oracle_s_step_l21(X, L, Theta, *rho, d, n, S);
    else oracle_s_step(X, L, Theta, *rho, N, S);
    /* Sec. 4.4: Theta and rho. */
    oracle_theta_step(X, L, S, *rho, N, Theta);

    double r2 = 0.0, dl2 = 0.0, ds2 = 0.0;
    for (int64_t k = 0; k < N; ++k) {
        const double res = X[k] - L[k] - S[k];
        const double dl = L[k] - Lprev[k];
        const double ds = S[k] - Sprev[k];
        r2 += res * res;
        dl2 += dl * dl;
        ds2 += ds * ds;
    }
    norms[0] = sqrt(r2);
    norms[1] = sqrt(dl2);
    norms[2] = sqrt(ds2);
    *rho = *rho * kappa;
    if (lloyd_out) *lloyd_out = steps;

    free(Lprev);
    free(Sprev);
    free(mu);
    free(cnt);
    free(active);
    return changed;
}

/* Eq. (8), with each trace term written as the within-cluster sum of squares
 * (Eq. (20)). */
double oracle_objective(const double *L, const double *S, const int32_t *labels,
                        int32_t c, double lambda, int64_t d, int64_t n)
{
    double *mu = (double *)calloc((size_t)(d * c), sizeof(double));
    oracle_cluster_means(L, d, n, labels, c, mu, NULL);
    double ss = 0.0, l1 = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        const int32_t i = labels[j];
        for (int64_t r = 0; r < d; ++r) {
            const double diff = L[j * d + r] - mu[i * d + r];
            ss += diff * diff;
        }
    }
    for (int64_t k = 0; k < d * n; ++k) l1 += fabs(S[k]);
    free(mu);
    return lambda * ss + l1;
}

/* Eq. (9). */
double oracle_lagrangian(const double *X, const double *L, const double *S,
                         const double *Theta, const int32_t *labels, int32_t c,
                         double lambda, double rho, int64_t d, int64_t n)
{
    double q = 0.0;
    for (int64_t k = 0; k < d * n; ++k) {
        const double v = X[k] - L[k] - S[k] + Theta[k] / rho;
        q += v * v;
    }
    return oracle_objective(L, S, labels, c, lambda, d, n) + 0.5 * rho * q;
}

/* Sec. 4 as a whole (ALM with the four updates) and the stopping rule of
 * Sec. 5: stop when max(||X-L-S||, ||L_{t+1}-L_t||, ||S_{t+1}-S_t||)/||X||
 * <= tol, or after max_iter iterations. */
int32_t oracle_solve(const double *X, int64_t d, int64_t n, int32_t c,
                     double lambda, double rho0, double kappa, double tol,
                     int32_t max_iter, int32_t km_max, uint64_t seed,
                     const int32_t *p0, int32_t warm, double *rho_io,
                     double *L, double *S, double *Theta, int32_t *labels,
                     oracle_stats *stats)
{
    return oracle_solve_ex(X, d, n, c, lambda, rho0, kappa, tol, max_iter, km_max, seed, p0, warm,
                           rho_io, L, S, Theta, labels, stats, 0);
}

int32_t oracle_solve_ex(const double *X, int64_t d, int64_t n, int32_t c,
                        double lambda, double rho0, double kappa, double tol,
                        int32_t max_iter, int32_t km_max, uint64_t seed,
                        const int32_t *p0, int32_t warm, double *rho_io,
                        double *L, double *S, double *Theta, int32_t *labels,
                        oracle_stats *stats, int32_t snorm)
{
    if (snorm != 0 && snorm != 1) return -1;
    if (d <= 0 || n <= 0 || c < 1 || c > n || max_iter < 0 || km_max < 1) return -1;
    if (!(tol >= 0.0) || !isfinite(tol) || !isfinite(lambda)) return -1;
    if (!(rho0 > 0.0) || !(kappa > 0.0)) return -1;
    const int64_t N = d * n;
    oracle_stats st;
    memset(&st, 0, sizeof(st));
    if (lambda <= 0.0) lambda = sqrt((double)(d > n ? d : n));

    const double nx = oracle_fro(X, N);
    double rho = (warm && rho_io && *rho_io > 0.0) ? *rho_io : rho0;

    if (!warm) {
        if (p0) {
            for (int64_t j = 0; j < n; ++j) {
                if (p0[j] < 0 || p0[j] >= c) return -1;
                labels[j] = p0[j];
            }
        } else if (nx > 0.0) {
            st.init_lloyd_steps = oracle_init_labels(X, d, n, c, seed, km_max, labels);
        } else {
            for (int64_t j = 0; j < n; ++j) labels[j] = 0;
        }
        memset(L, 0, (size_t)N * sizeof(double));
        memset(S, 0, (size_t)N * sizeof(double));
        memset(Theta, 0, (size_t)N * sizeof(double));
    }
    if (nx == 0.0) {
        memset(L, 0, (size_t)N * sizeof(double));
        memset(S, 0, (size_t)N * sizeof(double));
        st.converged = 1;
        st.rho_final = rho;
        if (stats) *stats = st;
        if (rho_io) *rho_io = rho;
        return 0;
    }

    double norms[3];
    for (int32_t t = 0; t < max_iter; ++t) {
        int32_t steps = 0;
        st.label_changes += oracle_iteration_ex(X, d, n, c, lambda, kappa, km_max, L, S,
                                                Theta, labels, &rho, norms, &steps, snorm);
        st.lloyd_steps += steps;
        st.iters = t + 1;
        st.err_resid = norms[0] / nx;
        st.err_dL = norms[1] / nx;
        st.err_dS = norms[2] / nx;
        st.err = st.err_resid;
        if (st.err_dL > st.err) st.err = st.err_dL;
        if (st.err_dS > st.err) st.err = st.err_dS;
        if (st.err <= tol) {
            st.converged = 1;
            break;
        }
    }
    st.rho_final = rho;
    if (stats) *stats = st;
    if (rho_io) *rho_io = rho;
    return 0;
}
