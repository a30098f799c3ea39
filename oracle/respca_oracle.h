/*
 * RES-PCA oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 CPU statement of the RES-PCA method
 * (Peng et al., "RES-PCA: A Scalable Approach to Recovering Low-rank
 * Matrices", arXiv 1904.07497).  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  The product library
 * shares no code, header, table or helper with this file and never calls it.
 *
 * Layout: every matrix is column-major, leading dimension = d (element
 * (r, j) of a d x n matrix A is A[j*d + r]).  Labels are int32 in [0, c).
 *
 * Parity notes (readings of the paper this oracle takes):
 *   - update order inside one iteration: L (Sec. 4.1), p (Sec. 4.2),
 *     S (Sec. 4.3), Theta and rho (Sec. 4.4);
 *   - "||p_i||_2" in Eq. (8)-(18) is read as the cluster size n_i;
 *   - the p step is Lloyd's K-means warm-started from the previous labels
 *     and the cluster means of D, stopped when no label changes (cap km_max);
 *     assignment ties go to the lowest cluster index; a cluster that becomes
 *     empty takes part in no later assignment;
 *   - the initial labels are k-means++ (splitmix64 draws) + Lloyd on X;
 *   - L, S, Theta start at zero; stopping test of Sec. 5 on post-update
 *     iterates, checked every iteration.
 */
#ifndef RESPCA_ORACLE_H
#define RESPCA_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t iters;          /* ALM iterations run */
    int32_t converged;      /* 1 if the Sec. 5 criterion reached tol */
    double err;             /* max of the three relative quantities */
    double err_resid;       /* ||X-L-S||_F / ||X||_F */
    double err_dL;          /* ||L_{t+1}-L_t||_F / ||X||_F */
    double err_dS;          /* ||S_{t+1}-S_t||_F / ||X||_F */
    double rho_final;       /* rho after the last update */
    int64_t label_changes;  /* labels changed by the p steps, summed */
    int64_t lloyd_steps;    /* assignment passes run by the p steps, summed */
    int32_t init_lloyd_steps; /* assignment passes of the initial K-means */
} oracle_stats;

/* splitmix64: advance *state and return the next 64-bit output. */
uint64_t oracle_splitmix64(uint64_t *state);
/* Uniform double in [0,1) from the top 53 bits of the next splitmix64 output. */
double oracle_uniform(uint64_t *state);

/* Frobenius norm, plain sequential sum of squares. */
double oracle_fro(const double *A, int64_t count);

/* Sec. 6 (anomaly detection): the l2 norm of every column of S, the score by
 * which columns whose S is large are flagged as outliers.  S is d x n
 * column-major; out has n entries. */
void oracle_column_norms(const double *S, int64_t d, int64_t n, double *out);

/* Cluster sizes and means of the columns of Y under labels (Eq. (18): the
 * vector 1^T P_i(D) / n_i).  Clusters with no member leave mu untouched and
 * get count 0. mu is d x c. */
void oracle_cluster_means(const double *Y, int64_t d, int64_t n,
                          const int32_t *labels, int32_t c,
                          double *mu, int64_t *counts);

/* L step, Eq. (18) with D = X - S + Theta/rho (Eq. (14)). mu_out (d x c,
 * nullable) receives the cluster means of D; counts_out (nullable) the n_i. */
void oracle_l_step(const double *X, const double *S, const double *Theta,
                   double rho, double lambda, const int32_t *labels, int32_t c,
                   int64_t d, int64_t n, double *L, double *mu_out,
                   int64_t *counts_out);

/* One K-means assignment, Eq. (21)-(22): labels[j] = argmin over active
 * clusters (active[i] != 0) of ||Y_j - mu_i||^2, direct difference form,
 * ties to the lowest index.  Returns the number of labels that changed. */
int64_t oracle_assign(const double *Y, int64_t d, int64_t n,
                      const double *mu, const uint8_t *active, int32_t c,
                      int32_t *labels);

/* Lloyd iterations from the given labels and centroids (active marks the
 * clusters that own a centroid).  Stops when an assignment changes nothing
 * or after km_max assignments.  On return labels hold the result; mu and
 * active hold the centroids used by the last assignment.  Returns the number
 * of assignment passes; *changed_out (nullable) = labels that differ from the
 * labels on entry. */
int32_t oracle_lloyd(const double *Y, int64_t d, int64_t n, int32_t c,
                     int32_t *labels, double *mu, uint8_t *active,
                     int32_t km_max, int64_t *changed_out);

/* k-means++ seeding of c centres among the columns of X. */
void oracle_kmeanspp(const double *X, int64_t d, int64_t n, int32_t c,
                     uint64_t seed, int64_t *centers);

/* Initial labels: k-means++ seeding, then Lloyd on X.  Returns the number of
 * assignment passes. */
int32_t oracle_init_labels(const double *X, int64_t d, int64_t n, int32_t c,
                           uint64_t seed, int32_t km_max, int32_t *labels);

/* S step, Eq. (24): S = sign(B) max(|B| - 1/rho, 0), B = X - L + Theta/rho. */
void oracle_s_step(const double *X, const double *L, const double *Theta,
                   double rho, int64_t count, double *S);

/* S step with the l2,1 norm on S, the alternative Sec. 3 names in place of
 * l1: S = argmin (1/rho)||S||_{2,1} + 1/2 ||S - B||_F^2, column by column
 * S_j = B_j max(0, 1 - 1/(rho ||B_j||_2)), B = X - L + Theta/rho. */
void oracle_s_step_l21(const double *X, const double *L, const double *Theta,
                       double rho, int64_t d, int64_t n, double *S);

/* Multiplier step, Eq. (25): Theta += rho (X - L - S). */
void oracle_theta_step(const double *X, const double *L, const double *S,
                       double rho, int64_t count, double *Theta);

/* One ALM iteration in the order L, p, S, Theta/rho from the state
 * (L, S, Theta, labels, *rho).  Updates everything in place, multiplies *rho
 * by kappa and writes the three Sec. 5 quantities (unnormalised Frobenius
 * norms) to norms[3] = {||X-L-S||, ||L-L_prev||, ||S-S_prev||}.
 * Returns the number of labels changed; *lloyd_out (nullable) = assignment
 * passes used. */
int64_t oracle_iteration(const double *X, int64_t d, int64_t n, int32_t c,
                         double lambda, double kappa, int32_t km_max,
                         double *L, double *S, double *Theta, int32_t *labels,
                         double *rho, double norms[3], int32_t *lloyd_out);
/* The same with the S norm chosen: snorm 0 = l1 (Eq. (24)), 1 = l2,1. */
int64_t oracle_iteration_ex(const double *X, int64_t d, int64_t n, int32_t c,
                            double lambda, double kappa, int32_t km_max,
                            double *L, double *S, double *Theta, int32_t *labels,
                            double *rho, double norms[3], int32_t *lloyd_out, int32_t snorm);

/* Model objective, Eq. (8), through the sum-of-squares identity of Eq. (20):
 * lambda * sum_i sum_{j in i} ||L_j - mean_i(L)||^2 + ||S||_1. */
double oracle_objective(const double *L, const double *S, const int32_t *labels,
                        int32_t c, double lambda, int64_t d, int64_t n);

/* Augmented Lagrangian, Eq. (9). */
double oracle_lagrangian(const double *X, const double *L, const double *S,
                         const double *Theta, const int32_t *labels, int32_t c,
                         double lambda, double rho, int64_t d, int64_t n);

/* Whole solver.  p0 (nullable) gives the initial labels; otherwise they come
 * from oracle_init_labels(seed).  If warm != 0, L, S, Theta and labels hold
 * the state to continue from and *rho_io its penalty; otherwise everything
 * starts at zero with rho = rho0.  lambda <= 0 selects sqrt(max(d, n)).
 * Theta (d x n) is caller storage.  Returns 0, or -1 on invalid arguments. */
int32_t oracle_solve(const double *X, int64_t d, int64_t n, int32_t c,
                     double lambda, double rho0, double kappa, double tol,
                     int32_t max_iter, int32_t km_max, uint64_t seed,
                     const int32_t *p0, int32_t warm, double *rho_io,
                     double *L, double *S, double *Theta, int32_t *labels,
                     oracle_stats *stats);
/* The same with the S norm chosen (snorm as in oracle_iteration_ex). */
int32_t oracle_solve_ex(const double *X, int64_t d, int64_t n, int32_t c,
                        double lambda, double rho0, double kappa, double tol,
                        int32_t max_iter, int32_t km_max, uint64_t seed,
                        const int32_t *p0, int32_t warm, double *rho_io,
                        double *L, double *S, double *Theta, int32_t *labels,
                        oracle_stats *stats, int32_t snorm);

#ifdef __cplusplus
}
#endif
#endif
