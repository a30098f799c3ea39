/*
 * respca.h -- C ABI of the GB300 RES-PCA solver (librespca.so).
 *
 * RES-PCA (Peng, Chen, Kang, Li, Cheng, "RES-PCA: A Scalable Approach to
 * Recovering Low-rank Matrices", arXiv 1904.07497) splits a data matrix
 * X (d x n, columns are samples) into X = L + S, L made of c groups of
 * nearly equal columns and S sparse, by solving Eq. (8):
 *
 *   min  lambda * sum_i Tr(L d(p_i) (I - 11^T/n_i) d(p_i) L^T) + ||S||_1
 *   s.t. X = L + S, p_i in {0,1}^n, sum_i p_i = 1
 *
 * with the augmented Lagrangian of Eq. (9) and, per iteration, the closed-form
 * L update of Eq. (18), K-means on the columns of L (Sec. 4.2, Eq. (21)-(22)),
 * soft-thresholding for S (Eq. (24)) and the multiplier update of Eq. (25),
 * stopped by the rule of Sec. 5.  Parameters default to Sec. 5.1:
 * lambda = sqrt(max(n, d)), rho0 = 1e-4, kappa = 1.5.
 *
 * Conventions for every entry point:
 *   - Matrices are column-major: element (r, j) of X is X[j*ldx + r].
 *   - Pointers are CUDA device pointers unless the entry point's name ends in
 *     _host; the caller owns all of them.  X is never written.
 *   - Work is queued on the handle's stream (respca_config.stream); the
 *     calls return after the solve has finished (they read the convergence
 *     test back every iteration) and the outputs are ready to use.
 *   - Errors are returned as respca_status; nothing is thrown across the ABI.
 *     After an error the outputs are unspecified; respca_last_error() gives
 *     a one-line description.  RESPCA_ERR_CUDA leaves the handle usable only
 *     if the CUDA context itself survived.
 *   - A handle is thread-compatible, not thread-safe: one call at a time.
 */
#ifndef RESPCA_H
#define RESPCA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RESPCA_ABI_VERSION 4

typedef struct respca_ctx *respca_handle;

typedef enum {
    RESPCA_OK = 0,
    RESPCA_ERR_INVALID_ARG = 1,     /* a size, pointer, label or parameter is out of range */
    RESPCA_ERR_NONFINITE_INPUT = 2, /* X holds NaN or Inf */
    RESPCA_ERR_OOM = 3,             /* device or pinned-host allocation failed */
    RESPCA_ERR_CUDA = 4,            /* a CUDA call failed */
    RESPCA_ERR_TIMEOUT = 5,         /* a bounded device-side wait gave up */
    RESPCA_ERR_UNSUPPORTED = 6      /* a valid request this build does not handle */
} respca_status;

/* Element type of X. */
typedef enum { RESPCA_F32 = 0, RESPCA_BF16 = 1, RESPCA_F16 = 2 } respca_dtype;

typedef struct {
    double rho0;             /* initial penalty rho (Sec. 5.1: 1e-4) */
    double kappa;            /* penalty growth factor, rho <- kappa rho (Eq. (25); Sec. 5.1: 1.5) */
    int32_t kmeans_max_iter; /* cap on Lloyd assignment passes per p step (default 100) */
    int32_t timing;          /* 1: time the fused iteration kernel with CUDA events
                                (respca_stats.ms_fused); default 0 */
    uint64_t seed;           /* seed of the k-means++ draws for the initial labels */
    void *stream;            /* cudaStream_t for all work; NULL = the legacy default stream */
    int32_t device;          /* CUDA device ordinal; -1 = the device current at respca_create */
    int32_t search_impl;     /* nearest-centroid search: 0 = tensor cores when c <= 256 (default;
                                with FP32 state and c <= 128 the fused iteration can also write
                                an FP16 copy fp16(s L) (s a power of two), which the all-column
                                search reads, widening each decision by ||L_j - fp16(s L_j)/s||
                                and re-deciding near ties from the FP32 L, so the labels are
                                unchanged; BF16 / FP16 data is searched directly), 1 = CUDA-core
                                kernel always, 2 = tensor cores on the FP32 operand only */
    int32_t ramp_skip;       /* 1 (default): compute the leading iterations in which S stays 0
                                and no label moves in closed form (exact; see respca_solve);
                                0: run every iteration */
    int32_t batch_lanes;     /* respca_solve_batched: problems solved at once, each lane with its
                                own stream and workspace (0 = default 8; 1 = one after another) */
    int32_t precision;       /* 0 (default): FP32 state throughout.  1: a bf16 phase first --
                                L, S, Theta (and an FP32 X, copied once) stored in BF16 in the
                                workspace, arithmetic in FP32, 14 instead of 28 bytes per
                                element and iteration -- until err <= switch_tol or err stops
                                falling; then the state is widened to FP32 and the iterations
                                continue on the FP32 X to tol.  Warm starts run in FP32. */
    int32_t s_norm;          /* norm on S: 0 (default) = l1, the paper's choice (Eq. (24));
                                1 = l2,1, the alternative Sec. 3 names: block soft-thresholding
                                S_j = B_j max(0, 1 - 1/(rho ||B_j||)) and Theta_j = rho B_j /
                                max(1, rho ||B_j||), in two passes per iteration (44 bytes per
                                element).  With 1 the closed-form leading iterations and the
                                bf16 phase are not used. */
    double switch_tol;       /* end of the bf16 phase (default 1e-2) */
    int32_t stop_after_ramp; /* 1: return after the closed-form leading iterations (ramp_skip;
                                cold starts), with L, Theta (respca_warm), p and rho of the
                                next iteration written out -- the state a learned warm start
                                (respca_net_forward) continues from; 0 (default): solve to tol */
    int32_t p_step;          /* clustering of the p step (Sec. 4.2): 0 (default) = K-means, the
                                paper's choice; 1 = spectral clustering, the nonlinear alternative
                                Sec. 4.2 names (see respca_spectral_labels).  With 1, X must be
                                FP32, precision must be 0, the closed-form leading iterations are
                                not used, and the initial labels (p0 = NULL) are the spectral
                                labels of the columns of X. */
    double spectral_scale;   /* p_step = 1: sigma^2 of the Gaussian affinity as a multiple of the
                                mean squared distance between columns (default 0.125) */
} respca_config;

typedef struct {
    int32_t iters;           /* ALM iterations run */
    int32_t converged;       /* 1 if the Sec. 5 criterion fell to tol */
    double err;              /* max(err_resid, err_dL, err_dS) at exit */
    double err_resid;        /* ||X - L - S||_F / ||X||_F */
    double err_dL;           /* ||L_{t+1} - L_t||_F / ||X||_F */
    double err_dS;           /* ||S_{t+1} - S_t||_F / ||X||_F */
    double rho_final;        /* rho after the last update */
    double lambda;           /* the lambda used */
    int64_t label_changes;   /* labels changed by the p steps, summed over iterations */
    int64_t lloyd_passes;    /* assignment passes run by the p steps */
    int64_t assigned_columns;/* columns whose nearest centroid had to be searched */
    int64_t rechecked_columns;/* near-tie columns re-decided in FP64 */
    int64_t kernel_launches; /* CUDA kernels this call launched */
    int32_t init_lloyd_passes;/* assignment passes of the initial K-means */
    int32_t fused_launches;  /* launches of the fused iteration kernel */
    float ms_total;          /* wall time of the call on the stream (CUDA events) */
    float ms_init;           /* part of ms_total spent before the first iteration */
    float ms_fused;          /* summed duration of the fused iteration kernel (cfg.timing = 1) */
    float ms_dense;          /* summed duration of the all-column tensor-core search kernel over
                                the passes in which it ran (cfg.timing = 1) */
    int32_t dense_passes;    /* passes in which that kernel searched every column */
    int32_t bf16_iters;      /* iterations run with BF16 state (precision = 1) */
    double x_norm;           /* ||X||_F, the denominator of the Sec. 5 quantities */
    float ms_dense16;        /* the part of ms_dense spent in passes that read 16-bit operands
                                (BF16 / FP16 data or the FP16 copy of L: 2 bytes per element) */
    int32_t dense16_passes;  /* the part of dense_passes that read 16-bit operands */
    int32_t copy16_iters;    /* fused iterations that also wrote the FP16 copy of L (2 bytes per
                                element more) */
} respca_stats;

/* Optional warm start / checkpoint-resume state (the paper starts from zero;
 * this hook lets a caller continue an earlier solve or supply a proposal). */
typedef struct {
    float *Theta;            /* d x n device multiplier Theta, leading dimension lds; in/out.
                                NULL: the handle keeps Theta and starts it at zero */
    double rho;              /* in: rho of the next iteration when warm != 0; out: rho_final */
    int32_t warm;            /* 1: L, S, Theta and p hold a state to continue from;
                                0: start from L = S = Theta = 0, rho = rho0 */
    int32_t reserved;
} respca_warm;

/* One problem of a batch (respca_solve_batched). Same meaning as the
 * arguments of respca_solve. */
typedef struct {
    int32_t x_dtype;
    int32_t c;
    const void *X;
    int64_t d, n, ldx;
    double lambda;
    double tol;
    int32_t max_iter;
    int32_t reserved;
    const int32_t *p0;
    float *L;
    float *S;
    int64_t lds;
    int32_t *p;
} respca_problem;

/* Fill *cfg with the defaults above. */
void respca_config_default(respca_config *cfg);

/* Create a solver handle bound to cfg->device and cfg->stream (cfg NULL =
 * defaults).  The handle owns its device workspace, grown on demand and freed
 * by respca_destroy.  Returns RESPCA_ERR_CUDA if no usable device exists. */
respca_status respca_create(respca_handle *h, const respca_config *cfg);

/* Free the handle and all of its device and pinned-host memory. NULL is a no-op. */
respca_status respca_destroy(respca_handle h);

/*
 * Solve Eq. (8) for one matrix (Sec. 4, all four updates per iteration, in the
 * order L (Sec. 4.1), p (Sec. 4.2), S (Sec. 4.3), Theta and rho (Sec. 4.4)).
 *
 *   x_dtype   element type of X (respca_dtype).
 *   X         d x n device matrix, leading dimension ldx >= d. Read only.
 *   lambda    weight of the variance term; <= 0 selects sqrt(max(d, n)) (Sec. 5.1).
 *   c         number of column groups (the rank or a bound on it), 1 <= c <= n.
 *   tol       stop when max(||X-L-S||, ||dL||, ||dS||)/||X|| <= tol (Sec. 5); >= 0.
 *   max_iter  iteration cap (>= 0; the paper uses 500).
 *   p0        optional initial labels (n int32 in [0, c), device); NULL = k-means++
 *             seeding (cfg.seed) followed by Lloyd on the columns of X.
 *   L, S      d x n device outputs (FP32), leading dimension lds >= d.
 *   p         n device int32 output labels (the groups of Eq. (8)).
 *   warm      optional warm start (see respca_warm); NULL = cold start.
 *   stats     optional host struct filled on return.
 * ||X||_F = 0 returns L = S = 0 at once.  Hitting max_iter is not an error
 * (stats->converged = 0).
 *
 * Ramp skip (cfg.ramp_skip, cold starts only): while every |B| <= 1/rho the S
 * step of Eq. (24) returns 0, and while no label moves the L step of Eq. (18)
 * maps X = X_m + X_r (cluster means + residual) to L_{t+1} = X_m + a_t g_t X_r,
 * Theta_{t+1} = rho_t b_t g_t X_r with g_0 = 1, g_{t+1} = 1 + (b_t/kappa) g_t,
 * a_t = rho_t/(2 lambda + rho_t), b_t = 1 - a_t.  Both conditions reduce to the
 * scalars max|X_r| and max_j ||r_j|| / sep(p_j) (sep = distance from a centroid
 * to the nearest other one), so the solver checks them for each leading
 * iteration (with a 1e-3 safety margin) and writes the state after the last
 * iteration that provably keeps S = 0 and every label.  The iterates equal
 * those of the step-by-step run up to FP32 rounding; stats count the skipped
 * iterations.
 */
respca_status respca_solve(respca_handle h, int32_t x_dtype, const void *X, int64_t d,
                           int64_t n, int64_t ldx, double lambda, int32_t c, double tol,
                           int32_t max_iter, const int32_t *p0, float *L, float *S,
                           int64_t lds, int32_t *p, respca_warm *warm, respca_stats *stats);

/* As respca_solve, but X, p0, L, S and p are HOST pointers (pageable or
 * pinned).  The handle stages them through its device workspace; the
 * host-to-device and device-to-host copies are part of the call. warm is not
 * accepted here (pass NULL). */
respca_status respca_solve_host(respca_handle h, int32_t x_dtype, const void *X, int64_t d,
                                int64_t n, int64_t ldx, double lambda, int32_t c, double tol,
                                int32_t max_iter, const int32_t *p0, float *L, float *S,
                                int64_t lds, int32_t *p, respca_stats *stats);

/* Initial labels alone: k-means++ seeding with cfg.seed (Arthur and
 * Vassilvitskii's D^2 sampling; splitmix64 uniforms) and Lloyd's method on the
 * columns of X until no label changes (cap cfg.kmeans_max_iter).  The paper
 * leaves the initial p open; this is the reading the solver uses when p0 is
 * NULL.  p: n device int32 output; *passes (nullable host) = assignment passes. */
respca_status respca_init_labels(respca_handle h, int32_t x_dtype, const void *X, int64_t d,
                                 int64_t n, int64_t ldx, int32_t c, int32_t *p,
                                 int32_t *passes);

/* Solve `batch` independent problems (device pointers as in respca_solve).
 * The problems run concurrently on cfg.batch_lanes lanes: each lane is an
 * internal solver with its own non-blocking stream and workspace, driven by
 * its own host thread, taking the largest remaining problem (d * n) next.
 * Every problem runs exactly the single-matrix path, so its results equal
 * those of respca_solve on it.  Work already queued on cfg.stream is waited
 * for first, and cfg.stream waits for the lanes when the call returns (it
 * blocks until all problems are done).  stats: optional host array of `batch`
 * entries.  The lowest-index failing problem's status is returned; the other
 * problems are still attempted.  The handle is not thread-safe; the lanes are
 * its own. */
respca_status respca_solve_batched(respca_handle h, int32_t batch, const respca_problem *probs,
                                   respca_stats *stats);

/* Options and results of respca_solve_batched_persistent. */
typedef struct {
    int32_t tile_rows;          /* in: rows per row-block work item, 64 or 128; 0 = autotuned
                                   (with two CTAs per SM the items are 64 rows) */
    int32_t ctas_per_sm;        /* in: resident CTAs per SM, 1 or 2; 0 = autotuned */
    int64_t spin_limit;         /* in: empty polls of the work queue after which a CTA gives up
                                   (RESPCA_ERR_TIMEOUT); 0 = default (2^23, about a second or more) */
    int32_t tuned_rows;         /* out: the rows per row item used */
    int32_t tuned_ctas_per_sm;  /* out: the CTAs per SM used */
    float ms_kernel;            /* out: duration of the persistent launch (CUDA events) */
    int32_t reserved;
} respca_batch_options;

/*
 * Solve `batch` independent problems (as respca_solve_batched) in ONE
 * persistent kernel launch, replayed from a CUDA graph while the batch's
 * pointers and sizes stay the same.  Each problem runs the iteration of
 * Sec. 4 -- Eq. (18), Lloyd's method for the p step of Sec. 4.2, Eq. (24),
 * Eq. (25) and the Sec. 5 stopping rule, every iteration (no closed-form
 * leading iterations) -- after k-means++ (cfg.seed, the same draws as
 * respca_init_labels) and Lloyd on X, or from the problem's p0.  The work of
 * all problems is split into row-block and column-block items that the
 * launch's CTAs (one or two per SM) pull from a per-problem claim word; the
 * CTA that completes a phase runs its serial tail and publishes the next
 * phase, so problems of any size mix in one launch.  Results match the FP64
 * oracle to FP32 rounding (labels identical to respca_solve's except where two
 * distances agree to about 1e-5); they are not bit-identical to respca_solve,
 * whose kernels sum in other orders.
 *
 * Limits: FP32 X, 1 <= c <= 64, d, n <= 2^22 (RESPCA_ERR_UNSUPPORTED beyond).
 * Tile rows and CTAs per SM are chosen by timing the candidates on a run of
 * the batch capped at 3 iterations, once per batch shape and handle, unless
 * opt fixes them.  A CTA that finds no work for spin_limit polls sets a
 * timeout flag; every CTA then leaves at its next item boundary and the call
 * returns RESPCA_ERR_TIMEOUT (outputs unspecified).  Per-problem errors (NaN
 * or Inf in X: RESPCA_ERR_NONFINITE_INPUT; p0 labels outside [0, c):
 * RESPCA_ERR_INVALID_ARG) end that problem only; the lowest-index one is
 * returned.  stats (optional, `batch` entries): per problem; kernel_launches
 * is 1 on entry 0 and ms_total the launch's duration on every entry.
 * opt: optional.  Synchronous: returns when every problem is done.
 */
respca_status respca_solve_batched_persistent(respca_handle h, int32_t batch, const respca_problem *probs,
                                              respca_stats *stats, respca_batch_options *opt);

/* Anomaly score of Sec. 6: out[j] = ||S_j||_2 for every column j of a d x n
 * device matrix S (leading dimension lds >= d), e.g. the S of a solve; the
 * columns with large scores are the outlying samples.  out: n device floats.
 * Runs on `stream` (cudaStream_t, NULL = legacy default stream); asynchronous.
 * Returns RESPCA_ERR_INVALID_ARG for null pointers or d, n < 1, lds < d. */
respca_status respca_column_norms(const float *S, int64_t d, int64_t n, int64_t lds, float *out,
                                  void *stream);

/*
 * Initial labels WITHOUT ANY ALLOCATION.  The paper has no counterpart: this
 * is a library convenience for callers that may not allocate device memory
 * while it runs: programs whose device memory belongs to their own pool
 * allocator or is capped by a hard budget, and hosts that forbid a plug-in
 * library from taking memory on its own.  No handle is used, because creating
 * one allocates.  It uses the same k-means++ draws (same seed) and the same
 * Lloyd rule as respca_init_labels; both take every assignment as the argmin
 * of the stored distances with near ties re-decided exactly (ties to the
 * lowest index), so the two give the same labels.  It runs on CUDA cores
 * (the handle path searches on tensor cores).
 *
 *   x_dtype, X, d, n, ldx, c  as in respca_init_labels (device X).
 *   seed             seed of the k-means++ draws (cfg.seed of the handle path).
 *   kmeans_max_iter  cap on Lloyd passes (values below 1 mean 1, as
 *                    cfg.kmeans_max_iter of the handle path).
 *   p                n device int32 output labels (caller-allocated).
 *   passes           optional host output: Lloyd assignment passes run.
 *   stream           cudaStream_t to run on (NULL = legacy default stream).
 *
 * X and p must be memory of the CUDA device that is current when the call is
 * made (or managed memory); otherwise RESPCA_ERR_INVALID_ARG.  All scratch
 * lives in one 32 MiB array in device global memory, declared at file scope
 * in the library; every GPU that loads the library holds it until the process
 * exits.  The call needs
 *   256-byte-aligned pieces totalling about 4 d (ceil(n/32) + c) + 4 c d + 12 n + 32 c bytes;
 * requests that do not fit (or c > 1024) return RESPCA_ERR_UNSUPPORTED
 * without touching the device.  The array's device address is looked up
 * once per device, on the first call made with that device current; make
 * that first call before any stream capture starts.  Calls share the array
 * (it keeps the previous call's contents; the call clears what must start at
 * zero), so calls that overlap on the GPU -- from two streams or two host
 * threads -- race and must be serialised by the caller.  The call is
 * synchronous: it reads its progress back from the device after every Lloyd
 * pass and returns when the labels are final.
 */
respca_status respca_init_labels_noalloc(int32_t x_dtype, const void *X, int64_t d, int64_t n,
                                         int64_t ldx, int32_t c, uint64_t seed,
                                         int32_t kmeans_max_iter, int32_t *p, int32_t *passes,
                                         void *stream);

/* Result of one spectral clustering (respca_spectral_labels). */
typedef struct {
    int32_t outer_iters;     /* Rayleigh-Ritz steps of the eigensolver */
    int32_t matvecs;         /* products of M with the search block */
    double residual;         /* max_j ||M u_j - theta_j u_j|| over the c eigenpairs kept */
    double sigma2;           /* the affinity's sigma^2 */
    double theta_c;          /* c-th largest Ritz value */
    double theta_next;       /* (c+1)-th largest Ritz value (eigen-gap = theta_c - theta_next) */
    int32_t lloyd_passes;    /* K-means passes on the embedding */
    int32_t converged;       /* 1 if residual <= 1e-5 within the iteration cap */
    double ms_gram;          /* with cfg.timing: device time of the Gram matrix Y^T Y (else 0) */
    double ms_products;      /* with cfg.timing: device time of the matvecs products with M (else 0) */
} respca_spectral_info;

/*
 * The spectral p step alone: labels of the n columns of Y (d x n device FP32,
 * leading dimension ldy >= d) in c groups by normalised spectral clustering
 * (Ng, Jordan and Weiss), the nonlinear clustering Sec. 4.2 offers in place of
 * K-means:
 *   A_ij = exp(-||y_i - y_j||^2 / (2 sigma^2)) for i != j, A_ii = 0, with
 *   sigma^2 = cfg.spectral_scale x the mean of ||y_i - y_j||^2 over i != j;
 *   M = D^{-1/2} A D^{-1/2} (D = row sums of A); U = the eigenvectors of M's
 *   c largest eigenvalues; rows of U scaled to unit length; K-means (k-means++
 *   with cfg.seed, then Lloyd, as respca_init_labels) on those rows.
 * The eigenvectors come from Chebyshev-filtered subspace iteration with
 * Rayleigh-Ritz on a block of c + 8 vectors (at most 100 steps of degree 8).
 * The handle keeps an n x n FP32 matrix in its workspace.  Limits: 1 <= c <= 64,
 * c < n <= 32768 (RESPCA_ERR_UNSUPPORTED beyond).  p: n device int32 outputs;
 * info: optional host output.  Synchronises the handle's stream.
 */
respca_status respca_spectral_labels(respca_handle h, const float *Y, int64_t d, int64_t n,
                                     int64_t ldy, int32_t c, int32_t *p,
                                     respca_spectral_info *info);

/*
 * Learned warm start.  Not in the paper: an unrolled continuation of the
 * Sec. 4 iteration that a caller trains to carry a state further than the
 * same number of plain iterations would, after which respca_solve continues
 * from its output (respca_warm).  The labels p are held fixed.  Layer k, with
 * its own step rho_k and soft threshold tau_k (all FP32 arithmetic):
 *   D = X - S + Theta/rho_k;  mu_i = mean of D over group i;  a = rho_k/(2 lambda + rho_k)
 *   L = a D + (1 - a) mu_p                                  (Eq. (18))
 *   B = X - L + Theta/rho_k;  S' = sign(B) max(|B| - tau_k, 0)  (Eq. (24), tau_k in place of 1/rho_k)
 *   Theta' = Theta + rho_k (X - L - S')                     (Eq. (25))
 * With tau_k = 1/rho_k and rho_{k+1} = kappa rho_k the layers are the plain
 * iterations with p fixed.  The parameters a caller learns are log
 * multipliers m = [theta_0..theta_{K-1}, phi_0..phi_{K-1}] on that schedule:
 * rho_k = rho kappa^k exp(theta_k), tau_k = exp(phi_k) / rho_k.
 */
typedef struct respca_net_s *respca_net;

/* Create a network context on `device` (-1 = current) working on `stream`
 * (cudaStream_t, NULL = legacy default).  It owns its device workspace: the
 * inputs of every layer (2 (K+1) d n floats) are kept for the backward pass. */
respca_status respca_net_create(respca_net *net, int32_t device, void *stream);
respca_status respca_net_destroy(respca_net net);

/* Host arithmetic: (rho_k, tau_k), k < layers, from rho, kappa and the 2 K
 * multipliers m (host floats, layout above).  rho > 0, kappa > 0. */
respca_status respca_net_schedule(double rho, double kappa, int32_t layers, const float *m,
                                  double *rho_k, double *tau_k);

/* Forward pass through `layers` layers from (S0, Theta0).
 *   X          d x n device FP32, leading dimension ldx >= d (read only).
 *   p          n device int32 labels in [0, c) (read only; fixed in every layer).
 *   lambda     weight of the variance term (> 0).
 *   S0, Theta0 d x n device FP32 input state, leading dimension lds >= d (copied).
 *   rho_k, tau_k  host arrays of `layers` positive values.
 *   L, S, Theta   d x n device FP32 outputs of the last layer (leading dimension
 *              lds; may be NULL).  The call waits once for the label check (after the
 *              label sort); the layers themselves are queued on the stream.
 * The context keeps the pointer X (not a copy): X must stay allocated and
 * unchanged until the matching respca_net_backward returns.
 * Errors: RESPCA_ERR_INVALID_ARG (null or inconsistent sizes, non-positive
 * scalars, layers < 1, labels outside [0, c)), RESPCA_ERR_OOM, RESPCA_ERR_CUDA. */
respca_status respca_net_forward(respca_net net, const float *X, int64_t d, int64_t n, int64_t ldx,
                                 const int32_t *p, int32_t c, double lambda, const float *S0,
                                 const float *Theta0, int64_t lds, int32_t layers,
                                 const double *rho_k, const double *tau_k, float *L, float *S,
                                 float *Theta);

/* Inference-only forward pass through the same layers (nothing is kept for
 * respca_net_backward, and a preceding forward pass is forgotten).
 *   x_dtype    element type of X (respca_dtype; FP32, BF16 or FP16), read as given.
 *   storage    0: the intermediate layers' S and Theta are stored in FP32;
 *              1: in BF16 (each stored value is the layer's FP32 result rounded to
 *              BF16; the layers then move 2 instead of 4 bytes per stored element).
 *              The arithmetic of every layer is FP32 either way.
 *   S0, Theta0 d x n device FP32 input state, leading dimension lds (read only).
 *   L, S, Theta d x n device FP32 outputs of the last layer (leading dimension lds),
 *              required; L of the intermediate layers is never formed.
 * Other arguments as respca_net_forward.  The call waits once for the label
 * check; the layers are queued on the stream.  Errors as respca_net_forward. */
respca_status respca_net_infer(respca_net net, int32_t x_dtype, const void *X, int64_t d, int64_t n,
                               int64_t ldx, const int32_t *p, int32_t c, double lambda,
                               const float *S0, const float *Theta0, int64_t lds, int32_t layers,
                               const double *rho_k, const double *tau_k, int32_t storage, float *L,
                               float *S, float *Theta);

/* Loss and exact gradient of the last forward pass:
 *   loss = scale (||L - Lt||_F^2 + ||S - St||_F^2)
 * for targets Lt, St (d x n device FP32, leading dimension ldt >= d).  Writes
 * host *loss, g_rho[k] = dloss/drho_k and g_tau[k] = dloss/dtau_k (FP32 sums
 * per element, FP64 across CTAs); g_m (optional, 2 K host floats) receives
 * dloss/dm for the multipliers of respca_net_schedule.  Synchronises the
 * stream.  RESPCA_ERR_INVALID_ARG without a preceding forward pass. */
respca_status respca_net_backward(respca_net net, const float *Lt, const float *St, int64_t ldt,
                                  double scale, double *loss, double *g_rho, double *g_tau,
                                  float *g_m);

/* The multipliers' predictor: a 2-layer MLP out = W2 tanh(W1 z + b1) + b2 on
 * nz statistics z of the state, hidden width H, nout outputs.  Parameters are
 * one device FP32 array [W1 (H x nz, row-major) | b1 (H) | W2 (nout x H) | b2
 * (nout)] of H nz + H + nout H + nout floats.  z, out, hidden (H floats, the
 * tanh activations kept for the backward pass) are device arrays.  Async on
 * `stream`.  nz, H, nout in [1, 1024]. */
respca_status respca_mlp_forward(const float *params, int32_t nz, int32_t H, int32_t nout,
                                 const float *z, float *out, float *hidden, void *stream);

/* Gradient of <gout, out> with respect to params into grad (same layout);
 * accumulate = 1 adds to grad instead of overwriting it. */
respca_status respca_mlp_backward(const float *params, int32_t nz, int32_t H, int32_t nout,
                                  const float *z, const float *hidden, const float *gout,
                                  float *grad, int32_t accumulate, void *stream);

/* One Adam step (Kingma and Ba) over `count` device floats: moments m, v
 * updated in place, bias correction for step t >= 1. */
respca_status respca_adam_step(float *params, const float *grad, float *m, float *v, int64_t count,
                               double lr, double beta1, double beta2, double eps, int32_t t,
                               void *stream);

/* Static description of a status code. */
const char *respca_status_string(respca_status s);

/* Description of the last error on this handle ("" if none). */
const char *respca_last_error(respca_handle h);

#ifdef __cplusplus
}
#endif
#endif /* RESPCA_H */
