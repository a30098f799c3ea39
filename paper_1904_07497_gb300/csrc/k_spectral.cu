// Kernels of the spectral p step (Sec. 4.2: spectral clustering in place of
// K-means on the columns of L).  Normalised spectral clustering:
//   A_ij = exp(-||y_i - y_j||^2 / (2 sigma^2)) (i != j), A_ii = 0,
//   sigma^2 = scale * mean_{i != j} ||y_i - y_j||^2,
//   M = D^{-1/2} A D^{-1/2},  U = top-c eigenvectors of M,  e_i = U_i / ||U_i||,
// then K-means on the e_i.  The eigenvectors come from Chebyshev-filtered
// subspace iteration with Rayleigh-Ritz (the spectrum of M lies in [-1, 1]).
#include "respca_internal.cuh"

namespace respca {

namespace {

constexpr int kGT = 64;     // GEMM output tile (rows and columns)
constexpr int kGK = 16;     // GEMM K step
constexpr int kGThreads = 256;

// C[i + j ldc] = alpha * sum_k A[k + i lda] B[k + j ldb]   (C = A^T B), FP32.
// 64 x 64 output tile per CTA, 4 x 4 per thread, K in steps of 16 through
// shared memory.
__global__ void __launch_bounds__(kGThreads)
    k_gemm_tn(const float* __restrict__ A, int64_t lda, const float* __restrict__ B, int64_t ldb,
              float* __restrict__ C, int64_t ldc, int64_t m, int64_t n, int64_t K, float alpha) {
    __shared__ float As[kGK][kGT + 1];
    __shared__ float Bs[kGK][kGT + 1];
    const int64_t i0 = (int64_t)blockIdx.x * kGT, j0 = (int64_t)blockIdx.y * kGT;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    for (int64_t k0 = 0; k0 < K; k0 += kGK) {
        // 16 x 64 elements of each operand: 4 per thread, k fastest (contiguous)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = threadIdx.x + q * kGThreads;
            const int kk = e & 15, ii = e >> 4;
            const int64_t k = k0 + kk;
            const int64_t ia = i0 + ii, jb = j0 + ii;
            As[kk][ii] = (k < K && ia < m) ? A[k + ia * lda] : 0.f;
            Bs[kk][ii] = (k < K && jb < n) ? B[k + jb * ldb] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][tx + 16 * q];
                b[q] = Bs[kk][ty + 16 * q];
            }
#pragma unroll
            for (int qa = 0; qa < 4; ++qa)
#pragma unroll
                for (int qb = 0; qb < 4; ++qb) acc[qa][qb] = fmaf(a[qa], b[qb], acc[qa][qb]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int qa = 0; qa < 4; ++qa)
#pragma unroll
        for (int qb = 0; qb < 4; ++qb) {
            const int64_t i = i0 + tx + 16 * qa, j = j0 + ty + 16 * qb;
            if (i < m && j < n) C[i + j * ldc] = alpha * acc[qa][qb];
        }
}

// Squared norm of every column (FP64 accumulation) and per-CTA partial sums of them.
__global__ void __launch_bounds__(kThreads)
    k_spec_norms(const float* __restrict__ Y, int64_t ldy, int64_t d, int64_t n, float* __restrict__ sqn,
                 double* __restrict__ sqn_sum_part) {
    __shared__ double red[kThreads / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double tot = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * (kThreads / 32) + warp; j < n; j += (int64_t)gridDim.x * (kThreads / 32)) {
        double s = 0.0;
        for (int64_t r = lane; r < d; r += 32) {
            const double v = Y[j * ldy + r];
            s += v * v;
        }
        s = warp_sum(s);
        if (lane == 0) sqn[j] = (float)s;
        tot += s;
    }
    if (lane == 0) red[warp] = tot;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        sqn_sum_part[blockIdx.x] = t;
    }
}

// Row sums of the Gram matrix (one CTA per row, FP64): sum_j G_ij = y_i . (sum_j y_j).
__global__ void __launch_bounds__(kThreads)
    k_spec_gsum(const float* __restrict__ G, int64_t n, double* __restrict__ gsum) {
    __shared__ double red[kThreads / 32];
    const int64_t i = blockIdx.x;
    double acc = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += kThreads) acc += (double)G[i * n + j];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        gsum[i] = t;
    }
}

// sigma^2 = scale * (2 n sum||y||^2 - 2 ||sum y||^2) / (n (n - 1)), with
// ||sum y||^2 = sum_ij G_ij; out[0] = sigma^2, out[1] = 1 / (2 sigma^2)  (one block).
__global__ void k_spec_sigma(const double* __restrict__ sqn_part, int parts, const double* __restrict__ gsum,
                             int64_t n, double scale, double* __restrict__ out) {
    __shared__ double red[2][kThreads / 32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < parts; i += kThreads) a += sqn_part[i];
    for (int64_t r = threadIdx.x; r < n; r += kThreads) b += gsum[r];
    a = warp_sum(a);
    b = warp_sum(b);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = a;
        red[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            ta += red[0][w];
            tb += red[1][w];
        }
        const double msd = (2.0 * (double)n * ta - 2.0 * tb) / ((double)n * (double)(n - 1));
        const double s2 = scale * msd;
        out[0] = s2;
        out[1] = s2 > 0.0 ? 0.5 / s2 : 0.0;
    }
}

// Row i (one CTA): G_ij -> A_ij in place and deg_i = sum_j A_ij (FP64, fixed order).
__global__ void __launch_bounds__(kThreads)
    k_spec_affinity(float* __restrict__ G, int64_t n, const float* __restrict__ sqn,
                    const double* __restrict__ sig, double* __restrict__ deg) {
    __shared__ double red[kThreads / 32];
    const int64_t i = blockIdx.x;
    const float inv2s2 = (float)sig[1];
    const float si = sqn[i];
    float* row = G + i * n;   // G is symmetric: row i = column i
    double acc = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += kThreads) {
        const float d2 = fmaxf(si + sqn[j] - 2.f * row[j], 0.f);
        const float a = (j == i || inv2s2 == 0.f) ? 0.f : expf(-d2 * inv2s2);
        row[j] = a;
        acc += (double)a;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        deg[i] = t;
    }
}

// r_j = deg_j^{-1/2} (FP64, rounded once; isolated points get 0).
__global__ void k_spec_rinv(const double* __restrict__ deg, int64_t n, float* __restrict__ r) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double dj = deg[j];
    r[j] = dj > 0.0 ? (float)(1.0 / sqrt(dj)) : 0.f;
}

// M_ij = A_ij r_i r_j.
__global__ void __launch_bounds__(kThreads)
    k_spec_normalise(float* __restrict__ A, int64_t n, const float* __restrict__ r) {
    const int64_t i = blockIdx.x;
    const float ri = r[i];
    for (int64_t j = threadIdx.x; j < n; j += kThreads) A[i * n + j] = A[i * n + j] * ri * r[j];
}

// splitmix64 (Steele, Lea, Flood 2014) of a counter: the start block.
__device__ __forceinline__ uint64_t spec_mix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__global__ void k_spec_start(float* __restrict__ Y, int64_t n, int b, uint64_t seed) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * b) return;
    const uint64_t u = spec_mix(seed * 0x100000001B3ULL + (uint64_t)e);
    Y[e] = (float)((double)(u >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
}

// Y_next = alpha T + beta Y + gamma Y_prev (elementwise over n x b).
__global__ void k_spec_axpby(float* __restrict__ out, const float* __restrict__ T, const float* __restrict__ Y,
                             const float* __restrict__ Yp, int64_t count, float alpha, float beta, float gamma) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    float v = alpha * T[e] + beta * Y[e];
    if (Yp) v += gamma * Yp[e];
    out[e] = v;
}

// W = M Y for the symmetric n x n matrix M and the n x b block Y (both
// column-major): one warp per row i of M (contiguous, = column i), lanes over
// k, the block's rows of Y staged in shared memory 128 at a time; M is read
// once.  BMAX >= b accumulators per lane, reduced across the warp at the end.
constexpr int kSymRows = 16;        // rows of M (warps) per CTA
constexpr int kSymK = 128;          // rows of Y per shared-memory stage
template <int BMAX>
__global__ void __launch_bounds__(kSymRows * 32)
    k_spec_symm(const float* __restrict__ M, int64_t n, const float* __restrict__ Y, int b,
                float* __restrict__ W) {
    __shared__ float ys[kSymK][BMAX + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * kSymRows + warp;
    const float* mrow = M + (i < n ? i : 0) * n;
    float acc[BMAX];
#pragma unroll
    for (int q = 0; q < BMAX; ++q) acc[q] = 0.f;
    for (int64_t k0 = 0; k0 < n; k0 += kSymK) {
        __syncthreads();
        for (int e = threadIdx.x; e < kSymK * BMAX; e += kSymRows * 32) {
            const int kk = e % kSymK, q = e / kSymK;
            ys[kk][q] = (q < b && k0 + kk < n) ? Y[k0 + kk + (int64_t)q * n] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < kSymK / 32; ++t) {
            const int kk = t * 32 + lane;
            const float m = (k0 + kk < n) ? mrow[k0 + kk] : 0.f;
#pragma unroll
            for (int q = 0; q < BMAX; ++q) acc[q] = fmaf(m, ys[kk][q], acc[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < BMAX; ++q) {
        const float v = warp_sum(acc[q]);
        if (lane == 0 && i < n && q < b) W[i + (int64_t)q * n] = v;
    }
}

// out[i + j b1] = sum_k A[k + i n] B[k + j n] in FP64 (one CTA per entry):
// the b1 x b2 Gram or Rayleigh-quotient matrices of n-row blocks.
__global__ void __launch_bounds__(kThreads)
    k_spec_gram_small(const float* __restrict__ A, const float* __restrict__ B, int64_t n, int b1,
                      double* __restrict__ out) {
    __shared__ double red[kThreads / 32];
    const int i = blockIdx.x, j = blockIdx.y;
    const float* a = A + (int64_t)i * n;
    const float* bb = B + (int64_t)j * n;
    double acc = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += kThreads) acc += (double)a[k] * (double)bb[k];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        out[i + (int64_t)j * b1] = t;
    }
}

// One step of Cholesky QR: G = Y^T Y (b x b, FP64) plus a shift of 1e-12
// times its largest diagonal entry (so that rounding cannot break the
// factorisation of a numerically rank-deficient block), G = R^T R, and
// Q = R^{-1} (upper triangular, column-major FP32) for Y <- Y Q.  One CTA.
constexpr int kCholThreads = 256;
__global__ void __launch_bounds__(kCholThreads)
    k_spec_chol_inv(const double* __restrict__ G, int b, float* __restrict__ Q) {
    extern __shared__ double cm[];
    double* R = cm;             // b x b, column-major, upper triangle used
    double* V = cm + b * b;     // R^{-1}
    __shared__ double shift;
    for (int e = threadIdx.x; e < b * b; e += kCholThreads) {
        R[e] = G[e];
        V[e] = 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int q = 0; q < b; ++q) mx = fmax(mx, R[q + q * b]);
        shift = 1e-12 * mx + 1e-300;
    }
    __syncthreads();
    // right-looking Cholesky on the upper triangle: R[k][j] for j >= k
    for (int k = 0; k < b; ++k) {
        __syncthreads();
        const double piv = sqrt(fmax(R[k + k * b] + shift, 1e-300));
        __syncthreads();
        for (int j = k + threadIdx.x; j < b; j += kCholThreads) R[k + j * b] = (j == k) ? piv : R[k + j * b] / piv;
        __syncthreads();
        // trailing update: R[i][j] -= R[k][i] R[k][j], k < i <= j
        for (int e = threadIdx.x; e < b * b; e += kCholThreads) {
            const int ii = e % b, jj = e / b;
            if (ii > k && jj >= ii) R[ii + jj * b] -= R[k + ii * b] * R[k + jj * b];
        }
    }
    __syncthreads();
    // V = R^{-1}, column by column: V[j][j] = 1/R[j][j], V[i][j] = -(sum_{k=i+1..j} R[i][k] V[k][j]) / R[i][i]
    for (int j = threadIdx.x; j < b; j += kCholThreads) {
        V[j + j * b] = 1.0 / R[j + j * b];
        for (int i = j - 1; i >= 0; --i) {
            double sacc = 0.0;
            for (int k = i + 1; k <= j; ++k) sacc += R[i + k * b] * V[k + j * b];
            V[i + j * b] = -sacc / R[i + i * b];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < b * b; e += kCholThreads) Q[e] = (float)V[e];
}

// Symmetric eigen-decomposition of H (b x b, FP32 in, symmetrised in FP64) by
// cyclic Jacobi with the round-robin pair order (b/2 disjoint rotations per
// step).  Writes the eigenvalues in descending order and the matching
// eigenvectors as the columns of Q (b x b, FP32, column-major).  One CTA.
constexpr int kJacThreads = 256;

__global__ void __launch_bounds__(kJacThreads)
    k_spec_jacobi(const double* __restrict__ H, int b, float* __restrict__ Q, double* __restrict__ evals,
                  int max_sweeps) {
    extern __shared__ double sm[];
    const int bp = b + (b & 1);          // padded to even (a zero row and column)
    double* a = sm;                      // bp x bp
    double* v = a + bp * bp;             // bp x bp
    double* cs = v + bp * bp;            // bp/2 cosines
    double* sn = cs + bp / 2;            // bp/2 sines
    int* pr = reinterpret_cast<int*>(sn + bp / 2);   // bp pair slots
    __shared__ double offn;
    for (int e = threadIdx.x; e < bp * bp; e += kJacThreads) {
        const int i = e % bp, j = e / bp;
        double x = 0.0;
        if (i < b && j < b) x = 0.5 * (H[i + j * b] + H[j + i * b]);
        a[e] = x;
        v[e] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    const int half = bp / 2;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) {
            double o = 0.0, t = 0.0;
            for (int j = 0; j < bp; ++j)
                for (int i = 0; i < bp; ++i) {
                    const double x = a[i + j * bp];
                    t += x * x;
                    if (i != j) o += x * x;
                }
            offn = (o <= 1e-24 * t || t == 0.0) ? -1.0 : o;   // off-diagonal below 1e-12 relative
        }
        __syncthreads();
        if (offn < 0.0) break;
        for (int step = 0; step < bp - 1; ++step) {
            // round-robin: slot 0 fixed, the others rotate by `step`
            if (threadIdx.x < bp) {
                int idx = threadIdx.x;
                int pos = (idx == 0) ? 0 : 1 + (idx - 1 + step) % (bp - 1);
                pr[pos] = idx;
            }
            __syncthreads();
            // pair k = (pr[k], pr[bp - 1 - k])
            if (threadIdx.x < half) {
                const int k = threadIdx.x;
                int p = pr[k], q = pr[bp - 1 - k];
                if (p > q) { const int t = p; p = q; q = t; }
                const double apq = a[p + q * bp];
                double c = 1.0, s = 0.0;
                if (fabs(apq) > 1e-300) {
                    const double app = a[p + p * bp], aqq = a[q + q * bp];
                    const double tau = (aqq - app) / (2.0 * apq);
                    const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    c = 1.0 / sqrt(1.0 + t * t);
                    s = t * c;
                }
                cs[k] = c;
                sn[k] = s;
            }
            __syncthreads();
            // rows: A <- J^T A (each pair updates its two rows, every column)
            for (int e = threadIdx.x; e < half * bp; e += kJacThreads) {
                const int k = e / bp, col = e % bp;
                int p = pr[k], q = pr[bp - 1 - k];
                if (p > q) { const int t = p; p = q; q = t; }
                const double c = cs[k], s = sn[k];
                const double xp = a[p + col * bp], xq = a[q + col * bp];
                a[p + col * bp] = c * xp - s * xq;
                a[q + col * bp] = s * xp + c * xq;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (int e = threadIdx.x; e < half * bp; e += kJacThreads) {
                const int k = e / bp, row = e % bp;
                int p = pr[k], q = pr[bp - 1 - k];
                if (p > q) { const int t = p; p = q; q = t; }
                const double c = cs[k], s = sn[k];
                const double xp = a[row + p * bp], xq = a[row + q * bp];
                a[row + p * bp] = c * xp - s * xq;
                a[row + q * bp] = s * xp + c * xq;
                const double vp = v[row + p * bp], vq = v[row + q * bp];
                v[row + p * bp] = c * vp - s * vq;
                v[row + q * bp] = s * vp + c * vq;
            }
            __syncthreads();
        }
    }
    // descending order of the first b eigenvalues (selection by rank; ties by index)
    for (int j = threadIdx.x; j < b; j += kJacThreads) {
        const double x = a[j + j * bp];
        int rank = 0;
        for (int k = 0; k < b; ++k) {
            const double y = a[k + k * bp];
            rank += (y > x) || (y == x && k < j);
        }
        evals[rank] = x;
        for (int i = 0; i < b; ++i) Q[i + rank * b] = (float)v[i + j * bp];
    }
}

// out = Y Q  (n x b times b x b; Q column-major), one thread per row.
__global__ void __launch_bounds__(kThreads)
    k_spec_rotate(const float* __restrict__ Y, const float* __restrict__ Q, float* __restrict__ out, int64_t n, int b) {
    extern __shared__ float qs[];
    for (int e = threadIdx.x; e < b * b; e += kThreads) qs[e] = Q[e];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    for (int j = 0; j < b; ++j) {
        float s = 0.f;
        for (int k = 0; k < b; ++k) s = fmaf(Y[i + (int64_t)k * n], qs[k + j * b], s);
        out[i + (int64_t)j * n] = s;
    }
}

// res[j] = ||W_j - theta_j Y_j||, j < c (one CTA per column).
__global__ void __launch_bounds__(kThreads)
    k_spec_residual(const float* __restrict__ W, const float* __restrict__ Y, const double* __restrict__ evals,
                    int64_t n, double* __restrict__ res) {
    __shared__ double red[kThreads / 32];
    const int j = blockIdx.x;
    const float th = (float)evals[j];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kThreads) {
        const double r = (double)W[i + (int64_t)j * n] - (double)th * Y[i + (int64_t)j * n];
        acc += r * r;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        res[j] = sqrt(t);
    }
}

// E (c x n, column-major): E[:, i] = U_i / ||U_i|| with U the first c columns of Y.
__global__ void __launch_bounds__(kThreads)
    k_spec_embed(const float* __restrict__ Y, int64_t n, int c, float* __restrict__ E) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int j = 0; j < c; ++j) {
        const double v = Y[i + (int64_t)j * n];
        s += v * v;
    }
    const double inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    for (int j = 0; j < c; ++j) E[(int64_t)j + i * c] = (float)((double)Y[i + (int64_t)j * n] * inv);
}

inline unsigned blocks_for(int64_t work, int per) { return (unsigned)((work + per - 1) / per); }

}  // namespace

cudaError_t launch_spec_affinity(const float* Y, int64_t ldy, int64_t d, int64_t n, double scale, float* G,
                                 float* sqn, double* part, int parts, double* gsum, double* sig, double* deg,
                                 float* rinv, cudaStream_t st) {
    count_launches(7);
    k_spec_norms<<<parts, kThreads, 0, st>>>(Y, ldy, d, n, sqn, part);
    const dim3 grid(blocks_for(n, kGT), blocks_for(n, kGT));
    k_gemm_tn<<<grid, kGThreads, 0, st>>>(Y, ldy, Y, ldy, G, n, n, n, d, 1.f);
    k_spec_gsum<<<(unsigned)n, kThreads, 0, st>>>(G, n, gsum);
    k_spec_sigma<<<1, kThreads, 0, st>>>(part, parts, gsum, n, scale, sig);
    k_spec_affinity<<<(unsigned)n, kThreads, 0, st>>>(G, n, sqn, sig, deg);
    k_spec_rinv<<<blocks_for(n, kThreads), kThreads, 0, st>>>(deg, n, rinv);
    k_spec_normalise<<<(unsigned)n, kThreads, 0, st>>>(G, n, rinv);
    return cudaGetLastError();
}

cudaError_t launch_spec_start(float* Y, int64_t n, int b, uint64_t seed, cudaStream_t st) {
    count_launches(1);
    k_spec_start<<<blocks_for(n * b, kThreads), kThreads, 0, st>>>(Y, n, b, seed);
    return cudaGetLastError();
}

cudaError_t launch_spec_axpby(float* out, const float* T, const float* Y, const float* Yp, int64_t count,
                              float alpha, float beta, float gamma, cudaStream_t st) {
    count_launches(1);
    k_spec_axpby<<<blocks_for(count, kThreads), kThreads, 0, st>>>(out, T, Y, Yp, count, alpha, beta, gamma);
    return cudaGetLastError();
}

cudaError_t launch_spec_symm(const float* M, int64_t n, const float* Y, int b, float* W, cudaStream_t st) {
    count_launches(1);
    const unsigned grid = blocks_for(n, kSymRows);
    if (b <= 16) k_spec_symm<16><<<grid, kSymRows * 32, 0, st>>>(M, n, Y, b, W);
    else if (b <= 32) k_spec_symm<32><<<grid, kSymRows * 32, 0, st>>>(M, n, Y, b, W);
    else if (b <= 48) k_spec_symm<48><<<grid, kSymRows * 32, 0, st>>>(M, n, Y, b, W);
    else k_spec_symm<72><<<grid, kSymRows * 32, 0, st>>>(M, n, Y, b, W);
    return cudaGetLastError();
}

cudaError_t launch_spec_gram_small(const float* A, const float* B, int64_t n, int b1, int b2, double* out,
                                   cudaStream_t st) {
    count_launches(1);
    k_spec_gram_small<<<dim3(b1, b2), kThreads, 0, st>>>(A, B, n, b1, out);
    return cudaGetLastError();
}

// Y <- Y R^{-1} twice (Cholesky QR2): Y becomes orthonormal with the span of
// its leading columns kept.  T is n x b scratch.
cudaError_t launch_spec_cholqr2(float* Y, float* T, int64_t n, int b, double* G, float* Q, cudaStream_t st) {
    for (int pass = 0; pass < 2; ++pass) {
        cudaError_t e = launch_spec_gram_small(Y, Y, n, b, b, G, st);
        if (e != cudaSuccess) return e;
        count_launches(1);
        e = allow_max_dynamic_smem((const void*)k_spec_chol_inv);
        if (e != cudaSuccess) return e;
        k_spec_chol_inv<<<1, kCholThreads, sizeof(double) * 2 * b * b, st>>>(G, b, Q);
        e = launch_spec_rotate(Y, Q, T, n, b, st);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(Y, T, sizeof(float) * (size_t)n * b, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

size_t spec_jacobi_smem(int b) {
    const int bp = b + (b & 1);
    return sizeof(double) * (2 * (size_t)bp * bp + bp) + sizeof(int) * bp;
}

cudaError_t launch_spec_jacobi(const double* H, int b, float* Q, double* evals, cudaStream_t st) {
    count_launches(1);
    const size_t smem = spec_jacobi_smem(b);
    cudaError_t e = allow_max_dynamic_smem((const void*)k_spec_jacobi);
    if (e != cudaSuccess) return e;
    k_spec_jacobi<<<1, kJacThreads, smem, st>>>(H, b, Q, evals, 60);
    return cudaGetLastError();
}

cudaError_t launch_spec_rotate(const float* Y, const float* Q, float* out, int64_t n, int b, cudaStream_t st) {
    count_launches(1);
    k_spec_rotate<<<blocks_for(n, kThreads), kThreads, sizeof(float) * b * b, st>>>(Y, Q, out, n, b);
    return cudaGetLastError();
}

cudaError_t launch_spec_residual(const float* W, const float* Y, const double* evals, int64_t n, int c,
                                 double* res, cudaStream_t st) {
    count_launches(1);
    k_spec_residual<<<c, kThreads, 0, st>>>(W, Y, evals, n, res);
    return cudaGetLastError();
}

cudaError_t launch_spec_embed(const float* Y, int64_t n, int c, float* E, cudaStream_t st) {
    count_launches(1);
    k_spec_embed<<<blocks_for(n, kThreads), kThreads, 0, st>>>(Y, n, c, E);
    return cudaGetLastError();
}

}  // namespace respca
