// Kernels of the spectral p step (Sec. 4.2: spectral clustering in place of
// K-means on the columns of L).  Normalised spectral clustering:
//   A_ij = exp(-||y_i - y_j||^2 / (2 sigma^2)) (i != j), A_ii = 0,
//   sigma^2 = scale * mean_{i != j} ||y_i - y_j||^2,
//   M = D^{-1/2} A D^{-1/2} (applied as a product, never formed),
//   U = top-c eigenvectors of M,  e_i = U_i / ||U_i||,
// then K-means on the e_i.  The eigenvectors come from Chebyshev-filtered
// subspace iteration with Rayleigh-Ritz (the spectrum of M lies in [-1, 1]).
#include <algorithm>

#include "respca_internal.cuh"

namespace respca {

namespace {

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

// Partial column sums of Y over column chunks (FP64): cs[ch d + r] = sum of
// Y[r + j ldy] over the chunk's columns j.  ||sum_j y_j||^2 = sum_ij y_i . y_j
// gives sigma^2 without a pass over the n x n Gram matrix.  Block (rb, ch):
// rows 32 rb .. 32 rb + 31 (lanes, coalesced), the chunk's columns split over
// the 8 warps, the warps' sums added in warp order.
constexpr int kSpecSumChunks = 64;
__global__ void __launch_bounds__(kThreads)
    k_spec_colsum(const float* __restrict__ Y, int64_t ldy, int64_t d, int64_t n, int64_t per,
                  double* __restrict__ cs) {
    __shared__ double part[kThreads / 32][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * 32 + lane;
    const int64_t j0 = (int64_t)blockIdx.y * per, j1 = j0 + per < n ? j0 + per : n;
    double acc = 0.0;
    if (r < d)
        for (int64_t j = j0 + warp; j < j1; j += kThreads / 32) acc += (double)Y[r + j * ldy];
    part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && r < d) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += part[w][lane];
        cs[(int64_t)blockIdx.y * d + r] = t;
    }
}

// sigma^2 = scale * (2 n sum||y||^2 - 2 ||sum y||^2) / (n (n - 1)), the mean
// over i != j of ||y_i - y_j||^2 scaled, with sum y from the chunk sums;
// out[0] = sigma^2, out[1] = 1 / (2 sigma^2)  (one block).
__global__ void k_spec_sigma(const double* __restrict__ sqn_part, int parts, const double* __restrict__ cs,
                             int64_t d, int64_t n, double scale, double* __restrict__ out) {
    __shared__ double red[2][kThreads / 32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < parts; i += kThreads) a += sqn_part[i];
    for (int64_t r = threadIdx.x; r < d; r += kThreads) {
        double v = 0.0;
        for (int ch = 0; ch < kSpecSumChunks; ++ch) v += cs[(int64_t)ch * d + r];
        b += v * v;
    }
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
    // each thread's entries summed in compensated FP32 (Kahan), then FP64 across threads:
    // one FP64 add per element would bound this pass by the FP64 pipe
    float acc = 0.f, comp = 0.f;
    for (int64_t j = threadIdx.x; j < n; j += kThreads) {
        const float d2 = fmaxf(si + sqn[j] - 2.f * row[j], 0.f);
        const float a = (j == i || inv2s2 == 0.f) ? 0.f : expf(-d2 * inv2s2);
        row[j] = a;
        const float y = a - comp;
        const float t = acc + y;
        comp = (t - acc) - y;
        acc = t;
    }
    double accd = (double)acc - (double)comp;
    accd = warp_sum(accd);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = accd;
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

// W = M Y for M = R A R (A the n x n affinity, column-major; R = diag(r),
// r_k = deg_k^{-1/2}) and the n x b block Y (column-major): the CTA stages
// its rows of R Y in shared memory and the reduction scales row i by r_i, so
// M itself is never formed.  Each warp takes 32 * CPL consecutive rows i (CPL per lane) and the CTA a
// chunk of k: for every k the lanes read one contiguous piece of column k of
// M, M[i + k n], and multiply it by Y[k][0..b), which all lanes read at the
// same shared-memory address (a broadcast).  M is read once, coalesced; the
// chunk's partial products go to P[chunk][q][i] and k_spec_symm_reduce adds
// them in chunk order (deterministic).  BMAX >= b accumulators per row.
constexpr int kSymWarps = 8;
constexpr int kSymSmemFloats = 12288;   // the CTA's rows of Y (48 KB)
constexpr int kSymBatch = 8;            // columns of A whose loads are issued together
// CPL rows per lane: lane-strided (rows i0 + 32 u) when VEC = false, or
// consecutive (one 16-byte load of rows 4 lane .. 4 lane + 3) when VEC = true
// (n % 4 == 0), which doubles the bytes each load instruction moves.
template <int BMAX, int CPL, bool VEC>
__global__ void __launch_bounds__(kSymWarps * 32, 2)
    k_spec_symm(const float* __restrict__ M, const float* __restrict__ r, int64_t n, const float* __restrict__ Y,
                int b, int64_t kc, float* __restrict__ P) {
    __shared__ __align__(16) float ys[kSymSmemFloats];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t k0 = (int64_t)blockIdx.y * kc;
    const int64_t kn = (k0 + kc < n ? k0 + kc : n) - k0;
    for (int64_t e = threadIdx.x; e < kc * BMAX; e += kSymWarps * 32) {
        const int64_t kk = e % kc;
        const int q = (int)(e / kc);
        ys[kk * BMAX + q] = (q < b && kk < kn) ? Y[k0 + kk + (int64_t)q * n] * r[k0 + kk] : 0.f;
    }
    __syncthreads();
    const int64_t wbase = ((int64_t)blockIdx.x * kSymWarps + warp) * 32 * CPL;
    // row of this lane's slot u
    auto row_of = [&](int u) -> int64_t { return VEC ? wbase + 4 * lane + u : wbase + lane + 32 * u; };
    // accumulators in pairs: one packed two-lane FMA (__ffma2_rn, rounding as two
    // fmaf) per pair halves the FMA instructions, which bound the issue rate here
    float2 acc[CPL][BMAX / 2];
#pragma unroll
    for (int u = 0; u < CPL; ++u)
#pragma unroll
        for (int q = 0; q < BMAX / 2; ++q) acc[u][q] = make_float2(0.f, 0.f);
    const bool all_live = row_of(CPL - 1) < n;
    // acc[u][q] += m[u] * y[q] for one row kk of Y (broadcast from shared memory)
    auto fma_row = [&](const float* m, int64_t kk) {
        const float4* yr = reinterpret_cast<const float4*>(ys + kk * BMAX);
#pragma unroll
        for (int q4 = 0; q4 < BMAX / 4; ++q4) {
            const float4 y = yr[q4];
            const float2 ya = make_float2(y.x, y.y), yb = make_float2(y.z, y.w);
#pragma unroll
            for (int u = 0; u < CPL; ++u) {
                const float2 mm = make_float2(m[u], m[u]);
                acc[u][2 * q4] = __ffma2_rn(mm, ya, acc[u][2 * q4]);
                acc[u][2 * q4 + 1] = __ffma2_rn(mm, yb, acc[u][2 * q4 + 1]);
            }
        }
    };
    int64_t kk = 0;
    if (VEC && all_live) {
        // kSymBatch columns' loads issued together, then their products: the loads of
        // one batch overlap each other (and other warps' products)
        const float* mc0 = M + k0 * n + row_of(0);
        for (; kk + kSymBatch <= kn; kk += kSymBatch) {
            float4 mv[kSymBatch];
#pragma unroll
            for (int t = 0; t < kSymBatch; ++t) mv[t] = __ldcs(reinterpret_cast<const float4*>(mc0 + (kk + t) * n));
#pragma unroll
            for (int t = 0; t < kSymBatch; ++t) {
                const float m4[4] = {mv[t].x, mv[t].y, mv[t].z, mv[t].w};
                fma_row(m4, kk + t);
            }
        }
    }
    for (; kk < kn; ++kk) {
        float m[CPL];
        const float* mc = M + (k0 + kk) * n;
#pragma unroll
        for (int u = 0; u < CPL; ++u) m[u] = row_of(u) < n ? __ldcs(mc + row_of(u)) : 0.f;
        fma_row(m, kk);
    }
    float* pc = P + (int64_t)blockIdx.y * b * n;
#pragma unroll
    for (int u = 0; u < CPL; ++u) {
        const int64_t i = row_of(u);
        if (i >= n) continue;
#pragma unroll
        for (int q = 0; q < BMAX; ++q)
            if (q < b) pc[(int64_t)q * n + i] = (q & 1) ? acc[u][q >> 1].y : acc[u][q >> 1].x;
    }
}

// W[i + q n] = r_i times the sum over chunks (in order) of P[chunk][q][i].
__global__ void __launch_bounds__(kThreads)
    k_spec_symm_reduce(const float* __restrict__ P, const float* __restrict__ r, int64_t n, int64_t nb, int chunks,
                       float* __restrict__ W) {
    const int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (e >= nb) return;
    float s = 0.f;
    for (int ch = 0; ch < chunks; ++ch) s += __ldcg(P + (int64_t)ch * nb + e);
    W[e] = s * r[e % n];
}

// out[i + j b1] = sum_k A[k + i n] B[k + j n] (one CTA per entry): the b1 x b2
// Gram or Rayleigh-quotient matrices of n-row blocks.  Each product is exact
// as an FP32 pair (hi = a b, lo = fma(a, b, -hi)); a thread adds its share in
// double-float FP32 (TwoSum on the hi parts, error about 2^-44 of the sum of
// |products|), and the threads' sums are added in FP64 in a fixed order.  One
// FP64 operation per element would be bound by this GPU's narrow FP64 pipe.
__global__ void __launch_bounds__(kThreads)
    k_spec_gram_small(const float* __restrict__ A, const float* __restrict__ B, int64_t n, int b1,
                      double* __restrict__ out) {
    __shared__ double red[kThreads / 32];
    const int i = blockIdx.x, j = blockIdx.y;
    const float* a = A + (int64_t)i * n;
    const float* bb = B + (int64_t)j * n;
    float sh = 0.f, sl = 0.f;
    for (int64_t k = threadIdx.x; k < n; k += kThreads) {
        const float x = a[k], y = bb[k];
        const float ph = x * y, pl = fmaf(x, y, -ph);
        const float t = sh + ph, bv = t - sh;
        float e = (sh - (t - bv)) + (ph - bv);
        e += sl + pl;
        sh = t + e;
        sl = e - (sh - t);
    }
    double acc = (double)sh + (double)sl;
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
// Each square root and reciprocal is taken once, by one thread: on this GPU
// the FP64 pipe is narrow, and the same operation in every thread would cost
// the whole block's worth of it.
constexpr int kCholThreads = 256;
__global__ void __launch_bounds__(kCholThreads)
    k_spec_chol_inv(const double* __restrict__ G, int b, float* __restrict__ Q) {
    extern __shared__ double cm[];
    double* R = cm;             // b x b, column-major, upper triangle used
    double* V = cm + b * b;     // R^{-1}
    double* rd = V + b * b;     // 1 / R[i][i]
    __shared__ double shift, pinv;
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
        if (threadIdx.x == 0) {
            const double piv = sqrt(fmax(R[k + k * b] + shift, 1e-300));
            R[k + k * b] = piv;
            pinv = 1.0 / piv;
            rd[k] = pinv;
        }
        __syncthreads();
        for (int j = k + 1 + threadIdx.x; j < b; j += kCholThreads) R[k + j * b] *= pinv;
        __syncthreads();
        // trailing update: R[i][j] -= R[k][i] R[k][j], k < i <= j (thread per (i, j) of the trailing block)
        const int m = b - k - 1;
        for (int e = threadIdx.x; e < m * m; e += kCholThreads) {
            const int ii = k + 1 + e % m, jj = k + 1 + e / m;
            if (jj >= ii) R[ii + jj * b] -= R[k + ii * b] * R[k + jj * b];
        }
        __syncthreads();
    }
    // V = R^{-1}, column by column: V[j][j] = 1/R[j][j], V[i][j] = -(sum_{k=i+1..j} R[i][k] V[k][j]) / R[i][i]
    for (int j = threadIdx.x; j < b; j += kCholThreads) {
        V[j + j * b] = rd[j];
        for (int i = j - 1; i >= 0; --i) {
            double sacc = 0.0;
            for (int k = i + 1; k <= j; ++k) sacc += R[i + k * b] * V[k + j * b];
            V[i + j * b] = -sacc * rd[i];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < b * b; e += kCholThreads) Q[e] = (float)V[e];
}

// Symmetric eigen-decomposition of H (b x b, FP64 in, symmetrised) by cyclic
// Jacobi with the round-robin pair order (bp/2 disjoint rotations per step,
// bp = b rounded up to even; the schedule of every step is tabulated once).
// The rotations run in FP32: on this GPU an FP64 operation costs tens of FP32
// ones, and the eigenvectors leave as FP32 anyway.  A pair is rotated only
// when |a_pq| > max(1e-6 sqrt(|a_pp a_qq|), 2e-7 ||A||_F); the loop ends after a sweep with no
// rotation, or when the off-diagonal part is below 1e-6 of the matrix
// (Frobenius).  The eigenvalues are the FP64 Rayleigh quotients
// v^T H v / v^T v of the FP32 eigenvector columns, whose error is second order
// in the vectors'.  Writes them in descending order (ties by index) and
// the matching vectors as the columns of Q (b x b, FP32, column-major).
// One CTA of NT threads.  A step is one phase after the angles: the pairs
// partition the indices, so every entry of A lies in exactly one 2 x 2 block
// (pair k1's rows, pair k2's columns), which a thread turns by both rotations
// (rows first, then columns, the same operations as two separate passes).
constexpr float kJacRel = 1e-6f, kJacAbs = 2e-7f;
template <int NT>
__global__ void __launch_bounds__(NT)
    k_spec_jacobi(const double* __restrict__ H, int b, float* __restrict__ Q, double* __restrict__ evals,
                  int max_sweeps) {
    extern __shared__ double sm[];
    const int bp = b + (b & 1);          // padded to even (a zero row and column)
    const int half = bp / 2;
    double* hs = sm;                     // b x b, the symmetrised H
    double* rq = hs + b * b;             // bp Rayleigh quotients
    float* a = reinterpret_cast<float*>(rq + bp);   // bp x bp
    float* v = a + bp * bp;              // bp x bp
    float* cs = v + bp * bp;             // half cosines
    float* sn = cs + half;               // half sines
    int2* sched = reinterpret_cast<int2*>(sn + half);   // (bp - 1) x half pairs (p < q); 8-byte aligned:
                                                       // 2 bp^2 + 2 half floats precede it
    __shared__ float red[NT / 32][2];
    __shared__ int stop, turned;
    __shared__ float anorm;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int e = tid; e < bp * bp; e += NT) {
        const int i = e % bp, j = e / bp;
        double x = 0.0;
        if (i < b && j < b) {
            x = 0.5 * (H[i + j * b] + H[j + i * b]);
            hs[i + j * b] = x;
        }
        a[e] = (float)x;
        v[e] = (i == j) ? 1.f : 0.f;
    }
    // step t: slot 0 holds index 0, slot s >= 1 holds 1 + (s - 1 - t) mod (bp - 1);
    // pair k joins slots k and bp - 1 - k
    for (int e = tid; e < (bp - 1) * half; e += NT) {
        const int t = e / half, k = e % half;
        auto at = [&](int slot) { return slot == 0 ? 0 : 1 + ((slot - 1 - t) % (bp - 1) + (bp - 1)) % (bp - 1); };
        int p = at(k), q = at(bp - 1 - k);
        if (p > q) { const int x = p; p = q; q = x; }
        sched[e] = make_int2(p, q);
    }
    __syncthreads();
    // each thread's 2 x 2 block and V entry, when one per thread covers them all
    // (the divisions then leave the step loop)
    const bool one_blk = half * half <= NT, one_v = bp * half <= NT;
    const int bk2 = tid / half, bk1 = tid - bk2 * half;
    const int vk = tid / bp, vi = tid - vk * bp;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        float o = 0.f, t2 = 0.f;
        for (int e = tid; e < bp * bp; e += NT) {
            const float x = a[e];
            t2 = fmaf(x, x, t2);
            if (e % bp != e / bp) o = fmaf(x, x, o);
        }
        o = warp_sum(o);
        t2 = warp_sum(t2);
        if (lane == 0) {
            red[warp][0] = o;
            red[warp][1] = t2;
        }
        __syncthreads();
        if (tid == 0) {
            float oo = 0.f, tt = 0.f;
            for (int w = 0; w < NT / 32; ++w) {
                oo += red[w][0];
                tt += red[w][1];
            }
            stop = (oo <= 1e-12f * tt || tt == 0.f) ? 1 : 0;
            turned = 0;
            anorm = sqrtf(tt);
        }
        __syncthreads();
        if (stop) break;
        for (int step = 0; step < bp - 1; ++step) {
            const int2* pairs = sched + step * half;
            for (int k = tid; k < half; k += NT) {
                const int p = pairs[k].x, q = pairs[k].y;
                const float apq = a[p + q * bp];
                const float app = a[p + p * bp], aqq = a[q + q * bp];
                float c = 1.f, s = 0.f;
                // rotate only where a_pq stands above FP32 rounding noise: relative to its
                // diagonal pair (the classical threshold for Jacobi in finite precision) and
                // to the whole matrix (rotations leave noise of that size in every entry)
                if (fabsf(apq) > fmaxf(kJacRel * sqrtf(fabsf(app) * fabsf(aqq)), kJacAbs * anorm)) {
                    // t = sign(tau) / (|tau| + sqrt(1 + tau^2)), the smaller root; for
                    // huge |tau| the rotation is below FP32 resolution and t = 1 / (2 tau).
                    // Approximate divisions: any (c, s) with c^2 + s^2 = 1 is a rotation,
                    // and one that leaves an ulp of a_pq behind is as good as exact here
                    const float tau = __fdividef(aqq - app, 2.f * apq);
                    const float at = fabsf(tau);
                    const float tr = at > 1e18f ? __fdividef(0.5f, at) : __fdividef(1.f, at + sqrtf(fmaf(at, at, 1.f)));
                    const float tt = tau >= 0.f ? tr : -tr;
                    c = rsqrtf(fmaf(tt, tt, 1.f));
                    s = tt * c;
                    turned = 1;
                }
                cs[k] = c;
                sn[k] = s;
            }
            __syncthreads();
            // A <- J^T A J by 2 x 2 blocks: rows of pair k1, columns of pair k2
            for (int e = tid; e < half * half; e += NT) {
                const int k2 = one_blk ? bk2 : e / half, k1 = one_blk ? bk1 : e - k2 * half;
                const int p1 = pairs[k1].x, q1 = pairs[k1].y, p2 = pairs[k2].x, q2 = pairs[k2].y;
                const float c1 = cs[k1], s1 = sn[k1], c2 = cs[k2], s2 = sn[k2];
                const float xpp = a[p1 + p2 * bp], xpq = a[p1 + q2 * bp];
                const float xqp = a[q1 + p2 * bp], xqq = a[q1 + q2 * bp];
                const float rpp = c1 * xpp - s1 * xqp, rqp = s1 * xpp + c1 * xqp;   // rows (J^T A)
                const float rpq = c1 * xpq - s1 * xqq, rqq = s1 * xpq + c1 * xqq;
                a[p1 + p2 * bp] = c2 * rpp - s2 * rpq;                                 // columns (. J)
                a[p1 + q2 * bp] = s2 * rpp + c2 * rpq;
                a[q1 + p2 * bp] = c2 * rqp - s2 * rqq;
                a[q1 + q2 * bp] = s2 * rqp + c2 * rqq;
            }
            // V <- V J (pair k's two columns, row i)
            for (int e = tid; e < bp * half; e += NT) {
                const int k = one_v ? vk : e / bp, i = one_v ? vi : e - k * bp;
                const int p = pairs[k].x, q = pairs[k].y;
                const float c = cs[k], s = sn[k];
                const float vp = v[i + p * bp], vq = v[i + q * bp];
                v[i + p * bp] = c * vp - s * vq;
                v[i + q * bp] = s * vp + c * vq;
            }
            __syncthreads();
        }
        // a sweep without a rotation changes nothing more
        if (!turned) break;
    }
    // Rayleigh quotients v^T H v / v^T v in FP64: one warp per column j, lanes over rows i
    for (int j = warp; j < bp; j += NT / 32) {
        double acc = 0.0, nrm = 0.0;
        if (j < b) {
            for (int i = lane; i < b; i += 32) {
                double hv = 0.0;
                for (int k = 0; k < b; ++k) hv = fma(hs[i + k * b], (double)v[k + j * bp], hv);
                const double vi = (double)v[i + j * bp];
                acc = fma(vi, hv, acc);
                nrm = fma(vi, vi, nrm);
            }
        }
        acc = warp_sum(acc);
        nrm = warp_sum(nrm);
        if (lane == 0) rq[j] = nrm > 0.0 ? acc / nrm : 0.0;
    }
    __syncthreads();
    // descending order of the first b eigenvalues (selection by rank; ties by index)
    for (int j = tid; j < b; j += NT) {
        const double x = rq[j];
        int rank = 0;
        for (int k = 0; k < b; ++k) {
            const double y = rq[k];
            rank += (y > x) || (y == x && k < j);
        }
        evals[rank] = x;
        for (int i = 0; i < b; ++i) Q[i + rank * b] = v[i + j * bp];
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
                                 float* sqn, double* part, int parts, double* colsum, double* sig, double* deg,
                                 float* rinv, DevStatus* status, cudaEvent_t g0, cudaEvent_t g1, cudaStream_t st) {
    count_launches(5);
    k_spec_norms<<<parts, kThreads, 0, st>>>(Y, ldy, d, n, sqn, part);
    const int64_t per = (n + kSpecSumChunks - 1) / kSpecSumChunks;
    k_spec_colsum<<<dim3(blocks_for(d, 32), kSpecSumChunks), kThreads, 0, st>>>(Y, ldy, d, n, per, colsum);
    k_spec_sigma<<<1, kThreads, 0, st>>>(part, parts, colsum, d, n, scale, sig);
    if (g0 && cudaEventRecord(g0, st) != cudaSuccess) return cudaGetLastError();
    const cudaError_t e = launch_gram_tc(Y, ldy, d, n, G, status, st);
    if (e != cudaSuccess) return e;
    if (g1 && cudaEventRecord(g1, st) != cudaSuccess) return cudaGetLastError();
    k_spec_affinity<<<(unsigned)n, kThreads, 0, st>>>(G, n, sqn, sig, deg);
    k_spec_rinv<<<blocks_for(n, kThreads), kThreads, 0, st>>>(deg, n, rinv);
    return cudaGetLastError();
}

size_t spec_colsum_doubles(int64_t d) { return (size_t)kSpecSumChunks * d; }

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

namespace {
int spec_bmax(int b) { return b <= 16 ? 16 : b <= 32 ? 32 : b <= 48 ? 48 : 72; }
int64_t spec_kc(int64_t n, int b) {
    const int bm = spec_bmax(b);
    const int cpl = (bm == 16 && n % 4 == 0) ? 4 : bm <= 16 ? 2 : 1;
    const int64_t iblocks = (n + kSymWarps * 32 * cpl - 1) / (kSymWarps * 32 * cpl);
    // about two (16-byte loads) or four CTAs per SM over the grid, each chunk a
    // multiple of 8 rows of Y: fewer chunks keep the partial products small
    const int64_t ctas = (cpl == 4 ? 2 : 4) * 152;
    const int64_t want = std::max<int64_t>(1, (ctas + iblocks - 1) / iblocks);
    int64_t kc = (n + want - 1) / want;
    kc = (kc + 7) / 8 * 8;
    return std::min<int64_t>(kc, kSymSmemFloats / bm / 8 * 8);
}
}  // namespace

int64_t spec_symm_chunks(int64_t n, int b) {
    const int64_t kc = spec_kc(n, b);
    return (n + kc - 1) / kc;
}

cudaError_t launch_spec_symm(const float* M, const float* r, int64_t n, const float* Y, int b, float* W, float* P,
                             cudaStream_t st) {
    count_launches(2);
    const int bm = spec_bmax(b);
    const bool vec = bm == 16 && n % 4 == 0;
    const int cpl = vec ? 4 : bm <= 16 ? 2 : 1;
    const int64_t kc = spec_kc(n, b), chunks = (n + kc - 1) / kc;
    const dim3 grid((unsigned)((n + kSymWarps * 32 * cpl - 1) / (kSymWarps * 32 * cpl)), (unsigned)chunks);
    const unsigned thr = kSymWarps * 32;
    if (vec) k_spec_symm<16, 4, true><<<grid, thr, 0, st>>>(M, r, n, Y, b, kc, P);
    else if (bm == 16) k_spec_symm<16, 2, false><<<grid, thr, 0, st>>>(M, r, n, Y, b, kc, P);
    else if (bm == 32) k_spec_symm<32, 1, false><<<grid, thr, 0, st>>>(M, r, n, Y, b, kc, P);
    else if (bm == 48) k_spec_symm<48, 1, false><<<grid, thr, 0, st>>>(M, r, n, Y, b, kc, P);
    else k_spec_symm<72, 1, false><<<grid, thr, 0, st>>>(M, r, n, Y, b, kc, P);
    const int64_t nb = n * (int64_t)b;
    k_spec_symm_reduce<<<blocks_for(nb, kThreads), kThreads, 0, st>>>(P, r, n, nb, (int)chunks, W);
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
        k_spec_chol_inv<<<1, kCholThreads, sizeof(double) * (2 * b * b + b), st>>>(G, b, Q);
        e = launch_spec_rotate(Y, Q, T, n, b, st);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(Y, T, sizeof(float) * (size_t)n * b, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

size_t spec_jacobi_smem(int b) {
    const int bp = b + (b & 1), half = bp / 2;
    return sizeof(double) * ((size_t)b * b + bp) + sizeof(float) * (2 * (size_t)bp * bp + 2 * half) +
           sizeof(int2) * (size_t)(bp - 1) * half;
}

cudaError_t launch_spec_jacobi(const double* H, int b, float* Q, double* evals, cudaStream_t st) {
    count_launches(1);
    const size_t smem = spec_jacobi_smem(b);
    const int bp = b + (b & 1);
    // threads: at least max(half^2, bp half) (one block entry or V entry each) where it fits
    if (bp <= 16) {
        cudaError_t e = allow_max_dynamic_smem((const void*)k_spec_jacobi<128>);
        if (e != cudaSuccess) return e;
        k_spec_jacobi<128><<<1, 128, smem, st>>>(H, b, Q, evals, 60);
    } else if (bp <= 32) {
        cudaError_t e = allow_max_dynamic_smem((const void*)k_spec_jacobi<512>);
        if (e != cudaSuccess) return e;
        k_spec_jacobi<512><<<1, 512, smem, st>>>(H, b, Q, evals, 60);
    } else {
        cudaError_t e = allow_max_dynamic_smem((const void*)k_spec_jacobi<1024>);
        if (e != cudaSuccess) return e;
        k_spec_jacobi<1024><<<1, 1024, smem, st>>>(H, b, Q, evals, 60);
    }
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
