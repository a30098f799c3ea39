// Streaming kernels around the RES-PCA iteration (HBM-bound work): ||X||_F,
// cluster sums and centroids, centroid statistics and separations, the
// pruning bounds of the K-means search, label bookkeeping and the closed-form
// ramp.  The fused iteration kernel itself is in k_iteration.cu.
#include <algorithm>
#include <cfloat>

#include "respca_internal.cuh"

namespace respca {

namespace {

// ---------------------------------------------------------------- ||X||_F
template <typename TX, bool VEC>
__global__ void __launch_bounds__(kThreads) k_fro2(const TX* __restrict__ X, int64_t d, int64_t n,
                                                   int64_t ldx, double* __restrict__ part,
                                                   DevStatus* __restrict__ status) {
    __shared__ double red[kThreads / 32];
    __shared__ float redm[kThreads / 32];
    const int64_t rows_per_unit = kThreads * 4;
    const int64_t seg = (d + rows_per_unit - 1) / rows_per_unit;
    const int64_t units = seg * n;
    // compensated FP32 per thread (an FP64 add per unit would bound this pass by the
    // FP64 pipe), FP64 across threads; and max |x|
    float acc = 0.f, comp = 0.f, mx = 0.f;
    bool bad = false;
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const int64_t j = units < 0x7fffffff ? (int64_t)((uint32_t)u / (uint32_t)seg) : u / seg;
        const int64_t r = (u - j * seg) * rows_per_unit + threadIdx.x * 4;
        const TX* col = X + j * ldx;
        float s = 0.f;
        if (VEC) {
            if (r < d) {
                const float4 v = XLoad<TX>::four(col + r);
                bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w));
                s = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, v.w * v.w)));
                mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (r + q < d) {
                    const float v = XLoad<TX>::one(col + r + q);
                    bad |= !isfinite(v);
                    s = fmaf(v, v, s);
                    mx = fmaxf(mx, fabsf(v));
                }
        }
        const float y = s - comp;
        const float t = acc + y;
        comp = (t - acc) - y;
        acc = t;
    }
    double accd = warp_sum((double)acc - (double)comp);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = accd;
        redm[threadIdx.x >> 5] = mx;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&status->nonfinite, 1);
    if (threadIdx.x == 0) {
        double t = 0.0;
        float m = 0.f;
        for (int w = 0; w < kThreads / 32; ++w) {
            t += red[w];
            m = fmaxf(m, redm[w]);
        }
        part[blockIdx.x] = t;
        atomicMax(&status->xmax_bits, __float_as_uint(m));   // non-negative floats order as their bits
    }
}

__global__ void k_sum_parts(const double* __restrict__ part, int nparts, double* __restrict__ out) {
    __shared__ double red[kThreads / 32];
    double t = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) t += part[i];
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
        *out = s;
    }
}

// ---------------------------------------------------------------- cluster sums
// Sum, per tile and row, the columns of X (kSumX), L (kSumL) or
// D = X - S + Theta * inv_rho (kSumD; S and Theta stored as TS).
template <int MODE, typename TX, typename TS, bool VEC>
__global__ void __launch_bounds__(kThreads)
    k_colsum(const TX* __restrict__ X, int64_t ldx, const float* __restrict__ L,
             const TS* __restrict__ S, const TS* __restrict__ Th, int64_t lds,
             float inv_rho, const int32_t* __restrict__ perm, const TileDesc* __restrict__ tiles,
             const DevStatus* __restrict__ status, int64_t d, float* __restrict__ Dpart) {
    __shared__ float red[kThreads / 32][kChunkRows];
    const int tile_idx = blockIdx.x;
    if (tile_idx >= status->ntiles) return;
    const TileDesc td = tiles[tile_idx];
    const int64_t r0 = (int64_t)blockIdx.y * kChunkRows;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    float4 acc[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[s] = make_float4(0.f, 0.f, 0.f, 0.f);

    for (int k = warp; k < td.len; k += kThreads / 32) {
        const int64_t col = perm[td.start + k];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int64_t rr = r0 + s * 128 + lane * 4;
            if (VEC) {
                if (rr < d) {
                    float4 v;
                    if (MODE == kSumX) {
                        v = XLoad<TX>::four(X + col * ldx + rr);
                    } else if (MODE == kSumL) {
                        v = *reinterpret_cast<const float4*>(L + col * lds + rr);
                    } else {
                        const float4 x = XLoad<TX>::four(X + col * ldx + rr);
                        const float4 sv = XLoad<TS>::four(S + col * lds + rr);
                        const float4 tv = XLoad<TS>::four(Th + col * lds + rr);
                        v = make_float4((x.x - sv.x) + tv.x * inv_rho, (x.y - sv.y) + tv.y * inv_rho,
                                        (x.z - sv.z) + tv.z * inv_rho, (x.w - sv.w) + tv.w * inv_rho);
                    }
                    acc[s].x += v.x;
                    acc[s].y += v.y;
                    acc[s].z += v.z;
                    acc[s].w += v.w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int64_t r = rr + q;
                    if (r < d) {
                        float v;
                        if (MODE == kSumX) v = XLoad<TX>::one(X + col * ldx + r);
                        else if (MODE == kSumL) v = L[col * lds + r];
                        else v = (XLoad<TX>::one(X + col * ldx + r) - XLoad<TS>::one(S + col * lds + r)) +
                                 XLoad<TS>::one(Th + col * lds + r) * inv_rho;
                        f4set(acc[s], q, f4get(acc[s], q) + v);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int q = 0; q < 4; ++q) red[warp][s * 128 + lane * 4 + q] = f4get(acc[s], q);
    __syncthreads();
    for (int i = threadIdx.x; i < kChunkRows; i += kThreads) {
        const int64_t r = r0 + i;
        if (r < d) {
            float v = 0.f;
#pragma unroll
            for (int w = 0; w < kThreads / 32; ++w) v += red[w][i];
            Dpart[(int64_t)tile_idx * d + r] = v;
        }
    }
}

// mu[i][r] = (sum over the tiles of cluster i of Dpart[t][r]) / n_i, summed in
// FP64 in tile order.  Empty clusters keep their old centroid (they take part
// in no assignment).
__global__ void __launch_bounds__(kThreads)
    k_centroids(const float* __restrict__ Dpart, const int32_t* __restrict__ tile_off,
                const int32_t* __restrict__ counts, int64_t d, float* __restrict__ mu,
                double* __restrict__ sums_out) {
    // 1 / n_i once per block: an FP64 division per thread would load this GPU's
    // narrow FP64 pipe with tens of operations per element
    __shared__ double inv_sh;
    const int i = blockIdx.y;
    const int cnt = counts[i];
    if (threadIdx.x == 0) inv_sh = cnt > 0 ? 1.0 / (double)cnt : 0.0;
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (r >= d) return;
    const int t0 = tile_off[i], t1 = tile_off[i + 1];
    // compensated FP32 sum of the tile partials (FP64 arithmetic is slow on this part),
    // four tiles' loads issued together, added in tile order
    float s = 0.f, comp = 0.f;
    auto add = [&](float x) {
        const float y = x - comp;
        const float u = s + y;
        comp = (u - s) - y;
        s = u;
    };
    int t = t0;
    for (; t + 4 <= t1; t += 4) {
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = Dpart[(int64_t)(t + q) * d + r];
#pragma unroll
        for (int q = 0; q < 4; ++q) add(v[q]);
    }
    for (; t < t1; ++t) add(Dpart[(int64_t)t * d + r]);
    const double sd = (double)s - (double)comp;
    if (sums_out) sums_out[(int64_t)i * d + r] = sd;
    if (cnt > 0) mu[(int64_t)i * d + r] = (float)(sd * inv_sh);
}

// Centroids from FP64 cluster sums (kept up to date incrementally).
__global__ void __launch_bounds__(kThreads)
    k_centroids_from_sums(const double* __restrict__ sums, const int32_t* __restrict__ counts,
                          int64_t d, float* __restrict__ mu, float* __restrict__ mu_old) {
    __shared__ double inv_sh;   // 1 / n_i once per block (see k_centroids)
    const int i = blockIdx.y;
    const int cnt = counts[i];
    if (threadIdx.x == 0) inv_sh = cnt > 0 ? 1.0 / (double)cnt : 0.0;
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (r >= d) return;
    const int64_t e = (int64_t)i * d + r;
    if (mu_old) mu_old[e] = mu[e];   // the previous centroids, for the drift
    if (cnt == 0) return;
    mu[e] = (float)(sums[e] * inv_sh);
}

// sums_i = n_i mu_i (FP64) for every row: the cluster sums that the centroids
// mu were formed from, recovered without reading the columns.
__global__ void __launch_bounds__(kThreads)
    k_sums_from_means(const float* __restrict__ mu, const int32_t* __restrict__ counts, int64_t d,
                      double* __restrict__ sums) {
    const int i = blockIdx.y;
    const int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (r >= d) return;
    sums[(int64_t)i * d + r] = (double)mu[(int64_t)i * d + r] * (double)counts[i];
}

// Cluster sums after a Lloyd pass moved some columns: sums_i += (columns that
// joined i) - (columns that left i), of X, L or D = X - S + Theta inv_rho.  k_moved lists each cluster's signed
// contributions contiguously (bucket i = contrib[boff[i] .. boff[i+1])).  A
// CTA takes 128 rows of one cluster and adds its bucket in double-float
// FP32 (TwoSum: the running sum is hi + lo to about 2^-44), then makes one
// FP64 update per row; FP64 adds per moved column would be bound by the slow
// FP64 pipe.
constexpr int kDeltaThreads = 128;
template <int MODE, typename TX>
__global__ void __launch_bounds__(kDeltaThreads)
    k_delta_sums(const TX* __restrict__ X, int64_t ldx, const float* __restrict__ L, int64_t lds,
                 const float* __restrict__ S, const float* __restrict__ Th, float inv_rho,
                 const int2* __restrict__ contrib, const int32_t* __restrict__ boff, int c, int64_t d,
                 double* __restrict__ sums) {
    const int64_t r = (int64_t)blockIdx.x * kDeltaThreads + threadIdx.x;
    if (r >= d) return;
    for (int i = blockIdx.y; i < c; i += gridDim.y) {
        const int b0 = boff[i], b1 = boff[i + 1];
        if (b0 == b1) continue;
        float hi = 0.f, lo = 0.f;
        // the value of bucket entry q at row r, signed
        auto value = [&](int2 e) -> float {   // (column, sign)
            const int64_t j = e.x;
            float x;
            if (MODE == kSumX) x = XLoad<TX>::one(X + j * ldx + r);
            else if (MODE == kSumL) x = L[j * lds + r];
            else x = (XLoad<TX>::one(X + j * ldx + r) - S[j * lds + r]) + Th[j * lds + r] * inv_rho;
            return e.y < 0 ? -x : x;
        };
        auto add = [&](float x) {   // TwoSum(hi, x)
            const float t = hi + x;
            const float bp = t - hi;
            lo += (hi - (t - bp)) + (x - bp);
            hi = t;
        };
        // eight entries' loads in flight at once, added in bucket order (a load per
        // entry in turn would cost a memory round trip each)
        int q = b0;
        for (; q + 8 <= b1; q += 8) {
            int2 e[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) e[u] = contrib[q + u];
            float x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = value(e[u]);
#pragma unroll
            for (int u = 0; u < 8; ++u) add(x[u]);
        }
        for (; q < b1; ++q) add(value(contrib[q]));
        sums[(int64_t)i * d + r] += (double)hi + (double)lo;
    }
}

constexpr int kCsThreads = 256;   // threads of the split centroid-statistics kernels

// ||mu_i||^2 and, when mu_old is given, the drift ||mu_i - mu_old_i||: centroid
// i's rows split over gridDim.y CTAs (one CTA per centroid would leave most SMs
// idle at small c); compensated FP32 sums per thread, an FP32 tree across the
// CTA (relative error ~1e-6, well inside the slack of the pruning bounds; the
// FP64 pipe of this part is too slow for a d-long FP64 reduction per centroid),
// and the CTA that finishes centroid i last adds the parts in split order.
__global__ void __launch_bounds__(kCsThreads)
    k_mu_stats(const float* __restrict__ mu, const float* __restrict__ mu_old, int64_t d, int64_t per,
               double* __restrict__ mu_norm2, float* __restrict__ mu_normf, double* __restrict__ drift,
               float2* __restrict__ part, int32_t* __restrict__ done) {
    __shared__ float red[kCsThreads / 32][2];
    __shared__ int last_sh;
    const int i = blockIdx.x;
    const int S = gridDim.y;
    const float* m = mu + (int64_t)i * d;
    const float* mo = mu_old ? mu_old + (int64_t)i * d : nullptr;
    const int64_t r0 = (int64_t)blockIdx.y * per, r1 = r0 + per < d ? r0 + per : d;
    float acc = 0.f, ca = 0.f, dr = 0.f, cd = 0.f;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += kCsThreads) {
        const float v = m[r];
        {
            const float y = v * v - ca;
            const float t = acc + y;
            ca = (t - acc) - y;
            acc = t;
        }
        if (mo) {
            const float e = v - mo[r];
            const float y = e * e - cd;
            const float t = dr + y;
            cd = (t - dr) - y;
            dr = t;
        }
    }
    acc = warp_sum(acc);
    dr = warp_sum(dr);
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5][0] = acc;
        red[threadIdx.x >> 5][1] = dr;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f, bsum = 0.f;
        for (int w = 0; w < kCsThreads / 32; ++w) {
            a += red[w][0];
            bsum += red[w][1];
        }
        part[(int64_t)i * S + blockIdx.y] = make_float2(a, bsum);
        __threadfence();
        last_sh = atomicAdd(&done[i], 1) == S - 1;
    }
    __syncthreads();
    if (!last_sh || threadIdx.x != 0) return;
    __threadfence();
    float a = 0.f, bsum = 0.f;
    for (int q = 0; q < S; ++q) {
        const float2 v = __ldcg(part + (int64_t)i * S + q);
        a += v.x;
        bsum += v.y;
    }
    mu_norm2[i] = (double)a;
    mu_normf[i] = a;
    if (drift) drift[i] = sqrt((double)bsum) * (1.0 + 1e-5);
    done[i] = 0;
}

// k_centroids_from_sums, the previous-centroid copy, k_mu_stats and the TF32
// split in one launch.  Centroid i's rows are split over gridDim.y CTAs of
// kCsThreads (one CTA per centroid would leave most SMs idle at small c, each
// doing two FP64 operations per element); each CTA reduces its rows' ||mu||^2
// and drift terms (compensated FP32 per thread, FP32 tree across the CTA) to
// part[i][s], and the CTA that finishes centroid i last (a counter, reset by
// it) adds the parts in split order.
__global__ void __launch_bounds__(kCsThreads)
    k_centroids_stats(const double* __restrict__ sums, const int32_t* __restrict__ counts, int64_t d,
                      int64_t per, float* __restrict__ mu, float* __restrict__ mu_old,
                      double* __restrict__ mu_norm2, float* __restrict__ mu_normf, double* __restrict__ drift,
                      MuSplitOut sp, float4* __restrict__ part, int32_t* __restrict__ done) {
    __shared__ float red[kCsThreads / 32][3];
    __shared__ int last_sh;
    __shared__ double inv_sh;   // 1 / n_i once per block (see k_centroids)
    const int i = blockIdx.x;
    const int S = gridDim.y;
    const int cnt = counts[i];
    if (threadIdx.x == 0) inv_sh = cnt != 0 ? 1.0 / (double)cnt : 0.0;
    __syncthreads();
    const double inv = inv_sh;
    float* m = mu + (int64_t)i * d;
    float* mo = mu_old + (int64_t)i * d;
    const int64_t r0 = (int64_t)blockIdx.y * per, r1 = r0 + per < d ? r0 + per : d;
    const float s16 = (sp.a16 && sp.a16_kind == 2) ? sp.status->sh_scale : 1.f;
    float acc = 0.f, ca = 0.f, dr = 0.f, cd = 0.f, e16 = 0.f;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += kCsThreads) {
        const float old = m[r];
        mo[r] = old;
        float v = old;
        if (cnt != 0) {
            v = (float)(sums[(int64_t)i * d + r] * inv);
            m[r] = v;
        }
        {
            const float y = v * v - ca;
            const float t = acc + y;
            ca = (t - acc) - y;
            acc = t;
        }
        {
            const float e = v - old;
            const float y = e * e - cd;
            const float t = dr + y;
            cd = (t - dr) - y;
            dr = t;
        }
        if (sp.hi) {
            const int64_t idx = (int64_t)i * sp.dpad + r;
            const float hi = tf32_hi(v);
            if (i < sp.Npad) {
                sp.hi[idx] = hi;
                sp.lo[idx] = v - hi;
            }
            if (sp.a) {
                sp.a[idx] = v;
                sp.a[(int64_t)sp.arows * sp.dpad + idx] = v - hi;
            }
            if (sp.a16) {   // the 16-bit split of k_mu_split
                const int64_t o = (int64_t)i * sp.dpad16 + r;
                uint16_t p1, p2;
                split16(v, sp.a16_kind, s16, p1, p2, e16);
                sp.a16[o] = p1;
                sp.a16[(int64_t)sp.arows * sp.dpad16 + o] = p2;
            }
        }
    }
    acc = warp_sum(acc);
    dr = warp_sum(dr);
    e16 = warp_sum(e16);
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5][0] = acc;
        red[threadIdx.x >> 5][1] = dr;
        red[threadIdx.x >> 5][2] = e16;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f, bsum = 0.f, esum = 0.f;
        for (int w = 0; w < kCsThreads / 32; ++w) {
            a += red[w][0];
            bsum += red[w][1];
            esum += red[w][2];
        }
        part[(int64_t)i * S + blockIdx.y] = make_float4(a, bsum, esum, 0.f);
        __threadfence();
        last_sh = atomicAdd(&done[i], 1) == S - 1;
    }
    __syncthreads();
    if (!last_sh || threadIdx.x != 0) return;
    __threadfence();
    float a = 0.f, bsum = 0.f, esum = 0.f;
    for (int q = 0; q < S; ++q) {
        const float4 v = __ldcg(part + (int64_t)i * S + q);
        a += v.x;
        bsum += v.y;
        esum += v.z;
    }
    mu_norm2[i] = (double)a;
    mu_normf[i] = a;
    drift[i] = sqrt((double)bsum) * (1.0 + 1e-5);
    if (sp.a16) sp.a16_err[i] = split16_err(esum, d, s16);
    done[i] = 0;
}

__global__ void __launch_bounds__(kThreads)
    k_mu_norms(const float* __restrict__ mu, int64_t d, double* __restrict__ mu_norm2,
               float* __restrict__ mu_normf) {
    __shared__ double red[kThreads / 32];
    const int i = blockIdx.x;
    const float* m = mu + (int64_t)i * d;
    double acc = 0.0;
    for (int64_t r = threadIdx.x; r < d; r += kThreads) acc += (double)m[r] * (double)m[r];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        mu_norm2[i] = t;
        mu_normf[i] = (float)t;
    }
}

// Pairwise squared centroid distances, one CTA per 64-row slab, staged in
// shared memory; partial sums are added into pair_ss (c x c, upper triangle).
constexpr int kSepRows = 64;
constexpr int kSepMaxC = 256;

__global__ void __launch_bounds__(kThreads)
    k_pair_dist(const float* __restrict__ mu, const int32_t* __restrict__ counts, int c, int64_t d,
                float* __restrict__ pair_ss) {
    // [c][kSepRows + 1]: the padded stride puts the rows that a warp's threads
    // read at once (different centroids j, same k) in different banks
    extern __shared__ __align__(16) float ms[];
    const int64_t r0 = (int64_t)blockIdx.x * kSepRows;
    for (int idx = threadIdx.x; idx < c * kSepRows; idx += kThreads) {
        const int i = idx / kSepRows, rr = idx % kSepRows;
        ms[i * (kSepRows + 1) + rr] = (r0 + rr < d) ? mu[(int64_t)i * d + r0 + rr] : 0.f;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < c * c; p += kThreads) {
        const int i = p / c, j = p % c;
        if (j <= i || counts[i] == 0 || counts[j] == 0) continue;
        const float* a = ms + i * (kSepRows + 1);
        const float* b = ms + j * (kSepRows + 1);
        float s = 0.f;
#pragma unroll 16
        for (int k = 0; k < kSepRows; ++k) {
            const float t = a[k] - b[k];
            s = fmaf(t, t, s);
        }
        atomicAdd(&pair_ss[p], s);
    }
}

// One warp per centroid, lanes over the other centroids.
__global__ void k_sep_min(const float* __restrict__ pair_ss, const int32_t* __restrict__ counts,
                          int c, double* __restrict__ sep2) {
    const int i = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= c) return;
    float best = INFINITY;
    if (counts[i] > 0)
        for (int j = lane; j < c; j += 32) {
            if (j == i || counts[j] == 0) continue;
            const int a = min(i, j), b = max(i, j);
            best = fminf(best, pair_ss[(int64_t)a * c + b]);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fminf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane == 0) sep2[i] = (double)best;
}

__global__ void k_fill_double(double* __restrict__ p, int count, double v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) p[i] = v;
}

// ---------------------------------------------------------------- finalisers
// The three Sec. 5 norms from the fused pass's per-(chunk, tile) partials,
// over kNormCtas CTAs (FP64 sums on one SM would be bound by its FP64 pipe):
// CTA g adds units u = g kThreads + tid + k kNormCtas kThreads in that order,
// its warps' and threads' sums in a fixed order, and the CTA that finishes
// last adds the CTAs' parts in CTA order (a counter in the status block,
// reset by that CTA).
constexpr int kNormCtas = 64;
__global__ void __launch_bounds__(kThreads)
    k_reduce_norms(const double* __restrict__ norm_part, int max_tiles, int nchunks,
                   DevStatus* __restrict__ status, double* __restrict__ part) {
    __shared__ double red[kThreads / 32][3];
    __shared__ int last_sh;
    const int ntiles = status->ntiles;
    const int64_t units = (int64_t)ntiles * nchunks;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    const int64_t stride = (int64_t)kNormCtas * kThreads;
    for (int64_t u = (int64_t)blockIdx.x * kThreads + threadIdx.x; u < units; u += stride) {
        const int64_t y = u / ntiles, t = u - y * ntiles;
        const double* p = norm_part + (y * max_tiles + t) * 3;
        a0 += p[0];
        a1 += p[1];
        a2 += p[2];
    }
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    a2 = warp_sum(a2);
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5][0] = a0;
        red[threadIdx.x >> 5][1] = a1;
        red[threadIdx.x >> 5][2] = a2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            t0 += red[w][0];
            t1 += red[w][1];
            t2 += red[w][2];
        }
        part[blockIdx.x * 3 + 0] = t0;
        part[blockIdx.x * 3 + 1] = t1;
        part[blockIdx.x * 3 + 2] = t2;
        __threadfence();
        last_sh = atomicAdd(&status->norms_done, 1) == kNormCtas - 1;
    }
    __syncthreads();
    if (!last_sh || threadIdx.x >= 3) return;
    __threadfence();
    double t = 0.0;
    for (int g = 0; g < kNormCtas; ++g) t += __ldcg(part + g * 3 + threadIdx.x);
    status->norm2[threadIdx.x] = t;
    __syncwarp(0x7u);
    if (threadIdx.x == 0) status->norms_done = 0;
}

// Hamerly-style exact pruning of the nearest-centroid search.  Per column j
// with label p: ub[j] >= ||L_j - mu_p|| and lb[j] <= min_{i != p} ||L_j - mu_i||.
// The own label is provably the strict nearest when ub < lb.
//   kBoundsIter (after the fused pass): ub = exact own distance to the new
//     centroids; lb degrades by the column's own movement and by the largest
//     drift of another centroid, and is raised to sep_p - ub when the
//     centroid separation gives more.
//   kBoundsLloyd (centroids moved, points fixed): ub grows by the own
//     centroid's drift, lb shrinks by the largest drift of another centroid.
// Columns that fail are queued; the search then resets both bounds exactly.
constexpr float kRelSlack = 1e-5f;

__global__ void __launch_bounds__(kThreads)
    k_flag_bounds(int mode, const float* __restrict__ own_part, const float* __restrict__ dl_part,
                  int nchunks, int64_t n, int c, const int32_t* __restrict__ labels,
                  const int32_t* __restrict__ counts, const double* __restrict__ sep2,
                  double safety, const double* __restrict__ drift, float* __restrict__ ub,
                  float* __restrict__ lb, int32_t* __restrict__ flag_list,
                  DevStatus* __restrict__ status, int32_t* __restrict__ labels_copy,
                  const float* __restrict__ ylo_part, float* __restrict__ ycol, float ycol_floor) {
    // ycol: [0, n) ||L_j - y~_j|| (bounded), [n, 2n) ||y~_j||^2 of the FP16 copy
    // largest and second largest drift over active clusters (per block)
    __shared__ double s_d1[kThreads], s_d2[kThreads];
    __shared__ int s_i1[kThreads];
    double d1 = 0.0, d2 = 0.0;
    int i1 = -1;
    if (drift) {
        for (int i = threadIdx.x; i < c; i += kThreads) {
            if (counts[i] == 0) continue;
            const double v = drift[i];
            if (v > d1) {
                d2 = d1;
                d1 = v;
                i1 = i;
            } else if (v > d2) {
                d2 = v;
            }
        }
    }
    s_d1[threadIdx.x] = d1;
    s_d2[threadIdx.x] = d2;
    s_i1[threadIdx.x] = i1;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const double a1 = s_d1[threadIdx.x], a2 = s_d2[threadIdx.x];
            const double b1 = s_d1[threadIdx.x + o], b2 = s_d2[threadIdx.x + o];
            if (b1 > a1) {
                s_d1[threadIdx.x] = b1;
                s_i1[threadIdx.x] = s_i1[threadIdx.x + o];
                s_d2[threadIdx.x] = fmax(a1, b2);
            } else {
                s_d2[threadIdx.x] = fmax(a2, b1);
            }
        }
        __syncthreads();
    }
    d1 = s_d1[0];
    d2 = s_d2[0];
    i1 = s_i1[0];

    const int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    bool flag = false;
    if (j < n) {
        const int p = labels[j];
        if (labels_copy) labels_copy[j] = p;   // the labels before this pass's search
        const double other = (p == i1) ? d2 : d1;
        double u, l;
        if (mode == kBoundsIter) {
            // the row chunks' partials in four compensated FP32 chains (an FP64 add per
            // chunk would bound this pass by the FP64 pipe at large d), joined in FP64;
            // their error, about 2^-23 relative, is far inside the 1e-5 slack below
            float so[4] = {0.f, 0.f, 0.f, 0.f}, co[4] = {0.f, 0.f, 0.f, 0.f};
            float sm[4] = {0.f, 0.f, 0.f, 0.f}, cm[4] = {0.f, 0.f, 0.f, 0.f};
            auto kahan = [](float& sum, float& comp, float x) {
                const float y = x - comp;
                const float t = sum + y;
                comp = (t - sum) - y;
                sum = t;
            };
            int ch = 0;
            for (; ch + 4 <= nchunks; ch += 4) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    kahan(so[q], co[q], own_part[(int64_t)(ch + q) * n + j]);
                    kahan(sm[q], cm[q], dl_part[(int64_t)(ch + q) * n + j]);
                }
            }
            for (; ch < nchunks; ++ch) {
                kahan(so[0], co[0], own_part[(int64_t)ch * n + j]);
                kahan(sm[0], cm[0], dl_part[(int64_t)ch * n + j]);
            }
            double own = 0.0, mv = 0.0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                own += (double)so[q] - (double)co[q];
                mv += (double)sm[q] - (double)cm[q];
            }
            const double eo = sqrt(own);
            u = eo * (1.0 + kRelSlack) + 1e-30;
            l = (double)lb[j] - sqrt(mv) * (1.0 + kRelSlack) - other * (1.0 + kRelSlack);
            const double sp = sep2[p];
            if (sp > 0.0) l = fmax(l, sqrt(sp * safety) - u);
            if (ycol) {
                // ||L_j - bf16(L_j)|| from the fused pass's chunk partials (the search of
                // this iteration's L runs on its 16-bit copy), same summation; the floor
                // covers squares that underflowed
                const float* yq_part = ylo_part + (int64_t)nchunks * n;
                float sy[4] = {0.f, 0.f, 0.f, 0.f}, cy[4] = {0.f, 0.f, 0.f, 0.f};
                float sq[4] = {0.f, 0.f, 0.f, 0.f}, cq[4] = {0.f, 0.f, 0.f, 0.f};
                int k = 0;
                for (; k + 4 <= nchunks; k += 4) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        kahan(sy[q], cy[q], ylo_part[(int64_t)(k + q) * n + j]);
                        kahan(sq[q], cq[q], yq_part[(int64_t)(k + q) * n + j]);
                    }
                }
                for (; k < nchunks; ++k) {
                    kahan(sy[0], cy[0], ylo_part[(int64_t)k * n + j]);
                    kahan(sq[0], cq[0], yq_part[(int64_t)k * n + j]);
                }
                double yl = 0.0, yq = 0.0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    yl += (double)sy[q] - (double)cy[q];
                    yq += (double)sq[q] - (double)cq[q];
                }
                ycol[j] = (float)(sqrt(yl) * (1.0 + kRelSlack)) + ycol_floor;
                ycol[n + j] = (float)yq;
            }
        } else {
            const double own_drift = drift ? drift[p] : 0.0;
            u = (double)ub[j] + own_drift * (1.0 + kRelSlack);
            l = (double)lb[j] - other * (1.0 + kRelSlack);
        }
        ub[j] = (float)(u * (1.0 + 1e-7));
        lb[j] = (float)(l > 0.0 ? l * (1.0 - 1e-7) : l);
        flag = !(u < l);
    }
    const unsigned mask = __ballot_sync(0xffffffffu, flag);
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0 && mask) base = atomicAdd(&status->flagged, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (flag) flag_list[base + __popc(mask & ((1u << lane) - 1u))] = (int32_t)j;
}

// FP16 copy fp16(s x) of FP32 columns for the all-column search over X (column
// stride ld16), with each column's ||x - y~|| (bounded: compensated FP32 sums,
// inflated, plus the underflow floor) in ycol[j] and ||y~||^2 in ycol[n + j],
// y~ = copy / s; the scale goes to the status for the centroid split and the
// finalize.  One warp per column, 16-byte rows (d % 4 == 0, aligned columns).
__global__ void __launch_bounds__(kThreads)
    k_copy16_cols(const float* __restrict__ X, int64_t ldx, int64_t d, int64_t n, float s,
                  __half* __restrict__ Y16, int64_t ld16, float* __restrict__ ycol, float floor,
                  DevStatus* __restrict__ status) {
    const float inv_s = 1.f / s;   // a power of two: exact
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        status->sh_scale = s;
        status->sh_inv2 = inv_s * inv_s;
    }
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    if (j >= n) return;
    const float* x = X + j * ldx;
    __half* y = Y16 + j * ld16;
    float se = 0.f, ce = 0.f, sq = 0.f, cq = 0.f;
    auto kahan = [](float& sum, float& comp, float v) {
        const float t = v - comp;
        const float u = sum + t;
        comp = (u - sum) - t;
        sum = u;
    };
    for (int64_t r = (int64_t)lane * 4; r < d; r += 128) {
        const float4 v = *reinterpret_cast<const float4*>(x + r);
        float e2 = 0.f, q2 = 0.f;
        __half2 h0, h1;
        h0.x = copy16(v.x, s, inv_s, e2, q2);
        h0.y = copy16(v.y, s, inv_s, e2, q2);
        h1.x = copy16(v.z, s, inv_s, e2, q2);
        h1.y = copy16(v.w, s, inv_s, e2, q2);
        uint2 u;
        u.x = *reinterpret_cast<const uint32_t*>(&h0);
        u.y = *reinterpret_cast<const uint32_t*>(&h1);
        *reinterpret_cast<uint2*>(y + r) = u;
        kahan(se, ce, e2);
        kahan(sq, cq, q2);
    }
    const double e = warp_sum((double)se - (double)ce), q = warp_sum((double)sq - (double)cq);
    if (lane == 0) {
        ycol[j] = (float)(sqrt(e) * (1.0 + 1e-5)) + floor;
        ycol[n + j] = (float)q;
    }
}

// The end of a device-run Lloyd pass's search: adds the pass counters, sets the
// loop's condition and clears the counters for the next pass (one thread).
__device__ void lloyd_pass_end(DevStatus* __restrict__ status, cudaGraphConditionalHandle cond,
                               int max_passes) {
    status->acc_flagged += status->flagged;
    status->acc_rechecked += status->rechecked;
    status->acc_changed += status->changed;
    const int passes = ++status->acc_passes;
    const bool more = status->changed != 0 && passes < max_passes && status->timeout == 0;
    cudaGraphSetConditional(cond, more ? 1u : 0u);
    // hand the pass's result to the host and clear the counters for the next pass
    status->last_changed = status->changed;
    status->flagged = 0;
    status->changed = 0;
    status->rechecked = 0;
    status->rc_pairs = 0;
}

// Columns whose label differs between `now` and `before`, in column order
// (single CTA; deterministic), as (column, old, new) triples; the cluster
// sizes follow the move.  Each thread takes kMovedK consecutive columns per
// round, so a round covers 8192 columns with one block-wide scan.  The moves
// are then bucketed by cluster as signed contributions (-1: left, +1:
// joined) in a fixed order, for k_delta_sums.
constexpr int kMovedThreads = 1024, kMovedK = 8;
__global__ void __launch_bounds__(kMovedThreads)
    k_moved(const int32_t* __restrict__ now, const int32_t* __restrict__ before, int64_t n, int c,
            int4* __restrict__ moved, int2* __restrict__ contrib, int32_t* __restrict__ boff,
            int32_t* __restrict__ counts, DevStatus* __restrict__ status, PassEnd pe) {
    __shared__ int wsum[32];
    __shared__ int base_sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // in a device-run Lloyd pass this kernel follows the search: it also ends it (the
    // fields it touches are read by none of the work below)
    if (pe.on && threadIdx.x == 0) lloyd_pass_end(status, pe.cond, pe.max_passes);
    if (threadIdx.x == 0) base_sh = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < n; b0 += (int64_t)kMovedThreads * kMovedK) {
        const int64_t j0 = b0 + (int64_t)threadIdx.x * kMovedK;
        int a[kMovedK], o[kMovedK];
        int cnt = 0;
#pragma unroll
        for (int e = 0; e < kMovedK; ++e) {
            const int64_t j = j0 + e;
            a[e] = j < n ? now[j] : 0;
            o[e] = j < n ? before[j] : 0;
            cnt += (a[e] != o[e]) ? 1 : 0;
        }
        int incl = cnt;   // inclusive scan over the warp
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int v = wsum[lane], inc = v;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, inc, off);
                if (lane >= off) inc += t;
            }
            wsum[lane] = inc - v;   // exclusive prefix of the warp totals
        }
        __syncthreads();
        const int base = base_sh;
        int pos = base + wsum[warp] + incl - cnt;
#pragma unroll
        for (int e = 0; e < kMovedK; ++e) {
            if (a[e] == o[e]) continue;
            moved[pos++] = make_int4((int)(j0 + e), o[e], a[e], 0);
            if (o[e] >= 0) atomicSub(&counts[o[e]], 1);
            atomicAdd(&counts[a[e]], 1);
        }
        __syncthreads();
        if (threadIdx.x == kMovedThreads - 1) base_sh = pos;   // the last thread ends the round
        __syncthreads();
    }
    __syncthreads();
    const int nm = base_sh;
    if (threadIdx.x == 0) status->moved = nm;

    // bucket the signed contributions by cluster: sizes, offsets, then a stable
    // placement by one warp (chunk by chunk, lanes ranked by __match_any_sync)
    __shared__ int off_sh[kMaxClusters + 1];
    for (int i = threadIdx.x; i <= c; i += kMovedThreads) off_sh[i] = 0;
    __syncthreads();
    for (int m = threadIdx.x; m < nm; m += kMovedThreads) {
        const int4 mv = moved[m];
        if (mv.y >= 0) atomicAdd(&off_sh[mv.y], 1);
        atomicAdd(&off_sh[mv.z], 1);
    }
    __syncthreads();
    if (warp == 0) {
        int carry = 0;
        for (int b = 0; b < c; b += 32) {
            const int v = (b + lane < c) ? off_sh[b + lane] : 0;
            int inc = v;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, inc, off);
                if (lane >= off) inc += t;
            }
            if (b + lane < c) off_sh[b + lane] = carry + inc - v;
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (lane == 0) off_sh[c] = carry;
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= c; i += kMovedThreads) boff[i] = off_sh[i];
    __syncthreads();
    if (warp == 0) {
        const unsigned below = (1u << lane) - 1u;
        for (int cb = 0; cb < nm; cb += 32) {
            const int m = cb + lane;
            const int4 mv = m < nm ? moved[m] : make_int4(0, -1, -1, 0);
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int key = side == 0 ? mv.y : mv.z;   // the cluster left, then the one joined
                const bool has = key >= 0;
                const unsigned act = __ballot_sync(0xffffffffu, has);
                unsigned peers = 0u;
                if (has) {
                    peers = __match_any_sync(act, key);
                    contrib[off_sh[key] + __popc(peers & below)] = make_int2(mv.x, side == 0 ? -1 : 1);
                }
                __syncwarp();
                if (has && (peers & below) == 0u) off_sh[key] += __popc(peers);
                __syncwarp();
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads)
    k_count_changed(const int32_t* __restrict__ labels, const int32_t* __restrict__ prev, int64_t n,
                    DevStatus* __restrict__ status) {
    const int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const bool ch = j < n && labels[j] != prev[j];
    const unsigned mask = __ballot_sync(0xffffffffu, ch);
    if ((threadIdx.x & 31) == 0 && mask) atomicAdd(&status->label_changes, __popc(mask));
}

// Ramp statistics of X against its cluster means (one warp per column):
// max |X - mu_p| over all elements and max_j ||X_j - mu_p(j)|| / sep(p(j)),
// with sep^2 = sep2 * safety; both non-negative, combined with integer max on
// their bit patterns (order-independent).  Also the FP64 sum of ||r_j||^2.
template <typename TX, bool VEC>
__global__ void __launch_bounds__(kThreads)
    k_ramp_stats(const TX* __restrict__ X, int64_t ldx, int64_t d, int64_t n,
                 const int32_t* __restrict__ labels, const float* __restrict__ mu,
                 const double* __restrict__ sep2, double safety,
                 unsigned int* __restrict__ max_abs_bits, unsigned long long* __restrict__ max_ratio_bits,
                 double* __restrict__ r2_part) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    double r2acc = 0.0;
    if (w < n) {
        const int p = labels[w];
        const TX* xc = X + w * ldx;
        const float* m = mu + (int64_t)p * d;
        float mx = 0.f, s2f = 0.f, c2 = 0.f;
        // compensated FP32 per lane (an FP64 multiply-add per element would bound this
        // pass by the FP64 pipe; the sums feed tests with 1e-3 margins), FP64 across lanes
        auto add = [&](float e) {
            mx = fmaxf(mx, fabsf(e));
            const float y = fmaf(e, e, -c2);
            const float t = s2f + y;
            c2 = (t - s2f) - y;
            s2f = t;
        };
        if (VEC) {   // four rows per lane and step (d % 4 == 0, 16-byte aligned rows)
            for (int64_t r = 4 * lane; r < d; r += 128) {
                const float4 x = XLoad<TX>::four(xc + r);
                const float4 mm = __ldg(reinterpret_cast<const float4*>(m + r));
                add(x.x - mm.x);
                add(x.y - mm.y);
                add(x.z - mm.z);
                add(x.w - mm.w);
            }
        } else {
            for (int64_t r = lane; r < d; r += 32) add(XLoad<TX>::one(xc + r) - m[r]);
        }
        double s2 = warp_sum((double)s2f - (double)c2);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) {
            atomicMax(max_abs_bits, __float_as_uint(mx));
            const double sp = sep2[p] * safety;
            const double ratio = sp > 0.0 ? sqrt(s2 / sp) : (s2 > 0.0 ? INFINITY : 0.0);
            atomicMax(max_ratio_bits, (unsigned long long)__double_as_longlong(ratio));
            r2acc = s2;
        }
    }
    if (lane == 0 && w < n) r2_part[w] = r2acc;
}

// State after the skipped ramp: L = mu_p + alpha (X - mu_p), Theta = beta (X - mu_p).
template <typename TX, typename TS, bool VEC>
__global__ void __launch_bounds__(kThreads)
    k_ramp_state(const TX* __restrict__ X, int64_t ldx, int64_t d, int64_t n,
                 const int32_t* __restrict__ labels, const float* __restrict__ mu, float alpha,
                 float beta, TS* __restrict__ L, TS* __restrict__ Th, int64_t lds) {
    // columns in turn per CTA, rows across its threads (four per thread and step when
    // rows are 16-byte aligned): no division per element
    for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
        const float* m = mu + (int64_t)labels[j] * d;
        const TX* xc = X + j * ldx;
        TS* lc = L + j * lds;
        TS* tc = Th + j * lds;
        if (VEC) {
            for (int64_t r = 4 * (int64_t)threadIdx.x; r < d; r += 4 * kThreads) {
                const float4 x = XLoad<TX>::four(xc + r);
                const float4 mm = __ldg(reinterpret_cast<const float4*>(m + r));
                const float4 e = make_float4(x.x - mm.x, x.y - mm.y, x.z - mm.z, x.w - mm.w);
                StateIO<TS>::store4(lc + r, make_float4(fmaf(alpha, e.x, mm.x), fmaf(alpha, e.y, mm.y),
                                                        fmaf(alpha, e.z, mm.z), fmaf(alpha, e.w, mm.w)));
                StateIO<TS>::store4(tc + r, make_float4(beta * e.x, beta * e.y, beta * e.z, beta * e.w));
            }
        } else {
            for (int64_t r = threadIdx.x; r < d; r += kThreads) {
                const float mr = m[r];
                const float e = XLoad<TX>::one(xc + r) - mr;
                StateIO<TS>::store1(lc + r, fmaf(alpha, e, mr));
                StateIO<TS>::store1(tc + r, beta * e);
            }
        }
    }
}

// Element-type conversion of a d x n column-major matrix (one CTA per column
// at a time): the BF16 copy of an FP32 X, and the BF16 state widened to FP32
// when the bf16 phase ends.
template <typename TI, typename TO>
__global__ void __launch_bounds__(kThreads)
    k_convert(const TI* __restrict__ src, int64_t lds, TO* __restrict__ dst, int64_t ldd, int64_t d,
              int64_t n) {
    for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
        const TI* s = src + j * lds;
        TO* o = dst + j * ldd;
        for (int64_t r = threadIdx.x; r < d; r += kThreads) StateIO<TO>::store1(o + r, XLoad<TI>::one(s + r));
    }
}

// Sec. 6 anomaly score ||S_j||_2, one warp per column: compensated FP32 sums
// per lane (d / 32 squares each), then a tree over the warp.
__global__ void __launch_bounds__(kThreads)
    k_column_norms(const float* __restrict__ S, int64_t lds, int64_t d, int64_t n,
                   float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (kThreads / 32);
    for (int64_t j = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5); j < n; j += warps) {
        const float* col = S + j * lds;
        float acc = 0.f, comp = 0.f;
        for (int64_t r = lane; r < d; r += 32) {
            const float v = col[r];
            const float y = fmaf(v, v, -comp);
            const float t = acc + y;
            comp = (t - acc) - y;
            acc = t;
        }
        acc = warp_sum(acc);
        if (lane == 0) out[j] = sqrtf(acc);
    }
}

__global__ void k_lloyd_init(DevStatus* __restrict__ status, int passes0) {
    status->acc_flagged = 0;
    status->acc_passes = passes0;
    status->acc_rechecked = 0;
    status->acc_changed = 0;
    status->flagged = 0;   // the per-pass counters start at zero (each pass's end re-zeroes them)
    status->changed = 0;
    status->rechecked = 0;
    status->rc_pairs = 0;
    status->last_changed = 0;
}


inline int grid_for(int64_t work, int per) { return (int)((work + per - 1) / per); }

}  // namespace

// ---------------------------------------------------------------- launchers
cudaError_t launch_fro2(int dtype, const void* X, int64_t d, int64_t n, int64_t ldx, double* part,
                        int nparts, DevStatus* status, cudaStream_t st) {
    count_launches(2);
    const int64_t seg = (d + kThreads * 4 - 1) / (kThreads * 4);
    const int64_t units = seg * n;
    const int grid = (int)(units < nparts ? units : nparts);
    RESPCA_DISPATCH_X(dtype, TX, {
        const bool vec = (ldx % 4 == 0) && (d % 4 == 0) &&
                         (reinterpret_cast<uintptr_t>(X) % (4 * sizeof(TX)) == 0);
        if (vec)
            k_fro2<TX, true><<<grid, kThreads, 0, st>>>((const TX*)X, d, n, ldx, part, status);
        else
            k_fro2<TX, false><<<grid, kThreads, 0, st>>>((const TX*)X, d, n, ldx, part, status);
    });
    k_sum_parts<<<1, kThreads, 0, st>>>(part, grid, &status->x_norm2);
    return cudaGetLastError();
}

template <int M, typename TX, typename TS>
void colsum_mode(dim3 grid, const TX* x, int64_t ldx, const float* L, const TS* S, const TS* Th,
                 int64_t lds, float inv_rho, const int32_t* perm, const TileDesc* tiles,
                 const DevStatus* status, int64_t d, float* Dpart, bool vec, cudaStream_t st) {
    if (vec)
        k_colsum<M, TX, TS, true><<<grid, kThreads, 0, st>>>(x, ldx, L, S, Th, lds, inv_rho, perm,
                                                             tiles, status, d, Dpart);
    else
        k_colsum<M, TX, TS, false><<<grid, kThreads, 0, st>>>(x, ldx, L, S, Th, lds, inv_rho, perm,
                                                              tiles, status, d, Dpart);
}

cudaError_t launch_colsum(int mode, int dtype, const void* X, int64_t ldx, const float* L,
                          const void* S, const void* Th, int64_t lds, float inv_rho,
                          const int32_t* perm, const TileDesc* tiles, int max_tiles,
                          const DevStatus* status, int64_t d, float* Dpart, bool vec,
                          cudaStream_t st, int sdtype) {
    count_launches(1);
    const dim3 grid(max_tiles, grid_for(d, kChunkRows));
    if (mode == kSumL) {
        colsum_mode<kSumL, float, float>(grid, nullptr, 0, L, nullptr, nullptr, lds, inv_rho, perm,
                                         tiles, status, d, Dpart, vec, st);
        return cudaGetLastError();
    }
    RESPCA_DISPATCH_X(dtype, TX, {
        if (mode == kSumX) {
            colsum_mode<kSumX, TX, float>(grid, (const TX*)X, ldx, L, nullptr, nullptr, lds, inv_rho,
                                          perm, tiles, status, d, Dpart, vec, st);
        } else {
            RESPCA_DISPATCH_S(sdtype, TS, {
                colsum_mode<kSumD, TX, TS>(grid, (const TX*)X, ldx, L, (const TS*)S, (const TS*)Th, lds,
                                           inv_rho, perm, tiles, status, d, Dpart, vec, st);
            });
        }
    });
    return cudaGetLastError();
}

cudaError_t launch_centroids(const float* Dpart, const int32_t* tile_off, const int32_t* counts,
                             int c, int64_t d, float* mu, cudaStream_t st, double* sums_out) {
    count_launches(1);
    const dim3 grid(grid_for(d, kThreads), c);
    k_centroids<<<grid, kThreads, 0, st>>>(Dpart, tile_off, counts, d, mu, sums_out);
    return cudaGetLastError();
}

cudaError_t launch_centroids_from_sums(const double* sums, const int32_t* counts, int c, int64_t d,
                                       float* mu, cudaStream_t st, float* mu_old) {
    count_launches(1);
    const dim3 grid(grid_for(d, kThreads), c);
    k_centroids_from_sums<<<grid, kThreads, 0, st>>>(sums, counts, d, mu, mu_old);
    return cudaGetLastError();
}

cudaError_t launch_delta_sums(int mode, int dtype, const void* X, int64_t ldx, const float* L,
                              int64_t lds, const int2* contrib, const int32_t* boff, int c, int64_t d,
                              double* sums, cudaStream_t st, const float* S, const float* Th,
                              float inv_rho) {
    count_launches(1);
    const dim3 grid((unsigned)grid_for(d, kDeltaThreads), (unsigned)std::min(c, 64));
    if (mode == kSumL) {
        k_delta_sums<kSumL, float><<<grid, kDeltaThreads, 0, st>>>(nullptr, 0, L, lds, nullptr, nullptr,
                                                                   0.f, contrib, boff, c, d, sums);
    } else {
        RESPCA_DISPATCH_X(dtype, TX, {
            if (mode == kSumX)
                k_delta_sums<kSumX, TX><<<grid, kDeltaThreads, 0, st>>>((const TX*)X, ldx, nullptr, 0, nullptr,
                                                                        nullptr, 0.f, contrib, boff, c, d,
                                                                        sums);
            else
                k_delta_sums<kSumD, TX><<<grid, kDeltaThreads, 0, st>>>((const TX*)X, ldx, nullptr, lds, S, Th,
                                                                        inv_rho, contrib, boff, c, d, sums);
        });
    }
    return cudaGetLastError();
}

cudaError_t launch_mu_stats(const float* mu, const float* mu_old, int c, int64_t d,
                            double* mu_norm2, float* mu_normf, double* drift, float2* part, int32_t* done,
                            cudaStream_t st) {
    count_launches(1);
    const int S = centroids_stats_splits(c, d);
    const int64_t per = (d + S - 1) / S;
    k_mu_stats<<<dim3(c, S), kCsThreads, 0, st>>>(mu, mu_old, d, per, mu_norm2, mu_normf, drift, part, done);
    return cudaGetLastError();
}

cudaError_t launch_sums_from_means(const float* mu, const int32_t* counts, int c, int64_t d, double* sums,
                                   cudaStream_t st) {
    count_launches(1);
    const dim3 grid(grid_for(d, kThreads), c);
    k_sums_from_means<<<grid, kThreads, 0, st>>>(mu, counts, d, sums);
    return cudaGetLastError();
}

int centroids_stats_splits(int c, int64_t d) {
    // about four CTAs per SM over the grid, at least 1024 rows per CTA
    const int64_t want = (4 * 152 + c - 1) / c;
    const int64_t most = (d + 1023) / 1024;
    return (int)std::max<int64_t>(1, std::min(want, most));
}

cudaError_t launch_centroids_stats(const double* sums, const int32_t* counts, int c, int64_t d, float* mu,
                                   float* mu_old, double* mu_norm2, float* mu_normf, double* drift,
                                   const MuSplitOut& sp, float4* part, int32_t* done, cudaStream_t st) {
    count_launches(1);
    const int S = centroids_stats_splits(c, d);
    const int64_t per = (d + S - 1) / S;
    k_centroids_stats<<<dim3(c, S), kCsThreads, 0, st>>>(sums, counts, d, per, mu, mu_old, mu_norm2, mu_normf,
                                                          drift, sp, part, done);
    return cudaGetLastError();
}

cudaError_t launch_flag_bounds(int mode, const float* own_part, const float* dl_part, int nchunks,
                               int64_t n, int c, const int32_t* labels, const int32_t* counts,
                               const double* sep2, double safety, const double* drift, float* ub,
                               float* lb, int32_t* flag_list, DevStatus* status, cudaStream_t st,
                               int32_t* labels_copy, const float* ylo_part, float* ycol, int64_t d) {
    count_launches(1);
    // |l - bf16(l)| below 2^-75 squares to zero in FP32: sqrt(d) 2^-74 covers all of them
    const float floor = ycol ? (float)(std::sqrt((double)d) * 5.29395592033938e-23) : 0.f;
    k_flag_bounds<<<grid_for(n, kThreads), kThreads, 0, st>>>(mode, own_part, dl_part, nchunks, n, c,
                                                              labels, counts, sep2, safety, drift,
                                                              ub, lb, flag_list, status, labels_copy,
                                                              ylo_part, ycol, floor);
    return cudaGetLastError();
}

cudaError_t launch_copy16_cols(const float* X, int64_t ldx, int64_t d, int64_t n, float s, void* Y16,
                              int64_t ld16, float* ycol, DevStatus* status, cudaStream_t st) {
    count_launches(1);
    // |x - y~| below 2^-75 squares to zero in FP32: sqrt(d) 2^-74 covers all of them
    const float floor = (float)(std::sqrt((double)d) * 5.29395592033938e-23);
    k_copy16_cols<<<grid_for(n, kThreads / 32), kThreads, 0, st>>>(X, ldx, d, n, s, static_cast<__half*>(Y16),
                                                                  ld16, ycol, floor, status);
    return cudaGetLastError();
}

cudaError_t launch_moved(const int32_t* now, const int32_t* before, int64_t n, int c, int4* moved,
                         int2* contrib, int32_t* boff, int32_t* counts, DevStatus* status,
                         cudaStream_t st, const PassEnd* pe) {
    count_launches(1);
    k_moved<<<1, kMovedThreads, 0, st>>>(now, before, n, c, moved, contrib, boff, counts, status,
                                         pe ? *pe : PassEnd{});
    return cudaGetLastError();
}

cudaError_t launch_mu_norms(const float* mu, int c, int64_t d, double* mu_norm2, float* mu_normf,
                            cudaStream_t st) {
    count_launches(1);
    k_mu_norms<<<c, kThreads, 0, st>>>(mu, d, mu_norm2, mu_normf);
    return cudaGetLastError();
}

cudaError_t launch_separation(const float* mu, const int32_t* counts, int c, int64_t d,
                              float* pair_ss, double* sep2, cudaStream_t st) {
    count_launches(c > kSepMaxC ? 1 : 2);
    if (c > kSepMaxC) {
        // No pruning for very many clusters: every column is searched.
        k_fill_double<<<grid_for(c, kThreads), kThreads, 0, st>>>(sep2, c, 0.0);
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(pair_ss, 0, sizeof(float) * (size_t)c * c, st);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(float) * (size_t)c * (kSepRows + 1);
    if (smem > 48 * 1024) {
        e = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_pair_dist));
        if (e != cudaSuccess) return e;
    }
    k_pair_dist<<<grid_for(d, kSepRows), kThreads, smem, st>>>(mu, counts, c, d, pair_ss);
    k_sep_min<<<grid_for(c, kThreads / 32), kThreads, 0, st>>>(pair_ss, counts, c, sep2);
    return cudaGetLastError();
}

cudaError_t launch_reduce_norms(const double* norm_part, int max_tiles, int nchunks,
                                DevStatus* status, double* part, cudaStream_t st) {
    count_launches(1);
    k_reduce_norms<<<kNormCtas, kThreads, 0, st>>>(norm_part, max_tiles, nchunks, status, part);
    return cudaGetLastError();
}

cudaError_t launch_ramp_stats(int dtype, const void* X, int64_t ldx, int64_t d, int64_t n,
                              const int32_t* labels, const float* mu, const double* sep2,
                              double safety, unsigned int* max_abs_bits,
                              unsigned long long* max_ratio_bits, double* r2_part, cudaStream_t st) {
    count_launches(1);
    const int grid = grid_for(n, kThreads / 32);
    RESPCA_DISPATCH_X(dtype, TX, {
        const bool vec = (ldx % 4 == 0) && (d % 4 == 0) && (reinterpret_cast<uintptr_t>(X) % (4 * sizeof(TX)) == 0) &&
                         (reinterpret_cast<uintptr_t>(mu) % 16 == 0);
        if (vec)
            k_ramp_stats<TX, true><<<grid, kThreads, 0, st>>>((const TX*)X, ldx, d, n, labels, mu, sep2, safety,
                                                              max_abs_bits, max_ratio_bits, r2_part);
        else
            k_ramp_stats<TX, false><<<grid, kThreads, 0, st>>>((const TX*)X, ldx, d, n, labels, mu, sep2, safety,
                                                               max_abs_bits, max_ratio_bits, r2_part);
    });
    return cudaGetLastError();
}

cudaError_t launch_ramp_state(int dtype, const void* X, int64_t ldx, int64_t d, int64_t n,
                              const int32_t* labels, const float* mu, float alpha, float beta,
                              void* L, void* Th, int64_t lds, cudaStream_t st, int sdtype) {
    count_launches(1);
    RESPCA_DISPATCH_X(dtype, TX, {
        RESPCA_DISPATCH_S(sdtype, TS, {
            const bool vec = (ldx % 4 == 0) && (lds % 4 == 0) && (d % 4 == 0) &&
                             (reinterpret_cast<uintptr_t>(X) % (4 * sizeof(TX)) == 0) &&
                             (reinterpret_cast<uintptr_t>(L) % (4 * sizeof(TS)) == 0) &&
                             (reinterpret_cast<uintptr_t>(Th) % (4 * sizeof(TS)) == 0) &&
                             (reinterpret_cast<uintptr_t>(mu) % 16 == 0);
            if (vec)
                k_ramp_state<TX, TS, true><<<152 * 8, kThreads, 0, st>>>((const TX*)X, ldx, d, n, labels, mu,
                                                                        alpha, beta, (TS*)L, (TS*)Th, lds);
            else
                k_ramp_state<TX, TS, false><<<152 * 8, kThreads, 0, st>>>((const TX*)X, ldx, d, n, labels, mu,
                                                                         alpha, beta, (TS*)L, (TS*)Th, lds);
        });
    });
    return cudaGetLastError();
}

cudaError_t launch_convert(int src_dtype, const void* src, int64_t lds, int dst_sdtype, void* dst,
                           int64_t ldd, int64_t d, int64_t n, cudaStream_t st) {
    count_launches(1);
    const int grid = (int)std::min<int64_t>(n, 152 * 16);
    RESPCA_DISPATCH_X(src_dtype, TI, {
        RESPCA_DISPATCH_S(dst_sdtype, TO, {
            k_convert<TI, TO><<<grid, kThreads, 0, st>>>((const TI*)src, lds, (TO*)dst, ldd, d, n);
        });
    });
    return cudaGetLastError();
}

cudaError_t launch_column_norms(const float* S, int64_t lds, int64_t d, int64_t n, float* out,
                                cudaStream_t st) {
    count_launches(1);
    const int grid = (int)std::min<int64_t>(grid_for(n, kThreads / 32), 152 * 32);
    k_column_norms<<<grid, kThreads, 0, st>>>(S, lds, d, n, out);
    return cudaGetLastError();
}

cudaError_t launch_lloyd_init(DevStatus* status, int passes0, cudaStream_t st) {
    count_launches(1);
    k_lloyd_init<<<1, 1, 0, st>>>(status, passes0);
    return cudaGetLastError();
}

cudaError_t launch_sum_doubles(const double* part, int64_t count, double* out, cudaStream_t st) {
    count_launches(1);
    k_sum_parts<<<1, kThreads, 0, st>>>(part, (int)count, out);
    return cudaGetLastError();
}

cudaError_t launch_count_changed(const int32_t* labels, const int32_t* prev, int64_t n,
                                 DevStatus* status, cudaStream_t st) {
    count_launches(1);
    k_count_changed<<<grid_for(n, kThreads), kThreads, 0, st>>>(labels, prev, n, status);
    return cudaGetLastError();
}

}  // namespace respca
