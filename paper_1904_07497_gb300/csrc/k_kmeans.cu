// K-means kernels of the RES-PCA p step (Sec. 4.2, Eq. (21)-(22)) and of the
// initial labels (k-means++ seeding, then Lloyd).
#include <cfloat>
#include <climits>

#include "respca_internal.cuh"

namespace respca {

namespace {

inline int grid_for(int64_t work, int per) { return (int)((work + per - 1) / per); }

// ---------------------------------------------------------------- label sort
constexpr int kSortParMaxC = 256;   // per-warp histograms fit shared memory up to here
// Stable counting sort of the columns by label (single CTA).  Produces the
// sorted column order perm, the cluster sizes n_i, and the label-pure tiles
// of at most kTileCols sorted columns; flags labels outside [0, c).
__global__ void __launch_bounds__(kSortThreads)
    k_sort_labels(const int32_t* __restrict__ labels, int64_t n, int c, int32_t* __restrict__ perm,
                  int32_t* __restrict__ counts, int32_t* __restrict__ tile_off,
                  TileDesc* __restrict__ tiles, DevStatus* __restrict__ status) {
    extern __shared__ int32_t sh[];
    int32_t* cnt = sh;            // [c]
    int32_t* run = sh + c;        // [c] running sorted position
    int32_t* toff = sh + 2 * c;   // [c + 1]
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    for (int i = threadIdx.x; i < c; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        const int32_t l = labels[j];
        if (l < 0 || l >= c) bad = 1;
        else atomicAdd(&cnt[l], 1);
    }
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0) {
            status->bad_labels = 1;
            status->ntiles = 0;
        }
        return;
    }
    // exclusive scans of the sizes and of the tile counts (warp 0)
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int32_t off = 0, toffs = 0;
        for (int base = 0; base < c; base += 32) {
            const int i = base + lane;
            const int32_t v = (i < c) ? cnt[i] : 0;
            const int32_t tv = (v + kTileCols - 1) / kTileCols;
            int32_t iv = v, it = tv;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t a = __shfl_up_sync(0xffffffffu, iv, o);
                const int32_t b = __shfl_up_sync(0xffffffffu, it, o);
                if (lane >= o) {
                    iv += a;
                    it += b;
                }
            }
            if (i < c) {
                run[i] = off + iv - v;
                toff[i] = toffs + it - tv;
            }
            off += __shfl_sync(0xffffffffu, iv, 31);
            toffs += __shfl_sync(0xffffffffu, it, 31);
        }
        if (lane == 0) {
            toff[c] = toffs;
            status->ntiles = toffs;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < c; i += blockDim.x) {
        counts[i] = cnt[i];
        tile_off[i] = toff[i];
        const int nt = toff[i + 1] - toff[i];
        for (int t = 0; t < nt; ++t) {
            TileDesc td;
            td.start = run[i] + t * kTileCols;
            td.len = min(kTileCols, cnt[i] - t * kTileCols);
            td.label = i;
            td.pad = 0;
            tiles[toff[i] + t] = td;
        }
    }
    if (threadIdx.x == 0) tile_off[c] = toff[c];
    __syncthreads();
    const int nwarps = blockDim.x / 32;
    if (c <= kSortParMaxC) {
        // stable scatter by all warps: warp w takes the w-th contiguous segment
        // of columns; its start for label l is run[l] plus the count of l in
        // the segments before it (per-warp histograms in hw[w][l])
        int32_t* hw = sh + 3 * c + 1;   // [nwarps][c]
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int64_t seg = (n + nwarps - 1) / nwarps;
        const int64_t j0 = (int64_t)warp * seg, j1 = min(n, j0 + seg);
        for (int i = lane; i < c; i += 32) hw[warp * c + i] = 0;
        __syncwarp();
        for (int64_t j = j0 + lane; j < j1; j += 32) atomicAdd(&hw[warp * c + labels[j]], 1);
        __syncthreads();
        for (int i = threadIdx.x; i < c; i += blockDim.x) {
            int32_t acc = run[i];
            for (int w = 0; w < nwarps; ++w) {
                const int32_t v = hw[w * c + i];
                hw[w * c + i] = acc;
                acc += v;
            }
        }
        __syncthreads();
        const unsigned lt = (1u << lane) - 1u;
        for (int64_t base = j0; base < j1; base += 32) {
            const int64_t j = base + lane;
            const int32_t l = (j < j1) ? labels[j] : -1;
            const unsigned peers = __match_any_sync(0xffffffffu, l);
            const int rank = __popc(peers & lt);
            int32_t pos = 0;
            if (l >= 0) pos = hw[warp * c + l] + rank;
            __syncwarp();
            if (l >= 0) {
                perm[pos] = (int32_t)j;
                if (rank == 0) hw[warp * c + l] += __popc(peers);
            }
            __syncwarp();
        }
        return;
    }
    // stable scatter, one warp, 32 columns at a time in column order
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const unsigned lt = (1u << lane) - 1u;
        for (int64_t base = 0; base < n; base += 32) {
            const int64_t j = base + lane;
            const int32_t l = (j < n) ? labels[j] : -1;
            const unsigned peers = __match_any_sync(0xffffffffu, l);
            const int rank = __popc(peers & lt);
            int32_t pos = 0;
            if (l >= 0) pos = run[l] + rank;
            __syncwarp();
            if (l >= 0) {
                perm[pos] = (int32_t)j;
                if (rank == 0) run[l] += __popc(peers);
            }
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------- assignment
// Nearest centroid for a set of columns of Y (all columns, or the queued list):
// scores s_i = ||mu_i||^2 - 2 mu_i . y_j over active clusters (n_i > 0), FP32
// products with Kahan-summed 64-row partials.  When the best two scores are
// closer than a bound on their rounding error, the candidates within the
// bound are re-decided with the exact squared distance in FP64, so every
// decision equals the argmin of the stored values (ties to the lowest index).
constexpr float kTieRel = 1e-5f;

template <typename TY>
__global__ void __launch_bounds__(kThreads)
    k_assign(const TY* __restrict__ Y, int64_t ldy, int64_t d, int64_t n,
             const int32_t* __restrict__ list, const float* __restrict__ mu,
             const float* __restrict__ mu_normf, const int32_t* __restrict__ counts, int c,
             int32_t* __restrict__ labels, DevStatus* __restrict__ status, float* __restrict__ ub,
             float* __restrict__ lb) {
    extern __shared__ __align__(16) float smem[];
    constexpr int LS = kAsgCols + 1;          // Ls row stride
    constexpr int MS = kAsgClusters + 4;      // Ms row stride (float4 aligned)
    float* Ls = smem;                          // [kAsgRows][LS]
    float* Ms = Ls + kAsgRows * LS;            // [kAsgRows][MS]
    float* scores = Ms + kAsgRows * MS;        // [c][LS]
    __shared__ int64_t colidx[kAsgCols];
    __shared__ float nrmL[kAsgCols];

    const int64_t total = list ? (int64_t)status->flagged : n;
    const int64_t base = (int64_t)blockIdx.x * kAsgCols;
    if (base >= total) return;
    const int tx = threadIdx.x & 31;
    const int ty = threadIdx.x >> 5;
    if (threadIdx.x < kAsgCols) {
        const int64_t q = base + threadIdx.x;
        colidx[threadIdx.x] = q < total ? (list ? (int64_t)list[q] : q) : -1;
    }
    __syncthreads();

    float nrm = 0.f, nrm_comp = 0.f;
    for (int cb = 0; cb < c; cb += kAsgClusters) {
        float acc[8], comp[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = comp[q] = 0.f;
        for (int64_t k0 = 0; k0 < d; k0 += kAsgRows) {
            for (int q = ty; q < kAsgCols; q += kThreads / 32) {
                const int64_t col = colidx[q];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int64_t r = k0 + h * 32 + tx;
                    float v = 0.f;
                    if (col >= 0 && r < d) v = XLoad<TY>::one(Y + col * ldy + r);
                    Ls[(h * 32 + tx) * LS + q] = v;
                }
            }
            for (int i = ty; i < kAsgClusters; i += kThreads / 32) {
                const int ci = cb + i;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int64_t r = k0 + h * 32 + tx;
                    Ms[(h * 32 + tx) * MS + i] = (ci < c && r < d) ? mu[(int64_t)ci * d + r] : 0.f;
                }
            }
            __syncthreads();
            float part[8];
            float npart = 0.f;
#pragma unroll
            for (int q = 0; q < 8; ++q) part[q] = 0.f;
#pragma unroll 8
            for (int k = 0; k < kAsgRows; ++k) {
                const float lv = Ls[k * LS + tx];
                const float4 m0 = *reinterpret_cast<const float4*>(&Ms[k * MS + ty * 8]);
                const float4 m1 = *reinterpret_cast<const float4*>(&Ms[k * MS + ty * 8 + 4]);
                part[0] = fmaf(m0.x, lv, part[0]);
                part[1] = fmaf(m0.y, lv, part[1]);
                part[2] = fmaf(m0.z, lv, part[2]);
                part[3] = fmaf(m0.w, lv, part[3]);
                part[4] = fmaf(m1.x, lv, part[4]);
                part[5] = fmaf(m1.y, lv, part[5]);
                part[6] = fmaf(m1.z, lv, part[6]);
                part[7] = fmaf(m1.w, lv, part[7]);
                if (cb == 0 && ty == 0) npart = fmaf(lv, lv, npart);
            }
            if (cb == 0 && ty == 0) {   // Kahan accumulation of ||y_j||^2
                const float y = npart - nrm_comp;
                const float t = nrm + y;
                nrm_comp = (t - nrm) - y;
                nrm = t;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {   // Kahan accumulation of the slab partials
                const float y = part[q] - comp[q];
                const float t = acc[q] + y;
                comp[q] = (t - acc[q]) - y;
                acc[q] = t;
            }
            __syncthreads();
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int ci = cb + ty * 8 + q;
            if (ci < c)
                scores[ci * LS + tx] = (counts[ci] > 0) ? fmaf(-2.f, acc[q], mu_normf[ci]) : INFINITY;
        }
    }
    if (ty == 0) nrmL[tx] = nrm;
    __syncthreads();

    const int lane = tx;
    for (int q = ty * (kAsgCols / 8); q < (ty + 1) * (kAsgCols / 8); ++q) {
        const int64_t col = colidx[q];
        if (col < 0) continue;
        float bs = INFINITY;
        int bi = INT_MAX;
        for (int i = lane; i < c; i += 32) {
            const float s = scores[i * LS + q];
            if (s < bs) {
                bs = s;
                bi = i;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float os = __shfl_xor_sync(0xffffffffu, bs, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (os < bs || (os == bs && oi < bi)) {
                bs = os;
                bi = oi;
            }
        }
        float ss = INFINITY;
        int si = INT_MAX;
        for (int i = lane; i < c; i += 32) {
            const float s = scores[i * LS + q];
            if (i != bi && s < ss) {
                ss = s;
                si = i;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float os = __shfl_xor_sync(0xffffffffu, ss, o);
            const int oi = __shfl_xor_sync(0xffffffffu, si, o);
            if (os < ss || (os == ss && oi < si)) {
                ss = os;
                si = oi;
            }
        }
        if (bi >= c) continue;   // no finite score: keep the label
        int newlab = bi;
        const float nl = nrmL[q];
        const float margin = kTieRel * (nl + fabsf(mu_normf[bi]));
        float ubv, lbv;
        if (ss - bs <= margin) {
            double best = INFINITY;
            int besti = bi;
            for (int i = 0; i < c; ++i) {
                if (!(scores[i * LS + q] <= bs + margin)) continue;
                double a = 0.0;
                const float* m = mu + (int64_t)i * d;
                for (int64_t r = lane; r < d; r += 32) {
                    const double diff = (double)XLoad<TY>::one(Y + col * ldy + r) - (double)m[r];
                    a = fma(diff, diff, a);
                }
                a = warp_sum(a);
                if (a < best) {
                    best = a;
                    besti = i;
                }
            }
            newlab = besti;
            ubv = (float)(sqrt(best) * (1.0 + 1e-6));
            lbv = 0.f;          // near tie: search this column again next time
            if (lane == 0) atomicAdd(&status->rechecked, 1);
        } else {
            // distances from the scores, widened by their rounding bound
            ubv = sqrtf(fmaxf(bs + nl + margin, 0.f)) * (1.f + 1e-6f);
            const float ms = si < c ? kTieRel * (nl + fabsf(mu_normf[si])) : 0.f;
            lbv = sqrtf(fmaxf(ss + nl - ms, 0.f)) * (1.f - 1e-6f);
        }
        if (lane == 0) {
            const int32_t old = labels[col];
            if (old != newlab) {
                labels[col] = newlab;
                atomicAdd(&status->changed, 1);
            }
            if (ub) {
                ub[col] = ubv;
                lb[col] = lbv;
            }
        }
    }
}

// ---------------------------------------------------------------- k-means++
// D2[j] (= or min=) squared distance of column j to the centre centers[k]:
// one warp per column, FP32 differences summed per lane with Kahan
// compensation over 8-element groups, FP64 across lanes.
template <typename TX, bool VEC>
__global__ void __launch_bounds__(kThreads)
    k_seed_dist(const TX* __restrict__ X, int64_t ldx, int64_t d, int64_t n,
                const int32_t* __restrict__ centers, int k, double* __restrict__ D2) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (kThreads / 32);
    const int64_t ctr = centers[k];
    const TX* xc = X + ctr * ldx;
    for (int64_t j = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5); j < n; j += warps) {
        const TX* xj = X + j * ldx;
        float s = 0.f, comp = 0.f;
        if (VEC) {
            // two 256-row steps per trip: all eight loads are issued first, then the
            // steps are added in the same order as one step per trip would add them
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int64_t r0 = lane * 4; r0 < d; r0 += 2 * 32 * 8) {
                float4 a[4], bq[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int64_t r = r0 + h * 128;
                    a[h] = r < d ? XLoad<TX>::four(xj + r) : z;
                    bq[h] = r < d ? XLoad<TX>::four(xc + r) : z;
                }
#pragma unroll
                for (int st = 0; st < 2; ++st) {
                    if (r0 + st * 256 >= d) break;
                    float part = 0.f, t;
                    const float4 a0 = a[2 * st], b0 = bq[2 * st], a1 = a[2 * st + 1], b1 = bq[2 * st + 1];
                    t = a0.x - b0.x; part = fmaf(t, t, part);
                    t = a0.y - b0.y; part = fmaf(t, t, part);
                    t = a0.z - b0.z; part = fmaf(t, t, part);
                    t = a0.w - b0.w; part = fmaf(t, t, part);
                    t = a1.x - b1.x; part = fmaf(t, t, part);
                    t = a1.y - b1.y; part = fmaf(t, t, part);
                    t = a1.z - b1.z; part = fmaf(t, t, part);
                    t = a1.w - b1.w; part = fmaf(t, t, part);
                    const float y = part - comp;
                    const float u = s + y;
                    comp = (u - s) - y;
                    s = u;
                }
            }
        } else {
            for (int64_t r0 = 0; r0 < d; r0 += 32 * 8) {
                float part = 0.f;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int64_t r = r0 + u * 32 + lane;
                    if (r < d) {
                        const float t = XLoad<TX>::one(xj + r) - XLoad<TX>::one(xc + r);
                        part = fmaf(t, t, part);
                    }
                }
                const float y = part - comp;
                const float u = s + y;
                comp = (u - s) - y;
                s = u;
            }
        }
        const double v = warp_sum((double)s);
        if (lane == 0) D2[j] = (k == 0) ? v : fmin(D2[j], v);
    }
}

// One k-means++ step in one launch: D2 against centre k (as k_seed_dist, one
// warp per column, grid = ceil(n / 8) so each warp takes one column), then
// centre kpick (kpick < 0: none) picked by the CTA that finishes last.  Each
// CTA writes the sum of its 8 columns' D2 (in column order) to part[b]; the
// last one (an atomic count of finished CTAs, reset for the next launch) finds
// the first column whose running sum exceeds u[kpick] times the total: the
// crossing block from the block sums (each thread scans a contiguous range
// of blocks, ranges in order), then the column inside it.  If rounding leaves
// no crossing, the last column with D2 > 0; with D2 all zero, floor(u n).
template <typename TX, bool VEC>
__global__ void __launch_bounds__(kThreads)
    k_seed_step(const TX* __restrict__ X, int64_t ldx, int64_t d, int64_t n,
                int32_t* __restrict__ centers, int k, int kpick, const double* __restrict__ u,
                double* __restrict__ D2, double* __restrict__ part, int32_t* __restrict__ done) {
    constexpr int W = kThreads / 32;
    __shared__ double colv[W];
    __shared__ double tsum[kThreads + 1];
    __shared__ long long s_block, s_pick;
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t ctr = centers[k];
    const TX* xc = X + ctr * ldx;
    const int64_t j = (int64_t)blockIdx.x * W + warp;
    double v = 0.0;
    if (j < n) {
        const TX* xj = X + j * ldx;
        float s = 0.f, comp = 0.f;
        if (VEC) {
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int64_t r0 = lane * 4; r0 < d; r0 += 2 * 32 * 8) {
                float4 a[4], bq[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int64_t r = r0 + h * 128;
                    a[h] = r < d ? XLoad<TX>::four(xj + r) : z;
                    bq[h] = r < d ? XLoad<TX>::four(xc + r) : z;
                }
#pragma unroll
                for (int st = 0; st < 2; ++st) {
                    if (r0 + st * 256 >= d) break;
                    float part8 = 0.f, t;
                    const float4 a0 = a[2 * st], b0 = bq[2 * st], a1 = a[2 * st + 1], b1 = bq[2 * st + 1];
                    t = a0.x - b0.x; part8 = fmaf(t, t, part8);
                    t = a0.y - b0.y; part8 = fmaf(t, t, part8);
                    t = a0.z - b0.z; part8 = fmaf(t, t, part8);
                    t = a0.w - b0.w; part8 = fmaf(t, t, part8);
                    t = a1.x - b1.x; part8 = fmaf(t, t, part8);
                    t = a1.y - b1.y; part8 = fmaf(t, t, part8);
                    t = a1.z - b1.z; part8 = fmaf(t, t, part8);
                    t = a1.w - b1.w; part8 = fmaf(t, t, part8);
                    const float y = part8 - comp;
                    const float uu = s + y;
                    comp = (uu - s) - y;
                    s = uu;
                }
            }
        } else {
            for (int64_t r0 = 0; r0 < d; r0 += 32 * 8) {
                float part8 = 0.f;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int64_t r = r0 + q * 32 + lane;
                    if (r < d) {
                        const float t = XLoad<TX>::one(xj + r) - XLoad<TX>::one(xc + r);
                        part8 = fmaf(t, t, part8);
                    }
                }
                const float y = part8 - comp;
                const float uu = s + y;
                comp = (uu - s) - y;
                s = uu;
            }
        }
        v = warp_sum((double)s);
        if (k > 0) v = fmin(D2[j], v);
        if (lane == 0) D2[j] = v;
    }
    if (kpick < 0) return;
    __threadfence();   // this warp's D2 is visible before the CTA counts as finished
    if (lane == 0) colv[warp] = (j < n) ? v : 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < W; ++w) b += colv[w];
        part[blockIdx.x] = b;
        __threadfence();
        s_last = (atomicAdd(done, 1) == (int)gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the last CTA: the pick
    const int64_t nb = gridDim.x;
    const int64_t chunk = (nb + kThreads - 1) / kThreads;
    const int64_t b0 = min(nb, (int64_t)threadIdx.x * chunk), b1 = min(nb, b0 + chunk);
    double t = 0.0;
    for (int64_t b = b0; b < b1; ++b) t += __ldcg(part + b);
    // exclusive prefix of the threads' range sums: a shuffle scan within each warp,
    // then the warps' totals in order (a chain of 5 + 8 FP64 additions instead of 256)
    double incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    double excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = 0.0;
    if (lane == 31) colv[warp] = incl;
    if (threadIdx.x == 0) {
        *done = 0;
        s_block = LLONG_MAX;
        s_pick = -1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double run = 0.0;
        for (int w = 0; w < W; ++w) {
            const double x = colv[w];
            colv[w] = run;
            run += x;
        }
        tsum[kThreads] = run;
    }
    __syncthreads();
    tsum[threadIdx.x] = colv[warp] + excl;
    __syncthreads();
    const double total = tsum[kThreads];
    const double uk = u[kpick];
    if (!(total > 0.0)) {
        if (threadIdx.x == 0) {
            int64_t pk = (int64_t)(uk * (double)n);
            centers[kpick] = (int32_t)(pk >= n ? n - 1 : pk);
        }
        return;
    }
    const double target = uk * total;
    double cum = tsum[threadIdx.x];
    for (int64_t b = b0; b < b1; ++b) {
        const double pb = __ldcg(part + b);
        if (cum + pb > target) {
            atomicMin(&s_block, (long long)b);
            break;
        }
        cum += pb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long pick = -1;
        if (s_block != LLONG_MAX) {
            // running sum up to the crossing block, in the same order as above
            const int64_t bq = s_block;
            const int owner = (int)(bq / chunk);
            double c2 = tsum[owner];
            for (int64_t b = (int64_t)owner * chunk; b < bq; ++b) c2 += __ldcg(part + b);
            long long lastpos = -1;
            for (int64_t jj = bq * W; jj < min(n, (bq + 1) * (int64_t)W); ++jj) {
                const double dj = __ldcg(D2 + jj);
                if (dj > 0.0) lastpos = jj;
                c2 += dj;
                if (c2 > target) {
                    pick = jj;
                    break;
                }
            }
            // the block's sum crossed but its running sum did not (rounding): the
            // crossing is at the block's end
            if (pick < 0) pick = lastpos;
        }
        if (pick < 0)
            for (int64_t jj = n - 1; jj >= 0; --jj)
                if (__ldcg(D2 + jj) > 0.0) {
                    pick = jj;
                    break;
                }
        centers[kpick] = (int32_t)(pick < 0 ? n - 1 : pick);
    }
}

// Pick centre k: the first column whose running sum of D2 exceeds u_k times
// the total (single CTA; FP64 block scans in column order).
__global__ void __launch_bounds__(1024)
    k_seed_pick(const double* __restrict__ D2, int64_t n, const double* __restrict__ u, int k,
                int32_t* __restrict__ centers) {
    __shared__ double wsum[32];
    __shared__ double s_total;
    __shared__ long long s_first;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double t = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) t += D2[j];
    t = warp_sum(t);
    if (lane == 0) wsum[warp] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 32; ++w) s += wsum[w];
        s_total = s;
        s_first = LLONG_MAX;
    }
    __syncthreads();
    const double total = s_total;
    const double uk = u[k];
    if (!(total > 0.0)) {
        if (threadIdx.x == 0) {
            int64_t pick = (int64_t)(uk * (double)n);
            if (pick >= n) pick = n - 1;
            centers[k] = (int32_t)pick;
        }
        return;
    }
    const double target = uk * total;
    double offset = 0.0;
    for (int64_t base = 0; base < n; base += blockDim.x) {
        const int64_t j = base + threadIdx.x;
        const double v = j < n ? D2[j] : 0.0;
        double incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double a = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += a;
        }
        __syncthreads();
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            double w = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double a = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += a;
            }
            wsum[lane] = w;   // inclusive over warps
        }
        __syncthreads();
        const double prefix = offset + (warp > 0 ? wsum[warp - 1] : 0.0) + incl;
        if (j < n && prefix > target) atomicMin(&s_first, (long long)j);
        __syncthreads();
        if (s_first != LLONG_MAX) break;
        offset += wsum[31];
    }
    if (s_first == LLONG_MAX) {
        // rounding left no crossing: the last column with positive mass
        if (threadIdx.x == 0) {
            int64_t pick = n - 1;
            for (int64_t j = n - 1; j >= 0; --j)
                if (D2[j] > 0.0) {
                    pick = j;
                    break;
                }
            centers[k] = (int32_t)pick;
        }
        return;
    }
    if (threadIdx.x == 0) centers[k] = (int32_t)s_first;
}

template <typename TX>
__global__ void __launch_bounds__(kThreads)
    k_gather_centers(const TX* __restrict__ X, int64_t ldx, int64_t d,
                     const int32_t* __restrict__ centers, float* __restrict__ mu,
                     int32_t* __restrict__ counts) {
    const int k = blockIdx.y;
    const int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) counts[k] = 1;
    if (r < d) mu[(int64_t)k * d + r] = XLoad<TX>::one(X + (int64_t)centers[k] * ldx + r);
}

}  // namespace

// ---------------------------------------------------------------- launchers
cudaError_t launch_sort_labels(const int32_t* labels, int64_t n, int c, int32_t* perm,
                               int32_t* counts, int32_t* tile_off, TileDesc* tiles,
                               DevStatus* status, cudaStream_t st) {
    count_launches(1);
    size_t smem = sizeof(int32_t) * (size_t)(3 * c + 1);
    if (c <= kSortParMaxC) smem += sizeof(int32_t) * (size_t)(kSortThreads / 32) * c;
    if (smem > 48 * 1024) {
        cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_sort_labels));
        if (e != cudaSuccess) return e;
    }
    k_sort_labels<<<1, kSortThreads, smem, st>>>(labels, n, c, perm, counts, tile_off, tiles, status);
    return cudaGetLastError();
}

size_t assign_smem_bytes(int c) {
    const int LS = kAsgCols + 1, MS = kAsgClusters + 4;
    return sizeof(float) * ((size_t)kAsgRows * LS + (size_t)kAsgRows * MS + (size_t)c * LS);
}

cudaError_t launch_assign(int dtype, const void* Y, int64_t ldy, int64_t d, int64_t n,
                          const int32_t* list, const float* mu, const float* mu_normf,
                          const int32_t* counts, int c, int32_t* labels, DevStatus* status,
                          cudaStream_t st, float* ub, float* lb) {
    count_launches(1);
    const size_t smem = assign_smem_bytes(c);
    const int grid = grid_for(n, kAsgCols);
    cudaError_t e = cudaSuccess;
    RESPCA_DISPATCH_X(dtype, TY, {
        e = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_assign<TY>));
        if (e == cudaSuccess)
            k_assign<TY><<<grid, kThreads, smem, st>>>((const TY*)Y, ldy, d, n, list, mu, mu_normf,
                                                       counts, c, labels, status, ub, lb);
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_seed_dist(int dtype, const void* X, int64_t ldx, int64_t d, int64_t n,
                             const int32_t* centers, int k, double* D2, cudaStream_t st) {
    count_launches(1);
    const int grid = grid_for(n, kThreads / 32);
    RESPCA_DISPATCH_X(dtype, TX, {
        const bool vec = (ldx % 4 == 0) && (d % 4 == 0) &&
                         (reinterpret_cast<uintptr_t>(X) % (4 * sizeof(TX)) == 0);
        if (vec)
            k_seed_dist<TX, true><<<grid, kThreads, 0, st>>>((const TX*)X, ldx, d, n, centers, k, D2);
        else
            k_seed_dist<TX, false><<<grid, kThreads, 0, st>>>((const TX*)X, ldx, d, n, centers, k, D2);
    });
    return cudaGetLastError();
}

cudaError_t launch_seed_step(int dtype, const void* X, int64_t ldx, int64_t d, int64_t n, int32_t* centers,
                             int k, int kpick, const double* u, double* D2, double* part, int32_t* done,
                             cudaStream_t st) {
    count_launches(1);
    const int grid = grid_for(n, kThreads / 32);
    RESPCA_DISPATCH_X(dtype, TX, {
        const bool vec = (ldx % 4 == 0) && (d % 4 == 0) &&
                         (reinterpret_cast<uintptr_t>(X) % (4 * sizeof(TX)) == 0);
        if (vec)
            k_seed_step<TX, true><<<grid, kThreads, 0, st>>>((const TX*)X, ldx, d, n, centers, k, kpick, u, D2,
                                                             part, done);
        else
            k_seed_step<TX, false><<<grid, kThreads, 0, st>>>((const TX*)X, ldx, d, n, centers, k, kpick, u, D2,
                                                              part, done);
    });
    return cudaGetLastError();
}

cudaError_t launch_seed_pick(const double* D2, int64_t n, const double* u, int k, int32_t* centers,
                             cudaStream_t st) {
    count_launches(1);
    k_seed_pick<<<1, 1024, 0, st>>>(D2, n, u, k, centers);
    return cudaGetLastError();
}

cudaError_t launch_gather_centers(int dtype, const void* X, int64_t ldx, int64_t d,
                                  const int32_t* centers, int c, float* mu, int32_t* counts,
                                  cudaStream_t st) {
    count_launches(1);
    const dim3 grid(grid_for(d, kThreads), c);
    RESPCA_DISPATCH_X(dtype, TX, {
        k_gather_centers<TX><<<grid, kThreads, 0, st>>>((const TX*)X, ldx, d, centers, mu, counts);
    });
    return cudaGetLastError();
}

}  // namespace respca
