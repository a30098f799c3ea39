// Nearest-centroid search on the 5th-generation tensor cores (sm_103a).
//
// The p step of Sec. 4.2 (Eq. (21)-(22)) needs, for every searched column y_j,
// the scores s_ij = ||mu_i||^2 - 2 mu_i . y_j over the c centroids: a
// (columns x d) . (d x c) product.  It runs on tcgen05.mma kind::tf32 with
// A = 128 columns (M = 128, K-major: a column of Y is contiguous along d),
// B = the centroids padded to Npad (K-major) and the FP32 accumulator in
// tensor memory.  FP32 accuracy comes from the 3-term split y = y_hi + y_lo,
// mu = mu_hi + mu_lo (hi = TF32-truncated):
//   y.mu ~ y_hi.mu_hi + y_hi.mu_lo + y_lo.mu_hi       (error ~ 2^-20 relative).
// kind::tf32 reads an FP32 operand by dropping its 13 low mantissa bits (a
// truncation, measured on this part with operands whose low bits tell
// truncation, rounding and full FP32 apart), so an unconverted FP32 tile in
// shared memory already is its hi part: the dense kernel writes only y_lo.
//
// Two kernels feed the tensor cores:
//  * k_search_dense (all columns, FP32 Y): stream-K over (column tile, 32-row
//    slab) work, split evenly over one CTA per SM.  Warp 0 issues TMA loads
//    (cp.async.bulk.tensor, 128-byte swizzle) into a ring of stages, warps 2-5
//    write the TF32 lo part of each Y tile to shared memory, one thread of
//    warp 1 issues the MMAs into two ping-pong TMEM accumulators, and warps
//    2-5 drain a finished accumulator to global partial sums.
//  * k_search_list (a queued subset of columns, or any element type): threads
//    gather the listed columns with plain loads, d split over gridDim.y.
// In both, the last CTA to finish a column tile adds the partial products in
// a fixed order, forms the scores, takes the argmin (ties to the lowest index)
// and updates the labels and pruning bounds; near ties go to k_search_recheck,
// which decides them with exact FP64 distances.
//
// Shared-memory operands use the canonical K-major 128-byte-swizzle layout:
// 8-row groups of 1024 bytes, 128 bytes (32 FP32) per row, 16-byte chunk q of
// row m stored at chunk q ^ (m % 8).  Every wait on an mbarrier is bounded; a
// wait that gives up sets status->timeout and the kernel drains its
// asynchronous work (with bounded waits), releases its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <mutex>
#include <type_traits>
#include <utility>
#include <vector>

#include "respca_internal.cuh"
#include "tc_ptx.cuh"

namespace respca {

namespace {

constexpr int kTcM = 128;             // columns per tile (UMMA M)
constexpr int kTcK = 32;              // d rows per slab: one 128-byte swizzle atom of FP32
constexpr int kTcStages = 2;          // stages of the list kernel
constexpr int kTcThreads = 256;       // threads of the list kernel
constexpr int kDnThreads = 224;       // dense kernel: 2 TMA warps, MMA warp, 4 split/epilogue warps
constexpr int kDnMaxY = 3;            // Y stages (row blocks)
constexpr int kDnMaxB = 6;            // centroid slab stages
constexpr int kTcMaxSplit = 16;       // largest d split of the list kernel
constexpr float kTieRelTc = 6e-5f;    // bound on the score rounding (see score_err)

// Score rounding bound of centroid i for a column y: e_i = kTieRelTc *
// (2 ||mu_i|| ||y|| + ||mu_i||^2) (Cauchy-Schwarz on the products' error).
// When the products use y truncated to TF32 (no y_lo term), ylo bounds
// ||y - tf32(y)|| and |mu_i . (y - tf32(y))| <= ||mu_i|| ylo adds 2 ||mu_i|| ylo.
__device__ __forceinline__ float score_err(float mu2, float y2, float ylo = 0.f) {
    const float mn = sqrtf(fmaxf(mu2, 0.f));
    return kTieRelTc * (2.f * mn * sqrtf(y2) + fabsf(mu2)) + 2.f * mn * ylo;
}

// Dot products g_i0 .. g_i0+7 of one column: sums over the nslots partial
// products (slot-major [slot][Npad][128], column m), loads issued together.
__device__ __forceinline__ void gather8(const float* __restrict__ gbase, int nslots, int Npad, int m,
                                        int i0, int c, float* g) {
#pragma unroll
    for (int q = 0; q < 8; ++q) g[q] = 0.f;
    for (int sl = 0; sl < nslots; ++sl) {
        const float* b = gbase + ((int64_t)sl * Npad + i0) * kTcM + m;
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = (i0 + q < c) ? __ldcg(b + (int64_t)q * kTcM) : 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) g[q] += v[q];
    }
}

// Scores s_i = ||mu_i||^2 - 2 g_i of one column from its dot products g_i
// (partial products summed in a fixed order), argmin with ties to the lowest
// index, and the update of the label and the bounds; a near tie is queued
// with its candidate set for the FP64 re-decision.
// gather(i0, g) fills g[0..7] with the dot products of centroids i0 .. i0+7.
template <typename Gather>
__device__ void finalize_scores(int64_t col, float y2, Gather gather,
                                const float* __restrict__ mu_normf,
                                const int32_t* __restrict__ counts, int c,
                                int32_t* __restrict__ labels, float* __restrict__ ub,
                                float* __restrict__ lb, DevStatus* __restrict__ status,
                                const RcQueue& rc, float ylo = 0.f) {
    float bs = INFINITY, ss = INFINITY, be = 0.f, se = 0.f;
    int bi = INT_MAX, si = INT_MAX;
    for (int i0 = 0; i0 < c; i0 += 8) {
        float g[8];
        gather(i0, g);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = i0 + q;
            if (i >= c || counts[i] == 0) continue;
            const float mu2 = mu_normf[i];
            const float sc = fmaf(-2.f, g[q], mu2);
            if (sc < bs) {
                ss = bs;
                se = be;
                si = bi;
                bs = sc;
                bi = i;
                be = score_err(mu2, y2, ylo);
            } else if (sc < ss) {
                ss = sc;
                si = i;
                se = score_err(mu2, y2, ylo);
            }
        }
    }
    if (bi >= c) return;
    if (ss - bs <= be + se) {
        // candidates: every centroid whose score interval reaches the lowest upper end
        float best_hi = INFINITY;
        for (int i0 = 0; i0 < c; i0 += 8) {
            float g[8];
            gather(i0, g);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int i = i0 + q;
                if (i >= c || counts[i] == 0) continue;
                const float mu2 = mu_normf[i];
                best_hi = fminf(best_hi, fmaf(-2.f, g[q], mu2) + score_err(mu2, y2, ylo));
            }
        }
        const int slot = atomicAdd(&status->rechecked, 1);
        RcRec* r = rc.rec + slot;
        for (int w = 0; w < kTcMaxClusters / 32; ++w) r->mask[w] = 0u;
        for (int i0 = 0; i0 < c; i0 += 8) {
            float g[8];
            gather(i0, g);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int i = i0 + q;
                if (i >= c || counts[i] == 0) continue;
                const float mu2 = mu_normf[i];
                if (fmaf(-2.f, g[q], mu2) - score_err(mu2, y2, ylo) <= best_hi)
                    r->mask[i >> 5] |= 1u << (i & 31);
            }
        }
        r->col = (int32_t)col;
        r->done = 0;
        if (slot < rc.cap) {
            int cnt = 0;
            for (int w = 0; w < kTcMaxClusters / 32; ++w) cnt += __popc(r->mask[w]);
            int at = atomicAdd(&status->rc_pairs, cnt);
            for (int i = 0; i < c; ++i)
                if ((r->mask[i >> 5] >> (i & 31)) & 1u) rc.pairs[at++] = slot * c + i;
        }
        return;
    }
    const float yerr = 1e-5f * y2;
    const int32_t old = labels[col];
    if (old != bi) {
        labels[col] = bi;
        atomicAdd(&status->changed, 1);
    }
    if (ub) {
        ub[col] = sqrtf(fmaxf(bs + y2 + be + yerr, 0.f)) * (1.f + 1e-6f);
        lb[col] = si < c ? sqrtf(fmaxf(ss + y2 - se - yerr, 0.f)) * (1.f - 1e-6f) : INFINITY;
    }
}

// The decision of finalize_scores by one warp for one column (c <= 128): lane
// l holds centroids l, l + 32, l + 64, l + 96.  Same scores, bounds and rules:
// best = the lowest score, ties to the lowest index; second = the lowest
// score among the others, ties to the lowest index; a near tie queues every
// centroid whose score interval reaches the lowest upper end.  g(i) returns
// the dot product of centroid i.
__device__ __forceinline__ void warp_best(float& v, int& i, float& e) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        const float oe = __shfl_xor_sync(0xffffffffu, e, o);
        if (ov < v || (ov == v && oi < i)) {
            v = ov;
            i = oi;
            e = oe;
        }
    }
}

// mu2v[q], okv[q], serr[q]: ||mu_i||^2, "cluster i is not empty" and the error
// norm of centroid i's 16-bit split (0 with FP32 operands) for i = lane + 32 q,
// loaded by the caller.  y2 is ||y~||^2 of the operand y~ the products use.
// ylo bounds ||y - tf32(y)|| when y2 is exact ||y||^2 (FP32 operand); ysh > 0
// (a 16-bit copy y~ of FP32 data) bounds ||y - y~||: the scores then widen by
// 2 ||mu_i|| ysh and the bounds are distances to y~ moved by ysh (triangle
// inequality).  The split adds |(mu_i - mu~_i) . y~| <= serr_i ||y~|| to each
// product.
__device__ __forceinline__ float pick4(const float (&v)[4], int q) {
    return q == 0 ? v[0] : q == 1 ? v[1] : q == 2 ? v[2] : v[3];
}

template <typename G>
__device__ void finalize_warp(int64_t col, float y2, float ylo, float ysh, G g, const float (&mu2v)[4],
                              const float (&serr)[4], const bool (&okv)[4],
                              int c, int32_t* __restrict__ labels, float* __restrict__ ub, float* __restrict__ lb,
                              DevStatus* __restrict__ status, const RcQueue& rc) {
    const int lane = threadIdx.x & 31;
    float sc[4], er[4];
    bool ok[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = lane + 32 * q;
        ok[q] = okv[q];
        sc[q] = INFINITY;
        er[q] = 0.f;
        if (ok[q]) {
            const float mu2 = mu2v[q];
            sc[q] = fmaf(-2.f, g(i), mu2);
            er[q] = score_err(mu2, y2, ylo + ysh) + 2.f * serr[q] * sqrtf(y2);
        }
    }
    float bs = INFINITY, be = 0.f;
    int bi = INT_MAX;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (ok[q] && sc[q] < bs) {
            bs = sc[q];
            bi = lane + 32 * q;
            be = er[q];
        }
    warp_best(bs, bi, be);
    if (bi >= c) return;
    float ss = INFINITY, se = 0.f;
    int si = INT_MAX;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (ok[q] && lane + 32 * q != bi && sc[q] < ss) {
            ss = sc[q];
            si = lane + 32 * q;
            se = er[q];
        }
    warp_best(ss, si, se);
    if (ss - bs <= be + se) {
        float hi = INFINITY;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (ok[q]) hi = fminf(hi, sc[q] + er[q]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) hi = fminf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        uint32_t m[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) m[q] = __ballot_sync(0xffffffffu, ok[q] && sc[q] - er[q] <= hi);
        int slot = 0, at = 0;
        if (lane == 0) {
            slot = atomicAdd(&status->rechecked, 1);
            RcRec* r = rc.rec + slot;
            for (int w = 0; w < kTcMaxClusters / 32; ++w) r->mask[w] = w < 4 ? m[w] : 0u;
            r->col = (int32_t)col;
            r->done = 0;
            if (slot < rc.cap) at = atomicAdd(&status->rc_pairs, __popc(m[0]) + __popc(m[1]) + __popc(m[2]) + __popc(m[3]));
        }
        slot = __shfl_sync(0xffffffffu, slot, 0);
        at = __shfl_sync(0xffffffffu, at, 0);
        if (slot < rc.cap) {
            // each lane its own candidates, in index order: lane + 32 q at its rank
            const uint32_t below = (1u << lane) - 1u;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if ((m[q] >> lane) & 1u) rc.pairs[at + __popc(m[q] & below)] = slot * c + lane + 32 * q;
                at += __popc(m[q]);
            }
        }
        return;
    }
    float bb = be, sb = se;
    if (ysh > 0.f) {   // uniform over the warp
        const float mu2b = __shfl_sync(0xffffffffu, pick4(mu2v, bi >> 5), bi & 31);
        const float mu2s = __shfl_sync(0xffffffffu, pick4(mu2v, si >> 5), si & 31);
        const float sb_ = __shfl_sync(0xffffffffu, pick4(serr, bi >> 5), bi & 31);
        const float ss_ = __shfl_sync(0xffffffffu, pick4(serr, si >> 5), si & 31);
        bb = score_err(mu2b, y2, ylo) + 2.f * sb_ * sqrtf(y2);
        sb = score_err(mu2s, y2, ylo) + 2.f * ss_ * sqrtf(y2);
    }
    if (lane != 0) return;
    const float yerr = 1e-5f * y2;
    const int32_t old = labels[col];
    if (old != bi) {
        labels[col] = bi;
        atomicAdd(&status->changed, 1);
    }
    if (ub) {
        ub[col] = (sqrtf(fmaxf(bs + y2 + bb + yerr, 0.f)) + ysh) * (1.f + 1e-6f);
        lb[col] = si < c ? fmaxf(sqrtf(fmaxf(ss + y2 - sb - yerr, 0.f)) - ysh, 0.f) * (1.f - 1e-6f) : INFINITY;
    }
}

// Partial products slot-major [slot][Npad][128], column m of a 128-column tile.
__device__ __forceinline__ void finalize_column(int64_t col, float y2, const float* __restrict__ gbase,
                                                int nslots, int Npad, int m,
                                                const float* __restrict__ mu_normf,
                                                const int32_t* __restrict__ counts, int c,
                                                int32_t* __restrict__ labels, float* __restrict__ ub,
                                                float* __restrict__ lb, DevStatus* __restrict__ status,
                                                const RcQueue& rc) {
    finalize_scores(col, y2, [&](int i0, float* g) { gather8(gbase, nslots, Npad, m, i0, c, g); },
                    mu_normf, counts, c, labels, ub, lb, status, rc);
}

// ============================================================== list kernel
template <typename TY, bool VEC>
__device__ __forceinline__ void load_col16(const TY* __restrict__ colp, int64_t r0, int64_t d,
                                           float4* v) {
    if (colp == nullptr) {
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t r = r0 + 4 * q;
        if (VEC) {
            v[q] = (r < d) ? XLoad<TY>::four(colp + r) : make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            float t[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) t[e] = (r + e < d) ? XLoad<TY>::one(colp + r + e) : 0.f;
            v[q] = make_float4(t[0], t[1], t[2], t[3]);
        }
    }
}

constexpr int kTcBMax = 4;   // prefetched 16-byte chunks of each centroid half per thread

template <typename TY, bool VEC>
__global__ void __launch_bounds__(kTcThreads, 2)
    k_search_list(const TY* __restrict__ Y, int64_t ldy, int64_t d, int64_t n,
                  const int32_t* __restrict__ list, int64_t list_max, DevStatus* __restrict__ status,
                  const float* __restrict__ mu_hi, const float* __restrict__ mu_lo, int64_t dpad,
                  int Npad, int max_split, const float* __restrict__ mu_normf,
                  const int32_t* __restrict__ counts, int c, int32_t* __restrict__ labels,
                  float* __restrict__ ub, float* __restrict__ lb, float* __restrict__ Gpart,
                  float* __restrict__ ynorm_part, int32_t* __restrict__ tile_count,
                  RcQueue rc_list) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t mbar[kTcStages];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int is_last_sh;

    const int64_t total = list ? (int64_t)status->flagged : n;
    if (list && total > list_max) return;   // the dense kernel searches every column instead
    const int64_t tile0 = (int64_t)blockIdx.x * kTcM;
    if (tile0 >= total) return;
    // d split: about two CTAs per SM over the tiles actually queued, every split non-empty
    const int64_t nslabs = (d + kTcK - 1) / kTcK;
    const int64_t tiles = (total + kTcM - 1) / kTcM;
    int64_t want = (2 * 152) / tiles;
    want = want < 1 ? 1 : (want > max_split ? max_split : want);
    if (want > nslabs) want = nslabs;
    const int64_t slabs_per_split = (nslabs + want - 1) / want;
    const int nsplit = (int)((nslabs + slabs_per_split - 1) / slabs_per_split);
    if ((int)blockIdx.y >= nsplit) return;
    const int64_t s_begin = (int64_t)blockIdx.y * slabs_per_split;
    const int64_t s_end = min(nslabs, s_begin + slabs_per_split);
    const int nq = (int)(s_end - s_begin);   // >= 1: every split is non-empty

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t a_bytes = kTcM * 128;
    const uint32_t b_bytes = (uint32_t)Npad * 128;
    const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
    auto a_hi = [&](int s) { return base + s * stage_bytes; };
    auto a_lo = [&](int s) { return base + s * stage_bytes + a_bytes; };
    auto b_hi = [&](int s) { return base + s * stage_bytes + 2 * a_bytes; };
    auto b_lo = [&](int s) { return base + s * stage_bytes + 2 * a_bytes + b_bytes; };

    uint32_t tmem_cols = 32;
    while ((int)tmem_cols < Npad) tmem_cols <<= 1;
    if (warp == 0) {
        tmem_alloc(&tmem_base_sh, tmem_cols);
        tc_fence_before();
    }
    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s) mbar_init(&mbar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    // A mapping: thread -> (column m of the tile, half h of the 32-row slab)
    const int m = tid >> 1, h = tid & 1;
    const int64_t pos = tile0 + m;
    const TY* colp = nullptr;
    if (pos < total) {
        const int64_t col = list ? (int64_t)list[pos] : pos;
        colp = Y + col * ldy;
    }
    const int bchunks = Npad * 8;
    const int bmine = (bchunks - tid + kTcThreads - 1) / kTcThreads;
    const uint32_t idesc = idesc_tf32(kTcM, Npad);

    float4 av[4], bh[kTcBMax], bl[kTcBMax];
    auto load_b = [&](int64_t k0) {
#pragma unroll
        for (int j = 0; j < kTcBMax; ++j) {
            if (j < bmine) {
                const int e = tid + j * kTcThreads;
                const int64_t g = (int64_t)(e >> 3) * dpad + k0 + (e & 7) * 4;
                bh[j] = __ldg(reinterpret_cast<const float4*>(mu_hi + g));
                bl[j] = __ldg(reinterpret_cast<const float4*>(mu_lo + g));
            }
        }
    };
    float ysq = 0.f, ycomp = 0.f;
    load_col16<TY, VEC>(colp, s_begin * kTcK + h * 16, d, av);
    load_b(s_begin * kTcK);
    bool failed = false;

    for (int q = 0; q < nq; ++q) {
        const int st = q & 1;
        const int64_t k0 = (s_begin + q) * kTcK;
        if (q >= kTcStages) {
            if (!mbar_wait(&mbar[st], (uint32_t)(((q - kTcStages) >> 1) & 1))) failed = true;
        }
        if (__syncthreads_or(failed)) {
            failed = true;
            break;
        }
        {
            float part = 0.f;
#pragma unroll
            for (int c4 = 0; c4 < 4; ++c4) {
                const float4 x = av[c4];
                const float4 hi = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
                const float4 lo = make_float4(x.x - hi.x, x.y - hi.y, x.z - hi.z, x.w - hi.w);
                const uint32_t off = sw128_off(m, h * 4 + c4);
                st_shared_v4(a_hi(st) + off, hi);
                st_shared_v4(a_lo(st) + off, lo);
                part = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, part))));
            }
            const float y = part - ycomp;   // Kahan accumulation of ||y_j||^2
            const float t = ysq + y;
            ycomp = (t - ysq) - y;
            ysq = t;
        }
#pragma unroll
        for (int j = 0; j < kTcBMax; ++j) {
            if (j < bmine) {
                const int e = tid + j * kTcThreads;
                const uint32_t off = sw128_off(e >> 3, e & 7);
                st_shared_v4(b_hi(st) + off, bh[j]);
                st_shared_v4(b_lo(st) + off, bl[j]);
            }
        }
        for (int e = tid + kTcBMax * kTcThreads; e < bchunks; e += kTcThreads) {   // Npad > 128
            const int64_t g = (int64_t)(e >> 3) * dpad + k0 + (e & 7) * 4;
            const uint32_t off = sw128_off(e >> 3, e & 7);
            st_shared_v4(b_hi(st) + off, __ldg(reinterpret_cast<const float4*>(mu_hi + g)));
            st_shared_v4(b_lo(st) + off, __ldg(reinterpret_cast<const float4*>(mu_lo + g)));
        }
        if (q + 1 < nq) {
            load_col16<TY, VEC>(colp, k0 + kTcK + h * 16, d, av);
            load_b(k0 + kTcK);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < kTcK / 8; ++ks) {
                const uint32_t koff = ks * 32;   // 8 TF32 = 32 bytes along K
                const uint64_t dah = sw128_desc(a_hi(st) + koff), dal = sw128_desc(a_lo(st) + koff);
                const uint64_t dbh = sw128_desc(b_hi(st) + koff), dbl = sw128_desc(b_lo(st) + koff);
                tc_mma(tmem, dah, dbh, idesc, (q > 0 || ks > 0) ? 1u : 0u);
                tc_mma(tmem, dah, dbl, idesc, 1u);
                tc_mma(tmem, dal, dbh, idesc, 1u);
            }
            tc_commit(&mbar[st]);
        }
    }

    {
        const int ql = failed ? -1 : nq - 1;
        if (ql >= 0) {
            if (!mbar_wait(&mbar[ql & 1], (uint32_t)((ql >> 1) & 1))) failed = true;
        } else {
            for (int s = 0; s < kTcStages; ++s) mbar_wait(&mbar[s], 0u);
        }
    }
    failed = __syncthreads_or(failed);
    tc_fence_after();
    float* gtile = Gpart + ((int64_t)blockIdx.x * max_split + blockIdx.y) * (int64_t)Npad * kTcM;
    if (!failed && warp < 4) {
        const int mm = warp * 32 + lane;
        for (int cb = 0; cb < Npad; cb += 16) {
            float v[16];
            tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) gtile[(int64_t)(cb + q) * kTcM + mm] = v[q];
        }
    }
    {
        const float other = __shfl_xor_sync(0xffffffffu, ysq, 1);
        if (h == 0) ynorm_part[((int64_t)blockIdx.x * max_split + blockIdx.y) * kTcM + m] = ysq + other;
    }
    if (failed && tid == 0) atomicOr(&status->timeout, 1);
    tc_fence_before();
    __threadfence();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, tmem_cols);
    if (tid == 0) {
        const int prev = atomicAdd(&tile_count[blockIdx.x], 1);
        is_last_sh = (prev == nsplit - 1);
    }
    __syncthreads();
    if (!is_last_sh) return;
    __threadfence();
    if (tid == 0) tile_count[blockIdx.x] = 0;
    if (tid >= kTcM) return;
    const int64_t p = tile0 + tid;
    if (p >= total) return;
    const int64_t col = list ? (int64_t)list[p] : p;
    const float* gt0 = Gpart + (int64_t)blockIdx.x * max_split * (int64_t)Npad * kTcM;
    const float* yt0 = ynorm_part + (int64_t)blockIdx.x * max_split * kTcM;
    float y2 = 0.f;
    for (int s = 0; s < nsplit; ++s) y2 += __ldcg(yt0 + (int64_t)s * kTcM + tid);
    finalize_column(col, y2, gt0, nsplit, Npad, tid, mu_normf, counts, c, labels, ub, lb, status,
                    rc_list);
}

// ============================================================== dense kernel
// Stream-K split of the (tile, slab) work: CTA b owns [w0(b), w0(b+1)),
// w0(b) = b W / G, W = tiles * slabs.  owner(w) is the CTA whose range holds w.
__host__ __device__ __forceinline__ int64_t sk_begin(int64_t b, int64_t W, int64_t G) {
    return (b * W) / G;
}
__host__ __device__ __forceinline__ int64_t sk_owner(int64_t w, int64_t W, int64_t G) {
    return ((w + 1) * G - 1) / W;
}

struct DenseArgs {
    int64_t d, n, Q, T, W;   // rows, columns, row blocks per tile, tiles, work units
    int64_t nslab;           // 32-row slabs in d
    int Npad, R, YS, BS;     // slabs per row block, Y stages (R slabs each), centroid stages
    int cmax, nacc;          // partial-sum slots per tile, accumulator buffers
    uint32_t lo_col;         // first TMEM column of the y_lo ring (BS x 32 columns)
    uint32_t tmem_cols;      // TMEM columns allocated
    int use_list;            // 1: a queued list was asked for (run only if it is long)
    int64_t list_min;
};

// A operand read from tensor memory (lane m = row m, column k = K index k).
__device__ __forceinline__ void tc_mma_tmem_a(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc,
                                              uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}"
        ::"r"(tmem_d), "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// 32 consecutive TMEM columns of this thread's lane.
__device__ __forceinline__ void tc_st32(uint32_t taddr, const uint32_t* r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
        ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
          "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
          "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),
          "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),
          "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

// Dense search.  A work unit is one row block (R slabs of 32 rows) of one
// 128-column tile; stream-K splits the units evenly over one CTA per SM.
// Y is staged a whole row block at a time (R boxes issued together, so each
// column is read in runs of R x 128 bytes), in YS stages; the centroid hi / lo
// slabs come through their own ring of BS stages, fed by a second producer
// warp.  The split warps write y_lo into a TMEM ring (BS x 32 columns), from
// where the third MMA of the split reads it as its A operand; the raw FP32
// tile in shared memory is the hi operand.
//   warp 0: Y producer, warp 1: MMA issuer, warps 2-5: split + epilogue,
//   warp 6: centroid producer.
// The MMA issuer is a single thread whose loop overhead bounds the tensor
// core's rate: stage indices and phases advance incrementally and the
// shared-memory descriptors are formed once and offset by addition (the
// address field of a descriptor is the byte address / 16).
__global__ void __launch_bounds__(kDnThreads, 1)
    k_search_dense(const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmBh,
                   const __grid_constant__ CUtensorMap tmBl, DenseArgs a,
                   DevStatus* __restrict__ status, const float* __restrict__ mu_normf,
                   const int32_t* __restrict__ counts, int c, int32_t* __restrict__ labels,
                   float* __restrict__ ub, float* __restrict__ lb, float* __restrict__ Gpart,
                   float* __restrict__ ynorm_part, int32_t* __restrict__ tile_count,
                   RcQueue rc_list) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t yfull[kDnMaxY], yempty[kDnMaxY];
    __shared__ uint64_t bfull[kDnMaxB], bempty[kDnMaxB], conv[kDnMaxB];
    __shared__ uint64_t acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_sh;
    __shared__ int is_last_sh;

    if (a.use_list && (int64_t)status->flagged < a.list_min) return;   // the list kernel handles it
    const int64_t G = gridDim.x, b = blockIdx.x;
    const int64_t w0 = sk_begin(b, a.W, G), w1 = sk_begin(b + 1, a.W, G);
    if (w0 >= w1) return;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int R = a.R, YS = a.YS, BS = a.BS, NA = a.nacc;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t a_bytes = kTcM * 128;
    const uint32_t b_bytes = (uint32_t)a.Npad * 128;
    const uint32_t y_stage = (uint32_t)R * a_bytes;
    const uint32_t b_base = base + (uint32_t)YS * y_stage;
    const int64_t w_tile0 = w0 / a.Q, w_blk0 = w0 % a.Q;
    // slabs of row block blk (the last block of d may be short)
    auto slabs_of = [&](int64_t blk) { return (int)min((int64_t)R, a.nslab - blk * R); };

    if (warp == 1) {
        tmem_alloc(&tmem_base_sh, a.tmem_cols);
        tc_fence_before();
    }
    if (tid == 0) {
        for (int s = 0; s < YS; ++s) {
            mbar_init(&yfull[s], 1);
            mbar_init(&yempty[s], 1);
        }
        for (int s = 0; s < BS; ++s) {
            mbar_init(&bfull[s], 1);
            mbar_init(&bempty[s], 1);
            mbar_init(&conv[s], 4);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&acc_full[s], 1);
            mbar_init(&acc_empty[s], 4);
        }
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    if (warp == 0) {
        // ---------------- Y producer: one row block per stage
        if (lane == 0) {
            RingPos yr(YS);
            int64_t k = 0, tile = w_tile0, blk = w_blk0;
            for (int64_t w = w0; w < w1; ++w, ++k) {
                if (k >= YS && !mbar_wait_or_abort(&yempty[yr.idx], yr.phase ^ 1u, &abort_sh)) {
                    abort_sh = 1;
                    break;
                }
                const int rs = slabs_of(blk);
                const uint32_t dst = base + (uint32_t)yr.idx * y_stage;
                mbar_expect_tx(&yfull[yr.idx], (uint32_t)rs * a_bytes);
                for (int q = 0; q < rs; ++q)
                    tma_load_2d(dst + (uint32_t)q * a_bytes, &tmY, &yfull[yr.idx],
                                (int32_t)((blk * R + q) * kTcK), (int32_t)(tile * kTcM));
                yr.next();
                if (++blk == a.Q) {
                    blk = 0;
                    ++tile;
                }
            }
            drain_ring(yfull, YS, k);   // no copy may be in flight when the CTA leaves
        }
    } else if (warp == 6) {
        // ---------------- centroid producer: one slab per stage
        if (lane == 0) {
            RingPos br(BS);
            int64_t j = 0, blk = w_blk0;
            bool ok = true;
            for (int64_t w = w0; w < w1 && ok; ++w) {
                const int rs = slabs_of(blk);
                for (int q = 0; q < rs; ++q, ++j) {
                    if (j >= BS && !mbar_wait_or_abort(&bempty[br.idx], br.phase ^ 1u, &abort_sh)) {
                        abort_sh = 1;
                        ok = false;
                        break;
                    }
                    const int32_t row = (int32_t)((blk * R + q) * kTcK);
                    const uint32_t dst = b_base + (uint32_t)br.idx * 2 * b_bytes;
                    mbar_expect_tx(&bfull[br.idx], 2 * b_bytes);
                    tma_load_2d(dst, &tmBh, &bfull[br.idx], row, 0);
                    tma_load_2d(dst + b_bytes, &tmBl, &bfull[br.idx], row, 0);
                    br.next();
                }
                if (++blk == a.Q) blk = 0;
            }
            drain_ring(bfull, BS, j);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(kTcM, a.Npad);
            const uint64_t dY = sw128_desc(base), dB = sw128_desc(b_base);
            const uint32_t y16 = y_stage >> 4, a16 = a_bytes >> 4, b16 = b_bytes >> 4;
            RingPos yr(YS), br(BS), ar(NA);
            int64_t g = 0, blk = w_blk0;
            bool ok = true;
            uint64_t* last_bar = nullptr;   // barrier of the latest commit and its phase
            uint32_t last_par = 0;
            for (int64_t w = w0; w < w1 && ok; ++w) {
                const int rs = slabs_of(blk);
                const bool seg_start = (w == w0) || (blk == 0);
                const bool seg_end = (w == w1 - 1) || (blk == a.Q - 1);
                if (seg_start && g >= NA &&
                    !mbar_wait_or_abort(&acc_empty[ar.idx], ar.phase ^ 1u, &abort_sh)) {
                    abort_sh = 1;
                    break;
                }
                if (!mbar_wait_or_abort(&yfull[yr.idx], yr.phase, &abort_sh)) {
                    abort_sh = 1;
                    break;
                }
                const uint32_t acc = tmem + (uint32_t)(ar.idx * a.Npad);
                uint64_t dA = dY + (uint64_t)(yr.idx * y16);
                for (int q = 0; q < rs; ++q, dA += a16) {
                    if (!mbar_wait_or_abort(&bfull[br.idx], br.phase, &abort_sh) ||
                        !mbar_wait_or_abort(&conv[br.idx], br.phase, &abort_sh)) {
                        abort_sh = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t dBh = dB + (uint64_t)(br.idx * 2 * b16), dBl = dBh + b16;
                    const uint32_t alo = tmem + a.lo_col + (uint32_t)(br.idx * 32);
                    const uint32_t first = (seg_start && q == 0) ? 0u : 1u;
#pragma unroll
                    for (int ks = 0; ks < kTcK / 8; ++ks) {
                        // 8 TF32 of K = 32 bytes = 2 descriptor address units
                        tc_mma(acc, dA + 2 * ks, dBh + 2 * ks, idesc, ks == 0 ? first : 1u);
                        tc_mma(acc, dA + 2 * ks, dBl + 2 * ks, idesc, 1u);
                        tc_mma_tmem_a(acc, alo + (uint32_t)(ks * 8), dBh + 2 * ks, idesc, 1u);
                    }
                    tc_commit(&bempty[br.idx]);
                    last_bar = &bempty[br.idx];
                    last_par = br.phase;
                    br.next();
                }
                if (!ok) break;
                tc_commit(&yempty[yr.idx]);
                last_bar = &yempty[yr.idx];
                last_par = yr.phase;
                yr.next();
                if (seg_end) {
                    tc_commit(&acc_full[ar.idx]);
                    ar.next();
                    ++g;
                }
                if (++blk == a.Q) blk = 0;
            }
            // drain: the last commit covers every MMA issued before it
            if (last_bar) mbar_wait(last_bar, last_par);
        }
    } else {
        // ---------------- TF32 lo split + epilogue (warps 2-5; row m = TMEM lane)
        const int m = 32 * (warp & 3) + lane;
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        const int et = tid - 64;   // 0..127
        RingPos yr(YS), br(BS), ar(NA);
        int64_t j = 0, tile = w_tile0, blk = w_blk0;
        float ysq = 0.f, ycomp = 0.f;
        bool ok = true;
        for (int64_t w = w0; w < w1 && ok; ++w) {
            const int rs = slabs_of(blk);
            const bool seg_start = (w == w0) || (blk == 0);
            const bool seg_end = (w == w1 - 1) || (blk == a.Q - 1);
            if (seg_start) ysq = ycomp = 0.f;
            if (!mbar_wait_or_abort(&yfull[yr.idx], yr.phase, &abort_sh)) {
                abort_sh = 1;
                break;
            }
            const uint32_t ybase = base + (uint32_t)yr.idx * y_stage;
            for (int q = 0; q < rs; ++q, ++j) {
                // the lo stage is free once the MMAs of slab j - BS are done
                if (j >= BS && !mbar_wait_or_abort(&bempty[br.idx], br.phase ^ 1u, &abort_sh)) {
                    abort_sh = 1;
                    ok = false;
                    break;
                }
                float part = 0.f;
                uint32_t r[32];
                const uint32_t src = ybase + (uint32_t)q * a_bytes;
#pragma unroll
                for (int qq = 0; qq < 8; ++qq) {
                    // the raw tile stays as the hi operand (the MMA truncates it)
                    const float4 x = ld_shared_v4(src + sw128_off(m, qq));
                    r[4 * qq + 0] = __float_as_uint(x.x - tf32_hi(x.x));
                    r[4 * qq + 1] = __float_as_uint(x.y - tf32_hi(x.y));
                    r[4 * qq + 2] = __float_as_uint(x.z - tf32_hi(x.z));
                    r[4 * qq + 3] = __float_as_uint(x.w - tf32_hi(x.w));
                    part = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, part))));
                }
                tc_st32(tmem + lane_base + a.lo_col + (uint32_t)(br.idx * 32), r);
                const float y = part - ycomp;   // Kahan accumulation of ||y_j||^2
                const float t = ysq + y;
                ycomp = (t - ysq) - y;
                ysq = t;
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&conv[br.idx]);
                br.next();
            }
            yr.next();
            const int64_t cur_tile = tile;
            if (++blk == a.Q) {
                blk = 0;
                ++tile;
            }
            if (!ok || !seg_end) continue;

            // a column tile segment is finished: drain its accumulator
            if (!mbar_wait_or_abort(&acc_full[ar.idx], ar.phase, &abort_sh)) {
                abort_sh = 1;
                break;
            }
            tc_fence_after();
            const int64_t bfirst = sk_owner(cur_tile * a.Q, a.W, G);
            const int64_t blast = sk_owner((cur_tile + 1) * a.Q - 1, a.W, G);
            const int slot = (int)(b - bfirst);
            const int ncontrib = (int)(blast - bfirst + 1);
            float* gslot = Gpart + ((int64_t)cur_tile * a.cmax + slot) * (int64_t)a.Npad * kTcM;
            const uint32_t acc = (uint32_t)(ar.idx * a.Npad);
            for (int cb = 0; cb < a.Npad; cb += 16) {
                float vv[16];
                tc_ld16(tmem + lane_base + acc + (uint32_t)cb, vv);
#pragma unroll
                for (int q = 0; q < 16; ++q) gslot[(int64_t)(cb + q) * kTcM + m] = vv[q];
            }
            ynorm_part[((int64_t)cur_tile * a.cmax + slot) * kTcM + m] = ysq;
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[ar.idx]);
            ar.next();
            __threadfence();
            named_sync(1, 128);
            if (et == 0) {
                const int prev = atomicAdd(&tile_count[cur_tile], 1);
                is_last_sh = (prev == ncontrib - 1);
            }
            named_sync(1, 128);
            const bool last = is_last_sh != 0;
            named_sync(1, 128);
            if (!last) continue;
            __threadfence();
            if (et == 0) tile_count[cur_tile] = 0;
            const int64_t p = cur_tile * kTcM + m;
            if (p < a.n) {
                const float* gt0 = Gpart + (int64_t)cur_tile * a.cmax * (int64_t)a.Npad * kTcM;
                const float* yt0 = ynorm_part + (int64_t)cur_tile * a.cmax * kTcM;
                float y2 = 0.f;
                for (int sl = 0; sl < ncontrib; ++sl) y2 += __ldcg(yt0 + (int64_t)sl * kTcM + m);
                finalize_column(p, y2, gt0, ncontrib, a.Npad, m, mu_normf, counts, c, labels, ub, lb,
                                status, rc_list);
            }
        }
    }
    __syncthreads();
    if (abort_sh && tid == 0) atomicOr(&status->timeout, 1);
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, a.tmem_cols);
}

// ============================================================== dense kernel, operands swapped
// For c <= 128 the centroids are the M = 128 operand and 256 data columns the
// N operand, so each MMA instruction covers four times the columns of the
// N = Npad form above (whose rate the issuing thread's per-instruction cost
// bounds).  A = mu_a slabs: for Npad <= 64 ("stacked") rows 0..63 hold the raw
// centroids (the MMA's hi part) and rows 64..127 their TF32 lo parts, and one
// MMA per 8 rows against the raw Y (which the MMA truncates to TF32) gives
//   D[i] + D[64 + i] = mu_hi.y_hi + mu_lo.y_hi;
// the missing mu.y_lo is at most ||mu|| ||y - tf32(y)|| (Cauchy-Schwarz; the
// split warps sum ||y - tf32(y)||^2 per column, at most 2^-10 ||y||) and widens
// the score bound (score_err's ylo), so the near ties it can hide are
// re-decided exactly.  For 64 < Npad <= 128 the A operand is two 128-row slabs
// per stage, A1 = raw centroids and A2 = their lo parts, and two MMAs per 8
// rows (A1.Y_raw, A2.Y_raw) give D[i] = mu_hi.y_hi + mu_lo.y_hi with the same
// bound.  No y_lo slab is formed, so the stages fill shared memory: four of
// 48 KB (stacked) or three of 64 KB.
//   warp 0: TMA producer (Y slab + A slab(s) per stage), warp 1: MMA issuer,
//   warps 2-5: ||y||^2 and ||y - tf32(y)||^2 sums (2 columns per thread) and
//   the epilogue (partials to Gpart).
// The scores, argmin and bounds follow in k_finalize_t, one thread per
// column: done by the last CTA of a tile, the slot sums of 256 columns sat
// on that CTA's critical path.
// A CTA's stream-K units [w0, w1), walked forward, or backward on alternate
// passes: a pass then starts on the units the previous one read last, which the
// L2 may still hold.  Tiles, 32-row blocks and the segment boundaries (the first
// and last unit of a tile in walking order) advance without divisions.
struct UnitWalk {
    int64_t tile, blk, left, Q;
    bool rev, first;
    __device__ UnitWalk(int64_t w0, int64_t w1, int64_t Q_, bool rev_)
        : left(w1 - w0), Q(Q_), rev(rev_), first(true) {
        const int64_t w = rev ? w1 - 1 : w0;
        tile = w / Q;
        blk = w - tile * Q;
    }
    __device__ __forceinline__ bool seg_start() const { return first || blk == (rev ? Q - 1 : 0); }
    __device__ __forceinline__ bool seg_end() const { return left == 1 || blk == (rev ? 0 : Q - 1); }
    __device__ __forceinline__ void next() {
        --left;
        first = false;
        if (rev) {
            if (blk == 0) {
                blk = Q - 1;
                --tile;
            } else {
                --blk;
            }
        } else if (++blk == Q) {
            blk = 0;
            ++tile;
        }
    }
};

constexpr int kTtN = 256;          // data columns per tile (MMA N)
constexpr int kTtThreads = 192;
constexpr int kTtMaxS = 4;

// ymode: what bounds ||y - y~|| for the operand y~ the products use.
//   0: FP32 operand truncated to TF32 by the MMA; the kernel sums ||y - tf32(y)||^2.
//   1: 16-bit operand that is the data itself (y~ = y).
//   2: FP16 copy fp16(s y) of FP32 data y, s = status->sh_scale; ycol[j] bounds
//      ||y_j - y~_j|| and ycol[n + j] is ||y~_j||^2 (y~ = copy / s; both formed where
//      the copy is written, so the kernel reads no norms from its stages), the
//      products carry s^2, and the distances are bounded through y~.
// With 16-bit operands the centroids are split into two 16-bit parts whose
// sum is within a16_err[i] of mu_i (exact norm of the split's error, bounded).
struct DenseTArgs {
    int64_t d, n, Q, T, W;   // rows, columns, slabs per tile, 256-column tiles, work units
    int Npad, stacked, S, cmax;
    int use_list;
    int64_t list_min;
    int ymode;
    const float* ycol;
    const float* a16_err;
};

// Adds the squares of the eight 16-bit values of a 16-byte chunk to acc.
template <typename TY>
__device__ __forceinline__ float sq8(const uint4 u, float acc) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float a, b;
        if constexpr (std::is_same<TY, __nv_bfloat16>::value) {
            a = __uint_as_float(w[k] << 16);
            b = __uint_as_float(w[k] & 0xFFFF0000u);
        } else {
            const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[k]));
            a = f.x;
            b = f.y;
        }
        acc = fmaf(a, a, fmaf(b, b, acc));
    }
    return acc;
}

template <typename TY>
__global__ void __launch_bounds__(kTtThreads, 1)
    k_search_dense_t(const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmA,
                     DenseTArgs a, DevStatus* __restrict__ status, const float* __restrict__ mu_normf,
                     const int32_t* __restrict__ counts, int c, int32_t* __restrict__ labels,
                     float* __restrict__ ub, float* __restrict__ lb, float* __restrict__ Gpart,
                     float* __restrict__ ynorm_part, int32_t* __restrict__ tile_count,
                     RcQueue rc_list) {
    extern __shared__ uint8_t smem_raw[];
    // conv: the norm warps are done with a stage (one per stage, so that a barrier can never
    // complete twice before the MMA warp waits on it)
    __shared__ uint64_t full[kTtMaxS], empty[kTtMaxS], conv[kTtMaxS], acc_full[2], acc_empty[2];
    __shared__ float xch[64][17];   // lo rows handed to the hi rows in the epilogue (stacked)
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_sh;

    if (a.use_list && (int64_t)status->flagged < a.list_min) return;   // the list kernel handles it
    const int64_t G = gridDim.x, b = blockIdx.x;
    const int64_t w0 = sk_begin(b, a.W, G), w1 = sk_begin(b + 1, a.W, G);
    if (w0 >= w1) return;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    constexpr bool k16 = sizeof(TY) == 2;
    constexpr int kRows = 128 / (int)sizeof(TY);      // d rows per slab: one 128-byte swizzle row
    const int S = a.S;
    const int na = a.stacked ? 1 : 2;                 // A slabs per stage
    const uint32_t y_bytes = kTtN * 128;              // 256 columns x 128 bytes
    const uint32_t a_bytes = 128 * 128;               // 128 centroid rows x 32 rows
    const uint32_t stage_bytes = y_bytes + (uint32_t)na * a_bytes;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    // walk backwards on every other all-column pass (the finalize counts them)
    const bool rev = (status->dense_passes & 1) != 0;
    constexpr uint32_t kTmemCols = 512;                // two 128 x 256 FP32 accumulators
    const bool norms = a.ymode != 2;                  // column norms from the stages (not given)

    if (warp == 1) {
        tmem_alloc(&tmem_base_sh, kTmemCols);
        tc_fence_before();
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
            mbar_init(&conv[s], 4);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&acc_full[s], 1);
            mbar_init(&acc_empty[s], 4);
        }
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            RingPos sr(S);
            UnitWalk uw(w0, w1, a.Q, rev);
            int64_t k = 0;
            for (int64_t w = w0; w < w1; ++w, ++k) {
                if (k >= S && !mbar_wait_or_abort(&empty[sr.idx], sr.phase ^ 1u, &abort_sh)) {
                    abort_sh = 1;
                    break;
                }
                const uint32_t dst = base + (uint32_t)sr.idx * stage_bytes;
                const int32_t row = (int32_t)(uw.blk * kRows);
                mbar_expect_tx(&full[sr.idx], stage_bytes);
                tma_load_2d(dst, &tmY, &full[sr.idx], row, (int32_t)(uw.tile * kTtN));
                tma_load_2d(dst + y_bytes, &tmA, &full[sr.idx], row, 0);
                if (na == 2) tma_load_2d(dst + y_bytes + a_bytes, &tmA, &full[sr.idx], row, 128);
                sr.next();
                uw.next();
            }
            drain_ring(full, S, k);   // no copy may be in flight when the CTA leaves
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = k16 ? idesc_f16(128, kTtN, std::is_same<TY, __nv_bfloat16>::value)
                                       : idesc_tf32(128, kTtN);
            const uint64_t dY0 = sw128_desc(base);
            const uint32_t st16 = stage_bytes >> 4, y16 = y_bytes >> 4, a16 = a_bytes >> 4;
            RingPos sr(S), ar(2);
            UnitWalk uw(w0, w1, a.Q, rev);
            int64_t g = 0;
            uint64_t* last_bar = nullptr;
            uint32_t last_par = 0;
            for (int64_t w = w0; w < w1; ++w) {
                const bool seg_start = uw.seg_start();
                const bool seg_end = uw.seg_end();
                if (seg_start && g >= 2 &&
                    !mbar_wait_or_abort(&acc_empty[ar.idx], ar.phase ^ 1u, &abort_sh)) {
                    abort_sh = 1;
                    break;
                }
                if (!mbar_wait_or_abort(&full[sr.idx], sr.phase, &abort_sh) ||
                    (norms && !mbar_wait_or_abort(&conv[sr.idx], sr.phase, &abort_sh))) {
                    abort_sh = 1;
                    break;
                }
                tc_fence_after();
                const uint64_t dY = dY0 + (uint64_t)(sr.idx * st16);
                const uint64_t dA1 = dY + y16, dA2 = dA1 + a16;
                const uint32_t acc = tmem + (uint32_t)(ar.idx * kTtN);
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    // 8 TF32 or 16 16-bit values of K = 32 bytes = 2 descriptor address units
                    if constexpr (k16) {
                        tc_mma_f16(acc, dA1 + 2 * ks, dY + 2 * ks, idesc, (seg_start && ks == 0) ? 0u : 1u);
                        if (na == 2) tc_mma_f16(acc, dA2 + 2 * ks, dY + 2 * ks, idesc, 1u);
                    } else {
                        tc_mma(acc, dA1 + 2 * ks, dY + 2 * ks, idesc, (seg_start && ks == 0) ? 0u : 1u);
                        if (na == 2) tc_mma(acc, dA2 + 2 * ks, dY + 2 * ks, idesc, 1u);
                    }
                }
                tc_commit(&empty[sr.idx]);
                last_bar = &empty[sr.idx];
                last_par = sr.phase;
                sr.next();
                if (seg_end) {
                    tc_commit(&acc_full[ar.idx]);
                    ar.next();
                    ++g;
                }
                uw.next();
            }
            // drain: the last commit covers every MMA issued before it
            if (last_bar) mbar_wait(last_bar, last_par);
        }
    } else {
        // ---------------- column norms + epilogue (warps 2-5)
        const int m = 32 * (warp & 3) + lane;          // this thread's columns: m and m + 128
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        RingPos sr(S), ar(2);
        UnitWalk uw(w0, w1, a.Q, rev);
        float ysq[2] = {0.f, 0.f}, ycomp[2] = {0.f, 0.f}, ylo2[2] = {0.f, 0.f};
        // drains a finished tile segment's accumulator (lane = A row) into Gpart, with
        // this thread's column-norm partials when the kernel forms them
        auto epilogue = [&](int64_t cur_tile) {
            const int slot = (int)(b - sk_owner(cur_tile * a.Q, a.W, G));
            // stacked: row i + 64 (lo part) is added into row i before the store
            const int rows_out = a.stacked ? 64 : 128;
            const bool lo_row = a.stacked && m >= 64;
            float* grow = Gpart + (((int64_t)cur_tile * a.cmax + slot) * rows_out + (m & (rows_out - 1))) * kTtN;
            for (int cb = 0; cb < kTtN; cb += 16) {
                float vv[16];
                tc_ld16(tmem + lane_base + (uint32_t)(ar.idx * kTtN + cb), vv);
                if (a.stacked) {
                    if (lo_row) {
#pragma unroll
                        for (int q = 0; q < 16; ++q) xch[m - 64][q] = vv[q];
                    }
                    named_sync(1, 128);
                    if (!lo_row) {
#pragma unroll
                        for (int q = 0; q < 16; ++q) vv[q] += xch[m][q];
                    }
                    named_sync(1, 128);
                }
                if (!lo_row) {
#pragma unroll
                    for (int q = 0; q < 16; q += 4)
                        *reinterpret_cast<float4*>(grow + cb + q) = make_float4(vv[q], vv[q + 1], vv[q + 2], vv[q + 3]);
                }
            }
            if (!norms) return;
            float* yn = ynorm_part + ((int64_t)cur_tile * a.cmax + slot) * kTtN;
            yn[m] = ysq[0];
            yn[m + 128] = ysq[1];
            if (!k16) {
                float* yl = yn + a.T * a.cmax * kTtN;   // ||y - tf32(y)||^2 partials in the second half
                yl[m] = ylo2[0];
                yl[m + 128] = ylo2[1];
            }
        };
        for (int64_t w = w0; w < w1; ++w) {
            const bool seg_start = uw.seg_start();
            const bool seg_end = uw.seg_end();
            if (seg_start) ysq[0] = ysq[1] = ycomp[0] = ycomp[1] = ylo2[0] = ylo2[1] = 0.f;
            if (!norms) {   // only the epilogue
                const int64_t cur_tile = uw.tile;
                uw.next();
                if (!seg_end) continue;
                if (!mbar_wait_or_abort(&acc_full[ar.idx], ar.phase, &abort_sh)) {
                    abort_sh = 1;
                    break;
                }
                tc_fence_after();
                epilogue(cur_tile);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[ar.idx]);
                ar.next();
                continue;
            }
            if (!mbar_wait_or_abort(&full[sr.idx], sr.phase, &abort_sh)) {
                abort_sh = 1;
                break;
            }
            const uint32_t ysrc = base + (uint32_t)sr.idx * stage_bytes;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = m + 128 * h;
                float part = 0.f;
                if constexpr (k16) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) part = sq8<TY>(ld_shared_u4(ysrc + sw128_off(row, q)), part);
                } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const uint32_t off = sw128_off(row, q);
                    const float4 x = ld_shared_v4(ysrc + off);
                    const float4 lo = make_float4(x.x - tf32_hi(x.x), x.y - tf32_hi(x.y), x.z - tf32_hi(x.z),
                                                  x.w - tf32_hi(x.w));
                    ylo2[h] = fmaf(lo.x, lo.x, fmaf(lo.y, lo.y, fmaf(lo.z, lo.z, fmaf(lo.w, lo.w, ylo2[h]))));
                    part = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, part))));
                }
                }
                const float y = part - ycomp[h];   // Kahan accumulation of ||y_j||^2
                const float t = ysq[h] + y;
                ycomp[h] = (t - ysq[h]) - y;
                ysq[h] = t;
            }
            // this stage's reads are ordered before the TMA overwrite the MMA's commit releases
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&conv[sr.idx]);
            sr.next();
            const int64_t cur_tile = uw.tile;
            uw.next();
            if (!seg_end) continue;

            // a tile segment is finished: drain its accumulator (lane = A row)
            if (!mbar_wait_or_abort(&acc_full[ar.idx], ar.phase, &abort_sh)) {
                abort_sh = 1;
                break;
            }
            tc_fence_after();
            epilogue(cur_tile);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[ar.idx]);
            ar.next();
        }
    }
    __syncthreads();
    if (abort_sh && tid == 0) atomicOr(&status->timeout, 1);
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, kTmemCols);
}

// Scores, argmin (ties to the lowest index), near-tie queue and bounds of
// every column from the swapped kernel's partials [tile][slot][rows][256]
// (rows = 64 when stacked, hi and lo parts already added; else 128).
// A block takes 16 columns of one tile: its 256 threads first sum the
// partials over the tile's slots (in slot order, hi and lo rows together)
// into shared memory, with coalesced and mutually independent loads; then one
// warp per column scores it from there.  Small blocks keep several per SM
// resident, so one wave covers n = 10^4 and their latencies overlap.
constexpr int kFinCols = 16, kFinThreads = 256;
// five blocks per SM (at most 48 registers): 625 blocks cover n = 10^4 in one wave
__global__ void __launch_bounds__(kFinThreads, 5)
    k_finalize_t(DenseTArgs a, int G, DevStatus* __restrict__ status, const float* __restrict__ mu_normf,
                 const int32_t* __restrict__ counts, int c, int32_t* __restrict__ labels,
                 float* __restrict__ ub, float* __restrict__ lb, const float* __restrict__ Gpart,
                 const float* __restrict__ ynorm_part, RcQueue rc_list) {
    constexpr int kGs = kFinCols + 1;       // row stride: the warps' lanes read down a column
    __shared__ float gs[128 * kGs];        // [centroid][column]
    __shared__ float ys[kFinCols], ylos[kFinCols], yshs[kFinCols];
    if (a.use_list && (int64_t)status->flagged < a.list_min) return;   // the dense kernel did not run
    if (blockIdx.x == 0 && threadIdx.x == 0) ++status->dense_passes;   // its walking direction alternates
    const int64_t col0 = (int64_t)blockIdx.x * kFinCols;
    const int64_t tile = col0 / kTtN;                 // kFinCols divides kTtN
    const int jc0 = (int)(col0 - tile * kTtN);
    const int64_t bfirst = sk_owner(tile * a.Q, a.W, G);
    const int64_t blast = sk_owner((tile + 1) * a.Q - 1, a.W, G);
    const int ncontrib = (int)(blast - bfirst + 1);
    const int t = threadIdx.x;
    const int jl = t % kFinCols;
    // the centroids' norms and counts first: their loads overlap the partial sums'
    float mu2v[4], serr[4];
    bool okv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = (t & 31) + 32 * q;
        okv[q] = i < c && __ldg(counts + i) != 0;
        mu2v[q] = i < c ? __ldg(mu_normf + i) : 0.f;
        serr[q] = (a.ymode != 0 && i < c) ? __ldg(a.a16_err + i) : 0.f;
    }
    // the FP16 copy's products carry s^2 (s a power of two: exact)
    const float inv2 = a.ymode == 2 ? status->sh_inv2 : 1.f;
    const int rows = a.stacked ? 64 : 128;   // the stacked kernel has added the lo rows in
    const float* gt = Gpart + (int64_t)tile * a.cmax * rows * kTtN + jc0 + jl;
    const int64_t slot_stride = (int64_t)rows * kTtN;
    for (int i = t / kFinCols; i < c; i += kFinThreads / kFinCols) {
        float v = 0.f;
#pragma unroll 4
        for (int sl = 0; sl < ncontrib; ++sl) v += __ldcg(gt + sl * slot_stride + (int64_t)i * kTtN);
        gs[i * kGs + jl] = v * inv2;
    }
    if (t < kFinCols) {
        const float* yt = ynorm_part + (int64_t)tile * a.cmax * kTtN + jc0 + t;
        float y2 = 0.f;
        if (a.ymode == 2) {   // ||y~||^2 formed with the copy
            if (col0 + t < a.n) y2 = __ldg(a.ycol + a.n + col0 + t);
        } else {
            for (int sl = 0; sl < ncontrib; ++sl) y2 += __ldcg(yt + (int64_t)sl * kTtN);
        }
        ys[t] = y2;
        if (a.ymode == 0) {
            // ||y - tf32(y)||: FP32 sums of at most d squares, so the norm is
            // inflated by d 2^-24 to stay an upper bound
            const float* ylt = yt + a.T * a.cmax * kTtN;
            float l2 = 0.f;
            for (int sl = 0; sl < ncontrib; ++sl) l2 += __ldcg(ylt + (int64_t)sl * kTtN);
            ylos[t] = sqrtf(l2) * (1.f + (float)(a.d + 64) * 5.9604645e-8f);
            yshs[t] = 0.f;
        } else {
            const int64_t col = col0 + t;
            ylos[t] = 0.f;
            yshs[t] = (a.ymode == 2 && col < a.n) ? __ldg(a.ycol + col) : 0.f;
        }
    }
    __syncthreads();
    // one warp per column (two columns per warp), lanes over the centroids
    constexpr int kColsPerWarp = kFinCols / (kFinThreads / 32);
    const int warp = t >> 5;
#pragma unroll
    for (int k2 = 0; k2 < kColsPerWarp; ++k2) {
        const int jw = warp * kColsPerWarp + k2;
        const int64_t p = col0 + jw;
        if (p >= a.n) break;
        finalize_warp(p, ys[jw], ylos[jw], yshs[jw], [&](int i) { return gs[i * kGs + jw]; }, mu2v, serr, okv, c,
                      labels, ub, lb,
                      status, rc_list);
    }
}

// ============================================================== exact recheck
// Squared distance ||y - mu_i||^2 by a whole CTA, to about 2^-43 relative, in
// double-float FP32 arithmetic (the FP64 pipe of this part runs about 2 FMA
// per clock per SM, 64 times below FP32):
//   e_h + e_l = y - mu exactly (Knuth's TwoSum), e_h^2 = p + p_err exactly
//   (product with an FMA), the rest 2 e_h e_l + e_l^2 + p_err is < 2^-22 of
//   p; the running sum is carried as s_h + s_l with TwoSum on s_h + p.
// The threads' (s_h, s_l) pairs meet across each warp in the same double-float
// form (TwoSum on the high parts, which is exact and symmetric, so every lane of
// the butterfly ends with the same pair); thread 0 adds the 8 warp totals in FP64.
// Equal inputs give bit-identical results, so exact ties (repeated columns)
// stay ties and go to the lowest index.
struct DfSum {
    float h = 0.f, l = 0.f;
    // explicitly rounded operations: a contraction into an FMA would break
    // the error-free transformations
    __device__ __forceinline__ void add_sq_diff(float yv, float mv) {
        const float e = __fsub_rn(yv, mv);
        const float bv = __fsub_rn(e, yv);
        const float el = __fadd_rn(__fsub_rn(yv, __fsub_rn(e, bv)), __fsub_rn(-mv, bv));  // e + el = yv - mv
        const float p = __fmul_rn(e, e);
        const float pe = fmaf(e, e, -p);                                               // e^2 = p + pe
        const float low = fmaf(2.f * e, el, pe) + el * el;
        const float t = __fadd_rn(h, p);                                               // TwoSum(h, p)
        const float bp = __fsub_rn(t, h);
        l += __fadd_rn(__fsub_rn(h, __fsub_rn(t, bp)), __fsub_rn(p, bp)) + low;
        h = t;
    }
    // (h, l) += (oh, ol): TwoSum on the high parts, the low parts added
    __device__ __forceinline__ void merge(float oh, float ol) {
        const float t = __fadd_rn(h, oh);
        const float bp = __fsub_rn(t, h);
        l = __fadd_rn(__fadd_rn(l, ol), __fadd_rn(__fsub_rn(h, __fsub_rn(t, bp)), __fsub_rn(oh, bp)));
        h = t;
    }
};

// 16-byte read-only global load that the compiler keeps in program order.
__device__ __forceinline__ float4 ld_nc_v4(const float4* p) {
    float4 v;
    asm volatile("ld.global.nc.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

// Returns the distance in thread 0 (0 in the other threads).
template <typename TY>
__device__ double block_dist2_exact(const TY* __restrict__ y, const float* __restrict__ mrow, int64_t d,
                                    bool vec, double* red) {
    DfSum a0, a1, a2, a3;
    if (vec && sizeof(TY) == 4) {
        const float4* y4 = reinterpret_cast<const float4*>(y);
        const float4* m4 = reinterpret_cast<const float4*>(mrow);
        const int64_t d4 = d / 4;
        // twelve 16-byte loads of each operand in flight per round: d up to 12288 is
        // one memory round trip; four independent TwoSum chains
        for (int64_t b0 = threadIdx.x; b0 < d4; b0 += 12 * kThreads) {
            float4 yv[12], mv[12];
            // volatile loads keep their order ahead of the arithmetic below, so all 24
            // are in flight together; out-of-range slots load the last vector and are
            // zeroed afterwards
#pragma unroll
            for (int u = 0; u < 12; ++u) {
                const int64_t j = min(b0 + u * kThreads, d4 - 1);
                yv[u] = ld_nc_v4(y4 + j);
                mv[u] = ld_nc_v4(m4 + j);
            }
#pragma unroll
            for (int u = 0; u < 12; ++u)
                if (b0 + u * kThreads >= d4) yv[u] = mv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 12; ++u) {
                a0.add_sq_diff(yv[u].x, mv[u].x);
                a1.add_sq_diff(yv[u].y, mv[u].y);
                a2.add_sq_diff(yv[u].z, mv[u].z);
                a3.add_sq_diff(yv[u].w, mv[u].w);
            }
        }
        for (int64_t r = d4 * 4 + threadIdx.x; r < d; r += kThreads) a0.add_sq_diff(XLoad<TY>::one(y + r), mrow[r]);
    } else {
        for (int64_t r = threadIdx.x; r < d; r += kThreads) a0.add_sq_diff(XLoad<TY>::one(y + r), mrow[r]);
    }
    a0.merge(a1.h, a1.l);
    a2.merge(a3.h, a3.l);
    // the threads' sums meet in double-float FP32 across the warp (FP64 per thread
    // would load this GPU's narrow FP64 pipe with a whole block's worth of work);
    // only the warps' totals are added in FP64, by thread 0
    a0.merge(a2.h, a2.l);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, a0.h, o);
        const float ol = __shfl_xor_sync(0xffffffffu, a0.l, o);
        a0.merge(oh, ol);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)a0.h + (double)a0.l;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    return s;
}

// Exact re-decision of near ties, one launch.  The candidate distances of the
// first rc_cap queued columns are spread over every SM from the queue's pair
// list, one CTA per (column, candidate) pair; the CTA that computes a column's last candidate
// (a counter in the column's record) decides that column over its candidates
// in increasing index (ties keep the lowest), so no single CTA decides them
// all.  Columns queued beyond rc_cap are decided by one CTA each, candidate
// after candidate.
template <typename TY>
__global__ void __launch_bounds__(kThreads)
    k_search_recheck(const TY* __restrict__ Y, int64_t ldy, int64_t d, bool vec,
                     DevStatus* __restrict__ status, const float* __restrict__ mu, int c,
                     int32_t* __restrict__ labels, float* __restrict__ ub, float* __restrict__ lb,
                     RcRec* __restrict__ rc_list, const int32_t* __restrict__ rc_pairs,
                     double* __restrict__ rc_dist, int64_t rc_cap) {
    __shared__ double red[kThreads / 32];
    const int64_t nall = status->rechecked;
    if (nall == 0) return;
    const int64_t npairs = status->rc_pairs;   // the candidates of the first rc_cap records
    for (int64_t v = blockIdx.x; v < npairs; v += gridDim.x) {
        const int64_t pr = __ldcg(rc_pairs + v);
        const int64_t k = pr / c;
        const int ci = (int)(pr - k * c);
        RcRec* rec = rc_list + k;
        const double dist = block_dist2_exact<TY>(Y + (int64_t)rec->col * ldy, mu + (int64_t)ci * d, d, vec, red);
        if (threadIdx.x == 0) {
            rc_dist[pr] = dist;
            __threadfence();   // the distance is visible before this candidate counts as done
            int cand = 0;
            for (int w = 0; w < kTcMaxClusters / 32; ++w) cand += __popc(rec->mask[w]);
            if (atomicAdd(&rec->done, 1) == cand - 1) {
                // this CTA computed the column's last candidate: it decides the column
                // (lowest distance, ties to the lowest index)
                __threadfence();
                const int64_t col = rec->col;
                double best = INFINITY;
                int besti = INT_MAX;
                for (int cj = 0; cj < c; ++cj) {
                    if (!((rec->mask[cj >> 5] >> (cj & 31)) & 1u)) continue;
                    const double dj = cj == ci ? dist : __ldcg(rc_dist + k * c + cj);
                    if (dj < best) {
                        best = dj;
                        besti = cj;
                    }
                }
                if (besti < c) {
                    if (labels[col] != besti) {
                        labels[col] = besti;
                        atomicAdd(&status->changed, 1);
                    }
                    if (ub) {
                        ub[col] = (float)(sqrt(best) * (1.0 + 1e-6));
                        lb[col] = 0.f;
                    }
                }
            }
        }
        __syncthreads();
    }
    // records beyond the distance buffer: one CTA per column, every candidate in turn
    for (int64_t k = rc_cap + blockIdx.x; k < nall; k += gridDim.x) {
        const RcRec& rec = rc_list[k];
        const int64_t col = rec.col;
        const TY* y = Y + col * ldy;
        double best = INFINITY;
        int besti = INT_MAX;
        for (int ci = 0; ci < c; ++ci) {
            if (!((rec.mask[ci >> 5] >> (ci & 31)) & 1u)) continue;
            const double dist = block_dist2_exact<TY>(y, mu + (int64_t)ci * d, d, vec, red);
            if (dist < best) {
                best = dist;
                besti = ci;
            }
        }
        if (threadIdx.x == 0 && besti < c) {
            if (labels[col] != besti) {
                labels[col] = besti;
                atomicAdd(&status->changed, 1);
            }
            if (ub) {
                ub[col] = (float)(sqrt(best) * (1.0 + 1e-6));
                lb[col] = 0.f;
            }
        }
        __syncthreads();
    }
}

// TF32 hi / lo parts of the centroids, zero-padded to Npad rows of dpad; and,
// when mu_a is given, the A operand of the swapped dense kernel: for
// stacked (Npad <= 64) rows i = raw mu_i and 64 + i = lo(mu_i) over 64 rows,
// otherwise rows i = raw mu_i and 128 + i = lo(mu_i) over 128 rows (rows
// beyond c zero).  With s16.a16: the same rows as the two 16-bit parts of
// split16 over dpad16, and a16_err[i] from the squared errors of row i, summed
// per CTA and then in CTA order by the CTA that finishes the row last.
// Grid: (rows, CTAs per row), kSplitPer elements of a row per CTA.
constexpr int kSplitPer = kThreads * 8;

__global__ void __launch_bounds__(kThreads)
    k_mu_split(const float* __restrict__ mu, int c, int64_t d, int Npad, int64_t dpad,
               float* __restrict__ mu_hi, float* __restrict__ mu_lo, float* __restrict__ mu_a,
               int arows, MuSplitOut s16, float* __restrict__ part, int32_t* __restrict__ done) {
    __shared__ float red[kThreads / 32];
    __shared__ int last_sh;
    const int i = blockIdx.x;
    const int64_t dw = (s16.a16 && s16.dpad16 > dpad) ? s16.dpad16 : dpad;
    const int64_t r0 = (int64_t)blockIdx.y * kSplitPer;
    const int64_t r1 = r0 + kSplitPer < dw ? r0 + kSplitPer : dw;
    const float s = (s16.a16 && s16.a16_kind == 2) ? s16.status->sh_scale : 1.f;
    float e2 = 0.f;
    // the row chunk's loads first, all in flight together
    constexpr int kPer = kSplitPer / kThreads;
    float vv[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int64_t r = r0 + threadIdx.x + (int64_t)k * kThreads;
        vv[k] = (i < c && r < d && r < r1) ? __ldg(mu + (int64_t)i * d + r) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int64_t r = r0 + threadIdx.x + (int64_t)k * kThreads;
        if (r >= r1) break;
        const float v = vv[k];
        if (r < dpad) {
            const int64_t o = (int64_t)i * dpad + r;
            const float hi = tf32_hi(v);
            if (i < Npad) {
                mu_hi[o] = hi;
                mu_lo[o] = v - hi;
            }
            if (mu_a) {
                mu_a[o] = v;
                mu_a[(int64_t)arows * dpad + o] = v - hi;
            }
        }
        if (s16.a16 && r < s16.dpad16) {
            uint16_t p1, p2;
            split16(v, s16.a16_kind, s, p1, p2, e2);
            const int64_t o = (int64_t)i * s16.dpad16 + r;
            s16.a16[o] = p1;
            s16.a16[(int64_t)arows * s16.dpad16 + o] = p2;
        }
    }
    if (!s16.a16) return;
    e2 = warp_sum(e2);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e2;
    __syncthreads();
    const int S = gridDim.y;
    if (threadIdx.x == 0) {
        float b = 0.f;
        for (int w = 0; w < kThreads / 32; ++w) b += red[w];
        part[(int64_t)i * S + blockIdx.y] = b;
        __threadfence();
        last_sh = atomicAdd(&done[i], 1) == S - 1;
    }
    __syncthreads();
    if (!last_sh || threadIdx.x != 0) return;
    __threadfence();
    float tot = 0.f;
    for (int q = 0; q < S; ++q) tot += __ldcg(part + (int64_t)i * S + q);
    s16.a16_err[i] = split16_err(tot, d, s);
    done[i] = 0;
}

inline int grid_for(int64_t work, int per) { return (int)((work + per - 1) / per); }

struct DensePlan {
    int R, YS, BS, nacc;
    uint32_t lo_col, tmem_cols;
    int64_t nslab, Q, T, W;
    int G, cmax;
    size_t smem;
};

// Shape of the dense kernel's pipeline: the longest row block (R slabs, at
// most 4) whose two Y stages leave room for at least three centroid stages in
// 200 KB of shared memory (else R = 1 with two), as many centroid stages as
// fit (at most kDnMaxB), and two accumulators when they fit next to the y_lo
// ring in 512 TMEM columns.
DensePlan dense_plan(int64_t n, int64_t d, int Npad, int r_pref = 4, int ys_pref = 2) {
    DensePlan p;
    const size_t budget = 200 * 1024, a_bytes = (size_t)kTcM * 128, b_stage = 2 * (size_t)Npad * 128;
    p.YS = ys_pref;
    p.R = 1;
    for (int R = r_pref; R >= 1; --R) {
        const size_t y = (size_t)p.YS * R * a_bytes;
        if (y < budget && (budget - y) / b_stage >= 3) {
            p.R = R;
            break;
        }
    }
    p.BS = (int)std::min<size_t>(kDnMaxB, (budget - (size_t)p.YS * p.R * a_bytes) / b_stage);
    if (p.BS < 2) p.BS = 2;   // Npad <= 256 keeps this inside 227 KB
    p.nacc = (((2 * Npad + 31) / 32) * 32 + p.BS * 32 <= 512) ? 2 : 1;
    p.lo_col = (uint32_t)(((p.nacc * Npad) + 31) / 32 * 32);
    const uint32_t used = p.lo_col + (uint32_t)(p.BS * 32);
    p.tmem_cols = 32;
    while (p.tmem_cols < used) p.tmem_cols <<= 1;
    p.nslab = (d + kTcK - 1) / kTcK;
    p.Q = (p.nslab + p.R - 1) / p.R;
    p.T = (n + kTcM - 1) / kTcM;
    p.W = p.Q * p.T;
    p.G = (int)std::min<int64_t>(num_sms(), p.W);
    p.cmax = 1;
    for (int64_t t = 0; t < p.T; ++t) {
        const int64_t nc = sk_owner((t + 1) * p.Q - 1, p.W, p.G) - sk_owner(t * p.Q, p.W, p.G) + 1;
        if (nc > p.cmax) p.cmax = (int)nc;
    }
    p.smem = (size_t)p.YS * p.R * a_bytes + (size_t)p.BS * b_stage + 1024;
    return p;
}

struct DenseTPlan {
    int stacked, S, G, cmax;
    int64_t Q, T, W;
    size_t smem;
};

// Swapped dense kernel: 256-column tiles, slabs of one 128-byte row per column
// (32 FP32 or 64 16-bit rows: slab_rows); stages of (Y slab, A slab(s)).
DenseTPlan dense_t_plan(int64_t n, int64_t d, int Npad, int slab_rows = kTcK) {
    DenseTPlan p;
    p.stacked = Npad <= 64 ? 1 : 0;
    // products with y truncated to TF32 only (no y_lo slabs): four stages of 48 KB
    // (stacked) or three of 64 KB (two A slabs)
    p.S = p.stacked ? 4 : 3;
    const size_t y_bytes = (size_t)kTtN * 128, a_bytes = 128 * 128;
    const size_t stage = y_bytes + (p.stacked ? 1 : 2) * a_bytes;
    p.Q = (d + slab_rows - 1) / slab_rows;
    p.T = (n + kTtN - 1) / kTtN;
    p.W = p.Q * p.T;
    p.G = (int)std::min<int64_t>(num_sms(), p.W);
    p.cmax = 1;
    for (int64_t t = 0; t < p.T; ++t) {
        const int64_t nc = sk_owner((t + 1) * p.Q - 1, p.W, p.G) - sk_owner(t * p.Q, p.W, p.G) + 1;
        if (nc > p.cmax) p.cmax = (int)nc;
    }
    p.smem = (size_t)p.S * stage + 1024;
    return p;
}

}  // namespace

cudaError_t allow_max_dynamic_smem(const void* func) {
    static std::mutex mu;
    static std::vector<std::pair<const void*, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (const auto& d : done)
        if (d.first == func && d.second == dev) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return e;
    done.emplace_back(func, dev);
    return cudaSuccess;
}

int tc_npad(int c) { return ((c + 15) / 16) * 16; }

TcPlan tc_plan(int64_t n, int64_t d, int c) {
    TcPlan t;
    t.Npad = tc_npad(c);
    t.dpad = (d + 31) / 32 * 32;
    t.tiles = (n + kTcM - 1) / kTcM;
    const DensePlan dp = dense_plan(n, d, t.Npad);
    const int64_t slots = std::max<int64_t>(kTcMaxSplit, dp.cmax);
    t.gpart = (size_t)slots * t.Npad * t.tiles * kTcM;
    t.ynorm = (size_t)slots * t.tiles * kTcM;
    if (t.Npad <= 128) {   // the swapped kernel's partials: [tile][slot][128 rows][256 columns]
        for (int rows : {kTcK, 2 * kTcK}) {   // FP32 and 16-bit operands
            const DenseTPlan tp = dense_t_plan(n, d, t.Npad, rows);
            t.gpart = std::max(t.gpart, (size_t)tp.T * tp.cmax * 128 * kTtN);
            // two halves: ||y||^2 and ||y - tf32(y)||^2 partials
            t.ynorm = std::max(t.ynorm, (size_t)tp.T * tp.cmax * kTtN * 2);
        }
    }
    t.mu_a = (size_t)256 * t.dpad;
    t.dpad16 = (d + 63) / 64 * 64;
    t.mu_a16 = (size_t)256 * t.dpad16;
    t.rc_cap = std::min<int64_t>(n, 2048);
    return t;
}

int mu_split16_splits(int64_t d) {
    const int64_t dw = (d + 63) / 64 * 64;
    return (int)((dw + kSplitPer - 1) / kSplitPer);
}

cudaError_t launch_mu_split(const float* mu, int c, int64_t d, int Npad, int64_t dpad, float* mu_hi,
                            float* mu_lo, cudaStream_t st, float* mu_a, const MuSplitOut* sp16, float* part,
                            int32_t* done) {
    count_launches(1);
    const int arows = Npad <= 64 ? 64 : 128;
    const bool with_a = mu_a != nullptr && Npad <= 128;
    const int rows = with_a ? arows : Npad;
    MuSplitOut s16;
    if (with_a && sp16 && sp16->a16) s16 = *sp16;
    const int64_t dw = (s16.a16 && s16.dpad16 > dpad) ? s16.dpad16 : dpad;
    const dim3 grid((unsigned)rows, (unsigned)((dw + kSplitPer - 1) / kSplitPer));
    k_mu_split<<<grid, kThreads, 0, st>>>(mu, c, d, Npad, dpad, mu_hi, mu_lo, with_a ? mu_a : nullptr, arows,
                                          s16, part, done);
    return cudaGetLastError();
}

int64_t search_list_max(int64_t n, int c, bool op16) {
    // for c <= 128 (256 columns per MMA) the all-column pass plus its finalize
    // (~97 us at d = n = 10^4 with FP32 operands, ~55 us with 16-bit ones) beats
    // the gathered list kernel (~0.8 TB/s) from about n / 6 (n / 10) queued columns on
    if (tc_npad(c) > 128) return n / 4;
    return op16 ? n / 10 : n / 6;
}

cudaError_t launch_search_tc(int dtype, const void* Y, int64_t ldy, int64_t d, int64_t n,
                             const int32_t* list, DevStatus* status, const float* mu,
                             const float* mu_hi, const float* mu_lo, int64_t dpad,
                             const float* mu_normf, const int32_t* counts, int c, int32_t* labels,
                             float* ub, float* lb, float* Gpart, float* ynorm_part,
                             int32_t* tile_count, RcRec* rc_list, int32_t* rc_pairs, double* rc_dist, int64_t rc_cap,
                             bool vec, cudaStream_t st, cudaEvent_t ev_dense0, cudaEvent_t ev_dense1,
                             bool* dense_launched_out, const float* mu_a, const Search16* s16) {
    const int Npad = tc_npad(c);
    cudaError_t e = cudaSuccess;
    const RcQueue rq{rc_list, rc_pairs, rc_cap};
    // dense TMA path: FP32 operand with 16-byte aligned columns
    const bool dense_ok = dtype == 0 && vec && (reinterpret_cast<uintptr_t>(Y) % 16 == 0) &&
                          ldy % 4 == 0 && (reinterpret_cast<uintptr_t>(mu_hi) % 16 == 0) &&
                          (reinterpret_cast<uintptr_t>(mu_lo) % 16 == 0);
    // 16-bit all-column path: BF16 or FP16 columns (the data, or the FP16 copy of
    // FP32 data) and the centroids' split of the same type, 16-byte aligned columns
    const bool dense16 = s16 && s16->y16 && s16->a16 && s16->a16_err && Npad <= 128 &&
                         (reinterpret_cast<uintptr_t>(s16->y16) % 16 == 0) && s16->ld16 % 8 == 0 &&
                         (reinterpret_cast<uintptr_t>(s16->a16) % 16 == 0) && s16->dpad16 % 64 == 0;
    // larger queued lists use the dense kernel
    const int64_t list_max = search_list_max(n, c, dense16);
    bool dense_launched = false;
    // The start event goes into the stream before the host-side preparation of
    // the launch (tensor-map encoding, attributes), so that it is reached while
    // the preceding kernel still runs and brackets this kernel, not the host.
    const bool dense_t_path =
        dense16 || (dense_ok && Npad <= 128 && mu_a && (reinterpret_cast<uintptr_t>(mu_a) % 16 == 0));
    if (ev_dense0 && (dense_ok || dense16)) cudaEventRecord(ev_dense0, st);
    if (dense_t_path) {
        CUtensorMap tmY, tmA;
        const DenseTPlan dp = dense_t_plan(n, d, Npad, dense16 ? 2 * kTcK : kTcK);
        const bool enc_ok =
            dense16 ? (encode_2d_16(&tmY, s16->y16, !s16->fp16, d, n, s16->ld16, 2 * kTcK, kTtN) &&
                       encode_2d_16(&tmA, s16->a16, !s16->fp16, s16->dpad16, 256, s16->dpad16, 2 * kTcK, 128))
                    : (encode_2d(&tmY, static_cast<const float*>(Y), d, n, ldy, kTcK, kTtN) &&
                       encode_2d(&tmA, mu_a, dpad, 256, dpad, kTcK, 128));
        if (enc_ok) {
            DenseTArgs a;
            a.d = d;
            a.n = n;
            a.Q = dp.Q;
            a.T = dp.T;
            a.W = dp.W;
            a.Npad = Npad;
            a.stacked = dp.stacked;
            a.S = dp.S;
            a.cmax = dp.cmax;
            a.use_list = list ? 1 : 0;
            a.list_min = list_max + 1;
            a.ymode = dense16 ? (s16->ycol ? 2 : 1) : 0;
            a.ycol = dense16 ? s16->ycol : nullptr;
            a.a16_err = dense16 ? s16->a16_err : nullptr;
            auto kern = !dense16 ? k_search_dense_t<float>
                                 : (s16->fp16 ? k_search_dense_t<__half> : k_search_dense_t<__nv_bfloat16>);
            e = allow_max_dynamic_smem(reinterpret_cast<const void*>(kern));
            if (e != cudaSuccess) return e;
            count_launches(1);
            kern<<<dp.G, kTtThreads, dp.smem, st>>>(tmY, tmA, a, status, mu_normf, counts, c, labels, ub, lb,
                                                    Gpart, ynorm_part, tile_count, rq);
            if (ev_dense1) cudaEventRecord(ev_dense1, st);
            count_launches(1);
            k_finalize_t<<<grid_for(n, kFinCols), kFinThreads, 0, st>>>(a, dp.G, status, mu_normf, counts, c,
                                                                        labels, ub, lb, Gpart, ynorm_part,
                                                                        rq);
            dense_launched = true;
        }
    } else if (dense_ok) {
        CUtensorMap tmY, tmBh, tmBl;
        const DensePlan dp = dense_plan(n, d, Npad);
        if (encode_2d(&tmY, static_cast<const float*>(Y), d, n, ldy, kTcK, kTcM) &&
            encode_2d(&tmBh, mu_hi, dpad, Npad, dpad, kTcK, (uint32_t)Npad) &&
            encode_2d(&tmBl, mu_lo, dpad, Npad, dpad, kTcK, (uint32_t)Npad)) {
            DenseArgs a;
            a.d = d;
            a.n = n;
            a.Q = dp.Q;
            a.T = dp.T;
            a.W = dp.W;
            a.nslab = dp.nslab;
            a.Npad = Npad;
            a.R = dp.R;
            a.YS = dp.YS;
            a.BS = dp.BS;
            a.cmax = dp.cmax;
            a.nacc = dp.nacc;
            a.lo_col = dp.lo_col;
            a.tmem_cols = dp.tmem_cols;
            a.use_list = list ? 1 : 0;
            a.list_min = list_max + 1;
            e = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_search_dense));
            if (e != cudaSuccess) return e;
            count_launches(1);
            k_search_dense<<<dp.G, kDnThreads, dp.smem, st>>>(tmY, tmBh, tmBl, a, status, mu_normf,
                                                              counts, c, labels, ub, lb, Gpart,
                                                              ynorm_part, tile_count, rq);
            if (ev_dense1) cudaEventRecord(ev_dense1, st);
            dense_launched = true;
        }
    }
    if (!dense_launched || list) {
        const int64_t nslabs = (d + kTcK - 1) / kTcK;
        const int max_split = (int)std::min<int64_t>(kTcMaxSplit, nslabs);
        const size_t smem = (size_t)kTcStages * (2 * kTcM * 128 + 2 * (size_t)Npad * 128) + 1024;
        const int64_t lmax = dense_launched ? list_max : n;
        // tiles for at most lmax queued columns: beyond them the kernel would only
        // start CTAs that return at once (in a pass the dense kernel takes, all do)
        const dim3 grid((unsigned)((std::min(n, lmax) + kTcM - 1) / kTcM), (unsigned)max_split);
        count_launches(1);
        RESPCA_DISPATCH_X(dtype, TY, {
            auto kern = vec ? k_search_list<TY, true> : k_search_list<TY, false>;
            e = allow_max_dynamic_smem(reinterpret_cast<const void*>(kern));
            if (e == cudaSuccess)
                kern<<<grid, kTcThreads, smem, st>>>((const TY*)Y, ldy, d, n, list, lmax, status, mu_hi,
                                                     mu_lo, dpad, Npad, kTcMaxSplit, mu_normf, counts,
                                                     c, labels, ub, lb, Gpart, ynorm_part, tile_count,
                                                     rq);
        });
        if (e != cudaSuccess) return e;
    }
    if (dense_launched_out) *dense_launched_out = dense_launched;
    count_launches(1);
    RESPCA_DISPATCH_X(dtype, TY, {
        // float4 rows need 16-byte aligned columns of Y and of the centroids (d % 4 == 0)
        const bool v4 = vec && sizeof(TY) == 4 && (reinterpret_cast<uintptr_t>(Y) % 16 == 0) &&
                        (reinterpret_cast<uintptr_t>(mu) % 16 == 0);
        // one resident wave (the pairs are taken grid-stride): further waves would be CTAs
        // that find no pair (the FP32 form holds 171 registers, one CTA per SM)
        static const int per_sm = [] {
            int b = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_search_recheck<TY>, kThreads, 0) != cudaSuccess)
                b = 1;
            return std::min(4, std::max(1, b));
        }();
        k_search_recheck<TY><<<per_sm * num_sms(), kThreads, 0, st>>>((const TY*)Y, ldy, d, v4, status, mu, c,
                                                               labels, ub, lb, rc_list, rc_pairs, rc_dist,
                                                               rc_cap);
    });
    return cudaGetLastError();
}

}  // namespace respca
