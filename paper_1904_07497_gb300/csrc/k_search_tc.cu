// Nearest-centroid search on the 5th-generation tensor cores (sm_103a).
//
// The p step of Sec. 4.2 (Eq. (21)-(22)) needs, for every searched column y_j,
// the scores s_ij = ||mu_i||^2 - 2 mu_i . y_j over the c centroids: a
// (columns x d) . (d x c) product.  k_search_tc computes it with
// tcgen05.mma kind::tf32: A = 128 columns (M = 128, K-major: a column of Y is
// contiguous along d), B = the centroids padded to Npad (K-major), the FP32
// accumulator in tensor memory.  FP32 accuracy comes from the 3-term split
// y = y_hi + y_lo, mu = mu_hi + mu_lo (hi = TF32-truncated):
//   y.mu ~ y_hi.mu_hi + y_hi.mu_lo + y_lo.mu_hi       (error ~ 2^-20 relative).
// The d dimension is split over gridDim.y CTAs; each writes its partial dot
// products, and k_search_finalize adds them, forms the scores, takes the
// argmin (ties to the lowest index), re-decides near ties in FP64 (through
// k_search_recheck) and updates the labels and the pruning bounds.
//
// Shared-memory operands use the canonical K-major 128-byte-swizzle layout:
// 8-row groups of 1024 bytes, 128 bytes (32 FP32) per row, 16-byte chunk q of
// row m stored at chunk q ^ (m % 8).  Every wait on an mbarrier is bounded; a
// wait that gives up sets status->timeout and the kernel returns after
// releasing its tensor memory.
#include <cfloat>
#include <climits>

#include "respca_internal.cuh"

namespace respca {

namespace {

constexpr int kTcM = 128;             // columns per CTA (UMMA M)
constexpr int kTcK = 32;              // d rows per slab: one 128-byte swizzle atom of FP32
constexpr int kTcStages = 2;
constexpr int kTcThreads = 256;
constexpr unsigned kSpinLimit = 1u << 22;
constexpr float kTieRelTc = 6e-5f;    // bound on the score rounding, relative to ||y||^2 + ||mu||^2

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (the stride-dimension byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t desc = 0;
    desc |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    desc |= (uint64_t)1 << 16;
    desc |= (uint64_t)(1024 >> 4) << 32;
    desc |= (uint64_t)1 << 46;
    desc |= (uint64_t)2 << 61;
    return desc;
}

// Instruction descriptor: FP32 accumulator, A and B TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (unsigned i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// byte offset of 16-byte chunk q of row m in a K-major 128-byte-swizzle tile
__device__ __forceinline__ uint32_t sw128_off(int m, int q) {
    return (uint32_t)((m >> 3) * 1024 + (m & 7) * 128 + ((q ^ (m & 7)) << 4));
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, float4 v) {
    asm volatile("st.shared.v4.f32 [%0], {%1,%2,%3,%4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}

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

// Score rounding bound of centroid i for a column y: e_i = kTieRelTc *
// (2 ||mu_i|| ||y|| + ||mu_i||^2) (Cauchy-Schwarz on the products' error).
__device__ __forceinline__ float score_err(float mu2, float y2) {
    return kTieRelTc * (2.f * sqrtf(fmaxf(mu2, 0.f) * y2) + fabsf(mu2));
}

constexpr int kTcBMax = 4;   // prefetched 16-byte chunks of each centroid half per thread

template <typename TY, bool VEC>
__global__ void __launch_bounds__(kTcThreads, 2)
    k_search_tc(const TY* __restrict__ Y, int64_t ldy, int64_t d, int64_t n,
                const int32_t* __restrict__ list, DevStatus* __restrict__ status,
                const float* __restrict__ mu_hi, const float* __restrict__ mu_lo, int64_t dpad,
                int Npad, int slabs_per_split, int nsplit, const float* __restrict__ mu_normf,
                const int32_t* __restrict__ counts, int c, int32_t* __restrict__ labels,
                float* __restrict__ ub, float* __restrict__ lb, float* __restrict__ Gpart,
                float* __restrict__ ynorm_part, int32_t* __restrict__ tile_count,
                int32_t* __restrict__ rc_list) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t mbar[kTcStages];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int is_last_sh;

    const int64_t total = list ? (int64_t)status->flagged : n;
    const int64_t tile0 = (int64_t)blockIdx.x * kTcM;
    if (tile0 >= total) return;
    const int64_t nslabs = (d + kTcK - 1) / kTcK;
    const int64_t s_begin = (int64_t)blockIdx.y * slabs_per_split;
    const int64_t s_end = min(nslabs, s_begin + slabs_per_split);
    const int nq = (int)(s_end - s_begin);   // >= 1: every split is non-empty

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    // 1024-byte aligned operand tiles
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
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base_sh)), "r"(tmem_cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
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
    // B mapping: 16-byte chunks e = tid + j * 256 of the Npad x 32 centroid slab
    const int bchunks = Npad * 8;
    const int bmine = (bchunks - tid + kTcThreads - 1) / kTcThreads;   // chunks of this thread
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
            // the MMAs that read this stage two slabs ago must have finished
            if (!mbar_wait(&mbar[st], (uint32_t)(((q - kTcStages) >> 1) & 1))) failed = true;
        }
        if (__syncthreads_or(failed)) {
            failed = true;
            break;
        }
        // A: split into TF32 hi / lo parts, store swizzled; ||y||^2 with Kahan
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
            const float y = part - ycomp;
            const float t = ysq + y;
            ycomp = (t - ysq) - y;
            ysq = t;
        }
        // B: centroid hi / lo slabs (split and zero-padded to Npad x dpad beforehand)
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
        // prefetch the next slab while the tensor cores work on this one
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

    // wait for the last commit (it covers every MMA issued before it)
    {
        const int ql = failed ? -1 : nq - 1;
        if (ql >= 0) {
            if (!mbar_wait(&mbar[ql & 1], (uint32_t)((ql >> 1) & 1))) failed = true;
        } else {
            // a wait gave up: give the tensor cores one more bounded chance to drain
            for (int s = 0; s < kTcStages; ++s) mbar_wait(&mbar[s], 0u);
        }
    }
    failed = __syncthreads_or(failed);
    tc_fence_after();
    // this split's partial dot products -> Gpart[tile][split][Npad][128]
    float* gtile = Gpart + ((int64_t)blockIdx.x * nsplit + blockIdx.y) * (int64_t)Npad * kTcM;
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
        if (h == 0) ynorm_part[((int64_t)blockIdx.x * nsplit + blockIdx.y) * kTcM + m] = ysq + other;
    }
    if (failed && tid == 0) atomicOr(&status->timeout, 1);
    tc_fence_before();
    __threadfence();
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols)
                     : "memory");
    }
    // the last split CTA of this column tile finishes the search for it
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
    const float* gt0 = Gpart + (int64_t)blockIdx.x * nsplit * (int64_t)Npad * kTcM;
    const float* yt0 = ynorm_part + (int64_t)blockIdx.x * nsplit * kTcM;
    float y2 = 0.f;
    for (int s = 0; s < nsplit; ++s) y2 += __ldcg(yt0 + (int64_t)s * kTcM + tid);
    float bs = INFINITY, ss = INFINITY, be = 0.f, se = 0.f;
    int bi = INT_MAX, si = INT_MAX;
    for (int i = 0; i < c; ++i) {
        if (counts[i] == 0) continue;
        float g = 0.f;
        for (int s = 0; s < nsplit; ++s) g += __ldcg(gt0 + ((int64_t)s * Npad + i) * kTcM + tid);
        const float mu2 = mu_normf[i];
        const float sc = fmaf(-2.f, g, mu2);
        if (sc < bs) {
            ss = bs;
            se = be;
            si = bi;
            bs = sc;
            bi = i;
            be = score_err(mu2, y2);
        } else if (sc < ss) {
            ss = sc;
            si = i;
            se = score_err(mu2, y2);
        }
    }
    if (bi >= c) return;
    const float yerr = 1e-5f * y2;
    if (ss - bs <= be + se) {   // near tie: FP64 re-decision
        const int slot = atomicAdd(&status->rechecked, 1);
        rc_list[slot] = (int32_t)p;
        return;
    }
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

// Exact squared distance ||y - mu_i||^2 in FP64 by a whole CTA (the FP32
// inputs convert exactly; four independent accumulators per thread).
template <typename TY>
__device__ double block_dist2_fp64(const TY* __restrict__ y, const float* __restrict__ mrow,
                                   int64_t d, double* red) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int64_t r = threadIdx.x;
    for (; r + 3 * kThreads < d; r += 4 * kThreads) {
        const double e0 = (double)XLoad<TY>::one(y + r) - (double)mrow[r];
        const double e1 = (double)XLoad<TY>::one(y + r + kThreads) - (double)mrow[r + kThreads];
        const double e2 = (double)XLoad<TY>::one(y + r + 2 * kThreads) - (double)mrow[r + 2 * kThreads];
        const double e3 = (double)XLoad<TY>::one(y + r + 3 * kThreads) - (double)mrow[r + 3 * kThreads];
        a0 = fma(e0, e0, a0);
        a1 = fma(e1, e1, a1);
        a2 = fma(e2, e2, a2);
        a3 = fma(e3, e3, a3);
    }
    for (; r < d; r += kThreads) {
        const double e0 = (double)XLoad<TY>::one(y + r) - (double)mrow[r];
        a0 = fma(e0, e0, a0);
    }
    double a = warp_sum((a0 + a1) + (a2 + a3));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    return t;
}

// FP64 re-decision of near ties (one CTA per queued column): every centroid
// whose score interval can reach the best one gets its exact squared distance.
template <typename TY>
__global__ void __launch_bounds__(kThreads)
    k_search_recheck(const TY* __restrict__ Y, int64_t ldy, int64_t d, int64_t n,
                     const int32_t* __restrict__ list, DevStatus* __restrict__ status,
                     const float* __restrict__ Gpart, const float* __restrict__ ynorm_part,
                     int nsplit, int Npad, const float* __restrict__ mu,
                     const float* __restrict__ mu_normf, const int32_t* __restrict__ counts, int c,
                     int32_t* __restrict__ labels, float* __restrict__ ub, float* __restrict__ lb,
                     const int32_t* __restrict__ rc_list) {
    __shared__ double red[kThreads / 32];
    __shared__ float fred[kThreads / 32];
    __shared__ uint8_t cand[kTcMaxClusters];
    const int nrc = status->rechecked;
    for (int64_t k = blockIdx.x; k < nrc; k += gridDim.x) {
        const int64_t p = rc_list[k];
        const int64_t col = list ? (int64_t)list[p] : p;
        const int64_t tile = p / kTcM, mm = p % kTcM;
        const float* gt0 = Gpart + tile * nsplit * (int64_t)Npad * kTcM;
        float y2 = 0.f;
        for (int s = 0; s < nsplit; ++s) y2 += ynorm_part[(tile * nsplit + s) * kTcM + mm];
        float sc = INFINITY, er = 0.f;
        const int i = threadIdx.x;   // c <= 256 = blockDim.x
        if (i < c && counts[i] > 0) {
            float g = 0.f;
            for (int s = 0; s < nsplit; ++s) g += gt0[((int64_t)s * Npad + i) * kTcM + mm];
            sc = fmaf(-2.f, g, mu_normf[i]);
            er = score_err(mu_normf[i], y2);
        }
        // lowest upper end of the score intervals
        float hi = sc + er;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) hi = fminf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        __syncthreads();
        if ((threadIdx.x & 31) == 0) fred[threadIdx.x >> 5] = hi;
        __syncthreads();
        float best_hi = INFINITY;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) best_hi = fminf(best_hi, fred[w]);
        if (i < c) cand[i] = (sc - er <= best_hi) ? 1 : 0;
        __syncthreads();
        double best = INFINITY;
        int besti = INT_MAX;
        const TY* y = Y + col * ldy;
        for (int ci = 0; ci < c; ++ci) {   // candidates in increasing index: ties keep the lowest
            if (!cand[ci]) continue;
            const double a = block_dist2_fp64<TY>(y, mu + (int64_t)ci * d, d, red);
            if (a < best) {
                best = a;
                besti = ci;
            }
        }
        if (threadIdx.x == 0 && besti < c) {
            const int32_t old = labels[col];
            if (old != besti) {
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

// TF32 hi / lo parts of the centroids, zero-padded to Npad rows of dpad.
__global__ void __launch_bounds__(kThreads)
    k_mu_split(const float* __restrict__ mu, int c, int64_t d, int Npad, int64_t dpad,
               float* __restrict__ mu_hi, float* __restrict__ mu_lo) {
    const int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (idx >= (int64_t)Npad * dpad) return;
    const int i = (int)(idx / dpad);
    const int64_t r = idx % dpad;
    const float v = (i < c && r < d) ? mu[(int64_t)i * d + r] : 0.f;
    const float hi = tf32_hi(v);
    mu_hi[idx] = hi;
    mu_lo[idx] = v - hi;
}

inline int grid_for(int64_t work, int per) { return (int)((work + per - 1) / per); }

}  // namespace

int tc_npad(int c) { return ((c + 15) / 16) * 16; }

size_t tc_smem_bytes(int Npad) {
    return (size_t)kTcStages * (2 * kTcM * 128 + 2 * (size_t)Npad * 128) + 1024;
}

// Number of d-splits: about two CTAs per SM in total, every split non-empty
// (the split count is derived back from the slabs per split).
static int64_t tc_slabs_per_split(int64_t n, int64_t d) {
    const int64_t tiles = (n + kTcM - 1) / kTcM;
    const int64_t nslabs = (d + kTcK - 1) / kTcK;
    int64_t s = (2 * 152) / (tiles > 0 ? tiles : 1);
    if (s < 1) s = 1;
    if (s > 16) s = 16;
    if (s > nslabs) s = nslabs;
    return (nslabs + s - 1) / s;
}

int tc_splits(int64_t n, int64_t d) {
    const int64_t nslabs = (d + kTcK - 1) / kTcK;
    const int64_t per = tc_slabs_per_split(n, d);
    return (int)((nslabs + per - 1) / per);
}

cudaError_t launch_mu_split(const float* mu, int c, int64_t d, int Npad, int64_t dpad, float* mu_hi,
                            float* mu_lo, cudaStream_t st) {
    count_launches(1);
    k_mu_split<<<grid_for((int64_t)Npad * dpad, kThreads), kThreads, 0, st>>>(mu, c, d, Npad, dpad,
                                                                            mu_hi, mu_lo);
    return cudaGetLastError();
}

cudaError_t launch_search_tc(int dtype, const void* Y, int64_t ldy, int64_t d, int64_t n,
                             const int32_t* list, DevStatus* status, const float* mu,
                             const float* mu_hi, const float* mu_lo, int64_t dpad,
                             const float* mu_normf, const int32_t* counts, int c, int32_t* labels,
                             float* ub, float* lb, float* Gpart, float* ynorm_part,
                             int32_t* tile_count, int32_t* rc_list, bool vec, cudaStream_t st) {
    const int Npad = tc_npad(c);
    const int nsplit = tc_splits(n, d);
    const int per = (int)tc_slabs_per_split(n, d);
    const size_t smem = tc_smem_bytes(Npad);
    const dim3 grid((unsigned)((n + kTcM - 1) / kTcM), (unsigned)nsplit);
    cudaError_t e = cudaSuccess;
    count_launches(2);
    RESPCA_DISPATCH_X(dtype, TY, {
        auto kern = vec ? k_search_tc<TY, true> : k_search_tc<TY, false>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) {
            kern<<<grid, kTcThreads, smem, st>>>((const TY*)Y, ldy, d, n, list, status, mu_hi, mu_lo,
                                                 dpad, Npad, per, nsplit, mu_normf, counts, c, labels,
                                                 ub, lb, Gpart, ynorm_part, tile_count, rc_list);
            k_search_recheck<TY><<<152, kThreads, 0, st>>>(
                (const TY*)Y, ldy, d, n, list, status, Gpart, ynorm_part, nsplit, Npad, mu, mu_normf,
                counts, c, labels, ub, lb, rc_list);
        }
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace respca
