// Gram matrix G = Y^T Y of the spectral p step (Sec. 4.2: the affinity of the
// columns of L needs every ||y_i - y_j||^2 = ||y_i||^2 + ||y_j||^2 - 2 y_i . y_j)
// on the 5th-generation tensor cores (sm_103a), tcgen05.mma kind::tf32.
//
// FP32 accuracy from the 3-term split y = hi + lo, hi = the TF32 truncation
// (the MMA reads an FP32 operand by truncating it to TF32, so a raw tile in
// shared memory already is its hi part):
//   y_i . y_j ~ hi_i . hi_j + hi_i . lo_j + lo_i . hi_j
// whose error, |lo_i . lo_j| <= 2^-20 ||y_i|| ||y_j|| plus the TF32 rounding
// of the lo parts and the FP32 accumulation, is of the order of FP32 rounding.
//
// Work: the upper triangle of 128 x 128 output tiles (block row <= block
// column), one CTA per SM taking tiles round-robin; per tile the d rows in
// 32-row slabs.  Each tile's values are written to both (i, j) and (j, i), so
// G is exactly symmetric; on a diagonal tile only entries with j >= i are
// written (the mirror supplies the rest).
//   warp 0: TMA producer (the A and B slabs of a stage: 128 columns x 32 rows
//           each, 128-byte swizzle), warp 1: MMA issuer (12 MMAs per slab into
//           one of two 128 x 128 FP32 accumulators in tensor memory),
//   warps 2-5: the lo parts of both slabs into a ring of 2 lo slots,
//   warps 6-9: epilogue (tensor memory -> G, both halves).
// Every mbarrier wait is bounded; a wait that gives up sets status->timeout,
// the CTA drains its copies and MMAs (bounded waits), frees its tensor memory
// and returns.
#include <algorithm>

#include "respca_internal.cuh"
#include "tc_ptx.cuh"

namespace respca {

namespace {

constexpr int kGmT = 128;          // output tile edge (MMA M = N = 128)
constexpr int kGmK = 32;           // rows of Y per slab (one 128-byte swizzle atom of FP32)
constexpr int kGmS = 4;            // stages of (A slab, B slab)
constexpr int kGmThreads = 320;    // 10 warps
constexpr uint32_t kGmSlab = kGmT * 128;           // 16 KB: 128 columns x 32 rows of FP32
constexpr uint32_t kGmStage = 2 * kGmSlab;          // A and B
constexpr uint32_t kGmLo = 2 * kGmSlab;             // lo parts of A and B
constexpr size_t kGmSmem = (size_t)kGmS * kGmStage + 2 * kGmLo + 1024;

struct GramArgs {
    int64_t n, Q;        // columns of Y (= order of G), slabs in d
    int64_t T, tiles;    // 128-column blocks, upper-triangle tiles
};

// (block row, block column) of upper-triangle tile t, row-major over bi <= bj.
__device__ __forceinline__ void tile_coords(int64_t t, int64_t T, int64_t* bi, int64_t* bj) {
    int64_t r = 0, left = t;
    while (left >= T - r) {
        left -= T - r;
        ++r;
    }
    *bi = r;
    *bj = r + left;
}

__global__ void __launch_bounds__(kGmThreads, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap tmY, GramArgs a, float* __restrict__ G,
              DevStatus* __restrict__ status) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full[kGmS], empty[kGmS], conv[2], loempty[2], acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_sh;

    const int64_t G0 = gridDim.x, b = blockIdx.x;
    if (b >= a.tiles) return;
    const int64_t my_tiles = (a.tiles - 1 - b) / G0 + 1;
    const int64_t units = my_tiles * a.Q;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t lo_base = base + (uint32_t)kGmS * kGmStage;
    constexpr uint32_t kTmemCols = 256;   // two 128 x 128 FP32 accumulators

    if (warp == 1) {
        tmem_alloc(&tmem_base_sh, kTmemCols);
        tc_fence_before();
    }
    if (tid == 0) {
        for (int s = 0; s < kGmS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&conv[s], 4);
            mbar_init(&loempty[s], 1);
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
            RingPos sr(kGmS);
            int64_t k = 0;
            for (int64_t u = 0; u < units; ++u, ++k) {
                const int64_t tl = u / a.Q, slab = u - tl * a.Q;
                int64_t bi, bj;
                tile_coords(b + tl * G0, a.T, &bi, &bj);
                if (k >= kGmS && !mbar_wait_or_abort(&empty[sr.idx], sr.phase ^ 1u, &abort_sh)) {
                    abort_sh = 1;
                    break;
                }
                const uint32_t dst = base + (uint32_t)sr.idx * kGmStage;
                const int32_t row = (int32_t)(slab * kGmK);
                mbar_expect_tx(&full[sr.idx], kGmStage);
                tma_load_2d(dst, &tmY, &full[sr.idx], row, (int32_t)(bi * kGmT));
                tma_load_2d(dst + kGmSlab, &tmY, &full[sr.idx], row, (int32_t)(bj * kGmT));
                sr.next();
            }
            drain_ring(full, kGmS, k);   // no copy may be in flight when the CTA leaves
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(kGmT, kGmT);
            const uint64_t d0 = sw128_desc(base), l0 = sw128_desc(lo_base);
            const uint32_t st16 = kGmStage >> 4, sl16 = kGmSlab >> 4, lo16 = kGmLo >> 4;
            RingPos sr(kGmS), lr(2), ar(2);
            int64_t g = 0, slab = 0;
            uint64_t* last_bar = nullptr;
            uint32_t last_par = 0;
            for (int64_t u = 0; u < units; ++u) {
                if (slab == 0 && g >= 2 &&
                    !mbar_wait_or_abort(&acc_empty[ar.idx], ar.phase ^ 1u, &abort_sh)) {
                    abort_sh = 1;
                    break;
                }
                if (!mbar_wait_or_abort(&full[sr.idx], sr.phase, &abort_sh) ||
                    !mbar_wait_or_abort(&conv[lr.idx], lr.phase, &abort_sh)) {
                    abort_sh = 1;
                    break;
                }
                tc_fence_after();
                const uint64_t dA = d0 + (uint64_t)(sr.idx * st16), dB = dA + sl16;
                const uint64_t dAl = l0 + (uint64_t)(lr.idx * lo16), dBl = dAl + sl16;
                const uint32_t acc = tmem + (uint32_t)(ar.idx * kGmT);
#pragma unroll
                for (int ks = 0; ks < kGmK / 8; ++ks) {
                    // 8 TF32 of K = 32 bytes = 2 descriptor address units
                    tc_mma(acc, dA + 2 * ks, dB + 2 * ks, idesc, (slab == 0 && ks == 0) ? 0u : 1u);
                    tc_mma(acc, dA + 2 * ks, dBl + 2 * ks, idesc, 1u);
                    tc_mma(acc, dAl + 2 * ks, dB + 2 * ks, idesc, 1u);
                }
                tc_commit(&empty[sr.idx]);
                tc_commit(&loempty[lr.idx]);
                last_bar = &loempty[lr.idx];
                last_par = lr.phase;
                sr.next();
                lr.next();
                if (++slab == a.Q) {
                    tc_commit(&acc_full[ar.idx]);
                    ar.next();
                    ++g;
                    slab = 0;
                }
            }
            // drain: the last commit covers every MMA issued before it
            if (last_bar) mbar_wait(last_bar, last_par);
        }
    } else if (warp < 6) {
        // ---------------- lo parts of the A and B slabs (row m of each)
        const int m = 32 * (warp - 2) + lane;
        RingPos sr(kGmS), lr(2);
        for (int64_t u = 0; u < units; ++u) {
            if (!mbar_wait_or_abort(&full[sr.idx], sr.phase, &abort_sh)) {
                abort_sh = 1;
                break;
            }
            // the lo slot is free once the MMAs of unit u - 2 are done
            if (u >= 2 && !mbar_wait_or_abort(&loempty[lr.idx], lr.phase ^ 1u, &abort_sh)) {
                abort_sh = 1;
                break;
            }
            const uint32_t src = base + (uint32_t)sr.idx * kGmStage;
            const uint32_t dst = lo_base + (uint32_t)lr.idx * kGmLo;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const uint32_t off = (uint32_t)h * kGmSlab + sw128_off(m, q);
                    const float4 x = ld_shared_v4(src + off);
                    st_shared_v4(dst + off, make_float4(x.x - tf32_hi(x.x), x.y - tf32_hi(x.y),
                                                        x.z - tf32_hi(x.z), x.w - tf32_hi(x.w)));
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&conv[lr.idx]);
            sr.next();
            lr.next();
        }
    } else {
        // ---------------- epilogue: lane = accumulator row (tensor-memory lane quarter warp % 4)
        const int quarter = warp & 3;
        const int r = 32 * quarter + lane;
        const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
        RingPos ar(2);
        for (int64_t tl = 0; tl < my_tiles; ++tl) {
            int64_t bi, bj;
            tile_coords(b + tl * G0, a.T, &bi, &bj);
            if (!mbar_wait_or_abort(&acc_full[ar.idx], ar.phase, &abort_sh)) {
                abort_sh = 1;
                break;
            }
            tc_fence_after();
            const int64_t i = bi * kGmT + r;
            const bool diag = bi == bj;
            for (int cb = 0; cb < kGmT; cb += 16) {
                float v[16];
                tc_ld16(tmem + lane_base + (uint32_t)(ar.idx * kGmT + cb), v);
                if (i >= a.n) continue;
                const int64_t j0 = bj * kGmT + cb;
                // (i, j) for the j of this chunk: lanes are consecutive i (coalesced per j)
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int64_t j = j0 + q;
                    if (j < a.n && (!diag || j >= i)) G[i + j * a.n] = v[q];
                }
                // (j, i): row i of the mirror, contiguous in j
                float* mrow = G + i * a.n + j0;
                if (j0 + 16 <= a.n && !diag && ((a.n & 3) == 0)) {
#pragma unroll
                    for (int q = 0; q < 16; q += 4)
                        *reinterpret_cast<float4*>(mrow + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int64_t j = j0 + q;
                        if (j < a.n && (!diag || j > i)) mrow[q] = v[q];
                    }
                }
            }
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

}  // namespace

bool gram_tc_ok(const float* Y, int64_t ldy) {
    return ((reinterpret_cast<uintptr_t>(Y) & 15u) == 0) && (ldy % 4 == 0) && encoder() != nullptr;
}

cudaError_t launch_gram_tc(const float* Y, int64_t ldy, int64_t d, int64_t n, float* G, DevStatus* status,
                           cudaStream_t st) {
    CUtensorMap tmY;
    if (!encode_2d(&tmY, Y, d, n, ldy, kGmK, kGmT)) return cudaErrorInvalidValue;
    GramArgs a;
    a.n = n;
    a.Q = (d + kGmK - 1) / kGmK;
    a.T = (n + kGmT - 1) / kGmT;
    a.tiles = a.T * (a.T + 1) / 2;
    const cudaError_t attr = allow_max_dynamic_smem((const void*)k_gram_tc);
    if (attr != cudaSuccess) return attr;
    const int grid = (int)std::min<int64_t>(num_sms(), a.tiles);
    count_launches(1);
    k_gram_tc<<<grid, kGmThreads, kGmSmem, st>>>(tmY, a, G, status);
    return cudaGetLastError();
}

}  // namespace respca
