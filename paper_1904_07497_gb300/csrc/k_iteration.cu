// The fused RES-PCA iteration kernel (the hot path).
//
// One pass over X, S, Theta and L_prev per ALM iteration computes D, the L
// step (Eq. (18)), the S step (Eq. (24)), the multiplier step (Eq. (25)), the
// three Frobenius quantities of the Sec. 5 stopping rule, each column's
// squared distance to its own centroid (for the exact pruning of the K-means
// search) and the cluster sums of the NEXT iteration's D under the current
// labels, which become the next centroids whenever the p step keeps every
// label.  28 bytes move per element (4 loads, 3 stores of 4 bytes) with FP32
// state; 14 with BF16 X and BF16 state (TS), where every stored value is the
// FP32 result rounded to BF16 and the norms, own distances and next sums are
// formed from the stored values (so the state is exactly what is stored).
// With FP32 state the pass can also write a BF16 copy of L (2 more bytes per
// element) and each column chunk's ||L_j - bf16(L_j)||^2: the nearest-centroid
// search of this iteration then reads half the bytes and widens its decisions
// by that norm.
#include <type_traits>

#include "respca_internal.cuh"

namespace respca {

namespace {

// ---------------------------------------------------------------- fused iteration
// One element of one ALM iteration.  l, sn, tn are the new L, S, Theta as
// stored (rounded to TS).
template <typename TS>
__device__ __forceinline__ void alm_element(float x, float s, float t, float l0, float m,
                                            const IterScalars& sc, float& l, float& sn, float& tn,
                                            float& own, float& nr, float& dlc, float& nds,
                                            float& dnext) {
    const float tr = t * sc.inv_rho;
    const float dv = (x - s) + tr;                    // D = X - S + Theta/rho (after Eq. (14))
    l = StateIO<TS>::round(fmaf(sc.a, dv, sc.b * m)); // Eq. (18): a D_j + (1-a) mean of cluster
    const float bb = (x - l) + tr;                    // B = X - L + Theta/rho
    const float mag = fabsf(bb) - sc.inv_rho;
    sn = StateIO<TS>::round(mag > 0.f ? copysignf(mag, bb) : 0.f);   // Eq. (24), sign(0) = 0
    tn = StateIO<TS>::round(fminf(fmaxf(sc.rho * bb, -1.f), 1.f));   // Eq. (25): clip(rho B)
    const float res = (x - l) - sn;
    const float dl = l - l0;
    const float ds = sn - s;
    const float e = l - m;
    own = fmaf(e, e, own);
    nr = fmaf(res, res, nr);
    dlc = fmaf(dl, dl, dlc);
    nds = fmaf(ds, ds, nds);
    dnext = (x - sn) + tn * sc.inv_rho_next;          // D of the next iteration
}

// SH: also the BF16 copy Lsh (column stride ldsh) and ylo_part.
template <typename TX, typename TS, bool VEC, bool SH>
__global__ void __launch_bounds__(kThreads, 2)
    k_iteration(const TX* __restrict__ X, int64_t ldx, TS* __restrict__ L, TS* __restrict__ S,
                TS* __restrict__ Th, int64_t lds, const float* __restrict__ mu,
                const int32_t* __restrict__ perm, const TileDesc* __restrict__ tiles,
                const DevStatus* __restrict__ status, int64_t d, int64_t n, IterScalars sc,
                float* __restrict__ Dpart, float* __restrict__ own_part,
                float* __restrict__ dl_part, double* __restrict__ norm_part,
                __nv_bfloat16* __restrict__ Lsh, int64_t ldsh, float* __restrict__ ylo_part) {
    __shared__ float red[kThreads / 32][kChunkRows];
    __shared__ double nred[kThreads / 32][3];
    const int tile_idx = blockIdx.x;
    if (tile_idx >= status->ntiles) return;
    const TileDesc td = tiles[tile_idx];
    const int64_t r0 = (int64_t)blockIdx.y * kChunkRows;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const float* mup = mu + (int64_t)td.label * d;

    float4 m[4], acc[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int64_t rr = r0 + s * 128 + lane * 4;
        acc[s] = make_float4(0.f, 0.f, 0.f, 0.f);
        m[s] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (VEC) {
            if (rr < d) m[s] = *reinterpret_cast<const float4*>(mup + rr);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (rr + q < d) f4set(m[s], q, mup[rr + q]);
        }
    }
    float nr = 0.f, ndl = 0.f, nds = 0.f;

    for (int k = warp; k < td.len; k += kThreads / 32) {
        const int64_t col = perm[td.start + k];
        const TX* xc = X + col * ldx;
        TS* lc = L + col * lds;
        TS* scol = S + col * lds;
        TS* tc = Th + col * lds;
        float own = 0.f, dlc = 0.f, yl = 0.f;
        if (VEC) {
            float4 xv[4], sv[4], tv[4], lv[4];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int64_t rr = r0 + s * 128 + lane * 4;
                if (rr < d) {
                    xv[s] = XLoad<TX>::four(xc + rr);
                    sv[s] = StateIO<TS>::load4(scol + rr);
                    tv[s] = StateIO<TS>::load4(tc + rr);
                    lv[s] = StateIO<TS>::load4(lc + rr);
                }
            }
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int64_t rr = r0 + s * 128 + lane * 4;
                if (rr < d) {
                    float4 lo, so, to;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float l, sn, tn, dn;
                        alm_element<TS>(f4get(xv[s], q), f4get(sv[s], q), f4get(tv[s], q),
                                    f4get(lv[s], q), f4get(m[s], q), sc, l, sn, tn, own, nr, dlc,
                                    nds, dn);
                        f4set(lo, q, l);
                        f4set(so, q, sn);
                        f4set(to, q, tn);
                        f4set(acc[s], q, f4get(acc[s], q) + dn);
                    }
                    StateIO<TS>::store4(lc + rr, lo);
                    StateIO<TS>::store4(scol + rr, so);
                    StateIO<TS>::store4(tc + rr, to);
                    if constexpr (SH) {
                        const __nv_bfloat162 b0 = __floats2bfloat162_rn(lo.x, lo.y);
                        const __nv_bfloat162 b1 = __floats2bfloat162_rn(lo.z, lo.w);
                        uint2 u;
                        u.x = *reinterpret_cast<const uint32_t*>(&b0);
                        u.y = *reinterpret_cast<const uint32_t*>(&b1);
                        *reinterpret_cast<uint2*>(Lsh + col * ldsh + rr) = u;
                        // l - bf16(l) is exact in FP32
                        const float2 f0 = __bfloat1622float2(b0), f1 = __bfloat1622float2(b1);
                        const float e0 = lo.x - f0.x, e1 = lo.y - f0.y, e2 = lo.z - f1.x, e3 = lo.w - f1.y;
                        yl = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, fmaf(e3, e3, yl))));
                    }
                }
            }
        } else {
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int64_t rr = r0 + s * 128 + lane * 4;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (rr + q < d) {
                        float l, sn, tn, dn;
                        alm_element<TS>(XLoad<TX>::one(xc + rr + q), StateIO<TS>::load1(scol + rr + q),
                                        StateIO<TS>::load1(tc + rr + q), StateIO<TS>::load1(lc + rr + q),
                                        f4get(m[s], q), sc, l, sn, tn, own, nr, dlc, nds, dn);
                        StateIO<TS>::store1(lc + rr + q, l);
                        StateIO<TS>::store1(scol + rr + q, sn);
                        StateIO<TS>::store1(tc + rr + q, tn);
                        f4set(acc[s], q, f4get(acc[s], q) + dn);
                    }
                }
            }
        }
        ndl += dlc;
        own = warp_sum(own);
        dlc = warp_sum(dlc);
        if constexpr (SH) yl = warp_sum(yl);
        if (lane == 0) {
            own_part[(int64_t)blockIdx.y * n + col] = own;
            dl_part[(int64_t)blockIdx.y * n + col] = dlc;
            if constexpr (SH) ylo_part[(int64_t)blockIdx.y * n + col] = yl;
        }
    }

#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int q = 0; q < 4; ++q) red[warp][s * 128 + lane * 4 + q] = f4get(acc[s], q);
    const double w0 = warp_sum((double)nr), w1 = warp_sum((double)ndl), w2 = warp_sum((double)nds);
    if (lane == 0) {
        nred[warp][0] = w0;
        nred[warp][1] = w1;
        nred[warp][2] = w2;
    }
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
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += nred[w][threadIdx.x];
        norm_part[((int64_t)blockIdx.y * gridDim.x + tile_idx) * 3 + threadIdx.x] = t;
    }
}

inline int grid_for(int64_t work, int per) { return (int)((work + per - 1) / per); }

}  // namespace

cudaError_t launch_iteration(int dtype, int sdtype, const void* X, int64_t ldx, void* L, void* S,
                             void* Th, int64_t lds, const float* mu, const int32_t* perm,
                             const TileDesc* tiles, int max_tiles, const DevStatus* status,
                             int64_t d, int64_t n, IterScalars sc, float* Dpart, float* own_part,
                             float* dl_part, double* norm_part, bool vec, cudaStream_t st, void* Lsh,
                             int64_t ldsh, float* ylo_part) {
    count_launches(1);
    const dim3 grid(max_tiles, grid_for(d, kChunkRows));
    auto* sh = static_cast<__nv_bfloat16*>(Lsh);
    RESPCA_DISPATCH_X(dtype, TX, {
        RESPCA_DISPATCH_S(sdtype, TS, {
            bool done = false;
            if constexpr (std::is_same<TS, float>::value) {
                if (vec && sh) {
                    k_iteration<TX, TS, true, true><<<grid, kThreads, 0, st>>>(
                        (const TX*)X, ldx, (TS*)L, (TS*)S, (TS*)Th, lds, mu, perm, tiles, status, d, n, sc,
                        Dpart, own_part, dl_part, norm_part, sh, ldsh, ylo_part);
                    done = true;
                }
            }
            if (!done) {
                if (vec)
                    k_iteration<TX, TS, true, false><<<grid, kThreads, 0, st>>>(
                        (const TX*)X, ldx, (TS*)L, (TS*)S, (TS*)Th, lds, mu, perm, tiles, status, d, n, sc,
                        Dpart, own_part, dl_part, norm_part, nullptr, 0, nullptr);
                else
                    k_iteration<TX, TS, false, false><<<grid, kThreads, 0, st>>>(
                        (const TX*)X, ldx, (TS*)L, (TS*)S, (TS*)Th, lds, mu, perm, tiles, status, d, n, sc,
                        Dpart, own_part, dl_part, norm_part, nullptr, 0, nullptr);
            }
        });
    });
    return cudaGetLastError();
}

}  // namespace respca
