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
// With FP32 state the pass also finds max |L| and can write an FP16 copy of L,
// fp16(s L) with s a power of two (2 more bytes per element), and each column
// chunk's ||L_j - fp16(s L_j) / s||^2: the nearest-centroid search of this
// iteration then reads half the bytes and widens its decisions by that norm.
// Values beyond the FP16 range are clamped; the norm counts them as they are
// stored, so the widening stays a bound whatever s is.
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

// SH: also the FP16 copy Lsh (column stride ldsh, scale sc.sh_scale) and, per
// row chunk and column, ||L_j - y~_j||^2 in ylo_part[chunk][col] and ||y~_j||^2 in
// ylo_part[nchunks + chunk][col] (y~ = copy / s).
template <typename TX, typename TS, bool VEC, bool SH>
__global__ void __launch_bounds__(kThreads, 2)
    k_iteration(const TX* __restrict__ X, int64_t ldx, TS* __restrict__ L, TS* __restrict__ S,
                TS* __restrict__ Th, int64_t lds, const float* __restrict__ mu,
                const int32_t* __restrict__ perm, const TileDesc* __restrict__ tiles,
                DevStatus* __restrict__ status, int64_t d, int64_t n, IterScalars sc,
                float* __restrict__ Dpart, float* __restrict__ own_part,
                float* __restrict__ dl_part, double* __restrict__ norm_part,
                __half* __restrict__ Lsh, int64_t ldsh, float* __restrict__ ylo_part) {
    constexpr bool kMax = std::is_same<TS, float>::value;   // max |L| for the copy's next scale
    __shared__ float red[kThreads / 32][kChunkRows];
    __shared__ double nred[kThreads / 32][3];
    __shared__ float mred[kThreads / 32];
    const int tile_idx = blockIdx.x;
    if (tile_idx >= status->ntiles) return;
    const TileDesc td = tiles[tile_idx];
    const int64_t r0 = (int64_t)blockIdx.y * kChunkRows;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const float* mup = mu + (int64_t)td.label * d;

    // the tile's centroid rows in shared memory (constant over the CTA's columns;
    // in registers they would push the loads in flight into local memory)
    __shared__ __align__(16) float msh[kChunkRows];
    for (int i = threadIdx.x; i < kChunkRows; i += kThreads) msh[i] = (r0 + i < d) ? mup[r0 + i] : 0.f;
    float4 acc[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    float nr = 0.f, ndl = 0.f, nds = 0.f, lmax = 0.f;
    const float inv_s = 1.f / sc.sh_scale;   // a power of two: exact
    if (SH && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        status->sh_scale = sc.sh_scale;
        status->sh_inv2 = inv_s * inv_s;
    }

    for (int k = warp; k < td.len; k += kThreads / 32) {
        const int64_t col = perm[td.start + k];
        const TX* xc = X + col * ldx;
        TS* lc = L + col * lds;
        TS* scol = S + col * lds;
        TS* tc = Th + col * lds;
        float own = 0.f, dlc = 0.f, yl = 0.f, yq = 0.f;
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
                    const float4 ms = *reinterpret_cast<const float4*>(msh + s * 128 + lane * 4);
                    float4 lo, so, to;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float l, sn, tn, dn;
                        alm_element<TS>(f4get(xv[s], q), f4get(sv[s], q), f4get(tv[s], q),
                                    f4get(lv[s], q), f4get(ms, q), sc, l, sn, tn, own, nr, dlc,
                                    nds, dn);
                        f4set(lo, q, l);
                        f4set(so, q, sn);
                        f4set(to, q, tn);
                        f4set(acc[s], q, f4get(acc[s], q) + dn);
                    }
                    StateIO<TS>::store4(lc + rr, lo);
                    StateIO<TS>::store4(scol + rr, so);
                    StateIO<TS>::store4(tc + rr, to);
                    if constexpr (kMax)
                        lmax = fmaxf(lmax, fmaxf(fmaxf(fabsf(lo.x), fabsf(lo.y)), fmaxf(fabsf(lo.z), fabsf(lo.w))));
                    if constexpr (SH) {
                        __half2 h0, h1;
                        h0.x = copy16(lo.x, sc.sh_scale, inv_s, yl, yq);
                        h0.y = copy16(lo.y, sc.sh_scale, inv_s, yl, yq);
                        h1.x = copy16(lo.z, sc.sh_scale, inv_s, yl, yq);
                        h1.y = copy16(lo.w, sc.sh_scale, inv_s, yl, yq);
                        uint2 u;
                        u.x = *reinterpret_cast<const uint32_t*>(&h0);
                        u.y = *reinterpret_cast<const uint32_t*>(&h1);
                        *reinterpret_cast<uint2*>(Lsh + col * ldsh + rr) = u;
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
                                        msh[s * 128 + lane * 4 + q], sc, l, sn, tn, own, nr, dlc, nds, dn);
                        StateIO<TS>::store1(lc + rr + q, l);
                        StateIO<TS>::store1(scol + rr + q, sn);
                        StateIO<TS>::store1(tc + rr + q, tn);
                        if constexpr (kMax) lmax = fmaxf(lmax, fabsf(l));
                        f4set(acc[s], q, f4get(acc[s], q) + dn);
                    }
                }
            }
        }
        ndl += dlc;
        own = warp_sum(own);
        dlc = warp_sum(dlc);
        if constexpr (SH) {
            yl = warp_sum(yl);
            yq = warp_sum(yq);
        }
        if (lane == 0) {
            own_part[(int64_t)blockIdx.y * n + col] = own;
            dl_part[(int64_t)blockIdx.y * n + col] = dlc;
            if constexpr (SH) {
                ylo_part[(int64_t)blockIdx.y * n + col] = yl;
                ylo_part[((int64_t)gridDim.y + blockIdx.y) * n + col] = yq;
            }
        }
    }

#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int q = 0; q < 4; ++q) red[warp][s * 128 + lane * 4 + q] = f4get(acc[s], q);
    const double w0 = warp_sum((double)nr), w1 = warp_sum((double)ndl), w2 = warp_sum((double)nds);
    if constexpr (kMax) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    }
    if (lane == 0) {
        nred[warp][0] = w0;
        nred[warp][1] = w1;
        nred[warp][2] = w2;
        mred[warp] = lmax;
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
    if (kMax && threadIdx.x == 32) {
        float m = 0.f;
        for (int w = 0; w < kThreads / 32; ++w) m = fmaxf(m, mred[w]);
        atomicMax(&status->lmax_bits, __float_as_uint(m));   // non-negative floats order as their bits
    }
}

inline int grid_for(int64_t work, int per) { return (int)((work + per - 1) / per); }

}  // namespace

cudaError_t launch_iteration(int dtype, int sdtype, const void* X, int64_t ldx, void* L, void* S,
                             void* Th, int64_t lds, const float* mu, const int32_t* perm,
                             const TileDesc* tiles, int max_tiles, DevStatus* status,
                             int64_t d, int64_t n, IterScalars sc, float* Dpart, float* own_part,
                             float* dl_part, double* norm_part, bool vec, cudaStream_t st, void* Lsh,
                             int64_t ldsh, float* ylo_part) {
    count_launches(1);
    const dim3 grid(max_tiles, grid_for(d, kChunkRows));
    auto* sh = static_cast<__half*>(Lsh);
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
