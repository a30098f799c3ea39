// The RES-PCA iteration with the l2,1 norm on S (the alternative to l1 that
// Sec. 3 names; model Eq. (8) with ||S||_{2,1}), FP32 state.
//
// The S step becomes block soft-thresholding of every column,
//   S_j = B_j max(0, 1 - 1/(rho ||B_j||)),  B = X - L + Theta/rho,
// and the multiplier step Eq. (25), Theta + rho (X - L - S) = rho (B - S),
// becomes rho B_j / max(1, rho ||B_j||): the projection of rho B_j onto the
// unit l2 ball.  ||B_j|| needs the whole column before any element of S_j can
// be written, so an iteration takes two passes over the label-sorted tiles:
//   A: the L step (Eq. (18)), each column's ||B_j||^2, distance to its own
//      centroid and movement, ||L - L_prev||^2       (reads X, S, Theta, L_prev; writes L)
//   B: S, Theta, ||X - L - S||^2, ||S - S_prev||^2 and the next D sums
//                                                    (reads X, S, Theta, L; writes S, Theta)
// 44 bytes per element instead of the l1 form's 28.
#include "respca_internal.cuh"

namespace respca {

namespace {

template <typename TX, bool VEC>
__global__ void __launch_bounds__(kThreads, 2)
    k_l21_pass_a(const TX* __restrict__ X, int64_t ldx, float* __restrict__ L,
                 const float* __restrict__ S, const float* __restrict__ Th, int64_t lds,
                 const float* __restrict__ mu, const int32_t* __restrict__ perm,
                 const TileDesc* __restrict__ tiles, const DevStatus* __restrict__ status, int64_t d,
                 int64_t n, IterScalars sc, float* __restrict__ own_part, float* __restrict__ dl_part,
                 float* __restrict__ bn_part, double* __restrict__ norm_part) {
    __shared__ double nred[kThreads / 32];
    const int tile_idx = blockIdx.x;
    if (tile_idx >= status->ntiles) return;
    const TileDesc td = tiles[tile_idx];
    const int64_t r0 = (int64_t)blockIdx.y * kChunkRows;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float* mup = mu + (int64_t)td.label * d;
    float ndl = 0.f;
    for (int k = warp; k < td.len; k += kThreads / 32) {
        const int64_t col = perm[td.start + k];
        const TX* xc = X + col * ldx;
        float* lc = L + col * lds;
        const float* scol = S + col * lds;
        const float* tc = Th + col * lds;
        float own = 0.f, dlc = 0.f, bsq = 0.f;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int64_t rr = r0 + s * 128 + lane * 4;
            if (VEC) {
                if (rr >= d) continue;
                const float4 x = XLoad<TX>::four(xc + rr);
                const float4 sv = __ldcs(reinterpret_cast<const float4*>(scol + rr));
                const float4 tv = __ldcs(reinterpret_cast<const float4*>(tc + rr));
                const float4 l0 = __ldcs(reinterpret_cast<const float4*>(lc + rr));
                const float4 m = *reinterpret_cast<const float4*>(mup + rr);
                float4 lo;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float tr = f4get(tv, q) * sc.inv_rho;
                    const float dv = (f4get(x, q) - f4get(sv, q)) + tr;     // D (Eq. (14))
                    const float l = fmaf(sc.a, dv, sc.b * f4get(m, q));       // Eq. (18)
                    const float bb = (f4get(x, q) - l) + tr;                  // B
                    const float e = l - f4get(m, q), dl = l - f4get(l0, q);
                    own = fmaf(e, e, own);
                    dlc = fmaf(dl, dl, dlc);
                    bsq = fmaf(bb, bb, bsq);
                    f4set(lo, q, l);
                }
                __stcs(reinterpret_cast<float4*>(lc + rr), lo);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int64_t r = rr + q;
                    if (r >= d) continue;
                    const float x = XLoad<TX>::one(xc + r);
                    const float tr = tc[r] * sc.inv_rho;
                    const float l = fmaf(sc.a, (x - scol[r]) + tr, sc.b * mup[r]);
                    const float bb = (x - l) + tr;
                    const float e = l - mup[r], dl = l - lc[r];
                    own = fmaf(e, e, own);
                    dlc = fmaf(dl, dl, dlc);
                    bsq = fmaf(bb, bb, bsq);
                    lc[r] = l;
                }
            }
        }
        ndl += dlc;
        own = warp_sum(own);
        dlc = warp_sum(dlc);
        bsq = warp_sum(bsq);
        if (lane == 0) {
            own_part[(int64_t)blockIdx.y * n + col] = own;
            dl_part[(int64_t)blockIdx.y * n + col] = dlc;
            bn_part[(int64_t)blockIdx.y * n + col] = bsq;
        }
    }
    const double w1 = warp_sum((double)ndl);
    if (lane == 0) nred[warp] = w1;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += nred[w];
        norm_part[((int64_t)blockIdx.y * gridDim.x + tile_idx) * 3 + 1] = t;
    }
}

template <typename TX, bool VEC>
__global__ void __launch_bounds__(kThreads, 2)
    k_l21_pass_b(const TX* __restrict__ X, int64_t ldx, const float* __restrict__ L,
                 float* __restrict__ S, float* __restrict__ Th, int64_t lds,
                 const int32_t* __restrict__ perm, const TileDesc* __restrict__ tiles,
                 const DevStatus* __restrict__ status, int64_t d, int64_t n, IterScalars sc,
                 const float* __restrict__ bn_part, float* __restrict__ Dpart,
                 double* __restrict__ norm_part) {
    __shared__ float red[kThreads / 32][kChunkRows];
    __shared__ double nred[kThreads / 32][2];
    const int tile_idx = blockIdx.x;
    if (tile_idx >= status->ntiles) return;
    const TileDesc td = tiles[tile_idx];
    const int64_t r0 = (int64_t)blockIdx.y * kChunkRows;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nch = gridDim.y;
    float4 acc[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    float nr = 0.f, nds = 0.f;
    for (int k = warp; k < td.len; k += kThreads / 32) {
        const int64_t col = perm[td.start + k];
        // ||B_j||^2 over every row chunk of pass A, then the column's factors
        float nb2 = 0.f;
        for (int ch = lane; ch < nch; ch += 32) nb2 += bn_part[(int64_t)ch * n + col];
        nb2 = warp_sum(nb2);
        const float nb = sqrtf(nb2);
        const bool shrink = nb > sc.inv_rho;
        const float f = shrink ? 1.f - sc.inv_rho / nb : 0.f;     // S_j = f B_j
        const float g = shrink ? 1.f / nb : sc.rho;                // Theta_j = g B_j
        const TX* xc = X + col * ldx;
        const float* lc = L + col * lds;
        float* scol = S + col * lds;
        float* tc = Th + col * lds;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int64_t rr = r0 + s * 128 + lane * 4;
            if (VEC) {
                if (rr >= d) continue;
                const float4 x = XLoad<TX>::four(xc + rr);
                const float4 sv = __ldcs(reinterpret_cast<const float4*>(scol + rr));
                const float4 tv = __ldcs(reinterpret_cast<const float4*>(tc + rr));
                const float4 lv = __ldcs(reinterpret_cast<const float4*>(lc + rr));
                float4 so, to;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float bb = (f4get(x, q) - f4get(lv, q)) + f4get(tv, q) * sc.inv_rho;
                    const float sn = f * bb, tn = g * bb;
                    const float res = (f4get(x, q) - f4get(lv, q)) - sn;
                    const float ds = sn - f4get(sv, q);
                    nr = fmaf(res, res, nr);
                    nds = fmaf(ds, ds, nds);
                    f4set(so, q, sn);
                    f4set(to, q, tn);
                    f4set(acc[s], q, f4get(acc[s], q) + ((f4get(x, q) - sn) + tn * sc.inv_rho_next));
                }
                __stcs(reinterpret_cast<float4*>(scol + rr), so);
                __stcs(reinterpret_cast<float4*>(tc + rr), to);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int64_t r = rr + q;
                    if (r >= d) continue;
                    const float x = XLoad<TX>::one(xc + r);
                    const float bb = (x - lc[r]) + tc[r] * sc.inv_rho;
                    const float sn = f * bb, tn = g * bb;
                    const float res = (x - lc[r]) - sn;
                    const float ds = sn - scol[r];
                    nr = fmaf(res, res, nr);
                    nds = fmaf(ds, ds, nds);
                    scol[r] = sn;
                    tc[r] = tn;
                    f4set(acc[s], q, f4get(acc[s], q) + ((x - sn) + tn * sc.inv_rho_next));
                }
            }
        }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int q = 0; q < 4; ++q) red[warp][s * 128 + lane * 4 + q] = f4get(acc[s], q);
    const double w0 = warp_sum((double)nr), w2 = warp_sum((double)nds);
    if (lane == 0) {
        nred[warp][0] = w0;
        nred[warp][1] = w2;
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
    if (threadIdx.x < 2) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += nred[w][threadIdx.x];
        norm_part[((int64_t)blockIdx.y * gridDim.x + tile_idx) * 3 + (threadIdx.x == 0 ? 0 : 2)] = t;
    }
}

inline int grid_for(int64_t work, int per) { return (int)((work + per - 1) / per); }

}  // namespace

cudaError_t launch_iteration_l21(int dtype, const void* X, int64_t ldx, float* L, float* S, float* Th,
                                 int64_t lds, const float* mu, const int32_t* perm,
                                 const TileDesc* tiles, int max_tiles, const DevStatus* status,
                                 int64_t d, int64_t n, IterScalars sc, float* Dpart, float* own_part,
                                 float* dl_part, float* bn_part, double* norm_part, bool vec,
                                 cudaStream_t st) {
    count_launches(2);
    const dim3 grid(max_tiles, grid_for(d, kChunkRows));
    RESPCA_DISPATCH_X(dtype, TX, {
        if (vec) {
            k_l21_pass_a<TX, true><<<grid, kThreads, 0, st>>>((const TX*)X, ldx, L, S, Th, lds, mu, perm,
                                                              tiles, status, d, n, sc, own_part, dl_part,
                                                              bn_part, norm_part);
            k_l21_pass_b<TX, true><<<grid, kThreads, 0, st>>>((const TX*)X, ldx, L, S, Th, lds, perm, tiles,
                                                              status, d, n, sc, bn_part, Dpart, norm_part);
        } else {
            k_l21_pass_a<TX, false><<<grid, kThreads, 0, st>>>((const TX*)X, ldx, L, S, Th, lds, mu, perm,
                                                               tiles, status, d, n, sc, own_part, dl_part,
                                                               bn_part, norm_part);
            k_l21_pass_b<TX, false><<<grid, kThreads, 0, st>>>((const TX*)X, ldx, L, S, Th, lds, perm, tiles,
                                                               status, d, n, sc, bn_part, Dpart, norm_part);
        }
    });
    return cudaGetLastError();
}

}  // namespace respca
