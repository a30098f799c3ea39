// Kernels of the learned warm start: an unrolled continuation of the
// iteration of Sec. 4 with the labels held fixed and learned per-layer steps
// rho_k and soft thresholds tau_k, its exact gradient, a width-64 MLP and an
// Adam step.  Layer k (Eq. (18), (24) with tau_k, (25)):
//   D = X - S + Theta/rho,  mu = cluster means of D,  a = rho/(2 lambda + rho)
//   L = a D + (1 - a) mu_p,  B = X - L + Theta/rho,  S' = soft(B, tau)
//   Theta' = Theta + rho (X - L - S')
// Reverse mode, given gS', gTheta' (and gL on the last layer):
//   gS~ = gS' - rho gTheta'             (S' enters Theta')
//   gB = gS~ [|B| > tau],  gtau = -sum gS~ sign(B) [|B| > tau]
//   gL = gL_ext - rho gTheta' - gB
//   gmu_i = (1 - a) sum_{j in i} gL_j,  gD = a gL + gmu_p / n_p
//   gS = -gD,  gTheta = gTheta' + (gB + gD) / rho
//   grho = sum gTheta' (X - L - S') + ga 2 lambda / (2 lambda + rho)^2
//          - (sum (gB + gD) Theta) / rho^2,      ga = sum gL (D - mu_p)
// Columns are visited through the label-sorted tiles, so the cluster sums of
// D (next layer's means) and of gL come out per tile like Dpart.
#include "respca_internal.cuh"

namespace respca {

namespace {

constexpr int kNetRows = 512;   // rows per CTA (one chunk), as the fused iteration

// Row mapping of a CTA's 512-row chunk: with VEC (d, the leading dimensions
// and the bases 16-byte aligned) each lane takes 4 slots of 4 consecutive rows
// through 16-byte accesses, otherwise 16 slots of one row; the arithmetic per
// element is the same either way.
template <bool VEC>
struct NetRows {
    static constexpr int kSlots = VEC ? 4 : 16;
    static constexpr int kW = VEC ? 4 : 1;
    static __device__ __forceinline__ int row(int q, int lane) { return VEC ? (q * 32 + lane) * 4 : q * 32 + lane; }
    static __device__ __forceinline__ void ld(const float* p, float* v) {
        if (VEC) {
            const float4 t = *reinterpret_cast<const float4*>(p);
            v[0] = t.x;
            v[1] = t.y;
            v[2] = t.z;
            v[3] = t.w;
        } else {
            v[0] = *p;
        }
    }
    static __device__ __forceinline__ void st(float* p, const float* v) {
        if (VEC) *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
        else *p = v[0];
    }
};

// ---------------------------------------------------------------- forward
template <bool VEC>
__global__ void __launch_bounds__(kThreads)
    k_net_layer(const float* __restrict__ X, int64_t ldx, const float* __restrict__ S,
                const float* __restrict__ Th, float* __restrict__ L, float* __restrict__ Sn,
                float* __restrict__ Thn, int64_t lds, const float* __restrict__ mu,
                const int32_t* __restrict__ perm, const TileDesc* __restrict__ tiles,
                const DevStatus* __restrict__ status, int64_t d, NetScalars sc,
                float* __restrict__ Dpart) {
    using RM = NetRows<VEC>;
    constexpr int W = RM::kW;
    __shared__ float red[kThreads / 32][kNetRows];
    const int tile_idx = blockIdx.x;
    if (tile_idx >= status->ntiles) return;
    const TileDesc td = tiles[tile_idx];
    const int64_t r0 = (int64_t)blockIdx.y * kNetRows;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float* mup = mu + (int64_t)td.label * d;
    float acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.f;
    for (int k = warp; k < td.len; k += kThreads / 32) {
        const int64_t col = perm[td.start + k];
#pragma unroll
        for (int q = 0; q < RM::kSlots; ++q) {
            const int64_t r = r0 + RM::row(q, lane);
            if (r >= d) continue;
            float x[W], s[W], t[W], m[W], l[W], sn[W], tn[W];
            RM::ld(X + col * ldx + r, x);
            RM::ld(S + col * lds + r, s);
            RM::ld(Th + col * lds + r, t);
            RM::ld(mup + r, m);
#pragma unroll
            for (int e = 0; e < W; ++e) {
                const float dv = (x[e] - s[e]) + t[e] * sc.inv_rho;
                l[e] = fmaf(sc.a, dv, sc.b * m[e]);
                const float bb = (x[e] - l[e]) + t[e] * sc.inv_rho;
                const float mag = fabsf(bb) - sc.tau;
                sn[e] = mag > 0.f ? copysignf(mag, bb) : 0.f;
                tn[e] = t[e] + sc.rho * ((x[e] - l[e]) - sn[e]);
                acc[q * W + e] += (x[e] - sn[e]) + tn[e] * sc.inv_rho_next;   // D of the next layer
            }
            RM::st(L + col * lds + r, l);
            RM::st(Sn + col * lds + r, sn);
            RM::st(Thn + col * lds + r, tn);
        }
    }
#pragma unroll
    for (int q = 0; q < RM::kSlots; ++q)
#pragma unroll
        for (int e = 0; e < W; ++e) red[warp][RM::row(q, lane) + e] = acc[q * W + e];
    __syncthreads();
    for (int i = threadIdx.x; i < kNetRows; i += kThreads) {
        const int64_t r = r0 + i;
        if (r >= d) continue;
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) v += red[w][i];
        Dpart[(int64_t)tile_idx * d + r] = v;
    }
}

// ---------------------------------------------------------------- inference forward
// The layer of k_net_layer for inference (no state is kept for a reverse
// pass): X is read in its own type, the input state (S, Theta) and the output
// state (S', Theta') are stored as TIN / TOUT (FP32, or BF16 holding the FP32
// result rounded once), and L is written only when WRITE_L (the last layer;
// the intermediate layers' L is never read).  Arithmetic is FP32 and the same
// as k_net_layer's per element.  With VEC (d, the leading dimensions and the
// bases aligned to 4 elements) each lane takes 4 slots of 4 consecutive rows.
template <bool VEC, typename TX, typename TIN, typename TOUT, bool WRITE_L>
__global__ void __launch_bounds__(kThreads)
    k_net_infer(const TX* __restrict__ X, int64_t ldx, const TIN* __restrict__ S,
                const TIN* __restrict__ Th, int64_t ldin, float* __restrict__ L,
                TOUT* __restrict__ Sn, TOUT* __restrict__ Thn, int64_t ldout,
                const float* __restrict__ mu, const int32_t* __restrict__ perm,
                const TileDesc* __restrict__ tiles, const DevStatus* __restrict__ status, int64_t d,
                NetScalars sc, float* __restrict__ Dpart) {
    constexpr int kSlots = VEC ? 4 : 16;
    constexpr int W = VEC ? 4 : 1;
    __shared__ float red[kThreads / 32][kNetRows];
    const int tile_idx = blockIdx.x;
    if (tile_idx >= status->ntiles) return;
    const TileDesc td = tiles[tile_idx];
    const int64_t r0 = (int64_t)blockIdx.y * kNetRows;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float* mup = mu + (int64_t)td.label * d;
    float acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.f;
    for (int k = warp; k < td.len; k += kThreads / 32) {
        const int64_t col = perm[td.start + k];
#pragma unroll
        for (int q = 0; q < kSlots; ++q) {
            const int64_t r = r0 + (VEC ? (q * 32 + lane) * 4 : q * 32 + lane);
            if (r >= d) continue;
            float x[W], s[W], t[W], m[W], l[W], sn[W], tn[W];
            if (VEC) {
                const float4 xv = XLoad<TX>::four(X + col * ldx + r);
                const float4 sv = StateIO<TIN>::load4(S + col * ldin + r);
                const float4 tv = StateIO<TIN>::load4(Th + col * ldin + r);
                const float4 mv = *reinterpret_cast<const float4*>(mup + r);
#pragma unroll
                for (int e = 0; e < W; ++e) {
                    x[e] = f4get(xv, e);
                    s[e] = f4get(sv, e);
                    t[e] = f4get(tv, e);
                    m[e] = f4get(mv, e);
                }
            } else {
                x[0] = XLoad<TX>::one(X + col * ldx + r);
                s[0] = StateIO<TIN>::load1(S + col * ldin + r);
                t[0] = StateIO<TIN>::load1(Th + col * ldin + r);
                m[0] = mup[r];
            }
#pragma unroll
            for (int e = 0; e < W; ++e) {
                const float dv = (x[e] - s[e]) + t[e] * sc.inv_rho;
                l[e] = fmaf(sc.a, dv, sc.b * m[e]);
                const float bb = (x[e] - l[e]) + t[e] * sc.inv_rho;
                const float mag = fabsf(bb) - sc.tau;
                sn[e] = mag > 0.f ? copysignf(mag, bb) : 0.f;
                tn[e] = t[e] + sc.rho * ((x[e] - l[e]) - sn[e]);
                // the next layer reads the stored values: sum its D from them
                acc[q * W + e] += (x[e] - StateIO<TOUT>::round(sn[e])) +
                                  StateIO<TOUT>::round(tn[e]) * sc.inv_rho_next;
            }
            if (VEC) {
                float4 lv, sv, tv;
#pragma unroll
                for (int e = 0; e < W; ++e) {
                    f4set(lv, e, l[e]);
                    f4set(sv, e, sn[e]);
                    f4set(tv, e, tn[e]);
                }
                if (WRITE_L) StateIO<float>::store4(L + col * ldout + r, lv);
                StateIO<TOUT>::store4(Sn + col * ldout + r, sv);
                StateIO<TOUT>::store4(Thn + col * ldout + r, tv);
            } else {
                if (WRITE_L) L[col * ldout + r] = l[0];
                StateIO<TOUT>::store1(Sn + col * ldout + r, sn[0]);
                StateIO<TOUT>::store1(Thn + col * ldout + r, tn[0]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kSlots; ++q)
#pragma unroll
        for (int e = 0; e < W; ++e) red[warp][(VEC ? (q * 32 + lane) * 4 : q * 32 + lane) + e] = acc[q * W + e];
    __syncthreads();
    for (int i = threadIdx.x; i < kNetRows; i += kThreads) {
        const int64_t r = r0 + i;
        if (r >= d) continue;
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) v += red[w][i];
        Dpart[(int64_t)tile_idx * d + r] = v;
    }
}

// ---------------------------------------------------------------- backward
// Per-CTA partial sums of the scalar gradients: 0: sum gTheta' R, 1: gtau,
// 2: ga, 3: sum (gB + gD) Theta (pass 2 adds its gD part).
constexpr int kNetScal = 4;

template <int PASS, bool VEC>
__global__ void __launch_bounds__(kThreads)
    k_net_back(const float* __restrict__ X, int64_t ldx, const float* __restrict__ S,
               const float* __restrict__ Th, int64_t lds, const float* __restrict__ mu,
               const int32_t* __restrict__ perm, const TileDesc* __restrict__ tiles,
               const DevStatus* __restrict__ status, int64_t d,
               NetScalars sc, const float* __restrict__ gLext, float* __restrict__ gS,
               float* __restrict__ gT, const float* __restrict__ gmean, float* __restrict__ Gpart,
               double* __restrict__ scal_part) {
    using RM = NetRows<VEC>;
    constexpr int W = RM::kW;
    __shared__ float red[kThreads / 32][kNetRows];
    __shared__ double sred[kThreads / 32][kNetScal];
    const int tile_idx = blockIdx.x;
    const int64_t part = ((int64_t)blockIdx.y * gridDim.x + tile_idx) * kNetScal;
    if (tile_idx >= status->ntiles) {
        if (threadIdx.x < kNetScal) scal_part[part + threadIdx.x] = 0.0;
        return;
    }
    const TileDesc td = tiles[tile_idx];
    const int64_t r0 = (int64_t)blockIdx.y * kNetRows;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float* mup = mu + (int64_t)td.label * d;
    const float* gmp = gmean ? gmean + (int64_t)td.label * d : nullptr;
    float acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.f;
    float s_tr = 0.f, s_tau = 0.f, s_a = 0.f, s_rt = 0.f;
    for (int k = warp; k < td.len; k += kThreads / 32) {
        const int64_t col = perm[td.start + k];
#pragma unroll
        for (int q = 0; q < RM::kSlots; ++q) {
            const int64_t r = r0 + RM::row(q, lane);
            if (r >= d) continue;
            const int64_t e0 = col * lds + r;
            float x[W], s[W], t[W], m[W], gso[W], gto[W], gle[W], gm[W];
            RM::ld(X + col * ldx + r, x);
            RM::ld(S + e0, s);
            RM::ld(Th + e0, t);
            RM::ld(mup + r, m);
            RM::ld(gS + e0, gso);
            RM::ld(gT + e0, gto);
            if (gLext) RM::ld(gLext + e0, gle);
            else
#pragma unroll
                for (int e = 0; e < W; ++e) gle[e] = 0.f;
            if (PASS == 2) RM::ld(gmp + r, gm);
#pragma unroll
            for (int e = 0; e < W; ++e) {
                const float dv = (x[e] - s[e]) + t[e] * sc.inv_rho;
                const float l = fmaf(sc.a, dv, sc.b * m[e]);
                const float bb = (x[e] - l) + t[e] * sc.inv_rho;
                const bool on = fabsf(bb) > sc.tau;
                const float sn = on ? copysignf(fabsf(bb) - sc.tau, bb) : 0.f;
                const float gsc = gso[e] - sc.rho * gto[e];
                const float gb = on ? gsc : 0.f;
                const float gl = gle[e] - sc.rho * gto[e] - gb;
                if (PASS == 1) {
                    s_tr = fmaf(gto[e], (x[e] - l) - sn, s_tr);
                    if (on) s_tau -= gsc * (bb > 0.f ? 1.f : -1.f);
                    s_a = fmaf(gl, dv - m[e], s_a);
                    s_rt = fmaf(gb, t[e], s_rt);
                    acc[q * W + e] += gl;
                } else {
                    const float gd = fmaf(sc.a, gl, sc.b * gm[e]);
                    s_rt = fmaf(gd, t[e], s_rt);
                    gso[e] = -gd;                                   // becomes dloss/dS of the layer input
                    gto[e] = gto[e] + (gb + gd) * sc.inv_rho;       // and dloss/dTheta
                }
            }
            if (PASS == 2) {
                RM::st(gS + e0, gso);
                RM::st(gT + e0, gto);
            }
        }
    }
    if (PASS == 1) {
#pragma unroll
        for (int q = 0; q < RM::kSlots; ++q)
#pragma unroll
            for (int e = 0; e < W; ++e) red[warp][RM::row(q, lane) + e] = acc[q * W + e];
    }
    const double w0 = warp_sum((double)s_tr), w1 = warp_sum((double)s_tau), w2 = warp_sum((double)s_a),
                 w3 = warp_sum((double)s_rt);
    if (lane == 0) {
        sred[warp][0] = w0;
        sred[warp][1] = w1;
        sred[warp][2] = w2;
        sred[warp][3] = w3;
    }
    __syncthreads();
    if (PASS == 1) {
        for (int i = threadIdx.x; i < kNetRows; i += kThreads) {
            const int64_t r = r0 + i;
            if (r >= d) continue;
            float v = 0.f;
#pragma unroll
            for (int w = 0; w < kThreads / 32; ++w) v += red[w][i];
            Gpart[(int64_t)tile_idx * d + r] = v;
        }
    }
    if (threadIdx.x < kNetScal) {
        double v = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) v += sred[w][threadIdx.x];
        scal_part[part + threadIdx.x] = v;
    }
}

// Sum of `parts` rows of kNetScal partials (fixed order) into out[kNetScal].
__global__ void k_net_scal_sum(const double* __restrict__ part, int64_t parts, double* __restrict__ out) {
    __shared__ double red[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int s = 0; s < kNetScal; ++s) {
        double v = 0.0;
        for (int64_t i = threadIdx.x; i < parts; i += kThreads) v += part[i * kNetScal + s];
        v = warp_sum(v);
        if (lane == 0) red[warp] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) t += red[w];
            out[s] = t;
        }
        __syncthreads();
    }
}

// loss = scale (||L - Lt||^2 + ||S - St||^2) and its gradient gL, gS; gT = 0.
// One CTA column-slab per blockIdx.x, rows over the threads.
__global__ void __launch_bounds__(kThreads)
    k_net_loss(const float* __restrict__ L, const float* __restrict__ S, int64_t lds,
               const float* __restrict__ Lt, const float* __restrict__ St, int64_t ldt, int64_t d, int64_t n,
               float scale, float* __restrict__ gL, float* __restrict__ gS, float* __restrict__ gT,
               double* __restrict__ part) {
    __shared__ double red[kThreads / 32];
    double acc = 0.0;
    for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
        float cs = 0.f;
        for (int64_t r = threadIdx.x; r < d; r += kThreads) {
            const int64_t e = j * lds + r;
            const float el = L[e] - Lt[j * ldt + r], es = S[e] - St[j * ldt + r];
            cs = fmaf(el, el, fmaf(es, es, cs));
            gL[e] = 2.f * scale * el;
            gS[e] = 2.f * scale * es;
            gT[e] = 0.f;
        }
        acc += (double)cs;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        part[blockIdx.x] = t * (double)scale;
    }
}

// out[0] = sum of part[0 .. count) (fixed order: strided per thread, then the warps).
__global__ void k_net_sum(const double* __restrict__ part, int64_t count, double* __restrict__ out) {
    __shared__ double red[kThreads / 32];
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < count; i += kThreads) v += part[i];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        out[0] = t;
    }
}

// ---------------------------------------------------------------- MLP
// out = W2 tanh(W1 z + b1) + b2; params packed [W1 (H x nz) | b1 (H) | W2 (nout x H) | b2 (nout)].
__global__ void k_mlp_forward(const float* __restrict__ P, int nz, int H, int nout,
                              const float* __restrict__ z, float* __restrict__ out,
                              float* __restrict__ hidden) {
    extern __shared__ float h[];
    const float* W1 = P;
    const float* b1 = W1 + (int64_t)H * nz;
    const float* W2 = b1 + H;
    const float* b2 = W2 + (int64_t)nout * H;
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        float s = b1[i];
        for (int k = 0; k < nz; ++k) s = fmaf(W1[i * nz + k], z[k], s);
        h[i] = tanhf(s);
        if (hidden) hidden[i] = h[i];
    }
    __syncthreads();
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        float s = b2[o];
        for (int i = 0; i < H; ++i) s = fmaf(W2[o * H + i], h[i], s);
        out[o] = s;
    }
}

// Gradient of <gout, out> with respect to the packed parameters.
__global__ void k_mlp_backward(const float* __restrict__ P, int nz, int H, int nout,
                               const float* __restrict__ z, const float* __restrict__ hidden,
                               const float* __restrict__ gout, float* __restrict__ G, int accumulate) {
    extern __shared__ float gh[];
    const float* W2 = P + (int64_t)H * nz + H;
    float* gW1 = G;
    float* gb1 = gW1 + (int64_t)H * nz;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + (int64_t)nout * H;
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        gb2[o] = (accumulate ? gb2[o] : 0.f) + gout[o];
        for (int i = 0; i < H; ++i) gW2[o * H + i] = (accumulate ? gW2[o * H + i] : 0.f) + gout[o] * hidden[i];
    }
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        float s = 0.f;
        for (int o = 0; o < nout; ++o) s = fmaf(W2[o * H + i], gout[o], s);
        gh[i] = s * (1.f - hidden[i] * hidden[i]);   // through tanh
    }
    __syncthreads();
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        gb1[i] = (accumulate ? gb1[i] : 0.f) + gh[i];
        for (int k = 0; k < nz; ++k) gW1[i * nz + k] = (accumulate ? gW1[i * nz + k] : 0.f) + gh[i] * z[k];
    }
}

__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                       float* __restrict__ V, int64_t count, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float g = G[i];
    const float m = b1 * M[i] + (1.f - b1) * g;
    const float v = b2 * V[i] + (1.f - b2) * g * g;
    M[i] = m;
    V[i] = v;
    P[i] -= lr * (m * c1) / (sqrtf(v * c2) + eps);
}

inline int grid_for(int64_t work, int per) { return (int)((work + per - 1) / per); }

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// 16-byte row accesses: d and both leading dimensions multiples of 4 floats and
// every base 16-byte aligned (the rows of mu are then aligned too).
template <typename... Ptrs>
bool net_vec(int64_t d, int64_t ldx, int64_t lds, const Ptrs*... ptrs) {
    if (d % 4 != 0 || ldx % 4 != 0 || lds % 4 != 0) return false;
    bool ok = true;
    ((ok = ok && aligned16(ptrs)), ...);
    return ok;
}

}  // namespace

int net_row_chunks(int64_t d) { return grid_for(d, kNetRows); }

cudaError_t launch_net_layer(const float* X, int64_t ldx, const float* S, const float* Th, float* L,
                             float* Sn, float* Thn, int64_t lds, const float* mu, const int32_t* perm,
                             const TileDesc* tiles, int max_tiles, const DevStatus* status, int64_t d,
                             const NetScalars& sc, float* Dpart, cudaStream_t st) {
    count_launches(1);
    const dim3 grid(max_tiles, grid_for(d, kNetRows));
    if (net_vec(d, ldx, lds, X, S, Th, L, Sn, Thn, mu))
        k_net_layer<true><<<grid, kThreads, 0, st>>>(X, ldx, S, Th, L, Sn, Thn, lds, mu, perm, tiles, status, d,
                                                     sc, Dpart);
    else
        k_net_layer<false><<<grid, kThreads, 0, st>>>(X, ldx, S, Th, L, Sn, Thn, lds, mu, perm, tiles, status, d,
                                                      sc, Dpart);
    return cudaGetLastError();
}

template <typename TX, typename TI, typename TO, bool WL>
void net_infer_go(bool vec, dim3 grid, cudaStream_t st, const void* X, int64_t ldx, const void* S,
                  const void* Th, int64_t ldin, float* L, void* Sn, void* Thn, int64_t ldout, const float* mu,
                  const int32_t* perm, const TileDesc* tiles, const DevStatus* status, int64_t d,
                  const NetScalars& sc, float* Dpart) {
    const TX* x = static_cast<const TX*>(X);
    const TI* s = static_cast<const TI*>(S);
    const TI* t = static_cast<const TI*>(Th);
    TO* sn = static_cast<TO*>(Sn);
    TO* tn = static_cast<TO*>(Thn);
    if (vec)
        k_net_infer<true, TX, TI, TO, WL><<<grid, kThreads, 0, st>>>(x, ldx, s, t, ldin, L, sn, tn, ldout, mu,
                                                                      perm, tiles, status, d, sc, Dpart);
    else
        k_net_infer<false, TX, TI, TO, WL><<<grid, kThreads, 0, st>>>(x, ldx, s, t, ldin, L, sn, tn, ldout, mu,
                                                                       perm, tiles, status, d, sc, Dpart);
}

// Inference layer: xdt / sin / sout are the element types of X (0 f32, 1 bf16,
// 2 f16), of the input state and of the output state (0 f32, 1 bf16); L
// (FP32, leading dimension ldout) is written when non-null, which requires
// sout = 0.
cudaError_t launch_net_infer(int xdt, int sin, int sout, const void* X, int64_t ldx, const void* S,
                             const void* Th, int64_t ldin, float* L, void* Sn, void* Thn, int64_t ldout,
                             const float* mu, const int32_t* perm, const TileDesc* tiles, int max_tiles,
                             const DevStatus* status, int64_t d, const NetScalars& sc, float* Dpart,
                             cudaStream_t st) {
    if (L && sout != 0) return cudaErrorInvalidValue;
    count_launches(1);
    const dim3 grid(max_tiles, grid_for(d, kNetRows));
    auto al = [](const void* p, size_t esz) { return (reinterpret_cast<uintptr_t>(p) % (4 * esz)) == 0; };
    const size_t ex = xdt == 0 ? 4 : 2, ei = sin == 0 ? 4 : 2, eo = sout == 0 ? 4 : 2;
    const bool vec = (d % 4 == 0) && (ldx % 4 == 0) && (ldin % 4 == 0) && (ldout % 4 == 0) && al(X, ex) &&
                     al(S, ei) && al(Th, ei) && al(Sn, eo) && al(Thn, eo) && (!L || al(L, 4)) && al(mu, 4);
    using BF = __nv_bfloat16;
    RESPCA_DISPATCH_X(xdt, TX, {
        if (sin == 0 && sout == 0) {
            if (L)
                net_infer_go<TX, float, float, true>(vec, grid, st, X, ldx, S, Th, ldin, L, Sn, Thn, ldout, mu,
                                                     perm, tiles, status, d, sc, Dpart);
            else
                net_infer_go<TX, float, float, false>(vec, grid, st, X, ldx, S, Th, ldin, L, Sn, Thn, ldout, mu,
                                                      perm, tiles, status, d, sc, Dpart);
        } else if (sin == 0) {
            net_infer_go<TX, float, BF, false>(vec, grid, st, X, ldx, S, Th, ldin, L, Sn, Thn, ldout, mu, perm,
                                               tiles, status, d, sc, Dpart);
        } else if (sout == 1) {
            net_infer_go<TX, BF, BF, false>(vec, grid, st, X, ldx, S, Th, ldin, L, Sn, Thn, ldout, mu, perm,
                                            tiles, status, d, sc, Dpart);
        } else if (L) {
            net_infer_go<TX, BF, float, true>(vec, grid, st, X, ldx, S, Th, ldin, L, Sn, Thn, ldout, mu, perm,
                                              tiles, status, d, sc, Dpart);
        } else {
            net_infer_go<TX, BF, float, false>(vec, grid, st, X, ldx, S, Th, ldin, L, Sn, Thn, ldout, mu, perm,
                                               tiles, status, d, sc, Dpart);
        }
    });
    return cudaGetLastError();
}

cudaError_t launch_net_back(int pass, const float* X, int64_t ldx, const float* S, const float* Th,
                            int64_t lds, const float* mu, const int32_t* perm, const TileDesc* tiles,
                            int max_tiles, const DevStatus* status, int64_t d, const NetScalars& sc,
                            const float* gLext, float* gS, float* gT, const float* gmean, float* Gpart,
                            double* scal_part, double* scal_out, cudaStream_t st) {
    count_launches(2);
    const dim3 grid(max_tiles, grid_for(d, kNetRows));
    const bool vec = net_vec(d, ldx, lds, X, S, Th, gS, gT, mu) && (!gLext || aligned16(gLext)) &&
                     (!gmean || aligned16(gmean));
    if (pass == 1 && vec)
        k_net_back<1, true><<<grid, kThreads, 0, st>>>(X, ldx, S, Th, lds, mu, perm, tiles, status, d, sc, gLext,
                                                       gS, gT, nullptr, Gpart, scal_part);
    else if (pass == 1)
        k_net_back<1, false><<<grid, kThreads, 0, st>>>(X, ldx, S, Th, lds, mu, perm, tiles, status, d, sc, gLext,
                                                        gS, gT, nullptr, Gpart, scal_part);
    else if (vec)
        k_net_back<2, true><<<grid, kThreads, 0, st>>>(X, ldx, S, Th, lds, mu, perm, tiles, status, d, sc, gLext,
                                                       gS, gT, gmean, nullptr, scal_part);
    else
        k_net_back<2, false><<<grid, kThreads, 0, st>>>(X, ldx, S, Th, lds, mu, perm, tiles, status, d, sc, gLext,
                                                        gS, gT, gmean, nullptr, scal_part);
    k_net_scal_sum<<<1, kThreads, 0, st>>>(scal_part, (int64_t)grid.x * grid.y, scal_out);
    return cudaGetLastError();
}

cudaError_t launch_net_loss(const float* L, const float* S, int64_t lds, const float* Lt, const float* St,
                            int64_t ldt, int64_t d, int64_t n, float scale, float* gL, float* gS, float* gT,
                            double* part, int parts, double* out, cudaStream_t st) {
    count_launches(2);
    k_net_loss<<<parts, kThreads, 0, st>>>(L, S, lds, Lt, St, ldt, d, n, scale, gL, gS, gT, part);
    k_net_sum<<<1, kThreads, 0, st>>>(part, parts, out);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float* P, int nz, int H, int nout, const float* z, float* out,
                               float* hidden, cudaStream_t st) {
    count_launches(1);
    k_mlp_forward<<<1, 128, sizeof(float) * H, st>>>(P, nz, H, nout, z, out, hidden);
    return cudaGetLastError();
}

cudaError_t launch_mlp_backward(const float* P, int nz, int H, int nout, const float* z, const float* hidden,
                                const float* gout, float* G, int accumulate, cudaStream_t st) {
    count_launches(1);
    k_mlp_backward<<<1, 128, sizeof(float) * H, st>>>(P, nz, H, nout, z, hidden, gout, G, accumulate);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* P, const float* G, float* M, float* V, int64_t count, float lr, float b1,
                        float b2, float eps, float c1, float c2, cudaStream_t st) {
    count_launches(1);
    k_adam<<<grid_for(count, kThreads), kThreads, 0, st>>>(P, G, M, V, count, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace respca
