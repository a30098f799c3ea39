// Batched RES-PCA in one persistent launch (respca_solve_batched_persistent,
// include/respca.h).
//
// Every problem of the batch runs the iteration of Sec. 4 -- the L step of
// Eq. (18), Lloyd's method for the p step (Sec. 4.2), the S step of Eq. (24),
// the Theta and rho updates of Eq. (25) and the Sec. 5 stopping rule -- after
// initial labels by k-means++ and Lloyd on X (or the caller's p0).  The work
// of one problem is a sequence of phases; each phase is split into work items
// over row blocks (cluster sums, element-wise updates: a row block sees every
// column, so its cluster sums are complete without cross-CTA reduction) or
// column blocks (the L step and the nearest-centroid search: a column block
// sees whole columns, so its distances are complete).
//
// Scheduling: one CTA per slot on every SM pulls items from a device-side
// claim word per problem (generation | item count | next item).  The CTA that
// completes the last item of a phase runs the phase's serial tail (fixed-order
// reductions, the label sort, the k-means++ pick, the stopping test) and
// publishes the next phase by swapping in a new claim word.  No CTA ever
// waits for another: a CTA with nothing to claim polls (a bounded number of
// times; then it sets the timeout flag, and every CTA leaves at its next
// item boundary).  Data that other CTAs write during the launch is read with
// L2-only loads, so no stale L1 line is ever used.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/respca.h"
#include "respca_internal.cuh"

namespace respca {
namespace batched {

constexpr int kBT = 256;                 // threads per CTA
constexpr int kBW = kBT / 32;            // warps per CTA
constexpr int kChunk = 128;              // rows per chunk of a column item (4 per lane)
constexpr int kMaxC = 64;                // largest c of this path

enum Phase : int32_t {
    PH_FRO = 0,      // row: ||X||^2, non-finite scan, L = S = Theta = 0
    PH_SEED,         // col: D2 against centre k (k-means++)
    PH_ASSIGN_X,     // col: nearest centroid of the columns of X (initial Lloyd)
    PH_MEANS_X,      // row: cluster means of X
    PH_SUMS_D,       // row: cluster means of D = X - S + Theta/rho (start of the iterations)
    PH_LSTEP,        // row: L step (Eq. (18)), ||L_{t+1} - L_t||^2
    PH_MEANS_L,      // row: cluster means of L (further Lloyd passes)
    PH_ASSIGN_L,     // col: nearest centroid of the columns of L (every pass of the p step)
    PH_STHETA,       // row: S step, Theta step, norms, means of the next D
    PH_DONE
};

enum BStatus : int32_t { BS_OK = 0, BS_NONFINITE = 1, BS_BAD_LABELS = 2 };

// Per-problem description (read-only during the launch).
struct BProb {
    const float* X;
    float* L;
    float* S;
    float* Th;
    int32_t* p;
    const int32_t* p0;
    int64_t ldx, lds, ldt;
    int32_t d, n, c, max_iter, km_max, W, cmax, row_items, col_items;
    double lam, tol, kappa;
    // workspace
    float* mu;            // c x d, centroid i at mu + i d
    int32_t* perm;        // n: columns sorted by label (stable)
    int32_t* offs;        // c + 1: start of each label's run in perm
    int32_t* pstart;      // n: labels at the start of the p step
    uint8_t* active;      // c: cluster takes part in assignments
    double* D2;           // n: k-means++ squared distances
    int32_t* centers;     // c
    const double* u;      // c draws in [0, 1)
    double* rpart;        // row_items x 3: item partial sums
    double* cpart;        // col_items x 2: item partial sums (dL^2, changes)
};

// Per-problem mutable control block (device).
struct BCtl {
    unsigned long long claim;   // gen:16 | nitems:24 | next:24
    int32_t done;               // completed items of the current phase
    int32_t phase;
    int32_t iter;               // ALM iterations completed
    int32_t passes;             // Lloyd passes of the current p step
    int32_t init_passes;
    int32_t seed_k;
    int32_t status;
    int32_t converged;
    double rho;
    double nx2;
    double dl2;                 // ||L_{t+1} - L_t||^2 of the current iteration
    double err, e_res, e_dl, e_ds;
    long long label_changes;
    long long lloyd_passes;
    long long last_changes;
};

// Launch-wide control.
struct BGlobal {
    int32_t finished;           // problems done
    int32_t abort;              // a CTA gave up waiting
    int32_t timeout;
    int32_t pad;
};

// Field-wise copies of a control block through volatile (L2-coherent)
// accesses: another SM may have written it during the launch.
__device__ void load_ctl(const BCtl* g, BCtl& o) {
    const volatile BCtl* v = g;
    o.phase = v->phase;
    o.iter = v->iter;
    o.passes = v->passes;
    o.init_passes = v->init_passes;
    o.seed_k = v->seed_k;
    o.status = v->status;
    o.converged = v->converged;
    o.rho = v->rho;
    o.nx2 = v->nx2;
    o.dl2 = v->dl2;
    o.err = v->err;
    o.e_res = v->e_res;
    o.e_dl = v->e_dl;
    o.e_ds = v->e_ds;
    o.label_changes = v->label_changes;
    o.lloyd_passes = v->lloyd_passes;
    o.last_changes = v->last_changes;
}

__device__ void store_ctl(BCtl* g, const BCtl& o) {
    volatile BCtl* v = g;
    v->iter = o.iter;
    v->passes = o.passes;
    v->init_passes = o.init_passes;
    v->seed_k = o.seed_k;
    v->status = o.status;
    v->converged = o.converged;
    v->rho = o.rho;
    v->nx2 = o.nx2;
    v->dl2 = o.dl2;
    v->err = o.err;
    v->e_res = o.e_res;
    v->e_dl = o.e_dl;
    v->e_ds = o.e_ds;
    v->label_changes = o.label_changes;
    v->lloyd_passes = o.lloyd_passes;
    v->last_changes = o.last_changes;
}

__device__ __forceinline__ unsigned long long make_claim(unsigned gen, unsigned nitems) {
    return ((unsigned long long)(gen & 0xFFFFu) << 48) | ((unsigned long long)(nitems & 0xFFFFFFu) << 24);
}
__device__ __forceinline__ unsigned claim_gen(unsigned long long w) { return (unsigned)(w >> 48); }
__device__ __forceinline__ unsigned claim_n(unsigned long long w) { return (unsigned)((w >> 24) & 0xFFFFFFu); }
__device__ __forceinline__ unsigned claim_next(unsigned long long w) { return (unsigned)(w & 0xFFFFFFu); }

// L2-only loads of data other CTAs write during the launch.
__device__ __forceinline__ float ldf(const float* p) { return __ldcg(p); }
__device__ __forceinline__ double ldd(const double* p) { return __ldcg(p); }
__device__ __forceinline__ int32_t ldi(const int32_t* p) { return __ldcg(p); }
__device__ __forceinline__ uint8_t ldu8(const uint8_t* p) {
    return (uint8_t)__ldcg(reinterpret_cast<const signed char*>(p));
}

__device__ __forceinline__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < kBW; ++w) t += red[w];
        red[kBW] = t;
    }
    __syncthreads();
    t = red[kBW];
    __syncthreads();
    return t;
}

// Shared memory of the persistent kernel (dynamic): a centroid chunk of the
// column items, per-warp row partials of the row items, scan scratch.
struct BSmem {
    union {
        struct {
            float cs[kMaxC * kChunk];    // 32 KB: centroid chunk of a column item
            double red[kBW][kChunk];     // 8 KB: per-warp row partials
        } it;
        float slot[(kMaxC + kBW) * kChunk];   // 36 KB: run sums of a row item, slot = label + warp
        int32_t hist[kMaxC * kBT];       // 64 KB: per-thread label histograms of the sort
    };
    double dscan[kBT + 1];
    double dred[kBW + 1];
    double inv_n[kMaxC];                 // 1 / n_i of the item's problem (0: empty cluster)
    int32_t offs_s[kMaxC + 1];
    int32_t wlo[kBW], whi[kBW];          // first and last label of each warp's range (row items)
    int32_t pick;
    int32_t item;
    int32_t nitems;
    int32_t pid;
    int32_t flag;
    int32_t next;
    int32_t aux;
    BCtl lc;                             // the finishing problem's control block (tail)
};

// ---------------------------------------------------------------- row items
// Rows [r0, r0 + KR*32) of every column; lane l takes rows r0 + l + 32 q.
// Cluster sums visit the columns in label-sorted order: for each cluster, warp
// w takes its columns in groups of kRG (loads of the group issued before the
// arithmetic), groups w, w + 8, ...; per-lane FP32 sums are flushed to FP64
// after every group and the 8 warps' partials are added in warp order, so
// every sum has one fixed order.  The descriptor's fields are copied to
// locals first: a store through L, S or Theta could otherwise alias them and
// force a reload after every store.
constexpr int kRG = 4;

template <int KR>
__device__ void row_item(const BProb& pbr, double rho, int phase, int item, BSmem& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)item * KR * 32;
    const float* __restrict__ X = pbr.X;
    float* __restrict__ L = pbr.L;
    float* __restrict__ S = pbr.S;
    float* __restrict__ Th = pbr.Th;
    float* __restrict__ mu = pbr.mu;
    const int32_t* __restrict__ perm = pbr.perm;
    const int32_t* __restrict__ offs = pbr.offs;
    const int64_t ldx = pbr.ldx, lds = pbr.lds, ldt = pbr.ldt;
    const int d = pbr.d, n = pbr.n, c = pbr.c;
    double* __restrict__ rpart = pbr.rpart;
    const double kappa = pbr.kappa;
    if (phase == PH_FRO) {
        // FP32 squares summed per lane, flushed to FP64 every 8 columns (the FP64
        // pipe is far slower than the FP32 one)
        double acc = 0.0, bad = 0.0;
        float fa = 0.f;
        int cols = 0;
        for (int j = warp; j < n; j += kBW) {
#pragma unroll
            for (int q = 0; q < KR; ++q) {
                const int64_t r = r0 + lane + 32 * q;
                if (r >= d) continue;
                const float x = __ldg(X + (int64_t)j * ldx + r);
                if (!isfinite(x)) bad += 1.0;
                fa = fmaf(x, x, fa);
                L[(int64_t)j * lds + r] = 0.f;
                S[(int64_t)j * lds + r] = 0.f;
                Th[(int64_t)j * ldt + r] = 0.f;
            }
            if (++cols == 8) {
                acc += (double)fa;
                fa = 0.f;
                cols = 0;
            }
        }
        acc += (double)fa;
        acc = block_sum(acc, sm.dred);
        bad = block_sum(bad, sm.dred);
        if (threadIdx.x == 0) {
            rpart[item * 3 + 0] = acc;
            rpart[item * 3 + 1] = bad;
        }
        return;
    }
    // phases over the label-sorted columns: warp w streams positions
    // [w n / 8, (w + 1) n / 8) of perm in groups of kRG, keeps the run sum of
    // the current label per lane (FP32, into FP64 every 8 groups) and stores
    // it to shared slot (label + w) when the label changes; labels never
    // decrease inside a warp's range, so each (warp, label) pair has its own
    // slot.  The slots of a label are then added in warp order.
    const float inv_rho = (float)(1.0 / rho);
    const float inv_rho_next = (float)(1.0 / (rho * kappa));   // D of the next iteration (PH_STHETA)
    const float rho_f = (float)fmin(rho, (double)FLT_MAX);
    const double lam = pbr.lam;
    const float a_f = (float)(rho / (2.0 * lam + rho)), b_f = (float)(2.0 * lam / (2.0 * lam + rho));
    const bool sums = phase != PH_LSTEP;
    double r2 = 0.0, ds2 = 0.0;
    float r2f = 0.f, ds2f = 0.f;
    const int p0 = (int)(((int64_t)warp * n) / kBW), p1 = (int)(((int64_t)(warp + 1) * n) / kBW);
    int l = 0;                      // label of position p0 (uniform over the warp)
    while (l + 1 < c && ldi(offs + l + 1) <= p0) ++l;
    int lend = ldi(offs + l + 1);
    if (lane == 0) {
        sm.wlo[warp] = (p0 < p1) ? l : 1 << 30;
        sm.whi[warp] = -1;
    }
    float mp[KR];                   // mu_p rows of the current label (PH_LSTEP)
    auto load_mu = [&]() {
#pragma unroll
        for (int q = 0; q < KR; ++q) {
            const int64_t r = r0 + lane + 32 * q;
            mp[q] = (phase == PH_LSTEP && r < d) ? ldf(mu + (int64_t)l * d + r) : 0.f;
        }
    };
    load_mu();
    float facc[KR];
    double dacc[KR];
#pragma unroll
    for (int q = 0; q < KR; ++q) {
        facc[q] = 0.f;
        dacc[q] = 0.0;
    }
    auto flush_run = [&]() {       // the run of label l ends
        if (sums) {
#pragma unroll
            for (int q = 0; q < KR; ++q)
                sm.slot[(l + warp) * kChunk + lane + 32 * q] = (float)(dacc[q] + (double)facc[q]);
        }
#pragma unroll
        for (int q = 0; q < KR; ++q) {
            facc[q] = 0.f;
            dacc[q] = 0.0;
        }
    };
    int groups = 0;
    for (int k0 = p0; k0 < p1; k0 += kRG) {
        int64_t js[kRG];
#pragma unroll
        for (int g = 0; g < kRG; ++g) js[g] = (k0 + g < p1) ? (int64_t)ldi(perm + k0 + g) : -1;
        // loads of the group (issued together)
        float x[kRG][KR], s1[kRG][KR], s2[kRG][KR], s3[kRG][KR];
#pragma unroll
        for (int g = 0; g < kRG; ++g)
#pragma unroll
            for (int q = 0; q < KR; ++q) {
                const int64_t r = r0 + lane + 32 * q;
                const bool ok = js[g] >= 0 && r < d;
                const int64_t j = js[g];
                x[g][q] = (ok && phase != PH_MEANS_L) ? __ldg(X + j * ldx + r) : 0.f;
                s1[g][q] = (ok && (phase == PH_MEANS_L || phase == PH_LSTEP || phase == PH_STHETA))
                               ? ldf(L + j * lds + r) : 0.f;
                s2[g][q] = (ok && phase != PH_MEANS_X && phase != PH_MEANS_L) ? ldf(S + j * lds + r) : 0.f;
                s3[g][q] = (ok && phase != PH_MEANS_X && phase != PH_MEANS_L) ? ldf(Th + j * ldt + r) : 0.f;
            }
#pragma unroll
        for (int g = 0; g < kRG; ++g) {
            if (js[g] < 0) break;
            const int k = k0 + g;
            if (k >= lend) {        // label boundary (uniform over the warp)
                flush_run();
                while (k >= lend) {
                    ++l;
                    lend = ldi(offs + l + 1);
                }
                load_mu();
            }
            const int64_t j = js[g];
#pragma unroll
            for (int q = 0; q < KR; ++q) {
                const int64_t r = r0 + lane + 32 * q;
                if (r >= d) continue;
                float v;
                if (phase == PH_MEANS_X) {
                    v = x[g][q];
                } else if (phase == PH_MEANS_L) {
                    v = s1[g][q];
                } else if (phase == PH_SUMS_D) {
                    v = (x[g][q] - s2[g][q]) + s3[g][q] * inv_rho;
                } else if (phase == PH_LSTEP) {   // Eq. (18): L = a D + (1 - a) mu_p
                    const float dv = (x[g][q] - s2[g][q]) + s3[g][q] * inv_rho;
                    const float lv = fmaf(a_f, dv, b_f * mp[q]);
                    r2f = fmaf(lv - s1[g][q], lv - s1[g][q], r2f);     // ||L_{t+1} - L_t||^2
                    L[j * lds + r] = lv;
                    v = 0.f;
                } else {   // PH_STHETA: Eq. (24), Eq. (25) as clip(rho B, -1, 1), norms, next D
                    const float xl = x[g][q] - s1[g][q];
                    const float B = xl + s3[g][q] * inv_rho;
                    const float mag = fabsf(B) - inv_rho;
                    const float sn = mag > 0.f ? copysignf(mag, B) : 0.f;
                    const float tn = fminf(1.f, fmaxf(-1.f, rho_f * B));
                    const float res = xl - sn;
                    r2f = fmaf(res, res, r2f);
                    ds2f = fmaf(sn - s2[g][q], sn - s2[g][q], ds2f);
                    S[j * lds + r] = sn;
                    Th[j * ldt + r] = tn;
                    v = (x[g][q] - sn) + tn * inv_rho_next;
                }
                facc[q] += v;
            }
        }
        if (++groups == 8) {   // FP32 over 32 columns, then FP64
#pragma unroll
            for (int q = 0; q < KR; ++q) {
                dacc[q] += (double)facc[q];
                facc[q] = 0.f;
            }
            r2 += (double)r2f;
            ds2 += (double)ds2f;
            r2f = ds2f = 0.f;
            groups = 0;
        }
    }
    if (p0 < p1) {
        flush_run();
        if (lane == 0) sm.whi[warp] = l;
    }
    r2 += (double)r2f;
    ds2 += (double)ds2f;
    __syncthreads();
    if (sums) {
        // 1 / n_i once per cluster and item (an FP64 division per element would
        // load the narrow FP64 pipe with tens of operations each)
        for (int i = threadIdx.x; i < c; i += kBT) {
            const int cnt = ldi(offs + i + 1) - ldi(offs + i);
            sm.inv_n[i] = cnt > 0 ? 1.0 / (double)cnt : 0.0;
        }
        __syncthreads();
        // mean of label i over rows: its slots (i + w) for the warps whose range held i
        for (int e = threadIdx.x; e < c * KR * 32; e += kBT) {
            const int i = e / (KR * 32), t = e - i * (KR * 32);
            const int64_t r = r0 + t;
            const double inv = sm.inv_n[i];
            if (inv == 0.0 || r >= d) continue;
            double sum = 0.0;
#pragma unroll
            for (int w = 0; w < kBW; ++w)
                if (sm.wlo[w] <= i && i <= sm.whi[w]) sum += (double)sm.slot[(i + w) * kChunk + t];
            mu[(int64_t)i * d + r] = (float)(sum * inv);
        }
    }
    __syncthreads();
    if (phase == PH_STHETA || phase == PH_LSTEP) {
        r2 = block_sum(r2, sm.dred);
        ds2 = block_sum(ds2, sm.dred);
        if (threadIdx.x == 0) {
            rpart[item * 3 + 0] = r2;
            rpart[item * 3 + 1] = ds2;
        }
    }
}

// ---------------------------------------------------------------- column items
// Columns [item W, item W + W): warp w takes CPW = 64 / CMAX consecutive
// columns; the rows are visited in chunks of 128 (lane l: rows l + 32 q), with
// the chunk of every centroid (or, for k-means++, of the centre column)
// staged in shared memory.  Software pipelined one chunk ahead: the next
// chunk's column values and staged values are loaded into registers while the
// current chunk is computed.  Rows past d and columns past n read as 0 on
// both sides, so they add nothing.  Squared distances are summed per lane in
// FP32 (ceil(d/32) terms at most) and across lanes by an FP32 tree (FP64 runs
// far slower), so each carries a relative error below eps = (ceil(d/32) + 9)
// 2^-23; candidates whose distance
// lies within that bound of the best one are re-decided in FP64 from the
// stored values (the plain sum of squared differences, ties to the lowest
// index).
template <int CMAX, int CPW, bool PREF>
__device__ void col_item(const BProb& pbr, int seed_k, int phase, int item, BSmem& sm) {
    constexpr int NQ = kChunk / 32;
    constexpr int MS = (CMAX * kChunk) / kBT;        // staged values per thread
    constexpr int MP = PREF ? MS : 1;                // of them prefetched into registers
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float* __restrict__ X = pbr.X;
    const float* __restrict__ Lm = pbr.L;
    const float* __restrict__ mu = pbr.mu;
    int32_t* __restrict__ lbl = pbr.p;
    double* __restrict__ D2 = pbr.D2;
    double* __restrict__ cpart = pbr.cpart;
    const int64_t ldx = pbr.ldx, lds = pbr.lds;
    const int W = pbr.W;
    const int d = pbr.d, n = pbr.n;
    const bool seed = phase == PH_SEED, fromL = phase == PH_ASSIGN_L;
    const int ce = seed ? 1 : pbr.c;
    const int64_t center = seed ? (int64_t)ldi(pbr.centers + seed_k) : 0;
    unsigned long long amask = 0ull;
    if (!seed)
        for (int i = 0; i < pbr.c; ++i)
            if (ldu8(pbr.active + i)) amask |= 1ull << i;
    int64_t col[CPW];
    int lab[CPW];
    float acc[CPW][CMAX];
#pragma unroll
    for (int k = 0; k < CPW; ++k) {
        col[k] = (int64_t)item * W + warp * CPW + k;
        lab[k] = (col[k] < n && !seed) ? ldi(lbl + col[k]) : 0;
#pragma unroll
        for (int i = 0; i < CMAX; ++i) acc[k][i] = 0.f;
    }
    float cur[CPW][NQ], nxt[CPW][NQ], mp[MP];
    auto data_load = [&](int64_t r0, float (&v)[CPW][NQ]) {
#pragma unroll
        for (int k = 0; k < CPW; ++k)
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int64_t r = r0 + lane + 32 * q;
                const bool ok = col[k] < n && r < d;
                v[k][q] = !ok ? 0.f : (fromL ? ldf(Lm + col[k] * lds + r) : __ldg(X + col[k] * ldx + r));
            }
    };
    auto stage_load = [&](int64_t r0) {
#pragma unroll
        for (int u = 0; u < MP; ++u) {
            const int idx = threadIdx.x + u * kBT;
            const int i = idx / kChunk, t = idx - i * kChunk;
            const int64_t r = r0 + t;
            float v = 0.f;
            if (i < ce && r < d) v = seed ? __ldg(X + center * ldx + r) : ldf(mu + (int64_t)i * d + r);
            mp[u] = v;
        }
    };
    auto stage_store = [&]() {
#pragma unroll
        for (int u = 0; u < MP; ++u) sm.it.cs[threadIdx.x + u * kBT] = mp[u];
    };
    // without the prefetch (too many registers), the chunk is staged directly
    auto stage_direct = [&](int64_t r0) {
#pragma unroll 4
        for (int u = 0; u < MS; ++u) {
            const int idx = threadIdx.x + u * kBT;
            const int i = idx / kChunk, t = idx - i * kChunk;
            const int64_t r = r0 + t;
            float v = 0.f;
            if (i < ce && r < d) v = seed ? __ldg(X + center * ldx + r) : ldf(mu + (int64_t)i * d + r);
            sm.it.cs[idx] = v;
        }
    };
    data_load(0, cur);
    if (PREF) {
        stage_load(0);
        stage_store();
    } else {
        stage_direct(0);
    }
    __syncthreads();
    for (int64_t r0 = 0; r0 < d; r0 += kChunk) {
        const bool more = r0 + kChunk < d;
        if (more) {
            data_load(r0 + kChunk, nxt);
            if (PREF) stage_load(r0 + kChunk);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int t = lane + 32 * q;
#pragma unroll
            for (int i = 0; i < CMAX; ++i) {
                if (i < ce) {
                    const float m = sm.it.cs[i * kChunk + t];
#pragma unroll
                    for (int k = 0; k < CPW; ++k) {
                        const float df = cur[k][q] - m;
                        acc[k][i] = fmaf(df, df, acc[k][i]);
                    }
                }
            }
        }
        __syncthreads();
        if (more) {
            if (PREF) stage_store();
            else stage_direct(r0 + kChunk);
#pragma unroll
            for (int k = 0; k < CPW; ++k)
#pragma unroll
                for (int q = 0; q < NQ; ++q) cur[k][q] = nxt[k][q];
        }
        __syncthreads();
    }
    // per-lane FP32 sums (ceil(d/32) terms), a 5-level FP32 tree across lanes
    const double eps = (double)((d + 31) / 32 + 9) * 1.1920928955078125e-7;
    double changes = 0.0;
#pragma unroll
    for (int k = 0; k < CPW; ++k) {
        const int64_t j = col[k];
        // distance of centroid i lands in lane (i & 31), slot i >> 5
        double mine[2] = {INFINITY, INFINITY};
#pragma unroll
        for (int i = 0; i < CMAX; ++i) {
            if (i < ce) {
                const double v = (double)warp_sum(acc[k][i]);
                if (lane == (i & 31)) mine[i >> 5] = v;
            }
        }
        if (j >= n) continue;
        if (seed) {
            if (lane == 0) {
                const double v = mine[0];
                D2[j] = (seed_k == 0) ? v : fmin(ldd(D2 + j), v);
            }
            continue;
        }
        // best active centroid (ties to the lowest index)
        double bv = INFINITY;
        int bi = -1;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = lane + 32 * h;
            if (i < ce && ((amask >> i) & 1ull) && mine[h] < bv) {
                bv = mine[h];
                bi = i;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (oi >= 0 && (bi < 0 || ov < bv || (ov == bv && oi < bi))) {
                bv = ov;
                bi = oi;
            }
        }
        // near-tie candidates
        unsigned long long cand = 0ull;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = lane + 32 * h;
            const bool is = i < ce && ((amask >> i) & 1ull) && (mine[h] - bv <= eps * (mine[h] + bv));
            const unsigned bal = __ballot_sync(0xffffffffu, is);
            cand |= (unsigned long long)bal << (32 * h);
        }
        if (__popcll(cand) > 1) {
            // re-decide in FP64 from the stored values
            double best = INFINITY;
            int besti = -1;
            unsigned long long m = cand;
            while (m) {
                const int i = __ffsll((long long)m) - 1;
                m &= m - 1;
                double sacc = 0.0;
                for (int64_t r = lane; r < d; r += 32) {
                    const double y = fromL ? (double)ldf(Lm + j * lds + r) : (double)__ldg(X + j * ldx + r);
                    const double df = y - (double)ldf(mu + (int64_t)i * d + r);
                    sacc += df * df;
                }
                sacc = warp_sum(sacc);
                if (sacc < best) {
                    best = sacc;
                    besti = i;
                }
            }
            bi = besti;
        }
        if (bi < 0) bi = lab[k] >= 0 ? lab[k] : 0;   // no active centroid cannot occur; keep labels in range
        if (lane == 0) {
            if (bi != lab[k]) {
                lbl[j] = bi;
                changes += 1.0;
            }
        }
    }
    changes = block_sum(changes, sm.dred);
    if (threadIdx.x == 0) {
        cpart[item * 2 + 0] = 0.0;
        cpart[item * 2 + 1] = changes;
    }
}

// ---------------------------------------------------------------- serial tails
// Stable counting sort of the labels (one CTA): thread t counts the labels of
// its contiguous chunk of columns; the label runs start at offs; column j goes
// to offs[p_j] + (columns with the same label before it).  Clusters with
// columns are the active ones.
__device__ void sort_labels(const BProb& pb, BSmem& sm) {
    const int n = pb.n, c = pb.c, t = threadIdx.x;
    const int chunk = (n + kBT - 1) / kBT;
    const int j0 = min(n, t * chunk), j1 = min(n, j0 + chunk);
    for (int i = 0; i < c; ++i) sm.hist[i * kBT + t] = 0;
    for (int j = j0; j < j1; ++j) sm.hist[ldi(pb.p + j) * kBT + t] += 1;
    __syncthreads();
    if (t < c) {   // prefix within the label's row
        int run = 0;
        for (int u = 0; u < kBT; ++u) {
            const int v = sm.hist[t * kBT + u];
            sm.hist[t * kBT + u] = run;
            run += v;
        }
        sm.offs_s[t + 1] = run;
    }
    __syncthreads();
    if (t == 0) {
        sm.offs_s[0] = 0;
        for (int i = 0; i < c; ++i) sm.offs_s[i + 1] += sm.offs_s[i];
    }
    __syncthreads();
    for (int j = j0; j < j1; ++j) {
        const int l = ldi(pb.p + j);
        const int pos = sm.offs_s[l] + sm.hist[l * kBT + t];
        sm.hist[l * kBT + t] += 1;
        pb.perm[pos] = j;
    }
    if (t <= c) pb.offs[t] = sm.offs_s[t];
    if (t < c) pb.active[t] = (sm.offs_s[t + 1] > sm.offs_s[t]) ? 1 : 0;
    __syncthreads();
}

// Sum of a per-item partial array in item order (thread 0; a few hundred
// items at most).
__device__ double item_sum(const double* part, int items, int stride, int off) {
    double s = 0.0;
    for (int i = 0; i < items; ++i) s += ldd(part + (int64_t)i * stride + off);
    return s;
}

// k-means++ pick with draw u: the first column whose running sum of D2
// exceeds u times the total (chunk sums in column order, then a running sum
// inside the chunk); if rounding leaves none, the last column with D2 > 0;
// with D2 all zero, floor(u n).
__device__ int kmpp_pick(const BProb& pb, double u, BSmem& sm) {
    const int n = pb.n, t = threadIdx.x;
    const int chunk = (n + kBT - 1) / kBT;
    const int j0 = min(n, t * chunk), j1 = min(n, j0 + chunk);
    double s = 0.0;
    for (int j = j0; j < j1; ++j) s += ldd(pb.D2 + j);
    sm.dscan[t] = s;
    if (t == 0) {
        sm.pick = INT32_MAX;
        sm.aux = -1;
    }
    __syncthreads();
    if (t == 0) {
        double run = 0.0;
        for (int v = 0; v < kBT; ++v) {
            const double x = sm.dscan[v];
            sm.dscan[v] = run;
            run += x;
        }
        sm.dscan[kBT] = run;
    }
    __syncthreads();
    const double total = sm.dscan[kBT];
    if (!(total > 0.0)) {
        int pk = (int)(u * (double)n);
        return pk >= n ? n - 1 : pk;
    }
    const double target = u * total;
    double cum = sm.dscan[t];
    for (int j = j0; j < j1; ++j) {
        const double v = ldd(pb.D2 + j);
        cum += v;
        if (cum > target) {
            atomicMin(&sm.pick, j);
            break;
        }
    }
    for (int j = j1 - 1; j >= j0; --j)
        if (ldd(pb.D2 + j) > 0.0) {
            atomicMax(&sm.aux, j);
            break;
        }
    __syncthreads();
    const int pk = (sm.pick != INT32_MAX) ? sm.pick : sm.aux;
    __syncthreads();
    return pk;
}

__device__ unsigned items_of(const BProb& pb, int phase) {
    switch (phase) {
        case PH_SEED:
        case PH_ASSIGN_X:
        case PH_ASSIGN_L: return (unsigned)pb.col_items;
        case PH_DONE: return 0u;
        default: return (unsigned)pb.row_items;
    }
}

// The tail of `phase` for one problem, run by the CTA that completed the
// phase's last item; ends by publishing the next phase.
__device__ void phase_tail(const BProb& pb, BCtl* gctl, BGlobal* g, int phase, BSmem& sm) {
    const int t = threadIdx.x;
    const int n = pb.n, c = pb.c;
    BCtl& ctl = sm.lc;
    if (t == 0) {
        load_ctl(gctl, ctl);
        sm.next = PH_DONE;
    }
    __syncthreads();
    if (phase == PH_FRO) {
        if (t == 0) {
            const double nx2 = item_sum(pb.rpart, pb.row_items, 3, 0);
            const double bad = item_sum(pb.rpart, pb.row_items, 3, 1);
            ctl.nx2 = nx2;
            sm.flag = bad > 0.0 ? 1 : (nx2 == 0.0 ? 2 : 0);
            sm.aux = 0;
        }
        __syncthreads();
        const int fl = sm.flag;
        if (fl == 1) {
            if (t == 0) ctl.status = BS_NONFINITE;
        } else {
            if (pb.p0) {
                for (int j = t; j < n; j += kBT) {
                    const int v = __ldg(pb.p0 + j);
                    if (v < 0 || v >= c) atomicExch(&sm.aux, 1);
                    pb.p[j] = v;
                }
            } else if (fl == 2) {
                for (int j = t; j < n; j += kBT) pb.p[j] = 0;
            }
            __syncthreads();
            if (sm.aux) {
                if (t == 0) ctl.status = BS_BAD_LABELS;
            } else if (fl == 2) {
                if (t == 0) ctl.converged = 1;
            } else if (pb.p0) {
                sort_labels(pb, sm);
                if (t == 0) sm.next = pb.max_iter > 0 ? PH_SUMS_D : PH_DONE;
            } else if (t == 0) {
                int first = (int)(__ldg(pb.u) * (double)n);
                if (first >= n) first = n - 1;
                pb.centers[0] = first;
                ctl.seed_k = 0;
                sm.next = PH_SEED;
            }
        }
    } else if (phase == PH_SEED) {
        const int k = ctl.seed_k;
        if (k + 1 < c) {
            const int pk = kmpp_pick(pb, __ldg(pb.u + k + 1), sm);
            if (t == 0) {
                pb.centers[k + 1] = pk;
                ctl.seed_k = k + 1;
                sm.next = PH_SEED;
            }
        } else {
            for (int64_t e = t; e < (int64_t)c * pb.d; e += kBT) {
                const int i = (int)(e / pb.d);
                const int64_t r = e - (int64_t)i * pb.d;
                pb.mu[e] = __ldg(pb.X + (int64_t)ldi(pb.centers + i) * pb.ldx + r);
            }
            for (int i = t; i < c; i += kBT) pb.active[i] = 1;
            for (int j = t; j < n; j += kBT) pb.p[j] = -1;
            if (t == 0) {
                ctl.init_passes = 0;
                sm.next = PH_ASSIGN_X;
            }
        }
    } else if (phase == PH_LSTEP) {
        // the labels the p step starts from
        for (int j = t; j < n; j += kBT) pb.pstart[j] = ldi(pb.p + j);
        if (t == 0) {
            ctl.dl2 = item_sum(pb.rpart, pb.row_items, 3, 0);
            ctl.passes = 0;
            sm.next = PH_ASSIGN_L;
        }
    } else if (phase == PH_ASSIGN_X || phase == PH_ASSIGN_L) {
        if (t == 0) {
            const double ch = item_sum(pb.cpart, pb.col_items, 2, 1);
            if (phase == PH_ASSIGN_L) {
                ctl.passes += 1;
            } else {
                ctl.init_passes += 1;
            }
            ctl.last_changes = (long long)ch;
        }
        __syncthreads();
        const bool moved = ctl.last_changes > 0;
        if (moved) sort_labels(pb, sm);
        if (t == 0) {
            if (phase == PH_ASSIGN_X) {
                if (moved && ctl.init_passes < pb.km_max) sm.next = PH_MEANS_X;
                else sm.next = pb.max_iter > 0 ? PH_SUMS_D : PH_DONE;
            } else {
                sm.next = (moved && ctl.passes < pb.km_max) ? PH_MEANS_L : PH_STHETA;
            }
        }
    } else if (phase == PH_MEANS_X) {
        if (t == 0) sm.next = PH_ASSIGN_X;
    } else if (phase == PH_SUMS_D) {
        if (t == 0) sm.next = PH_LSTEP;
    } else if (phase == PH_MEANS_L) {
        if (t == 0) sm.next = PH_ASSIGN_L;
    } else if (phase == PH_STHETA) {
        double mv = 0.0;
        for (int j = t; j < n; j += kBT) mv += (ldi(pb.pstart + j) != ldi(pb.p + j)) ? 1.0 : 0.0;
        mv = block_sum(mv, sm.dred);
        if (t == 0) {
            const double r2 = item_sum(pb.rpart, pb.row_items, 3, 0);
            const double ds2 = item_sum(pb.rpart, pb.row_items, 3, 1);
            const double nx = sqrt(ctl.nx2);
            ctl.label_changes += (long long)mv;
            ctl.lloyd_passes += ctl.passes;
            ctl.iter += 1;
            ctl.e_res = sqrt(r2) / nx;
            ctl.e_dl = sqrt(ctl.dl2) / nx;
            ctl.e_ds = sqrt(ds2) / nx;
            ctl.err = fmax(ctl.e_res, fmax(ctl.e_dl, ctl.e_ds));
            ctl.rho *= pb.kappa;
            if (ctl.err <= pb.tol) {
                ctl.converged = 1;
                sm.next = PH_DONE;
            } else {
                sm.next = ctl.iter >= pb.max_iter ? PH_DONE : PH_LSTEP;
            }
        }
    }
    __syncthreads();
    if (t == 0) {
        const int next = sm.next;
        const unsigned gen = claim_gen(*(volatile unsigned long long*)&gctl->claim) + 1u;
        store_ctl(gctl, ctl);
        *(volatile int32_t*)&gctl->done = 0;
        *(volatile int32_t*)&gctl->phase = next;
        __threadfence();
        atomicExch(&gctl->claim, make_claim(gen, items_of(pb, next)));
        if (next == PH_DONE) atomicAdd(&g->finished, 1);
    }
    __syncthreads();
}

// ---------------------------------------------------------------- the kernel
// One persistent launch for the whole batch.  Thread 0 of a CTA claims the
// next item of some problem (scanning the problems from where it last found
// work), the CTA runs it, and the CTA that completes a phase's last item runs
// that phase's tail.  A CTA that finds nothing polls again after a short
// sleep; after spin_limit empty scans it sets the timeout and abort flags.
// Every CTA leaves once all problems are done or the abort flag is set.
template <int MINB>
__global__ void __launch_bounds__(kBT, MINB)
    k_batched(const BProb* __restrict__ probs, BCtl* __restrict__ ctls, BGlobal* __restrict__ g, int P,
              int KR, long long spin_limit) {
    extern __shared__ __align__(16) unsigned char smraw[];
    BSmem& sm = *reinterpret_cast<BSmem*>(smraw);
    long long polls = 0;
    int start = (int)(blockIdx.x % (unsigned)P);
    for (;;) {
        if (threadIdx.x == 0) {
            int pid = -1;
            for (;;) {
                if (*(volatile int32_t*)&g->abort || *(volatile int32_t*)&g->finished >= P) break;
                for (int q = 0; q < P && pid < 0; ++q) {
                    const int cand = (start + q < P) ? start + q : start + q - P;
                    const unsigned long long w = *(volatile unsigned long long*)&ctls[cand].claim;
                    if (claim_next(w) < claim_n(w)) {
                        const unsigned long long old = atomicAdd(&ctls[cand].claim, 1ull);
                        if (claim_next(old) < claim_n(old)) {
                            pid = cand;
                            sm.item = (int32_t)claim_next(old);
                            sm.nitems = (int32_t)claim_n(old);
                        }
                    }
                }
                if (pid >= 0) {
                    start = pid;
                    polls = 0;
                    break;
                }
                if (++polls > spin_limit) {
                    atomicExch(&g->timeout, 1);
                    atomicExch(&g->abort, 1);
                    break;
                }
                __nanosleep(200);
            }
            sm.pid = pid;
            if (pid >= 0) {
                __threadfence();
                const volatile BCtl* v = ctls + pid;
                sm.next = v->phase;
                sm.lc.rho = v->rho;
                sm.lc.seed_k = v->seed_k;
            }
        }
        __syncthreads();
        const int pid = sm.pid;
        if (pid < 0) break;
        const BProb& pb = probs[pid];
        const int phase = sm.next, item = sm.item;
        const double rho = sm.lc.rho;
        const int seed_k = sm.lc.seed_k;
        __syncthreads();
        switch (phase) {
            case PH_SEED:
            case PH_ASSIGN_X:
            case PH_ASSIGN_L:
                // columns per warp: 64 / CMAX with one CTA per SM, half that with two
                // (the register budget halves); must match cpw_of on the host
                if (pb.cmax <= 16) {
                    if (MINB == 1) col_item<16, 4, true>(pb, seed_k, phase, item, sm);
                    else col_item<16, 2, true>(pb, seed_k, phase, item, sm);
                } else if (pb.cmax <= 32) {
                    if (MINB == 1) col_item<32, 2, true>(pb, seed_k, phase, item, sm);
                    else col_item<32, 1, true>(pb, seed_k, phase, item, sm);
                } else {
                    if (MINB == 1) col_item<64, 1, true>(pb, seed_k, phase, item, sm);
                    else col_item<64, 1, false>(pb, seed_k, phase, item, sm);
                }
                break;
            default:
                // two CTAs per SM take 64-row items only (the 128-row form's loads
                // do not fit their registers)
                if (MINB == 2 || KR == 2) row_item<2>(pb, rho, phase, item, sm);
                else row_item<4>(pb, rho, phase, item, sm);
                break;
        }
        __threadfence();   // this thread's writes are visible before the item counts as done
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const int prev = atomicAdd(&ctls[pid].done, 1);
            sm.flag = (prev + 1 == sm.nitems) ? 1 : 0;
        }
        __syncthreads();
        if (sm.flag) {
            __threadfence();
            phase_tail(pb, ctls + pid, g, phase, sm);
        }
        __syncthreads();
    }
}

}  // namespace batched

// ---------------------------------------------------------------- host driver
using namespace batched;

namespace {

struct HBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

cudaError_t hgrow(HBuf& b, size_t bytes, bool pinned) {
    if (b.p && b.bytes >= bytes) return cudaSuccess;
    if (b.p) {
        if (pinned) cudaFreeHost(b.p);
        else cudaFree(b.p);
    }
    b.p = nullptr;
    b.bytes = 0;
    const cudaError_t e = pinned ? cudaMallocHost(&b.p, bytes ? bytes : 16) : cudaMalloc(&b.p, bytes ? bytes : 16);
    if (e == cudaSuccess) b.bytes = bytes;
    return e;
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

int cmax_of(int c) { return c <= 16 ? 16 : (c <= 32 ? 32 : 64); }

// Columns per warp of a column item (the kernel's choice for MINB CTAs per SM).
int cpw_of(int cmax, int minb) { return minb == 1 ? 64 / cmax : std::max(1, 32 / cmax); }

struct Tuned {
    uint64_t key;
    int kr, minb;
};

}  // namespace

struct BatchedState {
    HBuf dprobs, dctl, dglob, work, draws;     // device
    HBuf hprobs, hctl, hglob;                  // pinned host
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    uint64_t graph_key = 0;
    std::vector<Tuned> tuned;
    cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
    cudaStream_t own = nullptr;                // launches and graph capture (never the legacy stream)
    bool attrs_set = false;
};

void batched_state_free(BatchedState* s) {
    if (!s) return;
    if (s->exec) cudaGraphExecDestroy(s->exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    for (HBuf* b : {&s->dprobs, &s->dctl, &s->dglob, &s->work, &s->draws})
        if (b->p) cudaFree(b->p);
    for (HBuf* b : {&s->hprobs, &s->hctl, &s->hglob})
        if (b->p) cudaFreeHost(b->p);
    if (s->e0) cudaEventDestroy(s->e0);
    if (s->e1) cudaEventDestroy(s->e1);
    if (s->e2) cudaEventDestroy(s->e2);
    if (s->own) cudaStreamDestroy(s->own);
    delete s;
}

namespace {

struct RunArgs {
    int device, sms;
    cudaStream_t st, own;
    uint64_t seed;
    double rho0, kappa;
    int km_max;
    long long spin_limit;
};

uint64_t fnv(uint64_t h, uint64_t v) { return (h ^ v) * 1099511628211ULL; }

// Workspace offsets of every problem (sized for the smallest row block, so
// every tile choice fits) and the table for one tile choice.
size_t layout(int32_t batch, const respca_problem* probs, char* base, int kr, int minb, int iter_cap,
              int km_max, double kappa, const double* draws, BProb* out) {
    size_t off = 0;
    for (int32_t b = 0; b < batch; ++b) {
        const respca_problem& q = probs[b];
        const int64_t d = q.d, n = q.n;
        const int c = q.c;
        const int cm = cmax_of(c);
        const int W = 8 * cpw_of(cm, minb);
        const int rows_min = 64;
        const int64_t ri_max = (d + rows_min - 1) / rows_min;
        const int64_t ci = (n + W - 1) / W;
        BProb pb;
        std::memset(&pb, 0, sizeof(pb));
        pb.X = static_cast<const float*>(q.X);
        pb.L = q.L;
        pb.S = q.S;
        pb.p = q.p;
        pb.p0 = q.p0;
        pb.ldx = q.ldx;
        pb.lds = q.lds;
        pb.ldt = d;
        pb.d = (int32_t)d;
        pb.n = (int32_t)n;
        pb.c = c;
        pb.max_iter = iter_cap >= 0 ? std::min(q.max_iter, iter_cap) : q.max_iter;
        pb.km_max = km_max;
        pb.W = W;
        pb.cmax = cm;
        pb.row_items = (int32_t)((d + 32 * kr - 1) / (32 * kr));
        pb.col_items = (int32_t)ci;
        pb.lam = q.lambda > 0.0 ? q.lambda : std::sqrt((double)std::max(d, n));
        pb.tol = q.tol;
        pb.kappa = kappa;
        pb.u = draws;
        auto take = [&](size_t bytes) {
            char* p = base ? base + off : nullptr;
            off = al256(off + bytes);
            return p;
        };
        pb.Th = reinterpret_cast<float*>(take(sizeof(float) * (size_t)d * n));
        pb.mu = reinterpret_cast<float*>(take(sizeof(float) * (size_t)c * d));
        pb.perm = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * n));
        pb.offs = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (c + 1)));
        pb.pstart = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * n));
        pb.active = reinterpret_cast<uint8_t*>(take(c));
        pb.D2 = reinterpret_cast<double*>(take(sizeof(double) * n));
        pb.centers = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * c));
        pb.rpart = reinterpret_cast<double*>(take(sizeof(double) * 3 * ri_max));
        pb.cpart = reinterpret_cast<double*>(take(sizeof(double) * 2 * ci));
        if (out) out[b] = pb;
    }
    return off;
}

}  // namespace

respca_status batched_persistent(BatchedState** sp, int device, cudaStream_t st, uint64_t seed, double rho0,
                                 double kappa, int km_max, int32_t batch, const respca_problem* probs,
                                 respca_stats* stats, respca_batch_options* opt, std::string* err) {
    auto fail = [&](respca_status s, const std::string& m) {
        if (err) *err = m;
        return s;
    };
    auto cfail = [&](cudaError_t e, const char* where) {
        if (err) *err = std::string(where) + ": " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? RESPCA_ERR_OOM : RESPCA_ERR_CUDA;
    };
#define BK(expr)                                   \
    do {                                           \
        const cudaError_t _e = (expr);             \
        if (_e != cudaSuccess) return cfail(_e, #expr); \
    } while (0)
    if (batch < 0 || (batch > 0 && !probs)) return fail(RESPCA_ERR_INVALID_ARG, "batch");
    if (opt && (opt->tile_rows != 0 && opt->tile_rows != 64 && opt->tile_rows != 128))
        return fail(RESPCA_ERR_INVALID_ARG, "tile_rows must be 0, 64 or 128");
    if (opt && (opt->ctas_per_sm < 0 || opt->ctas_per_sm > 2))
        return fail(RESPCA_ERR_INVALID_ARG, "ctas_per_sm must be 0, 1 or 2");
    if (batch == 0) return RESPCA_OK;
    for (int32_t b = 0; b < batch; ++b) {
        const respca_problem& q = probs[b];
        const std::string w = "problem " + std::to_string(b) + ": ";
        if (!q.X || !q.L || !q.S || !q.p || q.d < 1 || q.n < 1 || q.ldx < q.d || q.lds < q.d || q.c < 1 ||
            q.c > q.n || !(q.tol >= 0.0) || q.max_iter < 0 || !std::isfinite(q.lambda))
            return fail(RESPCA_ERR_INVALID_ARG, w + "invalid argument");
        if (q.x_dtype != RESPCA_F32) return fail(RESPCA_ERR_UNSUPPORTED, w + "the persistent path takes FP32 X");
        if (q.c > kMaxC) return fail(RESPCA_ERR_UNSUPPORTED, w + "the persistent path takes c <= 64");
        if (q.d > (int64_t)1 << 22 || q.n > (int64_t)1 << 22)
            return fail(RESPCA_ERR_UNSUPPORTED, w + "d and n up to 2^22 in the persistent path");
    }
    if (!*sp) {
        *sp = new (std::nothrow) BatchedState();
        if (!*sp) return fail(RESPCA_ERR_OOM, "batched state");
    }
    BatchedState& S = **sp;
    BK(cudaSetDevice(device));
    RunArgs ra;
    ra.device = device;
    BK(cudaDeviceGetAttribute(&ra.sms, cudaDevAttrMultiProcessorCount, device));
    ra.st = st;
    ra.seed = seed;
    ra.rho0 = rho0;
    ra.kappa = kappa;
    ra.km_max = std::max(1, km_max);
    ra.spin_limit = (opt && opt->spin_limit > 0) ? opt->spin_limit : (1LL << 23);
    if (!S.e0) {
        BK(cudaEventCreate(&S.e0));
        BK(cudaEventCreate(&S.e1));
        BK(cudaEventCreateWithFlags(&S.e2, cudaEventDisableTiming));
        BK(cudaStreamCreateWithFlags(&S.own, cudaStreamNonBlocking));
    }
    // the launch waits for the work already queued on the caller's stream
    BK(cudaEventRecord(S.e2, ra.st));
    BK(cudaStreamWaitEvent(S.own, S.e2, 0));
    st = S.own;
    if (!S.attrs_set) {
        BK(cudaFuncSetAttribute(k_batched<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BSmem)));
        BK(cudaFuncSetAttribute(k_batched<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BSmem)));
        S.attrs_set = true;
    }
    // device memory: workspace, the k-means++ draws (the same seed as the single path)
    // sized for the smallest items (64 rows, the narrower column items of two CTAs per SM)
    const size_t wbytes = layout(batch, probs, nullptr, 2, 2, -1, ra.km_max, kappa, nullptr, nullptr);
    BK(hgrow(S.work, wbytes, false));
    BK(hgrow(S.draws, sizeof(double) * kMaxC, false));
    BK(hgrow(S.dprobs, sizeof(BProb) * batch, false));
    BK(hgrow(S.dctl, sizeof(BCtl) * batch, false));
    BK(hgrow(S.dglob, sizeof(BGlobal), false));
    BK(hgrow(S.hprobs, sizeof(BProb) * batch, true));
    BK(hgrow(S.hctl, sizeof(BCtl) * batch, true));
    BK(hgrow(S.hglob, sizeof(BGlobal), true));
    {
        double u[kMaxC];
        uint64_t sst = seed;
        for (int k = 0; k < kMaxC; ++k) {
            sst += 0x9E3779B97F4A7C15ULL;   // splitmix64
            uint64_t z = sst;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
            z ^= z >> 31;
            u[k] = (double)(z >> 11) * (1.0 / 9007199254740992.0);
        }
        BK(cudaMemcpy(S.draws.p, u, sizeof(u), cudaMemcpyHostToDevice));
    }
    BProb* hp = static_cast<BProb*>(S.hprobs.p);
    BCtl* hc = static_cast<BCtl*>(S.hctl.p);
    BGlobal* hg = static_cast<BGlobal*>(S.hglob.p);
    const double* du = static_cast<const double*>(S.draws.p);
    // one launch of the whole batch with tile rows 32 kr, minb CTAs per SM
    auto run = [&](int kr, int minb, int iter_cap, bool use_graph, float* ms) -> respca_status {
        if (minb == 2) kr = 2;
        layout(batch, probs, static_cast<char*>(S.work.p), kr, minb, iter_cap, ra.km_max, kappa, du, hp);
        for (int32_t b = 0; b < batch; ++b) {
            std::memset(&hc[b], 0, sizeof(BCtl));
            hc[b].claim = ((unsigned long long)1 << 48) | ((unsigned long long)(hp[b].row_items & 0xFFFFFF) << 24);
            hc[b].phase = PH_FRO;
            hc[b].rho = rho0;
        }
        uint64_t key = 1469598103934665603ULL;
        key = fnv(key, (uint64_t)kr);
        key = fnv(key, (uint64_t)minb);
        key = fnv(key, (uint64_t)batch);
        key = fnv(key, (uint64_t)reinterpret_cast<uintptr_t>(S.work.p));
        key = fnv(key, (uint64_t)reinterpret_cast<uintptr_t>(S.dprobs.p));
        key = fnv(key, (uint64_t)reinterpret_cast<uintptr_t>(st));
        key = fnv(key, (uint64_t)ra.spin_limit);
        const unsigned char* tb = reinterpret_cast<const unsigned char*>(hp);
        for (size_t i = 0; i < sizeof(BProb) * batch; i += 8) {
            uint64_t v = 0;
            std::memcpy(&v, tb + i, std::min<size_t>(8, sizeof(BProb) * batch - i));
            key = fnv(key, v);
        }
        const bool have = use_graph && S.exec && S.graph_key == key;
        if (!have) BK(cudaMemcpyAsync(S.dprobs.p, hp, sizeof(BProb) * batch, cudaMemcpyHostToDevice, st));
        auto enqueue = [&]() -> cudaError_t {
            cudaError_t e = cudaMemcpyAsync(S.dctl.p, hc, sizeof(BCtl) * batch, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(S.dglob.p, 0, sizeof(BGlobal), st);
            if (e != cudaSuccess) return e;
            const dim3 grid(ra.sms * minb);
            if (minb == 2)
                k_batched<2><<<grid, kBT, sizeof(BSmem), st>>>(static_cast<const BProb*>(S.dprobs.p),
                                                              static_cast<BCtl*>(S.dctl.p),
                                                              static_cast<BGlobal*>(S.dglob.p), batch, kr,
                                                              ra.spin_limit);
            else
                k_batched<1><<<grid, kBT, sizeof(BSmem), st>>>(static_cast<const BProb*>(S.dprobs.p),
                                                              static_cast<BCtl*>(S.dctl.p),
                                                              static_cast<BGlobal*>(S.dglob.p), batch, kr,
                                                              ra.spin_limit);
            e = cudaGetLastError();
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(hc, S.dctl.p, sizeof(BCtl) * batch, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(hg, S.dglob.p, sizeof(BGlobal), cudaMemcpyDeviceToHost, st);
            return e;
        };
        count_launches(1);
        // timed around the whole launch (events inside a captured graph cannot be read back)
        BK(cudaEventRecord(S.e0, st));
        if (use_graph) {
            if (!have) {
                if (S.exec) cudaGraphExecDestroy(S.exec);
                if (S.graph) cudaGraphDestroy(S.graph);
                S.exec = nullptr;
                S.graph = nullptr;
                BK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                const cudaError_t e = enqueue();
                cudaGraph_t gph = nullptr;
                const cudaError_t e2 = cudaStreamEndCapture(st, &gph);
                if (e != cudaSuccess) {
                    if (gph) cudaGraphDestroy(gph);
                    return cfail(e, "capture of the batched launch");
                }
                BK(e2);
                S.graph = gph;
                BK(cudaGraphInstantiate(&S.exec, S.graph, 0));
                S.graph_key = key;
            }
            BK(cudaGraphLaunch(S.exec, st));
        } else {
            BK(enqueue());
        }
        BK(cudaEventRecord(S.e1, st));
        BK(cudaStreamSynchronize(st));
        if (ms) BK(cudaEventElapsedTime(ms, S.e0, S.e1));
        if (hg->timeout) return fail(RESPCA_ERR_TIMEOUT, "a CTA of the batched launch gave up waiting for work");
        return RESPCA_OK;
    };
#undef BK
    // tile choice: the caller's, a cached one for this batch shape, or the
    // fastest of the candidates on a run capped at 3 iterations
    int kr = 0, minb = 0;
    if (opt && opt->tile_rows) kr = opt->tile_rows / 32;
    if (opt && opt->ctas_per_sm) minb = opt->ctas_per_sm;
    if (!kr || !minb) {
        uint64_t skey = 1469598103934665603ULL;
        for (int32_t b = 0; b < batch; ++b) {
            skey = fnv(skey, (uint64_t)probs[b].d);
            skey = fnv(skey, (uint64_t)probs[b].n);
            skey = fnv(skey, (uint64_t)probs[b].c);
        }
        skey = fnv(skey, (uint64_t)(kr * 8 + minb));
        const Tuned* hit = nullptr;
        for (const Tuned& t : S.tuned)
            if (t.key == skey) hit = &t;
        if (hit) {
            kr = hit->kr;
            minb = hit->minb;
        } else {
            float best = INFINITY;
            int bk = 4, bm = 1;
            for (int ck : {2, 4}) {
                if (kr && ck != kr) continue;
                for (int cm : {1, 2}) {
                    if (minb && cm != minb) continue;
                    if (cm == 2 && ck == 4) continue;   // two CTAs per SM take 64-row items
                    float ms = 0.f;
                    respca_status rs = run(ck, cm, 3, false, &ms);
                    if (rs != RESPCA_OK) return rs;
                    rs = run(ck, cm, 3, false, &ms);
                    if (rs != RESPCA_OK) return rs;
                    if (ms < best) {
                        best = ms;
                        bk = ck;
                        bm = cm;
                    }
                }
            }
            kr = bk;
            minb = bm;
            S.tuned.push_back(Tuned{skey, kr, minb});
        }
    }
    if (minb == 2) kr = 2;
    float ms = 0.f;
    respca_status rs = run(kr, minb, -1, true, &ms);
    if (rs != RESPCA_OK) return rs;
    if (opt) {
        opt->tuned_rows = 32 * kr;
        opt->tuned_ctas_per_sm = minb;
        opt->ms_kernel = ms;
    }
    respca_status first = RESPCA_OK;
    for (int32_t b = 0; b < batch; ++b) {
        const BCtl& c = hc[b];
        if (stats) {
            respca_stats& o = stats[b];
            std::memset(&o, 0, sizeof(o));
            o.iters = c.iter;
            o.converged = c.converged;
            o.err = c.err;
            o.err_resid = c.e_res;
            o.err_dL = c.e_dl;
            o.err_dS = c.e_ds;
            o.rho_final = c.rho;
            o.lambda = hp[b].lam;
            o.label_changes = c.label_changes;
            o.lloyd_passes = c.lloyd_passes;
            o.init_lloyd_passes = c.init_passes;
            o.kernel_launches = b == 0 ? 1 : 0;
            o.ms_total = ms;
            o.x_norm = std::sqrt(c.nx2);
        }
        if (first == RESPCA_OK && c.status != BS_OK) {
            first = c.status == BS_NONFINITE ? RESPCA_ERR_NONFINITE_INPUT : RESPCA_ERR_INVALID_ARG;
            if (err)
                *err = "problem " + std::to_string(b) +
                       (c.status == BS_NONFINITE ? ": X holds NaN or Inf" : ": labels outside [0, c)");
        }
    }
    return first;
}

}  // namespace respca
