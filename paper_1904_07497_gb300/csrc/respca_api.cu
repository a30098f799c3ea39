// Host driver and C ABI of the RES-PCA solver (see include/respca.h).
//
// One solve = the initial labels (given, or k-means++ + Lloyd on X), then ALM
// iterations in the order of Sec. 4: L (Sec. 4.1), p (Sec. 4.2), S (Sec. 4.3),
// Theta and rho (Sec. 4.4), stopped by the rule of Sec. 5.  Every iteration is
// one fused HBM pass (k_iteration) plus small kernels; the host reads back a
// 64-byte status block once per iteration to run the stopping test and, when
// some labels moved, the remaining Lloyd passes of the p step.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/respca.h"
#include "respca_internal.cuh"

using namespace respca;

namespace {

// splitmix64 (Steele, Lea, Flood 2014): the draws of the k-means++ seeding.
uint64_t splitmix64_next(uint64_t& s) {
    s += 0x9E3779B97F4A7C15ULL;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

double unit_draw(uint64_t& s) { return (double)(splitmix64_next(s) >> 11) * (1.0 / 9007199254740992.0); }

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct respca_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;      // a batch lane's stream, created and destroyed with it
    cudaStream_t cap_stream = nullptr;      // private stream the Lloyd-pass graph is captured on
    struct LloydGraph {                     // device-run Lloyd loop, reused while its key holds
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        uint64_t key = 0;
        int64_t launches_per_pass = 0;
    } lloyd_graph[2];
    int lloyd_graph_next = 0;               // slot the next new graph replaces
    std::vector<respca_ctx*> lanes;         // batch lanes (respca_solve_batched), made on first use
    respca_ctx* spec_km = nullptr;          // K-means on the spectral embedding (own workspace)
    respca::BatchedState* batched = nullptr; // the persistent batched solve's buffers and graph
    respca_config cfg{};
    std::string last_error;

    // device workspace, grown on demand
    DevBuf theta, mu, mu_norm2, mu_normf, pair_ss, sep2, perm, counts, tile_off, tiles, labels_prev,
        Dpart, own_part, norm_part, flag_list, seedD2, seed_part, centers, seed_u, fro_part, status,
        hX, hL, hS, hp, hp0,
        mu_next, mu_old, drift, ub, lb, dl_part, sums, moved, contrib, boff, labels_pass,
        mu_hi, mu_lo, Gpart, ynorm_part, rc_list, rc_plist, tile_count, rc_dist,
        L16, S16, T16, X16,   // BF16 state and X of the bf16 phase (precision = 1)
        mu_a,                 // centroid operand of the swapped dense search
        bn_part,              // per-chunk ||B_j||^2 of the l2,1 iteration
        sumsD,                // FP64 sums of the next D under the iteration's starting labels
        sp_M, sp_sqn, sp_part, sp_gsum, sp_sig, sp_deg, sp_Y, sp_W, sp_T, sp_Z, sp_H, sp_Q, sp_ev,
        cs_part, cs_done,     // per-split norms and counters of the centroid statistics
        norm_red,             // the norm reduction's per-CTA parts
        sp_res, sp_E, sp_P, sp_Ypad,   // spectral p step: affinity, search blocks, Rayleigh-Ritz, embedding,
                              // M Y partials, a 16-byte-aligned copy of Y for the tensor maps
        mu_a16, a16_err, a16_part, a16_done,   // the centroids' 16-bit split and its error norms
        Lsh, ylo_part, ycol;  // FP16 copy of the FP32 L, its per-chunk and per-column error norms
    DevStatus* hstat = nullptr;     // pinned mirror of the status block
    double* hseed_u = nullptr;      // pinned staging of the seeding draws
    size_t hseed_cap = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, evk0 = nullptr, evk1 = nullptr;
    cudaEvent_t evd0 = nullptr, evd1 = nullptr;   // around the all-column search (timing mode)
    bool dense_recorded = false;                  // evd0 / evd1 bracket the last search's dense launch
    float ms_dense = 0.f;                         // per-solve accumulators of that kernel's time
    int32_t dense_passes = 0;
    float ms_dense16 = 0.f;                       // the part of them that read 16-bit operands
    int32_t dense16_passes = 0;
    bool dense16 = false;                         // the last search's all-column kernel read 16 bits
    const void* sh_for = nullptr;                 // the FP32 L that Lsh / ycol currently mirror
    int64_t sh_ld = 0;                            // column stride of Lsh
};

namespace {

constexpr int kFroParts = 1216;  // 152 SMs x 8

respca_status fail(respca_ctx* h, respca_status s, const char* what) {
    if (h) h->last_error = what;
    return s;
}

respca_status cuda_fail(respca_ctx* h, cudaError_t e, const char* where) {
    if (h) h->last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return (e == cudaErrorMemoryAllocation) ? RESPCA_ERR_OOM : RESPCA_ERR_CUDA;
}

#define CK(expr)                                                   \
    do {                                                           \
        cudaError_t _e = (expr);                                   \
        if (_e != cudaSuccess) return cuda_fail(h, _e, #expr);     \
    } while (0)

cudaError_t ensure(DevBuf& b, size_t bytes) {
    if (b.bytes >= bytes && b.p) return cudaSuccess;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMalloc(&b.p, bytes > 0 ? bytes : 16);
    if (e == cudaSuccess) b.bytes = bytes;
    return e;
}

template <typename T>
T* P(DevBuf& b) { return reinterpret_cast<T*>(b.p); }

int max_tiles_for(int64_t n, int c) { return (int)((n + kTileCols - 1) / kTileCols) + c; }
int nchunks_for(int64_t d) { return (int)((d + kChunkRows - 1) / kChunkRows); }

size_t elem_size(int dtype) { return dtype == RESPCA_F32 ? 4 : 2; }

// Every device buffer of the workspace.
std::vector<DevBuf*> all_bufs(respca_ctx* h) {
    return {&h->theta, &h->mu, &h->mu_norm2, &h->mu_normf, &h->pair_ss, &h->sep2, &h->perm,
                      &h->counts, &h->tile_off, &h->tiles, &h->labels_prev, &h->Dpart, &h->own_part,
                      &h->norm_part, &h->flag_list, &h->seedD2, &h->seed_part, &h->centers, &h->seed_u,
                      &h->fro_part,
                      &h->status, &h->hX, &h->hL, &h->hS, &h->hp, &h->hp0, &h->mu_next, &h->mu_old,
                      &h->drift, &h->ub, &h->lb, &h->dl_part, &h->sums, &h->moved, &h->contrib, &h->boff,
                      &h->labels_pass,
                      &h->mu_hi, &h->mu_lo, &h->Gpart, &h->ynorm_part, &h->rc_list, &h->tile_count,
                      &h->rc_dist, &h->rc_plist, &h->L16, &h->S16, &h->T16, &h->X16, &h->mu_a,
                      &h->bn_part, &h->sumsD, &h->sp_M, &h->sp_sqn, &h->sp_part, &h->sp_gsum,
                      &h->sp_sig, &h->sp_deg, &h->sp_Y, &h->sp_W, &h->sp_T, &h->sp_Z, &h->sp_H, &h->sp_Q,
                      &h->sp_ev, &h->sp_res, &h->sp_E, &h->sp_P, &h->sp_Ypad, &h->cs_part, &h->cs_done, &h->norm_red,
                      &h->mu_a16, &h->a16_err, &h->a16_part, &h->a16_done, &h->Lsh, &h->ylo_part, &h->ycol};
}

respca_status ensure_workspace(respca_ctx* h, int64_t d, int64_t n, int c, int64_t lds,
                               bool need_theta) {
    const int mt = max_tiles_for(n, c);
    const int nch = nchunks_for(d);
    if (need_theta) CK(ensure(h->theta, sizeof(float) * (size_t)lds * n));
    CK(ensure(h->mu_norm2, sizeof(double) * c));
    CK(ensure(h->mu_normf, sizeof(float) * c));
    CK(ensure(h->pair_ss, sizeof(float) * (size_t)std::min(c, 256) * std::min(c, 256)));
    CK(ensure(h->sep2, sizeof(double) * c));
    CK(ensure(h->perm, sizeof(int32_t) * n));
    CK(ensure(h->counts, sizeof(int32_t) * c));
    CK(ensure(h->tile_off, sizeof(int32_t) * (c + 1)));
    CK(ensure(h->tiles, sizeof(TileDesc) * mt));
    CK(ensure(h->labels_prev, sizeof(int32_t) * n));
    CK(ensure(h->Dpart, sizeof(float) * (size_t)mt * d));
    CK(ensure(h->own_part, sizeof(float) * (size_t)nch * n));
    CK(ensure(h->bn_part, sizeof(float) * (size_t)nch * n));
    CK(ensure(h->norm_part, sizeof(double) * 3 * (size_t)mt * nch));
    CK(ensure(h->norm_red, sizeof(double) * 3 * 64));
    CK(ensure(h->flag_list, sizeof(int32_t) * n));
    CK(ensure(h->seedD2, sizeof(double) * n));
    CK(ensure(h->seed_part, sizeof(double) * ((n + 7) / 8 + 1)));
    CK(ensure(h->centers, sizeof(int32_t) * c));
    CK(ensure(h->seed_u, sizeof(double) * c));
    CK(ensure(h->fro_part, sizeof(double) * kFroParts));
    CK(ensure(h->status, sizeof(DevStatus)));
    {
        // the statistics kernel's per-centroid counters start at zero and it leaves them so
        const size_t need = sizeof(int32_t) * c;
        const bool fresh = !h->cs_done.p || h->cs_done.bytes < need;
        CK(ensure(h->cs_done, need));
        if (fresh) CK(cudaMemsetAsync(h->cs_done.p, 0, need, h->stream));
        CK(ensure(h->cs_part, sizeof(float4) * (size_t)c * centroids_stats_splits(c, d)));
    }
    // centroid buffers start zeroed so entries of clusters that never had a
    // member hold finite values
    for (DevBuf* b : {&h->mu, &h->mu_next, &h->mu_old}) {
        const bool fresh = b->bytes < sizeof(float) * (size_t)c * d;
        CK(ensure(*b, sizeof(float) * (size_t)c * d));
        if (fresh) CK(cudaMemsetAsync(b->p, 0, b->bytes, h->stream));
    }
    CK(ensure(h->drift, sizeof(double) * c));
    CK(ensure(h->ub, sizeof(float) * n));
    CK(ensure(h->lb, sizeof(float) * n));
    CK(ensure(h->dl_part, sizeof(float) * (size_t)nch * n));
    CK(ensure(h->sums, sizeof(double) * (size_t)c * d));
    CK(ensure(h->sumsD, sizeof(double) * (size_t)c * d));
    CK(ensure(h->moved, sizeof(int4) * n));
    CK(ensure(h->contrib, sizeof(int2) * 2 * (size_t)n));
    CK(ensure(h->boff, sizeof(int32_t) * ((size_t)c + 1)));
    CK(ensure(h->labels_pass, sizeof(int32_t) * n));
    if (c <= kTcMaxClusters) {
        const TcPlan tp = tc_plan(n, d, c);
        CK(ensure(h->mu_hi, sizeof(float) * (size_t)tp.Npad * tp.dpad));
        CK(ensure(h->mu_lo, sizeof(float) * (size_t)tp.Npad * tp.dpad));
        CK(ensure(h->Gpart, sizeof(float) * tp.gpart));
        CK(ensure(h->ynorm_part, sizeof(float) * tp.ynorm));
        CK(ensure(h->tile_count, sizeof(int32_t) * tp.tiles));
        CK(ensure(h->rc_dist, sizeof(double) * (size_t)tp.rc_cap * c));
        CK(ensure(h->rc_plist, sizeof(int32_t) * (size_t)tp.rc_cap * c));
        CK(ensure(h->mu_a, sizeof(float) * tp.mu_a));
        CK(ensure(h->mu_a16, sizeof(uint16_t) * tp.mu_a16));
        CK(ensure(h->a16_err, sizeof(float) * 256));
        CK(ensure(h->a16_part, sizeof(float) * 256 * (size_t)mu_split16_splits(d)));
        CK(ensure(h->a16_done, sizeof(int32_t) * 256));
        CK(cudaMemsetAsync(h->a16_done.p, 0, h->a16_done.bytes, h->stream));
        // per-tile arrival counters of the search kernels start every call at zero
        CK(cudaMemsetAsync(h->tile_count.p, 0, h->tile_count.bytes, h->stream));
    }
    CK(ensure(h->rc_list, sizeof(RcRec) * n));
    if (h->hseed_cap < (size_t)c) {
        if (h->hseed_u) cudaFreeHost(h->hseed_u);
        h->hseed_u = nullptr;
        h->hseed_cap = 0;
        CK(cudaMallocHost(&h->hseed_u, sizeof(double) * c));
        h->hseed_cap = c;
    }
    return RESPCA_OK;
}

respca_status read_status(respca_ctx* h) {
    CK(cudaMemcpyAsync(h->hstat, h->status.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (h->hstat->timeout) return fail(h, RESPCA_ERR_TIMEOUT, "a bounded device wait gave up");
    return RESPCA_OK;
}

// Zero the per-pass counters of the status block (not the running totals).
cudaError_t zero_counters(respca_ctx* h) {
    DevStatus* s = P<DevStatus>(h->status);
    return cudaMemsetAsync(&s->flagged, 0, 4 * sizeof(int32_t), h->stream);   // flagged .. rc_pairs
}

// Centroids (and their norms, drift from the centroids the last search used,
// and pairwise separations) from the tile sums in Dpart, written to `dst`;
// `prev` holds the centroids of the last search.
respca_status finish_centroids(respca_ctx* h, int c, int64_t d, float* dst, const float* prev,
                               double* sums_out = nullptr, bool with_separation = true) {
    CK(launch_centroids(P<float>(h->Dpart), P<int32_t>(h->tile_off), P<int32_t>(h->counts), c, d,
                        dst, h->stream, sums_out));
    CK(launch_mu_stats(dst, prev, c, d, P<double>(h->mu_norm2), P<float>(h->mu_normf),
                       prev ? P<double>(h->drift) : nullptr, P<float2>(h->cs_part), P<int32_t>(h->cs_done), h->stream));
    if (with_separation)
        CK(launch_separation(dst, P<int32_t>(h->counts), c, d, P<float>(h->pair_ss), P<double>(h->sep2),
                             h->stream));
    return RESPCA_OK;
}

// ---------------------------------------------------------------- spectral p step
// Normalised spectral clustering of the columns of Y (Sec. 4.2 alternative to
// K-means): affinity and M = D^{-1/2} A D^{-1/2} (k_spectral.cu), the top-c
// eigenvectors of M by Chebyshev-filtered subspace iteration with
// Rayleigh-Ritz, the row-normalised embedding, and K-means on it in a second
// context whose workspace does not disturb the solver's.
constexpr int kSpecMaxC = 64;
constexpr int64_t kSpecMaxN = 32768;
constexpr int kSpecGuard = 8;       // extra vectors in the search block
constexpr int kSpecDegree = 8;      // Chebyshev degree per Rayleigh-Ritz step
constexpr int kSpecMaxOuter = 100;
// residual ||M u - theta u|| of the kept eigenpairs at which the eigensolver
// stops: about ten times the FP32 rounding of one product with M
double spec_tol(int64_t n) { return std::max(1e-5, 1e-6 * std::sqrt((double)n)); }

respca_status spectral_labels_impl(respca_ctx* h, const float* Y, int64_t ldy, int64_t d, int64_t n, int c,
                                   int32_t* p, respca_spectral_info* info) {
    if (c < 1 || c > kSpecMaxC || n > kSpecMaxN || n <= c)
        return fail(h, RESPCA_ERR_UNSUPPORTED, "spectral p step: needs 1 <= c <= 64 and c < n <= 32768");
    const int b = (int)std::min<int64_t>(n, c + kSpecGuard);
    const int parts = 152;
    cudaStream_t st = h->stream;
    CK(ensure(h->sp_M, sizeof(float) * (size_t)n * n));
    CK(ensure(h->sp_sqn, sizeof(float) * n));
    CK(ensure(h->sp_part, sizeof(double) * parts));
    CK(ensure(h->sp_gsum, sizeof(double) * spec_colsum_doubles(d)));
    CK(ensure(h->sp_sig, sizeof(double) * 2));
    CK(ensure(h->sp_deg, sizeof(double) * n));
    for (DevBuf* bb : {&h->sp_Y, &h->sp_W, &h->sp_T, &h->sp_Z}) CK(ensure(*bb, sizeof(float) * (size_t)n * b));
    CK(ensure(h->sp_H, sizeof(double) * b * b));
    CK(ensure(h->sp_Q, sizeof(float) * b * b));
    CK(ensure(h->sp_ev, sizeof(double) * b));
    CK(ensure(h->sp_res, sizeof(double) * c));
    CK(ensure(h->sp_E, sizeof(float) * (size_t)n * c));
    CK(ensure(h->sp_P, sizeof(float) * (size_t)spec_symm_chunks(n, b) * n * b));
    if (!h->status.p) {
        // a handle whose first call is this one: the status block (timeout flag) starts zeroed
        CK(ensure(h->status, sizeof(DevStatus)));
        CK(cudaMemsetAsync(h->status.p, 0, sizeof(DevStatus), st));
    }
    if (!h->spec_km) {
        respca_config kc = h->cfg;
        kc.stream = h->stream;
        kc.device = h->device;
        kc.timing = 0;
        kc.p_step = 0;
        respca_status cs = respca_create(&h->spec_km, &kc);
        if (cs != RESPCA_OK) return fail(h, cs, "spectral p step: K-means context");
    }
    float* M = P<float>(h->sp_M);
    if (!gram_tc_ok(Y, ldy)) {
        // the Gram kernel reads Y through a tensor map: 16-byte base and column stride
        const int64_t ldp = (d + 3) / 4 * 4;
        CK(ensure(h->sp_Ypad, sizeof(float) * (size_t)ldp * n));
        CK(cudaMemcpy2DAsync(h->sp_Ypad.p, sizeof(float) * ldp, Y, sizeof(float) * ldy, sizeof(float) * d, n,
                             cudaMemcpyDeviceToDevice, st));
        Y = P<float>(h->sp_Ypad);
        ldy = ldp;
    }
    DevStatus* dstat = P<DevStatus>(h->status);
    CK(cudaMemsetAsync(&dstat->timeout, 0, sizeof(int32_t), st));
    // with cfg.timing, events around the Gram kernel and each product with M (a
    // synchronisation per product: timing mode only)
    const bool timing = h->cfg.timing != 0;
    double ms_gram = 0.0, ms_prod = 0.0;
    CK(launch_spec_affinity(Y, ldy, d, n, h->cfg.spectral_scale, M, P<float>(h->sp_sqn), P<double>(h->sp_part),
                            parts, P<double>(h->sp_gsum), P<double>(h->sp_sig), P<double>(h->sp_deg),
                            P<float>(h->sp_sqn), dstat, timing ? h->evk0 : nullptr, timing ? h->evk1 : nullptr,
                            st));
    if (timing) {
        float ms = 0.f;
        CK(cudaEventSynchronize(h->evk1));
        CK(cudaEventElapsedTime(&ms, h->evk0, h->evk1));
        ms_gram = ms;
    }
    const float* rinv = P<float>(h->sp_sqn);   // deg^{-1/2}, written over the column norms
    auto product = [&](const float* Yin, float* Wout) -> cudaError_t {
        if (timing) {
            cudaError_t e = cudaEventRecord(h->evk0, st);
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = launch_spec_symm(M, rinv, n, Yin, b, Wout, P<float>(h->sp_P), st);
        if (e != cudaSuccess || !timing) return e;
        if ((e = cudaEventRecord(h->evk1, st)) != cudaSuccess || (e = cudaEventSynchronize(h->evk1)) != cudaSuccess)
            return e;
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, h->evk0, h->evk1);
        ms_prod += ms;
        return e;
    };
    float* Yb = P<float>(h->sp_Y);   // current orthonormal block (n x b)
    float* W = P<float>(h->sp_W);    // M Yb
    float* T = P<float>(h->sp_T);    // scratch
    float* Z = P<float>(h->sp_Z);    // scratch
    const int64_t nb = n * (int64_t)b;
    CK(launch_spec_start(Yb, n, b, h->cfg.seed, st));
    CK(launch_spec_cholqr2(Yb, T, n, b, P<double>(h->sp_H), P<float>(h->sp_Q), st));
    std::vector<double> ev(b), res(c);
    double sig2 = 0.0;
    int outer = 0, matvecs = 0;
    double rmax = INFINITY;
    double lo = -1.0;   // the spectrum of M lies in [-1, 1]
    for (;;) {
        // Rayleigh-Ritz on span(Yb): H = Yb^T M Yb, rotate to the Ritz vectors
        CK(product(Yb, W));
        ++matvecs;
        CK(launch_spec_gram_small(Yb, W, n, b, b, P<double>(h->sp_H), st));
        CK(launch_spec_jacobi(P<double>(h->sp_H), b, P<float>(h->sp_Q), P<double>(h->sp_ev), st));
        CK(launch_spec_rotate(Yb, P<float>(h->sp_Q), T, n, b, st));
        CK(launch_spec_rotate(W, P<float>(h->sp_Q), Z, n, b, st));
        std::swap(Yb, T);
        std::swap(W, Z);
        CK(launch_spec_residual(W, Yb, P<double>(h->sp_ev), n, c, P<double>(h->sp_res), st));
        CK(cudaMemcpyAsync(ev.data(), h->sp_ev.p, sizeof(double) * b, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(res.data(), h->sp_res.p, sizeof(double) * c, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&sig2, h->sp_sig.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        rmax = 0.0;
        for (double r : res) rmax = std::max(rmax, r);
        if (!(rmax > spec_tol(n)) || outer >= kSpecMaxOuter || b == n) break;
        ++outer;
        // Chebyshev filter of degree kSpecDegree damping [lo, a], a = the smallest
        // Ritz value of the block: Y_{k+1} = (2/e)(M - cen) Y_k - Y_{k-1}
        const double a = std::max(ev[b - 1], lo + 0.05);
        const double e = 0.5 * (a - lo), cen = 0.5 * (a + lo);
        // Y1 = (M Y0 - cen Y0) / e, with M Y0 = W from the Rayleigh-Ritz step
        float* y0 = Yb;
        float* y1 = T;
        float* y2 = Z;
        CK(launch_spec_axpby(y1, W, y0, nullptr, nb, (float)(1.0 / e), (float)(-cen / e), 0.f, st));
        for (int k = 2; k <= kSpecDegree; ++k) {
            CK(product(y1, W));   // W as scratch: M y1
            ++matvecs;
            CK(launch_spec_axpby(y2, W, y1, y0, nb, (float)(2.0 / e), (float)(-2.0 * cen / e), -1.f, st));
            float* t = y0;
            y0 = y1;
            y1 = y2;
            y2 = t;
        }
        // the filtered block y1 becomes the new (orthonormalised) search block
        CK(launch_spec_cholqr2(y1, y2, n, b, P<double>(h->sp_H), P<float>(h->sp_Q), st));
        if (y1 != Yb) {
            // keep the buffer roles fixed: Yb holds the block, T and Z are scratch
            CK(cudaMemcpyAsync(Yb, y1, sizeof(float) * nb, cudaMemcpyDeviceToDevice, st));
        }
    }
    {
        const respca_status ts = read_status(h);   // the Gram kernel's bounded waits
        if (ts != RESPCA_OK) return ts;
    }
    CK(launch_spec_embed(Yb, n, c, P<float>(h->sp_E), st));
    int32_t passes = 0;
    respca_status ks = respca_init_labels(h->spec_km, RESPCA_F32, h->sp_E.p, c, n, c, c, p, &passes);
    if (ks != RESPCA_OK) return fail(h, ks, "spectral p step: K-means on the embedding");
    if (info) {
        info->outer_iters = outer;
        info->matvecs = matvecs;
        info->ms_gram = ms_gram;
        info->ms_products = ms_prod;
        info->residual = rmax;
        info->sigma2 = sig2;
        info->theta_c = ev[c - 1];
        info->theta_next = (c < b) ? ev[c] : NAN;
        info->lloyd_passes = passes;
        info->converged = (rmax <= spec_tol(n)) ? 1 : 0;
    }
    return RESPCA_OK;
}

struct Problem {
    int dtype;
    const void* X;
    int64_t d, n, ldx;
    int c;
    float* L;
    float* S;
    float* Th;
    int64_t lds;
    int32_t* p;
    bool vec;     // 16-byte vector path usable for X, L, S, Theta, mu
};

// Nearest-centroid search (Sec. 4.2 assignment) for the listed columns of Y
// (all columns when list is null) against the centroids in h->mu: tensor
// cores for c <= 256 unless the handle asks for the CUDA-core kernel.
bool tc_search(respca_ctx* h, int c) {
    return c <= kTcMaxClusters && (h->cfg.search_impl == 0 || h->cfg.search_impl == 2);
}

// Scale of the FP16 copy of L: the power of two s with s m in [2^10, 2^11) for
// the reference magnitude m (the previous iteration's max |L|), 32x inside the
// FP16 range (values that outgrow it are clamped and their columns' error
// norms show it, so any s keeps the search exact).
float copy_scale(float m) {
    if (!(m > 0.f) || !std::isfinite(m)) return 1.f;
    int e = 0;
    std::frexp(m, &e);   // m < 2^e
    return std::ldexp(1.f, std::min(100, std::max(-100, 11 - e)));
}

// The 16-bit operand of the all-column search of Y, if any: BF16 or FP16 data
// itself, or the FP16 copy of the FP32 L the fused iteration wrote
// (h->sh_for).  *kind: the centroid split it needs (split16: 1 BF16, 2 FP16
// of s mu with the copy's scale s, 3 FP16 of mu), or 0.
bool search16_for(respca_ctx* h, int dtype, const void* Y, int64_t ldy, int64_t d, int c, Search16* s,
                  int* kind) {
    *kind = 0;
    if (h->cfg.search_impl != 0 || tc_npad(c) > 128) return false;
    s->a16 = P<uint16_t>(h->mu_a16);
    s->a16_err = P<float>(h->a16_err);
    s->dpad16 = (d + 63) / 64 * 64;
    if (dtype == RESPCA_BF16 || dtype == RESPCA_F16) {
        s->y16 = Y;
        s->ld16 = ldy;
        s->fp16 = dtype == RESPCA_F16;
        s->ycol = nullptr;
        *kind = s->fp16 ? 3 : 1;
        return true;
    }
    if (dtype == RESPCA_F32 && Y && Y == h->sh_for) {
        s->y16 = h->Lsh.p;
        s->ld16 = h->sh_ld;
        s->fp16 = true;
        s->ycol = P<float>(h->ycol);
        *kind = 2;
        return true;
    }
    return false;
}

// The a16 fields of a split description for kind (0: none).
void set_split16(respca_ctx* h, int64_t d, int kind, MuSplitOut* sp) {
    if (!kind) return;
    sp->a16 = P<uint16_t>(h->mu_a16);
    sp->dpad16 = (d + 63) / 64 * 64;
    sp->a16_kind = kind;
    sp->a16_err = P<float>(h->a16_err);
    sp->status = P<DevStatus>(h->status);
}

// The TF32 split of the centroids in h->mu (for the tensor-core search), and
// the 16-bit one of kind (search16_for) if any.
respca_status split_centroids(respca_ctx* h, int c, int64_t d, int kind) {
    const int64_t dpad = (d + 31) / 32 * 32;
    MuSplitOut sp16;
    set_split16(h, d, kind, &sp16);
    CK(launch_mu_split(P<float>(h->mu), c, d, tc_npad(c), dpad, P<float>(h->mu_hi), P<float>(h->mu_lo),
                       h->stream, P<float>(h->mu_a), kind ? &sp16 : nullptr, P<float>(h->a16_part),
                       P<int32_t>(h->a16_done)));
    return RESPCA_OK;
}

// split_ready: the split of the current centroids is already in place (the
// device-run Lloyd loop's update writes it).
respca_status search(respca_ctx* h, int dtype, const void* Y, int64_t ldy, int64_t d, int64_t n,
                     const int32_t* list, int c, int32_t* p, bool vec, bool split_ready = false) {
    DevStatus* ds = P<DevStatus>(h->status);
    if (tc_search(h, c)) {
        const int64_t dpad = (d + 31) / 32 * 32;
        const int64_t rc_cap = tc_plan(n, d, c).rc_cap;
        Search16 s16;
        int kind = 0;
        const bool use16 = search16_for(h, dtype, Y, ldy, d, c, &s16, &kind);
        if (!split_ready) {
            const respca_status rs = split_centroids(h, c, d, kind);
            if (rs != RESPCA_OK) return rs;
        }
        const bool timing = h->cfg.timing != 0;
        h->dense16 = use16;
        CK(launch_search_tc(dtype, Y, ldy, d, n, list, ds, P<float>(h->mu), P<float>(h->mu_hi),
                            P<float>(h->mu_lo), dpad, P<float>(h->mu_normf), P<int32_t>(h->counts), c,
                            p, P<float>(h->ub), P<float>(h->lb), P<float>(h->Gpart),
                            P<float>(h->ynorm_part), P<int32_t>(h->tile_count), P<RcRec>(h->rc_list),
                            P<int32_t>(h->rc_plist), P<double>(h->rc_dist), rc_cap, vec, h->stream, timing ? h->evd0 : nullptr,
                            timing ? h->evd1 : nullptr, timing ? &h->dense_recorded : nullptr,
                            P<float>(h->mu_a), use16 ? &s16 : nullptr));
    } else {
        CK(launch_assign(dtype, Y, ldy, d, n, list, P<float>(h->mu), P<float>(h->mu_normf),
                         P<int32_t>(h->counts), c, p, ds, h->stream, P<float>(h->ub), P<float>(h->lb)));
    }
    return RESPCA_OK;
}

// Timing mode: after the status of a search pass is read, adds the dense
// kernel's duration if it searched every column in this pass (no queue given,
// or a queue longer than search_list_max: otherwise that kernel returned at once).
respca_status account_dense(respca_ctx* h, bool list_given, int64_t n, int c) {
    if (!h->dense_recorded) return RESPCA_OK;
    h->dense_recorded = false;
    if (list_given && (int64_t)h->hstat->flagged <= search_list_max(n, c, h->dense16)) return RESPCA_OK;
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->evd0, h->evd1));
    h->ms_dense += ms;
    h->dense_passes += 1;
    if (h->dense16) {
        h->ms_dense16 += ms;
        h->dense16_passes += 1;
    }
    return RESPCA_OK;
}

struct SearchCounts {
    int passes = 0;
    int64_t assigned = 0;
    int64_t rechecked = 0;
    int64_t changed = 0;   // labels changed, summed over the passes counted here
};

// One Lloyd pass, first half: degrade the bounds by the centroid drift,
// queue the columns they cannot settle, search them.
// In the device-run loop the counters are cleared by the previous pass's
// end (k_moved of its update) and by k_lloyd_init before the first, not here.
respca_status lloyd_pass_search(respca_ctx* h, int mode, int dtype, const void* Y, int64_t ldy,
                                int64_t d, int64_t n, int c, int32_t* p, bool vec, bool in_graph = false) {
    (void)mode;
    DevStatus* ds = P<DevStatus>(h->status);
    if (!in_graph) CK(zero_counters(h));
    CK(launch_flag_bounds(kBoundsLloyd, nullptr, nullptr, 0, n, c, p, P<int32_t>(h->counts), nullptr,
                          1.0, P<double>(h->drift), P<float>(h->ub), P<float>(h->lb),
                          P<int32_t>(h->flag_list), ds, h->stream, P<int32_t>(h->labels_pass)));
    return search(h, dtype, Y, ldy, d, n, P<int32_t>(h->flag_list), c, p, vec, in_graph);
}

// Second half: move the changed columns between the cluster sums and form the
// new centroids, their norms and drift.
respca_status lloyd_pass_update(respca_ctx* h, int mode, int dtype, const void* Y, int64_t ldy,
                                int64_t d, int64_t n, int c, int32_t* p, const PassEnd* pe = nullptr) {
    DevStatus* ds = P<DevStatus>(h->status);
    const float* Lp = (mode == kSumL) ? static_cast<const float*>(Y) : nullptr;
    CK(launch_moved(p, P<int32_t>(h->labels_pass), n, c, P<int4>(h->moved), P<int2>(h->contrib),
                    P<int32_t>(h->boff), P<int32_t>(h->counts), ds, h->stream, pe));
    CK(launch_delta_sums(mode, dtype, Y, ldy, Lp, ldy, P<int2>(h->contrib), P<int32_t>(h->boff), c, d,
                         P<double>(h->sums), h->stream));
    MuSplitOut sp;
    if (tc_search(h, c)) {
        sp.Npad = tc_npad(c);
        sp.dpad = (d + 31) / 32 * 32;
        sp.arows = sp.Npad <= 64 ? 64 : 128;
        sp.hi = P<float>(h->mu_hi);
        sp.lo = P<float>(h->mu_lo);
        sp.a = sp.Npad <= 128 ? P<float>(h->mu_a) : nullptr;
        Search16 s16;
        int kind = 0;
        search16_for(h, dtype, Y, ldy, d, c, &s16, &kind);
        if (sp.a) set_split16(h, d, kind, &sp);
    }
    CK(launch_centroids_stats(P<double>(h->sums), P<int32_t>(h->counts), c, d, P<float>(h->mu),
                              P<float>(h->mu_old), P<double>(h->mu_norm2), P<float>(h->mu_normf),
                              P<double>(h->drift), sp, P<float4>(h->cs_part), P<int32_t>(h->cs_done), h->stream));
    return RESPCA_OK;
}

// Fingerprint of everything a captured pass depends on: the call's arguments
// and every workspace pointer (a reallocation changes it).
uint64_t lloyd_key(respca_ctx* h, int mode, int dtype, const void* Y, int64_t ldy, int64_t d, int64_t n,
                   int c, const int32_t* p, bool vec, int max_passes) {
    uint64_t k = 1469598103934665603ULL;
    auto mix = [&](uint64_t v) { k = (k ^ v) * 1099511628211ULL; };
    mix((uint64_t)mode);
    mix((uint64_t)dtype);
    mix(reinterpret_cast<uintptr_t>(Y));
    mix((uint64_t)ldy);
    mix((uint64_t)d);
    mix((uint64_t)n);
    mix((uint64_t)c);
    mix(reinterpret_cast<uintptr_t>(p));
    mix(vec ? 1u : 0u);
    mix((uint64_t)max_passes);
    mix((uint64_t)h->cfg.search_impl);
    mix(Y == h->sh_for ? 1u : 0u);   // whether the searches read the FP16 copy
    mix(reinterpret_cast<uintptr_t>(h->stream));
    for (DevBuf* b : all_bufs(h)) mix(reinterpret_cast<uintptr_t>(b->p));
    return k;
}

// The Lloyd loop run on the device: one pass is captured once into the body
// of a conditional while node; the first kernel of each pass's update (k_moved)
// also adds the pass counters and sets the condition.  The host reads the
// status once, after the loop.  The centroid update runs after the last pass
// too; when the loop stopped at max_passes with labels still moving, the
// centroids of that pass's search are put back (the host loop stops before
// that update).  RESPCA_ERR_UNSUPPORTED: no graph could be made here.
respca_status lloyd_loop_on_device(respca_ctx* h, int mode, int dtype, const void* Y, int64_t ldy,
                                   int64_t d, int64_t n, int c, int32_t* p, bool vec, int max_passes,
                                   SearchCounts* sc) {
    const uint64_t key = lloyd_key(h, mode, dtype, Y, ldy, d, n, c, p, vec, max_passes);
    respca_ctx::LloydGraph* g = nullptr;
    for (auto& e : h->lloyd_graph)
        if (e.exec && e.key == key) g = &e;
    if (!g) {
        if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
            return RESPCA_ERR_UNSUPPORTED;
        g = &h->lloyd_graph[h->lloyd_graph_next];
        h->lloyd_graph_next ^= 1;
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        *g = respca_ctx::LloydGraph{};
        cudaGraph_t graph = nullptr;
        cudaGraphConditionalHandle cond;
        cudaGraphNodeParams cp = {};
        cudaGraphNode_t node;
        if (cudaGraphCreate(&graph, 0) != cudaSuccess) return RESPCA_ERR_UNSUPPORTED;
        if (cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
            cudaGraphDestroy(graph);
            return RESPCA_ERR_UNSUPPORTED;
        }
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp) != cudaSuccess) {
            cudaGraphDestroy(graph);
            return RESPCA_ERR_UNSUPPORTED;
        }
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        // capture one pass on the private stream
        cudaStream_t user = h->stream;
        h->stream = h->cap_stream;
        const int64_t l0 = t_kernel_launches;
        respca_status rs = RESPCA_OK;
        if (cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            rs = RESPCA_ERR_UNSUPPORTED;
        } else {
            rs = lloyd_pass_search(h, mode, dtype, Y, ldy, d, n, c, p, vec, true);
            // the update's first kernel ends the pass (counters, loop condition)
            PassEnd pe;
            pe.cond = cond;
            pe.max_passes = max_passes;
            pe.on = 1;
            if (rs == RESPCA_OK) rs = lloyd_pass_update(h, mode, dtype, Y, ldy, d, n, c, p, &pe);
            cudaGraph_t captured = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(h->stream, &captured);
            if (rs == RESPCA_OK && ec != cudaSuccess) rs = RESPCA_ERR_UNSUPPORTED;
        }
        h->stream = user;
        g->launches_per_pass = t_kernel_launches - l0;
        t_kernel_launches = l0;
        cudaGetLastError();
        if (rs == RESPCA_OK && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) rs = RESPCA_ERR_UNSUPPORTED;
        if (rs != RESPCA_OK) {
            cudaGetLastError();
            if (g->exec) cudaGraphExecDestroy(g->exec);
            cudaGraphDestroy(graph);
            *g = respca_ctx::LloydGraph{};
            return rs == RESPCA_ERR_CUDA ? RESPCA_ERR_UNSUPPORTED : rs;
        }
        g->graph = graph;
        g->key = key;
    }
    DevStatus* ds = P<DevStatus>(h->status);
    CK(launch_lloyd_init(ds, sc->passes, h->stream));
    if (tc_search(h, c)) {   // the loop's searches use the split its updates write
        Search16 s16;
        int kind = 0;
        search16_for(h, dtype, Y, ldy, d, c, &s16, &kind);
        const respca_status rs = split_centroids(h, c, d, kind);
        if (rs != RESPCA_OK) return rs;
    }
    CK(cudaGraphLaunch(g->exec, h->stream));
    respca_status rs = read_status(h);
    if (rs != RESPCA_OK) return rs;
    const int run = h->hstat->acc_passes - sc->passes;
    t_kernel_launches += (int64_t)run * g->launches_per_pass;
    sc->passes = h->hstat->acc_passes;
    sc->assigned += h->hstat->acc_flagged;
    sc->rechecked += h->hstat->acc_rechecked;
    sc->changed += h->hstat->acc_changed;
    if (h->hstat->last_changed != 0)   // stopped at max_passes: back to the last search's centroids
        CK(cudaMemcpyAsync(h->mu.p, h->mu_old.p, sizeof(float) * (size_t)c * d, cudaMemcpyDeviceToDevice,
                           h->stream));
    return RESPCA_OK;
}

// Lloyd passes after an assignment moved some labels (Sec. 4.2 p step, or
// the initial labels): centroids become the means of the columns of Y under
// the new labels (the first time from a full pass over Y, then by moving only
// the columns whose label changed), every column's bounds degrade by the
// centroid drift, and only the columns the bounds cannot settle are searched.
// Stops when a pass changes no label or after max_passes passes in total.
//
// from_means (the p step of an iteration, FP32 L): h->mu holds the means of D
// under the labels the iteration started with (h->labels_prev, h->counts), and
// the mean of L = a D + (1 - a) mu_p over a cluster is that same mean, so the
// cluster sums of L under those labels are n_i mu_i; the columns the first
// search moved are then added and removed, instead of reading L again.
respca_status lloyd_continue(respca_ctx* h, int mode, int dtype, const void* Y, int64_t ldy,
                             int64_t d, int64_t n, int c, int32_t* p, bool vec, int max_passes,
                             SearchCounts* sc, bool from_means = false) {
    DevStatus* ds = P<DevStatus>(h->status);
    const int mt = max_tiles_for(n, c);
    const float* Lp = (mode == kSumL) ? static_cast<const float*>(Y) : nullptr;
    if (from_means) {
        CK(launch_sums_from_means(P<float>(h->mu), P<int32_t>(h->counts), c, d, P<double>(h->sums), h->stream));
        CK(launch_moved(p, P<int32_t>(h->labels_prev), n, c, P<int4>(h->moved), P<int2>(h->contrib),
                        P<int32_t>(h->boff), P<int32_t>(h->counts), ds, h->stream));
        CK(launch_delta_sums(mode, dtype, Y, ldy, Lp, ldy, P<int2>(h->contrib), P<int32_t>(h->boff), c, d,
                             P<double>(h->sums), h->stream));
        MuSplitOut none;
        CK(launch_centroids_stats(P<double>(h->sums), P<int32_t>(h->counts), c, d, P<float>(h->mu),
                                  P<float>(h->mu_old), P<double>(h->mu_norm2), P<float>(h->mu_normf),
                                  P<double>(h->drift), none, P<float4>(h->cs_part), P<int32_t>(h->cs_done),
                                  h->stream));
    } else {
        CK(launch_sort_labels(p, n, c, P<int32_t>(h->perm), P<int32_t>(h->counts), P<int32_t>(h->tile_off),
                              P<TileDesc>(h->tiles), ds, h->stream));
        CK(launch_colsum(mode, dtype, Y, ldy, Lp, nullptr, nullptr, ldy, 0.f, P<int32_t>(h->perm),
                         P<TileDesc>(h->tiles), mt, ds, d, P<float>(h->Dpart), vec, h->stream));
        CK(cudaMemcpyAsync(h->mu_old.p, h->mu.p, sizeof(float) * (size_t)c * d, cudaMemcpyDeviceToDevice,
                           h->stream));
        CK(launch_centroids(P<float>(h->Dpart), P<int32_t>(h->tile_off), P<int32_t>(h->counts), c, d,
                            P<float>(h->mu), h->stream, P<double>(h->sums)));
        CK(launch_mu_stats(P<float>(h->mu), P<float>(h->mu_old), c, d, P<double>(h->mu_norm2),
                           P<float>(h->mu_normf), P<double>(h->drift), P<float2>(h->cs_part), P<int32_t>(h->cs_done), h->stream));
    }
    // the device loop pays off where a pass is long enough for the launches and
    // status reads it saves to matter; building the graph costs about as much
    // as a few passes of a small problem
    constexpr int64_t kDeviceLoopMinElems = int64_t(1) << 22;
    if (h->cfg.timing == 0 && sc->passes < max_passes && d * n >= kDeviceLoopMinElems) {
        const respca_status rs = lloyd_loop_on_device(h, mode, dtype, Y, ldy, d, n, c, p, vec, max_passes, sc);
        if (rs != RESPCA_ERR_UNSUPPORTED) return rs;
        h->last_error.clear();   // no graph on this setup: the host runs the loop below
    }
    while (sc->passes < max_passes) {
        respca_status rs = lloyd_pass_search(h, mode, dtype, Y, ldy, d, n, c, p, vec);
        if (rs != RESPCA_OK) return rs;
        rs = read_status(h);
        if (rs != RESPCA_OK) return rs;
        rs = account_dense(h, true, n, c);
        if (rs != RESPCA_OK) return rs;
        sc->passes += 1;
        sc->assigned += h->hstat->flagged;
        sc->rechecked += h->hstat->rechecked;
        sc->changed += h->hstat->changed;
        if (h->hstat->changed == 0 || sc->passes >= max_passes) break;
        rs = lloyd_pass_update(h, mode, dtype, Y, ldy, d, n, c, p);
        if (rs != RESPCA_OK) return rs;
    }
    return RESPCA_OK;
}

// Initial labels: k-means++ seeding (D^2 sampling with splitmix64 draws),
// then Lloyd on the columns of X until no label changes.
// xmax > 0 (max |X|, known to the solve): the all-column passes over an FP32 X
// read an FP16 copy of it, written once here (as the iterations' passes read L's).
respca_status init_labels_impl(respca_ctx* h, const Problem& pb, int* passes_out, float xmax = 0.f) {
    const int c = pb.c;
    uint64_t st = h->cfg.seed;
    for (int k = 0; k < c; ++k) h->hseed_u[k] = unit_draw(st);
    int first = (int)(h->hseed_u[0] * (double)pb.n);
    if (first >= pb.n) first = (int)pb.n - 1;
    CK(cudaMemcpyAsync(h->seed_u.p, h->hseed_u, sizeof(double) * c, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->centers.p, &first, sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    // step k: D2 against centre k, then the pick of centre k + 1 (one launch)
    CK(cudaMemsetAsync(&P<DevStatus>(h->status)->seed_done, 0, sizeof(int32_t), h->stream));
    for (int k = 0; k + 1 < c; ++k)
        CK(launch_seed_step(pb.dtype, pb.X, pb.ldx, pb.d, pb.n, P<int32_t>(h->centers), k, k + 1,
                            P<double>(h->seed_u), P<double>(h->seedD2), P<double>(h->seed_part),
                            &P<DevStatus>(h->status)->seed_done, h->stream));
    CK(launch_gather_centers(pb.dtype, pb.X, pb.ldx, pb.d, P<int32_t>(h->centers), c, P<float>(h->mu),
                             P<int32_t>(h->counts), h->stream));
    CK(launch_mu_stats(P<float>(h->mu), nullptr, c, pb.d, P<double>(h->mu_norm2), P<float>(h->mu_normf),
                       nullptr, P<float2>(h->cs_part), P<int32_t>(h->cs_done), h->stream));
    CK(cudaMemsetAsync(pb.p, 0xFF, sizeof(int32_t) * pb.n, h->stream));
    CK(cudaMemsetAsync(h->lb.p, 0, sizeof(float) * pb.n, h->stream));
    DevStatus* ds = P<DevStatus>(h->status);
    const int km = std::max(1, h->cfg.kmeans_max_iter);
    SearchCounts sc;
    // large enough that the passes' savings (2 B per element each) repay the copy's 6 B
    constexpr int64_t kCopyXMinElems = int64_t(1) << 22;
    const bool copy_x = xmax > 0.f && pb.dtype == RESPCA_F32 && pb.vec && h->cfg.search_impl == 0 &&
                        tc_npad(c) <= 128 && pb.d * pb.n >= kCopyXMinElems;
    if (copy_x) {
        h->sh_ld = (pb.d + 7) / 8 * 8;
        CK(ensure(h->Lsh, sizeof(uint16_t) * (size_t)h->sh_ld * pb.n));
        CK(ensure(h->ycol, sizeof(float) * 2 * (size_t)pb.n));
        CK(launch_copy16_cols(static_cast<const float*>(pb.X), pb.ldx, pb.d, pb.n, copy_scale(xmax), h->Lsh.p,
                              h->sh_ld, P<float>(h->ycol), P<DevStatus>(h->status), h->stream));
        h->sh_for = pb.X;
    }
    CK(zero_counters(h));
    respca_status rs = search(h, pb.dtype, pb.X, pb.ldx, pb.d, pb.n, nullptr, c, pb.p, pb.vec);
    if (rs != RESPCA_OK) return rs;
    rs = read_status(h);
    if (rs != RESPCA_OK) return rs;
    rs = account_dense(h, false, pb.n, pb.c);
    if (rs != RESPCA_OK) return rs;
    sc.passes = 1;
    if (h->hstat->changed > 0 && km > 1) {
        rs = lloyd_continue(h, kSumX, pb.dtype, pb.X, pb.ldx, pb.d, pb.n, c, pb.p, pb.vec, km, &sc);
        if (rs != RESPCA_OK) return rs;
    }
    if (copy_x) h->sh_for = nullptr;   // the buffer serves L's copy next
    if (passes_out) *passes_out = sc.passes;
    return RESPCA_OK;
}

bool vec_ok(const void* p, int64_t ld, size_t esz) {
    return (reinterpret_cast<uintptr_t>(p) % (4 * esz) == 0) && (ld % 4 == 0);
}

respca_status check_args(respca_ctx* h, int dtype, const void* X, int64_t d, int64_t n, int64_t ldx,
                         double lambda, int c, double tol, int max_iter, float* L, float* S,
                         int64_t lds, int32_t* p) {
    if (!h) return RESPCA_ERR_INVALID_ARG;
    if (dtype < 0 || dtype > 2) return fail(h, RESPCA_ERR_INVALID_ARG, "x_dtype must be 0, 1 or 2");
    if (!X || !L || !S || !p) return fail(h, RESPCA_ERR_INVALID_ARG, "null X, L, S or p");
    if (d <= 0 || n <= 0) return fail(h, RESPCA_ERR_INVALID_ARG, "d and n must be positive");
    if (n > INT32_MAX - 64) return fail(h, RESPCA_ERR_INVALID_ARG, "n too large");
    if (ldx < d || lds < d) return fail(h, RESPCA_ERR_INVALID_ARG, "leading dimension < d");
    if (c < 1 || c > n) return fail(h, RESPCA_ERR_INVALID_ARG, "c must satisfy 1 <= c <= n");
    if (c > kMaxClusters) return fail(h, RESPCA_ERR_UNSUPPORTED, "c above 1024 is not supported");
    if (!std::isfinite(lambda)) return fail(h, RESPCA_ERR_INVALID_ARG, "lambda not finite");
    if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(h, RESPCA_ERR_INVALID_ARG, "tol must be finite and >= 0");
    if (max_iter < 0) return fail(h, RESPCA_ERR_INVALID_ARG, "max_iter < 0");
    if ((int64_t)(d / kChunkRows) >= 65535) return fail(h, RESPCA_ERR_UNSUPPORTED, "d too large");
    return RESPCA_OK;
}

double safety_factor(int64_t d) {
    // relative rounding slack on the FP32 squared separations (sums of d
    // positive terms) used by the pruning test
    double s = 1.0 - 2.0 * (double)d * 6.0e-8 - 1e-6;
    return s < 0.5 ? 0.5 : s;
}

// End of the bf16 phase: the BF16 state becomes the caller's FP32 L and S and
// the FP32 Theta.
respca_status widen_state(respca_ctx* h, const void* L16, const void* S16, const void* T16,
                          int64_t ld16, float* L, float* S, float* Th, int64_t lds, int64_t d,
                          int64_t n) {
    CK(launch_convert(RESPCA_BF16, L16, ld16, 0, L, lds, d, n, h->stream));
    CK(launch_convert(RESPCA_BF16, S16, ld16, 0, S, lds, d, n, h->stream));
    CK(launch_convert(RESPCA_BF16, T16, ld16, 0, Th, lds, d, n, h->stream));
    return RESPCA_OK;
}

respca_status solve_impl(respca_ctx* h, int dtype, const void* X, int64_t d, int64_t n, int64_t ldx,
                         double lambda, int c, double tol, int max_iter, const int32_t* p0, float* L,
                         float* S, int64_t lds, int32_t* p, respca_warm* warm, respca_stats* stats) {
    respca_status rs = check_args(h, dtype, X, d, n, ldx, lambda, c, tol, max_iter, L, S, lds, p);
    if (rs != RESPCA_OK) return rs;
    const bool is_warm = warm && warm->warm;
    if (is_warm && !(warm->rho > 0.0)) return fail(h, RESPCA_ERR_INVALID_ARG, "warm start needs rho > 0");
    if (is_warm && !warm->Theta) return fail(h, RESPCA_ERR_INVALID_ARG, "warm start needs Theta");
    CK(cudaSetDevice(h->device));
    const bool user_theta = warm && warm->Theta;
    rs = ensure_workspace(h, d, n, c, lds, !user_theta);
    if (rs != RESPCA_OK) return rs;
    h->last_error.clear();

    respca_stats out{};
    const int64_t launches0 = t_kernel_launches;
    const bool timing = h->cfg.timing != 0;
    h->ms_dense = 0.f;
    h->dense_passes = 0;
    h->ms_dense16 = 0.f;
    h->dense16_passes = 0;
    h->dense_recorded = false;
    h->sh_for = nullptr;
    CK(cudaEventRecord(h->ev0, h->stream));
    DevStatus* ds = P<DevStatus>(h->status);
    CK(cudaMemsetAsync(ds, 0, sizeof(DevStatus), h->stream));
    CK(launch_fro2(dtype, X, d, n, ldx, P<double>(h->fro_part), kFroParts, ds, h->stream));
    rs = read_status(h);
    if (rs != RESPCA_OK) return rs;
    if (h->hstat->nonfinite) return fail(h, RESPCA_ERR_NONFINITE_INPUT, "X holds NaN or Inf");
    const double nx = std::sqrt(h->hstat->x_norm2);
    // max |L| of the last fused iteration (max |X| before the first): sets the FP16 copy's scale
    float lmax_ref;
    std::memcpy(&lmax_ref, &h->hstat->xmax_bits, sizeof(float));
    const double lam = lambda > 0.0 ? lambda : std::sqrt((double)std::max(d, n));
    out.lambda = lam;
    out.x_norm = nx;

    Problem pb;
    pb.dtype = dtype;
    pb.X = X;
    pb.d = d;
    pb.n = n;
    pb.ldx = ldx;
    pb.c = c;
    pb.L = L;
    pb.S = S;
    pb.Th = user_theta ? warm->Theta : P<float>(h->theta);
    pb.lds = lds;
    pb.p = p;
    pb.vec = vec_ok(X, ldx, elem_size(dtype)) && vec_ok(L, lds, 4) && vec_ok(S, lds, 4) &&
             vec_ok(pb.Th, lds, 4) && (d % 4 == 0);

    // The views the iterations run on: FP32 state in the caller's L, S and
    // Theta, or (precision = 1, not warm) BF16 state and X in the workspace
    // until the bf16 phase ends.
    struct View {
        int xd;            // element type of the X the iterations read
        const void* X;
        int64_t ldx;
        int sd;            // state storage: 0 FP32, 1 BF16
        void *L, *S, *Th;
        int64_t ld;
        bool vec;
    } v{dtype, X, ldx, 0, L, S, pb.Th, lds, pb.vec};
    const bool l21 = h->cfg.s_norm == 1;
    const bool spectral = h->cfg.p_step == 1;
    if (spectral && dtype != RESPCA_F32)
        return fail(h, RESPCA_ERR_UNSUPPORTED, "spectral p step: X must be FP32");
    if (h->cfg.precision == 1 && !is_warm && !l21) {
        const int64_t ld16 = (d + 7) / 8 * 8;
        const size_t bytes = sizeof(uint16_t) * (size_t)ld16 * n;
        CK(ensure(h->L16, bytes));
        CK(ensure(h->S16, bytes));
        CK(ensure(h->T16, bytes));
        if (dtype == RESPCA_F32) {
            CK(ensure(h->X16, bytes));
            CK(launch_convert(dtype, X, ldx, 1, h->X16.p, ld16, d, n, h->stream));
            v.xd = RESPCA_BF16;
            v.X = h->X16.p;
            v.ldx = ld16;
        }
        v.sd = 1;
        v.L = h->L16.p;
        v.S = h->S16.p;
        v.Th = h->T16.p;
        v.ld = ld16;
        v.vec = (d % 4 == 0) && vec_ok(v.X, v.ldx, elem_size(v.xd));
    }
    double rho = is_warm ? warm->rho : h->cfg.rho0;
    if (!is_warm) {
        if (p0) {
            CK(cudaMemcpyAsync(p, p0, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, h->stream));
        } else if (nx > 0.0 && spectral) {
            respca_spectral_info si{};
            rs = spectral_labels_impl(h, static_cast<const float*>(X), ldx, d, n, c, p, &si);
            if (rs != RESPCA_OK) return rs;
            out.init_lloyd_passes = si.lloyd_passes;
        } else if (nx > 0.0) {
            int passes = 0;
            rs = init_labels_impl(h, pb, &passes, lmax_ref);   // lmax_ref is max |X| here
            if (rs != RESPCA_OK) return rs;
            out.init_lloyd_passes = passes;
        } else {
            CK(cudaMemsetAsync(p, 0, sizeof(int32_t) * n, h->stream));
        }
        CK(cudaMemset2DAsync(L, sizeof(float) * lds, 0, sizeof(float) * d, n, h->stream));
        CK(cudaMemset2DAsync(S, sizeof(float) * lds, 0, sizeof(float) * d, n, h->stream));
        CK(cudaMemset2DAsync(pb.Th, sizeof(float) * lds, 0, sizeof(float) * d, n, h->stream));
        if (v.sd == 1) {
            const size_t es = sizeof(uint16_t);
            CK(cudaMemset2DAsync(v.L, es * v.ld, 0, es * d, n, h->stream));
            CK(cudaMemset2DAsync(v.S, es * v.ld, 0, es * d, n, h->stream));
            CK(cudaMemset2DAsync(v.Th, es * v.ld, 0, es * d, n, h->stream));
        }
    }
    // sort the labels into tiles (and validate caller labels)
    const int mt = max_tiles_for(n, c);
    const int nch = nchunks_for(d);
    CK(launch_sort_labels(p, n, c, P<int32_t>(h->perm), P<int32_t>(h->counts), P<int32_t>(h->tile_off),
                          P<TileDesc>(h->tiles), ds, h->stream));
    rs = read_status(h);
    if (rs != RESPCA_OK) return rs;
    if (h->hstat->bad_labels) return fail(h, RESPCA_ERR_INVALID_ARG, "labels outside [0, c)");

    if (nx == 0.0) {
        CK(cudaMemset2DAsync(L, sizeof(float) * lds, 0, sizeof(float) * d, n, h->stream));
        CK(cudaMemset2DAsync(S, sizeof(float) * lds, 0, sizeof(float) * d, n, h->stream));
        CK(cudaEventRecord(h->ev1, h->stream));
        CK(cudaEventSynchronize(h->ev1));
        out.converged = 1;
        out.rho_final = rho;
        out.kernel_launches = t_kernel_launches - launches0;
        out.ms_dense = h->ms_dense;
        out.dense_passes = h->dense_passes;
        cudaEventElapsedTime(&out.ms_total, h->ev0, h->ev1);
        if (warm) warm->rho = rho;
        if (stats) *stats = out;
        return RESPCA_OK;
    }

    // centroids of D = X - S + Theta/rho under the current labels; no bound
    // information yet (lb = 0, no drift)
    CK(launch_colsum(kSumD, v.xd, v.X, v.ldx, nullptr, v.S, v.Th, v.ld, (float)(1.0 / rho),
                     P<int32_t>(h->perm), P<TileDesc>(h->tiles), mt, ds, d, P<float>(h->Dpart), v.vec,
                     h->stream, v.sd));
    rs = finish_centroids(h, c, d, P<float>(h->mu), nullptr);
    if (rs != RESPCA_OK) return rs;
    CK(cudaMemsetAsync(h->lb.p, 0, sizeof(float) * n, h->stream));
    CK(cudaMemsetAsync(h->drift.p, 0, sizeof(double) * c, h->stream));

    const int km = std::max(1, h->cfg.kmeans_max_iter);
    const double kappa = h->cfg.kappa;
    const double safety = safety_factor(d);
    int t_start = 0;
    if (!is_warm && h->cfg.ramp_skip && max_iter > 0 && !l21 && !spectral) {
        // Leading iterations with S = 0 and no label move, in closed form:
        // L_{t+1} = X_m + a_t g_t X_r, Theta_{t+1} = rho_t b_t g_t X_r.
        CK(cudaMemsetAsync(&ds->ramp_r2, 0, sizeof(double) + sizeof(unsigned long long) + sizeof(unsigned int),
                           h->stream));
        CK(launch_ramp_stats(v.xd, v.X, v.ldx, d, n, p, P<float>(h->mu), P<double>(h->sep2), safety,
                             &ds->ramp_abs, &ds->ramp_ratio, P<double>(h->seedD2), h->stream));
        CK(launch_sum_doubles(P<double>(h->seedD2), n, &ds->ramp_r2, h->stream));
        rs = read_status(h);
        if (rs != RESPCA_OK) return rs;
        float mabs;
        std::memcpy(&mabs, &h->hstat->ramp_abs, sizeof(float));
        double ratio;
        std::memcpy(&ratio, &h->hstat->ramp_ratio, sizeof(double));
        const double xr2 = h->hstat->ramp_r2;
        const double xr = std::sqrt(xr2);
        const double M = (double)mabs, margin = 1e-3;
        double g = 1.0, r = rho, prev_ag = 0.0, alpha = 0.0, beta = 0.0;
        int T = 0;
        double e_res = 0.0, e_dl = 0.0;
        while (T < max_iter) {
            const double a = r / (2.0 * lam + r), b = 2.0 * lam / (2.0 * lam + r);
            if (!(r * b * g * M <= 1.0 - margin)) break;          // S stays 0 (Eq. (24))
            if (!(a * g * ratio <= 0.5 * (1.0 - margin))) break;  // own centroid stays nearest
            const double ag = a * g;
            const double er = (1.0 - ag) * xr / nx;
            // ||L_{t+1} - L_t||: from L_0 = 0 the first step moves by ||X_m + a g X_r||
            const double edl = (T == 0)
                                   ? std::sqrt(std::max(0.0, h->hstat->x_norm2 - xr2 + ag * ag * xr2)) / nx
                                   : std::fabs(ag - prev_ag) * xr / nx;
            if (std::max(er, edl) <= tol) break;                  // leave convergence to the loop
            alpha = ag;
            beta = r * b * g;
            e_res = er;
            e_dl = edl;
            prev_ag = ag;
            g = 1.0 + (b / kappa) * g;
            r *= kappa;
            ++T;
        }
        if (T > 0) {
            CK(launch_ramp_state(v.xd, v.X, v.ldx, d, n, p, P<float>(h->mu), (float)alpha, (float)beta,
                                 v.L, v.Th, v.ld, h->stream, v.sd));
            rho = r;
            t_start = T;
            out.iters = T;
            out.err_resid = e_res;
            out.err_dL = e_dl;
            out.err_dS = 0.0;
            out.err = std::max(e_res, e_dl);
        }
    }
    CK(cudaEventRecord(h->ev2, h->stream));
    // stop_after_ramp: the closed-form leading iterations only
    const int iter_cap = (h->cfg.stop_after_ramp && !is_warm) ? t_start : max_iter;

    double err_hist[2] = {INFINITY, INFINITY};   // err of the last two bf16 iterations
    // all-column search passes counted on the device up to the last status read: the
    // copy of L (2 B per element more in the fused pass) is written for an iteration
    // when the previous p step (or the initial labels) searched every column twice or
    // more, each such pass then reading 2 B per element less (the status was last
    // read after the initial labels, which are the only passes before this loop)
    int32_t dense_seen = 0;
    for (int t = t_start; t < iter_cap; ++t) {
        const double rho_next = rho * kappa;
        IterScalars sc;
        sc.a = (float)(rho / (2.0 * lam + rho));
        sc.b = (float)(2.0 * lam / (2.0 * lam + rho));
        sc.inv_rho = (float)(1.0 / rho);
        sc.rho = (float)std::min(rho, (double)FLT_MAX);
        sc.inv_rho_next = (float)(1.0 / rho_next);

        CK(zero_counters(h));
        CK(cudaMemcpyAsync(h->labels_prev.p, p, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, h->stream));
        // the K-means p step on FP32 L searches an FP16 copy of it written by the same pass
        const int32_t dense_now = h->hstat->dense_passes;
        const bool use_sh = !l21 && !spectral && v.sd == 0 && v.vec && h->cfg.search_impl == 0 &&
                            tc_npad(c) <= 128 && dense_now - dense_seen >= 2;
        dense_seen = dense_now;
        if (use_sh) {
            h->sh_ld = (d + 7) / 8 * 8;
            CK(ensure(h->Lsh, sizeof(uint16_t) * (size_t)h->sh_ld * n));
            CK(ensure(h->ylo_part, sizeof(float) * 2 * (size_t)nch * n));
            CK(ensure(h->ycol, sizeof(float) * 2 * (size_t)n));
            sc.sh_scale = copy_scale(lmax_ref);
            out.copy16_iters += 1;
        }
        CK(cudaMemsetAsync(&ds->lmax_bits, 0, sizeof(uint32_t), h->stream));
        // L, S, Theta, norms, own distances, column movement and next-D sums in one pass
        if (timing) CK(cudaEventRecord(h->evk0, h->stream));
        if (l21)
            CK(launch_iteration_l21(v.xd, v.X, v.ldx, L, S, pb.Th, lds, P<float>(h->mu),
                                    P<int32_t>(h->perm), P<TileDesc>(h->tiles), mt, ds, d, n, sc,
                                    P<float>(h->Dpart), P<float>(h->own_part), P<float>(h->dl_part),
                                    P<float>(h->bn_part), P<double>(h->norm_part), v.vec, h->stream));
        else
            CK(launch_iteration(v.xd, v.sd, v.X, v.ldx, v.L, v.S, v.Th, v.ld, P<float>(h->mu),
                                P<int32_t>(h->perm), P<TileDesc>(h->tiles), mt, ds, d, n, sc,
                                P<float>(h->Dpart), P<float>(h->own_part), P<float>(h->dl_part),
                                P<double>(h->norm_part), v.vec, h->stream, use_sh ? h->Lsh.p : nullptr,
                                h->sh_ld, P<float>(h->ylo_part)));
        h->sh_for = use_sh ? v.L : nullptr;
        if (timing) CK(cudaEventRecord(h->evk1, h->stream));
        out.fused_launches += 1;
        CK(launch_reduce_norms(P<double>(h->norm_part), mt, nch, ds, P<double>(h->norm_red), h->stream));
        double r2, dl2, ds2;
        if (spectral) {
            // p step by spectral clustering of the columns of L (Sec. 4.2), then the
            // next centroids: D = X - S + Theta/rho_{t+1} under the new labels
            respca_spectral_info si{};
            rs = spectral_labels_impl(h, L, lds, d, n, c, p, &si);
            if (rs != RESPCA_OK) return rs;
            CK(launch_sort_labels(p, n, c, P<int32_t>(h->perm), P<int32_t>(h->counts), P<int32_t>(h->tile_off),
                                  P<TileDesc>(h->tiles), ds, h->stream));
            CK(launch_colsum(kSumD, v.xd, v.X, v.ldx, nullptr, v.S, v.Th, v.ld, sc.inv_rho_next,
                             P<int32_t>(h->perm), P<TileDesc>(h->tiles), mt, ds, d, P<float>(h->Dpart), v.vec,
                             h->stream, v.sd));
            rs = finish_centroids(h, c, d, P<float>(h->mu), nullptr);
            if (rs != RESPCA_OK) return rs;
            rs = read_status(h);
            if (rs != RESPCA_OK) return rs;
            out.lloyd_passes += si.lloyd_passes;
            r2 = h->hstat->norm2[0];
            dl2 = h->hstat->norm2[1];
            ds2 = h->hstat->norm2[2];
        } else {
        // p step, first Lloyd assignment: search only the columns the bounds cannot settle
        CK(launch_flag_bounds(kBoundsIter, P<float>(h->own_part), P<float>(h->dl_part), nch, n, c, p,
                              P<int32_t>(h->counts), P<double>(h->sep2), safety, P<double>(h->drift),
                              P<float>(h->ub), P<float>(h->lb), P<int32_t>(h->flag_list), ds,
                              h->stream, nullptr, h->sh_for ? P<float>(h->ylo_part) : nullptr,
                              h->sh_for ? P<float>(h->ycol) : nullptr, d));
        rs = search(h, v.sd == 1 ? RESPCA_BF16 : RESPCA_F32, v.L, v.ld, d, n, P<int32_t>(h->flag_list),
                    c, p, v.vec);
        if (rs != RESPCA_OK) return rs;
        // next centroids if every label stays (queued before the check; discarded
        // otherwise, but its FP64 sums then start the incremental update below).
        // Their separations are formed only once the labels are known to stay:
        // when some move, the final centroids get theirs at the end.
        rs = finish_centroids(h, c, d, P<float>(h->mu_next), P<float>(h->mu),
                              v.sd == 0 ? P<double>(h->sumsD) : nullptr, false);
        if (rs != RESPCA_OK) return rs;
        rs = read_status(h);
        if (rs != RESPCA_OK) return rs;
        rs = account_dense(h, true, n, c);
        if (rs != RESPCA_OK) return rs;
        if (timing) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, h->evk0, h->evk1));
            out.ms_fused += ms;
        }
        out.lloyd_passes += 1;
        out.assigned_columns += h->hstat->flagged;
        out.rechecked_columns += h->hstat->rechecked;
        r2 = h->hstat->norm2[0];
        dl2 = h->hstat->norm2[1];
        ds2 = h->hstat->norm2[2];

        if (h->hstat->changed == 0) {
            CK(cudaMemcpyAsync(h->mu.p, h->mu_next.p, sizeof(float) * (size_t)c * d, cudaMemcpyDeviceToDevice, h->stream));
            CK(launch_separation(P<float>(h->mu), P<int32_t>(h->counts), c, d, P<float>(h->pair_ss),
                                 P<double>(h->sep2), h->stream));
        } else {
            // Lloyd on the columns of L until no label changes
            SearchCounts scount;
            scount.passes = 1;
            scount.changed = h->hstat->changed;   // the first search's
            // (BF16 L is summed as the "X" operand: the sums only need its element type)
            rs = v.sd == 1 ? lloyd_continue(h, kSumX, RESPCA_BF16, v.L, v.ld, d, n, c, p, v.vec, km, &scount)
                           : lloyd_continue(h, kSumL, RESPCA_F32, v.L, v.ld, d, n, c, p, v.vec, km, &scount,
                                            true);
            if (rs != RESPCA_OK) return rs;
            out.lloyd_passes += scount.passes - 1;
            out.assigned_columns += scount.assigned;
            out.rechecked_columns += scount.rechecked;
            // next centroids: D = X - S + Theta/rho_{t+1} under the final labels.  The
            // correction below reads D at each moved column twice (24 B per element and
            // moved column), the recount once for every column (12 B per element): it
            // takes over from n / 8 moves on (the summed label changes bound the moves)
            if (v.sd == 0 && scount.changed <= n / 8) {
                // the fused pass's sums under the starting labels, corrected by
                // the columns whose label the p step changed
                CK(launch_moved(p, P<int32_t>(h->labels_prev), n, c, P<int4>(h->moved),
                                P<int2>(h->contrib), P<int32_t>(h->boff), P<int32_t>(h->counts), ds,
                                h->stream));
                CK(launch_delta_sums(kSumD, v.xd, v.X, v.ldx, nullptr, v.ld, P<int2>(h->contrib),
                                     P<int32_t>(h->boff), c, d, P<double>(h->sumsD), h->stream,
                                     static_cast<const float*>(v.S), static_cast<const float*>(v.Th),
                                     sc.inv_rho_next));
                CK(launch_sort_labels(p, n, c, P<int32_t>(h->perm), P<int32_t>(h->counts),
                                      P<int32_t>(h->tile_off), P<TileDesc>(h->tiles), ds, h->stream));
                CK(launch_centroids_from_sums(P<double>(h->sumsD), P<int32_t>(h->counts), c, d,
                                              P<float>(h->mu_next), h->stream));
                CK(launch_mu_stats(P<float>(h->mu_next), P<float>(h->mu), c, d, P<double>(h->mu_norm2),
                                   P<float>(h->mu_normf), P<double>(h->drift), P<float2>(h->cs_part), P<int32_t>(h->cs_done), h->stream));
                CK(launch_separation(P<float>(h->mu_next), P<int32_t>(h->counts), c, d,
                                     P<float>(h->pair_ss), P<double>(h->sep2), h->stream));
            } else {
                CK(launch_sort_labels(p, n, c, P<int32_t>(h->perm), P<int32_t>(h->counts),
                                      P<int32_t>(h->tile_off), P<TileDesc>(h->tiles), ds, h->stream));
                CK(launch_colsum(kSumD, v.xd, v.X, v.ldx, nullptr, v.S, v.Th, v.ld, sc.inv_rho_next,
                                 P<int32_t>(h->perm), P<TileDesc>(h->tiles), mt, ds, d, P<float>(h->Dpart),
                                 v.vec, h->stream, v.sd));
                rs = finish_centroids(h, c, d, P<float>(h->mu_next), P<float>(h->mu));
                if (rs != RESPCA_OK) return rs;
            }
            CK(cudaMemcpyAsync(h->mu.p, h->mu_next.p, sizeof(float) * (size_t)c * d, cudaMemcpyDeviceToDevice, h->stream));
            CK(launch_count_changed(p, P<int32_t>(h->labels_prev), n, ds, h->stream));
        }
        }   // K-means p step
        {
            float m;   // this iteration's max |L| (FP32 state; read with the p step's status)
            std::memcpy(&m, &h->hstat->lmax_bits, sizeof(float));
            if (m > 0.f) lmax_ref = m;
        }
        rho = rho_next;
        out.iters = t + 1;
        out.err_resid = std::sqrt(r2) / nx;
        out.err_dL = std::sqrt(dl2) / nx;
        out.err_dS = std::sqrt(ds2) / nx;
        out.err = std::max(out.err_resid, std::max(out.err_dL, out.err_dS));
        if (out.err <= tol) {
            out.converged = 1;
            break;
        }
        if (v.sd == 1) {
            out.bf16_iters += 1;
            // the bf16 phase ends at switch_tol, or once err stops falling (BF16
            // rounding of the state puts a floor under it)
            const bool stalled = out.bf16_iters >= 3 && out.err >= err_hist[1];
            err_hist[1] = err_hist[0];
            err_hist[0] = out.err;
            if (out.err <= h->cfg.switch_tol || stalled) {
                rs = widen_state(h, v.L, v.S, v.Th, v.ld, L, S, pb.Th, lds, d, n);
                if (rs != RESPCA_OK) return rs;
                h->sh_for = nullptr;
                v = View{dtype, X, ldx, 0, L, S, pb.Th, lds, pb.vec};
                // centroids of the next iteration from the FP32 X and the widened state
                CK(launch_sort_labels(p, n, c, P<int32_t>(h->perm), P<int32_t>(h->counts),
                                      P<int32_t>(h->tile_off), P<TileDesc>(h->tiles), ds, h->stream));
                CK(launch_colsum(kSumD, v.xd, v.X, v.ldx, nullptr, v.S, v.Th, v.ld, (float)(1.0 / rho),
                                 P<int32_t>(h->perm), P<TileDesc>(h->tiles), mt, ds, d,
                                 P<float>(h->Dpart), v.vec, h->stream, 0));
                rs = finish_centroids(h, c, d, P<float>(h->mu_next), P<float>(h->mu));
                if (rs != RESPCA_OK) return rs;
                CK(cudaMemcpyAsync(h->mu.p, h->mu_next.p, sizeof(float) * (size_t)c * d, cudaMemcpyDeviceToDevice, h->stream));
            }
        }
    }
    if (v.sd == 1) {   // stopped inside the bf16 phase: the outputs are FP32
        rs = widen_state(h, v.L, v.S, v.Th, v.ld, L, S, pb.Th, lds, d, n);
        if (rs != RESPCA_OK) return rs;
    }
    CK(cudaEventRecord(h->ev1, h->stream));
    rs = read_status(h);
    if (rs != RESPCA_OK) return rs;
    out.label_changes = h->hstat->label_changes;
    out.rho_final = rho;
    out.kernel_launches = t_kernel_launches - launches0;
    out.ms_dense = h->ms_dense;
    out.dense_passes = h->dense_passes;
    out.ms_dense16 = h->ms_dense16;
    out.dense16_passes = h->dense16_passes;
    h->sh_for = nullptr;
    cudaEventElapsedTime(&out.ms_total, h->ev0, h->ev1);
    cudaEventElapsedTime(&out.ms_init, h->ev0, h->ev2);
    if (warm) warm->rho = rho;
    if (stats) *stats = out;
    return RESPCA_OK;
}

}  // namespace

// ============================================================== C ABI
extern "C" {

void respca_config_default(respca_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->rho0 = 1e-4;
    cfg->kappa = 1.5;
    cfg->kmeans_max_iter = 100;
    cfg->seed = 0;
    cfg->stream = nullptr;
    cfg->device = -1;
    cfg->search_impl = 0;
    cfg->ramp_skip = 1;
    cfg->precision = 0;
    cfg->switch_tol = 1e-2;
    cfg->p_step = 0;
    cfg->spectral_scale = 0.125;
}

respca_status respca_create(respca_handle* out, const respca_config* cfg) {
    if (!out) return RESPCA_ERR_INVALID_ARG;
    *out = nullptr;
    respca_config c;
    if (cfg) c = *cfg;
    else respca_config_default(&c);
    if (!(c.rho0 > 0.0) || !(c.kappa > 0.0) || !std::isfinite(c.rho0) || !std::isfinite(c.kappa))
        return RESPCA_ERR_INVALID_ARG;
    if (c.s_norm != 0 && c.s_norm != 1) return RESPCA_ERR_INVALID_ARG;
    if (c.precision != 0 && c.precision != 1) return RESPCA_ERR_INVALID_ARG;
    if (c.p_step != 0 && c.p_step != 1) return RESPCA_ERR_INVALID_ARG;
    if (c.p_step == 1 && (c.precision != 0 || !(c.spectral_scale > 0.0) || !std::isfinite(c.spectral_scale)))
        return RESPCA_ERR_INVALID_ARG;
    if (c.stop_after_ramp != 0 && c.stop_after_ramp != 1) return RESPCA_ERR_INVALID_ARG;
    int dev = c.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return RESPCA_ERR_CUDA;
    if (cudaSetDevice(dev) != cudaSuccess) return RESPCA_ERR_CUDA;
    respca_ctx* h = new (std::nothrow) respca_ctx();
    if (!h) return RESPCA_ERR_OOM;
    h->cfg = c;
    h->device = dev;
    h->stream = reinterpret_cast<cudaStream_t>(c.stream);
    if (cudaMallocHost(&h->hstat, sizeof(DevStatus)) != cudaSuccess ||
        cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess ||
        cudaEventCreate(&h->ev2) != cudaSuccess || cudaEventCreate(&h->evk0) != cudaSuccess ||
        cudaEventCreate(&h->evk1) != cudaSuccess || cudaEventCreate(&h->evd0) != cudaSuccess ||
        cudaEventCreate(&h->evd1) != cudaSuccess) {
        respca_destroy(h);
        return RESPCA_ERR_OOM;
    }
    *out = h;
    return RESPCA_OK;
}

respca_status respca_destroy(respca_handle h) {
    if (!h) return RESPCA_OK;
    for (respca_ctx* lane : h->lanes) respca_destroy(lane);
    h->lanes.clear();
    if (h->spec_km) respca_destroy(h->spec_km);
    h->spec_km = nullptr;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    for (DevBuf* b : all_bufs(h))
        if (b->p) cudaFree(b->p);
    respca::batched_state_free(h->batched);
    h->batched = nullptr;
    if (h->hstat) cudaFreeHost(h->hstat);
    if (h->hseed_u) cudaFreeHost(h->hseed_u);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->ev2) cudaEventDestroy(h->ev2);
    if (h->evk0) cudaEventDestroy(h->evk0);
    if (h->evk1) cudaEventDestroy(h->evk1);
    if (h->evd0) cudaEventDestroy(h->evd0);
    if (h->evd1) cudaEventDestroy(h->evd1);
    for (auto& g : h->lloyd_graph) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
    return RESPCA_OK;
}

respca_status respca_solve(respca_handle h, int32_t x_dtype, const void* X, int64_t d, int64_t n,
                           int64_t ldx, double lambda, int32_t c, double tol, int32_t max_iter,
                           const int32_t* p0, float* L, float* S, int64_t lds, int32_t* p,
                           respca_warm* warm, respca_stats* stats) {
    return solve_impl(h, x_dtype, X, d, n, ldx, lambda, c, tol, max_iter, p0, L, S, lds, p, warm, stats);
}

respca_status respca_solve_host(respca_handle h, int32_t x_dtype, const void* X, int64_t d, int64_t n,
                                int64_t ldx, double lambda, int32_t c, double tol, int32_t max_iter,
                                const int32_t* p0, float* L, float* S, int64_t lds, int32_t* p,
                                respca_stats* stats) {
    respca_status rs = check_args(h, x_dtype, X, d, n, ldx, lambda, c, tol, max_iter, L, S, lds, p);
    if (rs != RESPCA_OK) return rs;
    CK(cudaSetDevice(h->device));
    const size_t esz = elem_size(x_dtype);
    // device copies with leading dimension rounded up to 4 elements (16-byte columns)
    const int64_t dpad = (d + 3) / 4 * 4;
    CK(ensure(h->hX, esz * (size_t)dpad * n));
    CK(ensure(h->hL, sizeof(float) * (size_t)dpad * n));
    CK(ensure(h->hS, sizeof(float) * (size_t)dpad * n));
    CK(ensure(h->hp, sizeof(int32_t) * n));
    if (p0) CK(ensure(h->hp0, sizeof(int32_t) * n));
    CK(cudaMemcpy2DAsync(h->hX.p, esz * dpad, X, esz * ldx, esz * d, n, cudaMemcpyHostToDevice, h->stream));
    if (dpad != d) {
        // zero the padding rows so no uninitialised value is ever read
        CK(cudaMemset2DAsync((char*)h->hX.p + esz * d, esz * dpad, 0, esz * (dpad - d), n, h->stream));
    }
    if (p0) CK(cudaMemcpyAsync(h->hp0.p, p0, sizeof(int32_t) * n, cudaMemcpyHostToDevice, h->stream));
    rs = solve_impl(h, x_dtype, h->hX.p, d, n, dpad, lambda, c, tol, max_iter,
                    p0 ? P<int32_t>(h->hp0) : nullptr, P<float>(h->hL), P<float>(h->hS), dpad,
                    P<int32_t>(h->hp), nullptr, stats);
    if (rs != RESPCA_OK) return rs;
    CK(cudaMemcpy2DAsync(L, sizeof(float) * lds, h->hL.p, sizeof(float) * dpad, sizeof(float) * d, n,
                         cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpy2DAsync(S, sizeof(float) * lds, h->hS.p, sizeof(float) * dpad, sizeof(float) * d, n,
                         cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(p, h->hp.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return RESPCA_OK;
}

respca_status respca_init_labels(respca_handle h, int32_t x_dtype, const void* X, int64_t d, int64_t n,
                                 int64_t ldx, int32_t c, int32_t* p, int32_t* passes) {
    if (!h) return RESPCA_ERR_INVALID_ARG;
    if (x_dtype < 0 || x_dtype > 2 || !X || !p || d <= 0 || n <= 0 || ldx < d || c < 1 || c > n)
        return fail(h, RESPCA_ERR_INVALID_ARG, "invalid arguments");
    if (c > kMaxClusters) return fail(h, RESPCA_ERR_UNSUPPORTED, "c above 1024 is not supported");
    CK(cudaSetDevice(h->device));
    respca_status rs = ensure_workspace(h, d, n, c, d, false);
    if (rs != RESPCA_OK) return rs;
    Problem pb{};
    pb.dtype = x_dtype;
    pb.X = X;
    pb.d = d;
    pb.n = n;
    pb.ldx = ldx;
    pb.c = c;
    pb.p = p;
    pb.vec = vec_ok(X, ldx, elem_size(x_dtype)) && (d % 4 == 0);
    CK(cudaMemsetAsync(h->status.p, 0, sizeof(DevStatus), h->stream));
    int np = 0;
    rs = init_labels_impl(h, pb, &np);
    if (rs != RESPCA_OK) return rs;
    if (passes) *passes = np;
    return RESPCA_OK;
}

respca_status respca_solve_batched(respca_handle h, int32_t batch, const respca_problem* probs,
                                   respca_stats* stats) {
    if (!h || batch < 0 || (batch > 0 && !probs)) return RESPCA_ERR_INVALID_ARG;
    if (batch == 0) return RESPCA_OK;
    auto solve_one = [&](respca_ctx* ctx, int32_t b) {
        const respca_problem& q = probs[b];
        return respca_solve(ctx, q.x_dtype, q.X, q.d, q.n, q.ldx, q.lambda, q.c, q.tol, q.max_iter,
                            q.p0, q.L, q.S, q.lds, q.p, nullptr, stats ? &stats[b] : nullptr);
    };
    const int lanes = std::min<int>(h->cfg.batch_lanes > 0 ? h->cfg.batch_lanes : 8, batch);
    if (lanes <= 1) {
        respca_status first = RESPCA_OK;
        for (int32_t b = 0; b < batch; ++b) {
            const respca_status rs = solve_one(h, b);
            if (rs != RESPCA_OK && first == RESPCA_OK) first = rs;
        }
        return first;
    }
    if (cudaSetDevice(h->device) != cudaSuccess) return RESPCA_ERR_CUDA;
    while ((int)h->lanes.size() < lanes) {
        respca_config lc = h->cfg;
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return RESPCA_ERR_CUDA;
        lc.stream = s;
        lc.device = h->device;
        respca_handle lane = nullptr;
        const respca_status rs = respca_create(&lane, &lc);
        if (rs != RESPCA_OK) {
            cudaStreamDestroy(s);
            return rs;
        }
        lane->own_stream = s;
        h->lanes.push_back(lane);
    }
    // largest problems first, so the lanes finish together
    std::vector<int32_t> order(batch);
    for (int32_t b = 0; b < batch; ++b) order[b] = b;
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        return probs[x].d * probs[x].n > probs[y].d * probs[y].n;
    });
    // the lanes start after the work already queued on the caller's stream
    if (cudaEventRecord(h->ev0, h->stream) != cudaSuccess) return RESPCA_ERR_CUDA;
    for (int w = 0; w < lanes; ++w)
        if (cudaStreamWaitEvent(h->lanes[w]->stream, h->ev0, 0) != cudaSuccess) return RESPCA_ERR_CUDA;
    std::vector<respca_status> result(batch, RESPCA_OK);
    std::vector<std::string> message(batch);
    std::atomic<int32_t> next{0};
    auto run_lane = [&](int w) {
        cudaSetDevice(h->device);
        respca_ctx* ctx = h->lanes[w];
        for (;;) {
            const int32_t k = next.fetch_add(1);
            if (k >= batch) break;
            result[order[k]] = solve_one(ctx, order[k]);
            if (result[order[k]] != RESPCA_OK) message[order[k]] = ctx->last_error;
        }
    };
    std::vector<std::thread> threads;
    try {
        for (int w = 1; w < lanes; ++w) threads.emplace_back(run_lane, w);
    } catch (...) {
        // fewer host threads than lanes: the remaining lanes' share goes to the others
    }
    run_lane(0);
    for (std::thread& t : threads) t.join();
    // the caller's stream sees the lanes' work as done
    for (int w = 0; w < lanes; ++w) {
        if (cudaEventRecord(h->lanes[w]->ev1, h->lanes[w]->stream) != cudaSuccess ||
            cudaStreamWaitEvent(h->stream, h->lanes[w]->ev1, 0) != cudaSuccess)
            return RESPCA_ERR_CUDA;
    }
    for (int32_t b = 0; b < batch; ++b) {
        if (result[b] != RESPCA_OK) {
            h->last_error = std::string("problem ") + std::to_string(b) + ": " + message[b];
            return result[b];
        }
    }
    return RESPCA_OK;
}

respca_status respca_solve_batched_persistent(respca_handle h, int32_t batch, const respca_problem* probs,
                                              respca_stats* stats, respca_batch_options* opt) {
    if (!h) return RESPCA_ERR_INVALID_ARG;
    h->last_error.clear();
    return respca::batched_persistent(&h->batched, h->device, h->stream, h->cfg.seed, h->cfg.rho0, h->cfg.kappa,
                                      h->cfg.kmeans_max_iter, batch, probs, stats, opt, &h->last_error);
}

respca_status respca_column_norms(const float* S, int64_t d, int64_t n, int64_t lds, float* out,
                                  void* stream) {
    if (!S || !out || d < 1 || n < 1 || lds < d) return RESPCA_ERR_INVALID_ARG;
    if (launch_column_norms(S, lds, d, n, out, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
        return RESPCA_ERR_CUDA;
    return RESPCA_OK;
}

respca_status respca_spectral_labels(respca_handle h, const float* Y, int64_t d, int64_t n, int64_t ldy,
                                     int32_t c, int32_t* p, respca_spectral_info* info) {
    if (!h || !Y || !p || d < 1 || n < 1 || ldy < d || c < 1) return fail(h, RESPCA_ERR_INVALID_ARG, "bad arguments");
    if (!(h->cfg.spectral_scale > 0.0)) return fail(h, RESPCA_ERR_INVALID_ARG, "spectral_scale must be > 0");
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(h, RESPCA_ERR_CUDA, "cudaSetDevice");
    return spectral_labels_impl(h, Y, ldy, d, n, c, p, info);
}

const char* respca_status_string(respca_status s) {
    switch (s) {
        case RESPCA_OK: return "ok";
        case RESPCA_ERR_INVALID_ARG: return "invalid argument";
        case RESPCA_ERR_NONFINITE_INPUT: return "non-finite input";
        case RESPCA_ERR_OOM: return "out of memory";
        case RESPCA_ERR_CUDA: return "CUDA error";
        case RESPCA_ERR_TIMEOUT: return "device wait timed out";
        case RESPCA_ERR_UNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

const char* respca_last_error(respca_handle h) { return h ? h->last_error.c_str() : ""; }

}  // extern "C"
