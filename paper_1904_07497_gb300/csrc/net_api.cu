// Host driver and C ABI of the learned warm start (include/respca.h,
// respca_net_*, respca_mlp_*, respca_adam_step): an unrolled continuation of
// the Sec. 4 iteration with fixed labels and per-layer (rho_k, tau_k), its
// reverse pass, and the small MLP that predicts the per-layer multipliers.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/respca.h"
#include "respca_internal.cuh"

using namespace respca;

namespace {

struct NetBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

cudaError_t grow(NetBuf& b, size_t bytes) {
    if (b.p && b.bytes >= bytes) return cudaSuccess;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    const cudaError_t e = cudaMalloc(&b.p, bytes > 0 ? bytes : 16);
    if (e == cudaSuccess) b.bytes = bytes;
    return e;
}

template <typename T>
T* F(NetBuf& b) { return reinterpret_cast<T*>(b.p); }

constexpr int kLossParts = 1216;   // CTAs of the loss kernel (152 SMs x 8)

}  // namespace

struct respca_net_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    // the last forward pass, kept for the reverse pass
    bool have_forward = false;
    const float* X = nullptr;
    int64_t d = 0, n = 0, ldx = 0;
    int c = 0, layers = 0;
    double lambda = 0.0;
    std::vector<double> rho_k, tau_k;
    NetBuf state;           // (layers + 1) pairs (S, Theta), d x n each, leading dimension d
    NetBuf L;               // L of the last layer
    NetBuf mu;              // layers x c x d centroids of D, one set per layer
    NetBuf perm, counts, tile_off, tiles, status, part;   // label sort and tile partials
    NetBuf gS, gT, gL, gmean, scal_part, scal_out, loss_part, loss_out;
    NetBuf ping;            // inference: two (S, Theta) states of the intermediate layers
};

namespace {

float* S_of(respca_net_s* h, int k) { return F<float>(h->state) + (size_t)(2 * k) * h->d * h->n; }
float* T_of(respca_net_s* h, int k) { return F<float>(h->state) + (size_t)(2 * k + 1) * h->d * h->n; }
float* mu_of(respca_net_s* h, int k) { return F<float>(h->mu) + (size_t)k * h->c * h->d; }

NetScalars scalars(const respca_net_s* h, int k) {
    const double rho = h->rho_k[k];
    const double rho_next = (k + 1 < h->layers) ? h->rho_k[k + 1] : rho;
    NetScalars sc;
    sc.a = (float)(rho / (2.0 * h->lambda + rho));
    sc.b = (float)(2.0 * h->lambda / (2.0 * h->lambda + rho));
    sc.rho = (float)rho;
    sc.inv_rho = (float)(1.0 / rho);
    sc.tau = (float)h->tau_k[k];
    sc.inv_rho_next = (float)(1.0 / rho_next);
    return sc;
}

int max_tiles(const respca_net_s* h) { return (int)((h->n + kTileCols - 1) / kTileCols) + h->c; }

#define NK(expr)                                                                     \
    do {                                                                             \
        const cudaError_t _e = (expr);                                               \
        if (_e != cudaSuccess)                                                       \
            return _e == cudaErrorMemoryAllocation ? RESPCA_ERR_OOM : RESPCA_ERR_CUDA; \
    } while (0)

bool aligned16(const void* p, int64_t ld) {
    return (reinterpret_cast<uintptr_t>(p) & 15) == 0 && (ld % 4) == 0;
}

}  // namespace

extern "C" {

respca_status respca_net_create(respca_net* net, int32_t device, void* stream) {
    if (!net) return RESPCA_ERR_INVALID_ARG;
    *net = nullptr;
    int dev = device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return RESPCA_ERR_CUDA;
    if (cudaSetDevice(dev) != cudaSuccess) return RESPCA_ERR_CUDA;
    auto* h = new (std::nothrow) respca_net_s();
    if (!h) return RESPCA_ERR_OOM;
    h->device = dev;
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    *net = h;
    return RESPCA_OK;
}

respca_status respca_net_destroy(respca_net h) {
    if (!h) return RESPCA_OK;
    cudaSetDevice(h->device);
    for (NetBuf* b : {&h->state, &h->L, &h->mu, &h->perm, &h->counts, &h->tile_off, &h->tiles, &h->status,
                      &h->part, &h->gS, &h->gT, &h->gL, &h->gmean, &h->scal_part, &h->scal_out,
                      &h->loss_part, &h->loss_out, &h->ping})
        if (b->p) cudaFree(b->p);
    delete h;
    return RESPCA_OK;
}

respca_status respca_net_schedule(double rho, double kappa, int32_t layers, const float* m, double* rho_k,
                                  double* tau_k) {
    if (!m || !rho_k || !tau_k || layers < 1 || !(rho > 0.0) || !(kappa > 0.0)) return RESPCA_ERR_INVALID_ARG;
    double r = rho;
    for (int k = 0; k < layers; ++k) {
        rho_k[k] = r * std::exp((double)m[k]);
        tau_k[k] = std::exp((double)m[layers + k]) / rho_k[k];
        r *= kappa;
    }
    return RESPCA_OK;
}

respca_status respca_net_forward(respca_net h, const float* X, int64_t d, int64_t n, int64_t ldx,
                                 const int32_t* p, int32_t c, double lambda, const float* S0,
                                 const float* Theta0, int64_t lds, int32_t layers, const double* rho_k,
                                 const double* tau_k, float* L, float* S, float* Theta) {
    if (!h || !X || !p || !S0 || !Theta0 || !rho_k || !tau_k) return RESPCA_ERR_INVALID_ARG;
    if (d < 1 || n < 1 || ldx < d || lds < d || c < 1 || c > kMaxClusters || c > n || layers < 1 ||
        !(lambda > 0.0))
        return RESPCA_ERR_INVALID_ARG;
    if (n > INT32_MAX / 2) return RESPCA_ERR_UNSUPPORTED;
    for (int k = 0; k < layers; ++k)
        if (!(rho_k[k] > 0.0) || !(tau_k[k] >= 0.0) || !std::isfinite(rho_k[k])) return RESPCA_ERR_INVALID_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return RESPCA_ERR_CUDA;
    h->have_forward = false;
    h->X = X;
    h->d = d;
    h->n = n;
    h->ldx = ldx;
    h->c = c;
    h->layers = layers;
    h->lambda = lambda;
    h->rho_k.assign(rho_k, rho_k + layers);
    h->tau_k.assign(tau_k, tau_k + layers);
    const size_t dn = (size_t)d * n;
    const int mt = max_tiles(h);
    cudaStream_t st = h->stream;
    NK(grow(h->state, sizeof(float) * dn * 2 * (layers + 1)));
    NK(grow(h->L, sizeof(float) * dn));
    NK(grow(h->mu, sizeof(float) * (size_t)layers * c * d));
    NK(grow(h->perm, sizeof(int32_t) * n));
    NK(grow(h->counts, sizeof(int32_t) * c));
    NK(grow(h->tile_off, sizeof(int32_t) * (c + 1)));
    NK(grow(h->tiles, sizeof(TileDesc) * mt));
    NK(grow(h->status, sizeof(DevStatus)));
    NK(grow(h->part, sizeof(float) * (size_t)mt * d));
    DevStatus* ds = F<DevStatus>(h->status);
    NK(cudaMemsetAsync(ds, 0, sizeof(DevStatus), st));
    NK(launch_sort_labels(p, n, c, F<int32_t>(h->perm), F<int32_t>(h->counts), F<int32_t>(h->tile_off),
                          F<TileDesc>(h->tiles), ds, st));
    // labels outside [0, c) leave the group offsets unwritten: stop before any kernel reads them
    int32_t bad = 0;
    NK(cudaMemcpyAsync(&bad, &ds->bad_labels, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    NK(cudaStreamSynchronize(st));
    if (bad) return RESPCA_ERR_INVALID_ARG;
    NK(cudaMemcpy2DAsync(S_of(h, 0), sizeof(float) * d, S0, sizeof(float) * lds, sizeof(float) * d, n,
                         cudaMemcpyDeviceToDevice, st));
    NK(cudaMemcpy2DAsync(T_of(h, 0), sizeof(float) * d, Theta0, sizeof(float) * lds, sizeof(float) * d, n,
                         cudaMemcpyDeviceToDevice, st));
    // means of the first layer's D; each layer sums the next one's
    const bool vec = (d % 4 == 0) && aligned16(X, ldx) && aligned16(h->state.p, d);
    NK(launch_colsum(kSumD, RESPCA_F32, X, ldx, nullptr, S_of(h, 0), T_of(h, 0), d, (float)(1.0 / rho_k[0]),
                     F<int32_t>(h->perm), F<TileDesc>(h->tiles), mt, ds, d, F<float>(h->part), vec, st));
    for (int k = 0; k < layers; ++k) {
        NK(launch_centroids(F<float>(h->part), F<int32_t>(h->tile_off), F<int32_t>(h->counts), c, d,
                            mu_of(h, k), st));
        NK(launch_net_layer(X, ldx, S_of(h, k), T_of(h, k), F<float>(h->L), S_of(h, k + 1), T_of(h, k + 1), d,
                            mu_of(h, k), F<int32_t>(h->perm), F<TileDesc>(h->tiles), mt, ds, d, scalars(h, k),
                            F<float>(h->part), st));
    }
    if (L)
        NK(cudaMemcpy2DAsync(L, sizeof(float) * lds, h->L.p, sizeof(float) * d, sizeof(float) * d, n,
                             cudaMemcpyDeviceToDevice, st));
    if (S)
        NK(cudaMemcpy2DAsync(S, sizeof(float) * lds, S_of(h, layers), sizeof(float) * d, sizeof(float) * d, n,
                             cudaMemcpyDeviceToDevice, st));
    if (Theta)
        NK(cudaMemcpy2DAsync(Theta, sizeof(float) * lds, T_of(h, layers), sizeof(float) * d, sizeof(float) * d,
                             n, cudaMemcpyDeviceToDevice, st));
    h->have_forward = true;
    return RESPCA_OK;
}

respca_status respca_net_backward(respca_net h, const float* Lt, const float* St, int64_t ldt, double scale,
                                  double* loss, double* g_rho, double* g_tau, float* g_m) {
    if (!h || !Lt || !St || !loss || !g_rho || !g_tau) return RESPCA_ERR_INVALID_ARG;
    if (!h->have_forward || ldt < h->d || !(scale > 0.0)) return RESPCA_ERR_INVALID_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return RESPCA_ERR_CUDA;
    const int64_t d = h->d, n = h->n;
    const size_t dn = (size_t)d * n;
    const int K = h->layers, mt = max_tiles(h);
    const int parts = mt * net_row_chunks(d);
    cudaStream_t st = h->stream;
    NK(grow(h->gS, sizeof(float) * dn));
    NK(grow(h->gT, sizeof(float) * dn));
    NK(grow(h->gL, sizeof(float) * dn));
    NK(grow(h->gmean, sizeof(float) * (size_t)h->c * d));
    NK(grow(h->scal_part, sizeof(double) * 4 * parts));
    NK(grow(h->scal_out, sizeof(double) * 8 * K));
    NK(grow(h->loss_part, sizeof(double) * kLossParts));
    NK(grow(h->loss_out, sizeof(double)));
    const DevStatus* ds = F<DevStatus>(h->status);
    NK(launch_net_loss(F<float>(h->L), S_of(h, K), d, Lt, St, ldt, d, n, (float)scale, F<float>(h->gL),
                       F<float>(h->gS), F<float>(h->gT), F<double>(h->loss_part), kLossParts,
                       F<double>(h->loss_out), st));
    for (int k = K - 1; k >= 0; --k) {
        const NetScalars sc = scalars(h, k);
        const float* gLext = (k == K - 1) ? F<float>(h->gL) : nullptr;
        double* so = F<double>(h->scal_out) + 8 * k;
        NK(launch_net_back(1, h->X, h->ldx, S_of(h, k), T_of(h, k), d, mu_of(h, k), F<int32_t>(h->perm),
                           F<TileDesc>(h->tiles), mt, ds, d, sc, gLext, F<float>(h->gS), F<float>(h->gT),
                           nullptr, F<float>(h->part), F<double>(h->scal_part), so, st));
        NK(launch_centroids(F<float>(h->part), F<int32_t>(h->tile_off), F<int32_t>(h->counts), h->c, d,
                            F<float>(h->gmean), st));
        NK(launch_net_back(2, h->X, h->ldx, S_of(h, k), T_of(h, k), d, mu_of(h, k), F<int32_t>(h->perm),
                           F<TileDesc>(h->tiles), mt, ds, d, sc, gLext, F<float>(h->gS), F<float>(h->gT),
                           F<float>(h->gmean), nullptr, F<double>(h->scal_part), so + 4, st));
    }
    std::vector<double> sc_host(8 * K);
    NK(cudaMemcpyAsync(sc_host.data(), h->scal_out.p, sizeof(double) * 8 * K, cudaMemcpyDeviceToHost, st));
    NK(cudaMemcpyAsync(loss, h->loss_out.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    NK(cudaStreamSynchronize(st));
    for (int k = 0; k < K; ++k) {
        const double* s = sc_host.data() + 8 * k;
        const double rho = h->rho_k[k], lam2 = 2.0 * h->lambda;
        // s[0] sum gTheta' (X - L - S'), s[1] dloss/dtau, s[2] dloss/da,
        // s[3] + s[7] sum (gB + gD) Theta  (Theta/rho enters B and D)
        g_rho[k] = s[0] + s[2] * lam2 / ((lam2 + rho) * (lam2 + rho)) - (s[3] + s[7]) / (rho * rho);
        g_tau[k] = s[1];
        if (g_m) {
            g_m[k] = (float)(rho * g_rho[k] - h->tau_k[k] * g_tau[k]);
            g_m[K + k] = (float)(h->tau_k[k] * g_tau[k]);
        }
    }
    return RESPCA_OK;
}

respca_status respca_mlp_forward(const float* params, int32_t nz, int32_t H, int32_t nout, const float* z,
                                 float* out, float* hidden, void* stream) {
    if (!params || !z || !out || !hidden || nz < 1 || H < 1 || nout < 1 || nz > 1024 || H > 1024 ||
        nout > 1024)
        return RESPCA_ERR_INVALID_ARG;
    return launch_mlp_forward(params, nz, H, nout, z, out, hidden, reinterpret_cast<cudaStream_t>(stream)) ==
                   cudaSuccess
               ? RESPCA_OK
               : RESPCA_ERR_CUDA;
}

respca_status respca_mlp_backward(const float* params, int32_t nz, int32_t H, int32_t nout, const float* z,
                                  const float* hidden, const float* gout, float* grad, int32_t accumulate,
                                  void* stream) {
    if (!params || !z || !hidden || !gout || !grad || nz < 1 || H < 1 || nout < 1 || nz > 1024 || H > 1024 ||
        nout > 1024)
        return RESPCA_ERR_INVALID_ARG;
    return launch_mlp_backward(params, nz, H, nout, z, hidden, gout, grad, accumulate ? 1 : 0,
                               reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
               ? RESPCA_OK
               : RESPCA_ERR_CUDA;
}

respca_status respca_adam_step(float* params, const float* grad, float* m, float* v, int64_t count, double lr,
                               double beta1, double beta2, double eps, int32_t t, void* stream) {
    if (!params || !grad || !m || !v || count < 1 || t < 1 || !(beta1 >= 0.0 && beta1 < 1.0) ||
        !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
        return RESPCA_ERR_INVALID_ARG;
    const double c1 = 1.0 / (1.0 - std::pow(beta1, t)), c2 = 1.0 / (1.0 - std::pow(beta2, t));
    return launch_adam(params, grad, m, v, count, (float)lr, (float)beta1, (float)beta2, (float)eps, (float)c1,
                       (float)c2, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
               ? RESPCA_OK
               : RESPCA_ERR_CUDA;
}

respca_status respca_net_infer(respca_net h, int32_t x_dtype, const void* X, int64_t d, int64_t n, int64_t ldx,
                               const int32_t* p, int32_t c, double lambda, const float* S0, const float* Theta0,
                               int64_t lds, int32_t layers, const double* rho_k, const double* tau_k,
                               int32_t storage, float* L, float* S, float* Theta) {
    if (!h || !X || !p || !S0 || !Theta0 || !rho_k || !tau_k || !L || !S || !Theta)
        return RESPCA_ERR_INVALID_ARG;
    if (x_dtype < 0 || x_dtype > 2 || (storage != 0 && storage != 1)) return RESPCA_ERR_INVALID_ARG;
    if (d < 1 || n < 1 || ldx < d || lds < d || c < 1 || c > kMaxClusters || c > n || layers < 1 ||
        !(lambda > 0.0))
        return RESPCA_ERR_INVALID_ARG;
    if (n > INT32_MAX / 2) return RESPCA_ERR_UNSUPPORTED;
    for (int k = 0; k < layers; ++k)
        if (!(rho_k[k] > 0.0) || !(tau_k[k] >= 0.0) || !std::isfinite(rho_k[k])) return RESPCA_ERR_INVALID_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return RESPCA_ERR_CUDA;
    h->have_forward = false;     // nothing is kept for a reverse pass
    const int mt = (int)((n + kTileCols - 1) / kTileCols) + c;
    const int64_t ldm = (d + 7) / 8 * 8;             // intermediate states: 16-byte aligned columns
    const size_t esz = storage == 1 ? 2 : 4;
    cudaStream_t st = h->stream;
    NK(grow(h->ping, esz * (size_t)ldm * n * (layers > 1 ? 4 : 0) + 16));
    NK(grow(h->mu, sizeof(float) * (size_t)c * d));
    NK(grow(h->perm, sizeof(int32_t) * n));
    NK(grow(h->counts, sizeof(int32_t) * c));
    NK(grow(h->tile_off, sizeof(int32_t) * (c + 1)));
    NK(grow(h->tiles, sizeof(TileDesc) * mt));
    NK(grow(h->status, sizeof(DevStatus)));
    NK(grow(h->part, sizeof(float) * (size_t)mt * d));
    DevStatus* ds = F<DevStatus>(h->status);
    NK(cudaMemsetAsync(ds, 0, sizeof(DevStatus), st));
    NK(launch_sort_labels(p, n, c, F<int32_t>(h->perm), F<int32_t>(h->counts), F<int32_t>(h->tile_off),
                          F<TileDesc>(h->tiles), ds, st));
    int32_t bad = 0;
    NK(cudaMemcpyAsync(&bad, &ds->bad_labels, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    NK(cudaStreamSynchronize(st));
    if (bad) return RESPCA_ERR_INVALID_ARG;
    // buffer k of the ping-pong pair: (S, Theta) of an intermediate layer
    char* base = static_cast<char*>(h->ping.p);
    auto Sb = [&](int k) { return base + esz * (size_t)ldm * n * (2 * (k & 1)); };
    auto Tb = [&](int k) { return base + esz * (size_t)ldm * n * (2 * (k & 1) + 1); };
    const bool vec_in = (d % 4 == 0) && (lds % 4 == 0) && (reinterpret_cast<uintptr_t>(S0) % 16 == 0) &&
                        (reinterpret_cast<uintptr_t>(Theta0) % 16 == 0) && (ldx % 4 == 0) &&
                        (reinterpret_cast<uintptr_t>(X) % (x_dtype == 0 ? 16 : 8) == 0);
    NK(launch_colsum(kSumD, x_dtype, X, ldx, nullptr, S0, Theta0, lds, (float)(1.0 / rho_k[0]), F<int32_t>(h->perm),
                     F<TileDesc>(h->tiles), mt, ds, d, F<float>(h->part), vec_in, st));
    for (int k = 0; k < layers; ++k) {
        NetScalars sc;
        const double rho = rho_k[k], rho_next = (k + 1 < layers) ? rho_k[k + 1] : rho;
        sc.a = (float)(rho / (2.0 * lambda + rho));
        sc.b = (float)(2.0 * lambda / (2.0 * lambda + rho));
        sc.rho = (float)rho;
        sc.inv_rho = (float)(1.0 / rho);
        sc.tau = (float)tau_k[k];
        sc.inv_rho_next = (float)(1.0 / rho_next);
        NK(launch_centroids(F<float>(h->part), F<int32_t>(h->tile_off), F<int32_t>(h->counts), c, d,
                            F<float>(h->mu), st));
        const bool first = k == 0, last = k + 1 == layers;
        NK(launch_net_infer(x_dtype, first ? 0 : storage, last ? 0 : storage, X, ldx,
                            first ? static_cast<const void*>(S0) : Sb(k - 1),
                            first ? static_cast<const void*>(Theta0) : Tb(k - 1), first ? lds : ldm,
                            last ? L : nullptr, last ? static_cast<void*>(S) : Sb(k),
                            last ? static_cast<void*>(Theta) : Tb(k), last ? lds : ldm, F<float>(h->mu),
                            F<int32_t>(h->perm), F<TileDesc>(h->tiles), mt, ds, d, sc, F<float>(h->part), st));
    }
    return RESPCA_OK;
}

}  // extern "C"
