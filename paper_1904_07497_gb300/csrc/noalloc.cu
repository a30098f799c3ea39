// Allocation-free variant of the initial-labels computation
// (respca_init_labels_noalloc, declared in include/respca.h).
//
// Who needs it: callers that must not allocate device memory while they run
// this step -- applications whose device memory is owned by their own pool
// allocator or capped by a hard budget, and plug-in hosts that forbid a
// library from taking device memory behind their back.  Such callers cannot
// create a respca handle, whose workspace is cudaMalloc'ed on demand.  This
// entry point takes every bit of scratch from one file-scope __device__ array
// instead, sized once at library load.  The call is synchronous: it reads its
// progress back from the device after every Lloyd pass.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/respca.h"
#include "respca_internal.cuh"

using namespace respca;

namespace {

// 32 MiB of device memory per GPU that loads the library, held until exit.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Carves 256-byte aligned pieces out of the scratch array (base may be null
// to measure the total).
struct Carve {
    char* base;
    size_t off = 0;
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = reinterpret_cast<T*>(base + off);
        off += sizeof(T) * count;
        return p;
    }
};

struct Scratch {
    DevStatus* status;
    double* D2;
    int32_t* centers;
    double* u;
    float* mu;
    double* mu_norm2;
    float* mu_normf;
    int32_t* counts;
    int32_t* perm;
    int32_t* tile_off;
    TileDesc* tiles;
    float* Dpart;
};

size_t layout(char* base, int64_t d, int64_t n, int c, Scratch* s) {
    const int64_t mt = (n + kTileCols - 1) / kTileCols + c;
    Carve cv{base};
    Scratch t;
    t.status = cv.take<DevStatus>(1);
    t.D2 = cv.take<double>(n);
    t.centers = cv.take<int32_t>(c);
    t.u = cv.take<double>(c);
    t.mu = cv.take<float>((size_t)c * d);
    t.mu_norm2 = cv.take<double>(c);
    t.mu_normf = cv.take<float>(c);
    t.counts = cv.take<int32_t>(c);
    t.perm = cv.take<int32_t>(n);
    t.tile_off = cv.take<int32_t>(c + 1);
    t.tiles = cv.take<TileDesc>(mt);
    t.Dpart = cv.take<float>((size_t)mt * d);
    if (s) *s = t;
    return cv.off;
}

// Device address of the scratch array on the current device.  Looked up once
// per device (cudaGetSymbolAddress with that device current) and cached.
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// True when ptr is device memory of device dev (or managed memory, which
// every device can reach).
bool on_device(const void* ptr, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        (void)cudaGetLastError();   // clear the error this query may leave behind
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

uint64_t draw_bits(uint64_t& s) {   // splitmix64, as in the handle path
    s += 0x9E3779B97F4A7C15ULL;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" respca_status respca_init_labels_noalloc(int32_t x_dtype, const void* X, int64_t d,
                                                     int64_t n, int64_t ldx, int32_t c,
                                                     uint64_t seed, int32_t kmeans_max_iter,
                                                     int32_t* p, int32_t* passes, void* stream) {
    if (x_dtype < 0 || x_dtype > 2 || !X || !p || d <= 0 || n <= 0 || ldx < d || c < 1 || c > n ||
        n > INT32_MAX - 64)
        return RESPCA_ERR_INVALID_ARG;
    if (c > kMaxClusters) return RESPCA_ERR_UNSUPPORTED;
    if (layout(nullptr, d, n, c, nullptr) > kNoAllocScratchBytes) return RESPCA_ERR_UNSUPPORTED;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // The scratch array and every launch belong to the current device, so X
    // and p must live there too (a kernel given another GPU's pointer faults).
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return RESPCA_ERR_CUDA;
    if (!on_device(X, cur) || !on_device(p, cur)) return RESPCA_ERR_INVALID_ARG;
    void* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return RESPCA_ERR_CUDA;
    Scratch s;
    layout(static_cast<char*>(base), d, n, c, &s);

#define NA_CK(expr)                                   \
    do {                                              \
        if ((expr) != cudaSuccess) return RESPCA_ERR_CUDA; \
    } while (0)

    // The array keeps the previous call's contents: zero the status block.
    NA_CK(cudaMemsetAsync(s.status, 0, sizeof(DevStatus), st));
    double u[kMaxClusters];          // host stack, no heap
    uint64_t state = seed;
    for (int k = 0; k < c; ++k) u[k] = (double)(draw_bits(state) >> 11) * (1.0 / 9007199254740992.0);
    int32_t first = (int32_t)(u[0] * (double)n);
    if (first >= n) first = (int32_t)n - 1;
    NA_CK(cudaMemcpyAsync(s.u, u, sizeof(double) * c, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(s.centers, &first, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    NA_CK(launch_seed_dist(x_dtype, X, ldx, d, n, s.centers, 0, s.D2, st));
    for (int k = 1; k < c; ++k) {
        NA_CK(launch_seed_pick(s.D2, n, s.u, k, s.centers, st));
        if (k + 1 < c) NA_CK(launch_seed_dist(x_dtype, X, ldx, d, n, s.centers, k, s.D2, st));
    }
    NA_CK(launch_gather_centers(x_dtype, X, ldx, d, s.centers, c, s.mu, s.counts, st));
    NA_CK(launch_mu_norms(s.mu, c, d, s.mu_norm2, s.mu_normf, st));
    NA_CK(cudaMemsetAsync(p, 0xFF, sizeof(int32_t) * n, st));
    const size_t esz = x_dtype == RESPCA_F32 ? 4 : 2;
    const bool vec = (reinterpret_cast<uintptr_t>(X) % (4 * esz) == 0) && (ldx % 4 == 0) && (d % 4 == 0);
    const int mt = (int)((n + kTileCols - 1) / kTileCols) + c;
    const int km = kmeans_max_iter > 1 ? kmeans_max_iter : 1;   // as the handle path
    int np = 0;
    DevStatus hs;
    while (np < km) {
        NA_CK(cudaMemsetAsync(&s.status->flagged, 0, 3 * sizeof(int32_t), st));
        NA_CK(launch_assign(x_dtype, X, ldx, d, n, nullptr, s.mu, s.mu_normf, s.counts, c, p,
                            s.status, st));
        ++np;
        NA_CK(cudaMemcpyAsync(&hs, s.status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
        NA_CK(cudaStreamSynchronize(st));
        if (hs.changed == 0) break;
        NA_CK(launch_sort_labels(p, n, c, s.perm, s.counts, s.tile_off, s.tiles, s.status, st));
        NA_CK(launch_colsum(kSumX, x_dtype, X, ldx, nullptr, nullptr, nullptr, 0, 0.f, s.perm,
                            s.tiles, mt, s.status, d, s.Dpart, vec, st));
        NA_CK(launch_centroids(s.Dpart, s.tile_off, s.counts, c, d, s.mu, st));
        NA_CK(launch_mu_norms(s.mu, c, d, s.mu_norm2, s.mu_normf, st));
    }
#undef NA_CK
    if (passes) *passes = np;
    return RESPCA_OK;
}
