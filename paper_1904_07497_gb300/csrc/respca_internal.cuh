// Internal declarations shared by the RES-PCA CUDA translation units.
//
// Data layout in HBM (all column-major, a column = one sample):
//   X      d x n, leading dim ldx, FP32 / BF16 / FP16 (read only)
//   L, S   d x n FP32, leading dim lds (caller's outputs, updated in place)
//   Theta  d x n FP32, leading dim lds (handle workspace or caller's)
//   mu     c x d FP32, cluster i's centroid contiguous: mu[i*d + r]
//   labels n int32
// Columns are visited in label-sorted order (perm) through "tiles": runs of
// at most kTileCols consecutive sorted columns that share one label, so a
// thread can sum a row of one cluster in a register.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <string>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/respca.h"

namespace respca {

constexpr int kThreads = 256;       // threads per CTA of the streaming kernels
constexpr int kTileCols = 32;       // columns per label-pure tile
constexpr int kChunkRows = 512;     // rows per CTA in the streaming kernels
constexpr int kAsgCols = 32;        // columns per CTA in the assignment kernel
constexpr int kAsgRows = 64;        // rows staged per step in the assignment kernel
constexpr int kAsgClusters = 64;    // centroids per register block in the assignment kernel
constexpr int kMaxClusters = 1024;  // largest c this build accepts
constexpr int kSortThreads = 1024;

// Per-iteration scalars, derived in FP64 on the host and rounded once.
struct IterScalars {
    float a;             // rho / (2 lambda + rho)          (Eq. (18), first term)
    float b;             // 2 lambda / (2 lambda + rho)      (Eq. (18), mean term)
    float inv_rho;       // 1 / rho_t
    float rho;           // rho_t, capped at FLT_MAX
    float inv_rho_next;  // 1 / rho_{t+1}
    float sh_scale = 1.f;  // scale s of the FP16 copy of L the pass writes (if any)
};

struct TileDesc {
    int32_t start;  // first sorted position
    int32_t len;    // columns in the tile (1..kTileCols)
    int32_t label;  // cluster of every column in the tile
    int32_t pad;
};

// Device-side status block, read back once per iteration.
struct DevStatus {
    double norm2[3];        // sums of squares of X-L-S, L-L_prev, S-S_prev
    double x_norm2;         // ||X||_F^2
    double ramp_r2;         // ||X - mu_p||_F^2 (ramp statistics)
    unsigned long long ramp_ratio;  // bits of max_j ||X_j - mu_p|| / sep(p)
    unsigned int ramp_abs;  // bits of max |X - mu_p|
    int32_t flagged;        // columns queued for a nearest-centroid search
    int32_t changed;        // labels changed by the last assignment pass
    int32_t rechecked;      // near-tie columns re-decided in FP64
    int32_t rc_pairs;       // (column, candidate) pairs queued for the re-decision
    int32_t nonfinite;      // X holds NaN/Inf
    int32_t ntiles;         // tiles of the current sort
    int32_t bad_labels;     // labels outside [0, c)
    int32_t label_changes;  // running total of changed labels (vs. start of iteration)
    int32_t moved;          // entries of the last moved-column list
    int32_t timeout;        // a bounded device-side wait gave up
    int32_t last_changed;   // device-run Lloyd loop: labels changed by its last pass
    int64_t acc_flagged;    // device-run Lloyd loop: columns searched over its passes
    int32_t acc_passes;     //   passes run (including those before the loop)
    int32_t acc_rechecked;  //   near ties re-decided
    int32_t acc_changed;    //   labels changed (summed over passes)
    int32_t seed_done;      // CTAs of the current k-means++ step that finished (reset by the last)
    int32_t dense_passes;   // all-column search passes so far (their parity sets the walking direction)
    int32_t norms_done;     // CTAs of the norm reduction that finished (reset by the last)
    float sh_scale;         // power-of-two scale s of the FP16 copy of L (stores fp16(s l)) and of the
    float sh_inv2;          //   centroids' FP16 split; 1 / s^2 (set by the fused iteration that wrote it)
    uint32_t lmax_bits;     // bits of max |L| over the last fused iteration (FP32 state)
    uint32_t xmax_bits;     // bits of max |X| (the norm pass over X)
};

// Modes of the bound-based pruning kernel.
enum BoundsMode : int { kBoundsIter = 0, kBoundsLloyd = 1 };

// Mode of the column-group sum kernel.
enum SumMode : int { kSumX = 0, kSumL = 1, kSumD = 2 };

// Kernels launched by this thread (each launcher adds its count); a solve
// reports the difference across its body.
inline thread_local int64_t t_kernel_launches = 0;
inline void count_launches(int k) { t_kernel_launches += k; }

// ---------------------------------------------------------------- launchers
// (each returns the launch status; all run on `st`)
// One k-means++ step: D2 against centre k, then centre kpick (< 0: none)
// picked by the CTA that finishes last.  part: ceil(n / 8) doubles.
cudaError_t launch_seed_step(int dtype, const void* X, int64_t ldx, int64_t d, int64_t n, int32_t* centers,
                             int k, int kpick, const double* u, double* D2, double* part, int32_t* done,
                             cudaStream_t st);
cudaError_t launch_fro2(int dtype, const void* X, int64_t d, int64_t n, int64_t ldx,
                        double* part, int nparts, DevStatus* status, cudaStream_t st);

cudaError_t launch_sort_labels(const int32_t* labels, int64_t n, int c, int32_t* perm,
                               int32_t* counts, int32_t* tile_off, TileDesc* tiles,
                               DevStatus* status, cudaStream_t st);

cudaError_t launch_colsum(int mode, int dtype, const void* X, int64_t ldx, const float* L,
                          const void* S, const void* Th, int64_t lds, float inv_rho,
                          const int32_t* perm, const TileDesc* tiles, int max_tiles,
                          const DevStatus* status, int64_t d, float* Dpart, bool vec,
                          cudaStream_t st, int sdtype = 0);

cudaError_t launch_centroids(const float* Dpart, const int32_t* tile_off, const int32_t* counts,
                             int c, int64_t d, float* mu, cudaStream_t st,
                             double* sums_out = nullptr);

cudaError_t launch_centroids_from_sums(const double* sums, const int32_t* counts, int c, int64_t d,
                                       float* mu, cudaStream_t st, float* mu_old = nullptr);

cudaError_t launch_delta_sums(int mode, int dtype, const void* X, int64_t ldx, const float* L,
                              int64_t lds, const int2* contrib, const int32_t* boff, int c, int64_t d,
                              double* sums, cudaStream_t st, const float* S = nullptr,
                              const float* Th = nullptr, float inv_rho = 0.f);

// part / done: as for launch_centroids_stats (the two never run at once on a stream)
cudaError_t launch_mu_stats(const float* mu, const float* mu_old, int c, int64_t d,
                            double* mu_norm2, float* mu_normf, double* drift, float2* part, int32_t* done,
                            cudaStream_t st);

// TF32 split of the centroids for the tensor-core search (layout of launch_mu_split).
struct MuSplitOut {
    float* hi = nullptr;   // Npad x dpad
    float* lo = nullptr;   // Npad x dpad
    float* a = nullptr;    // 2 arows x dpad (raw rows, then lo rows), or null
    int64_t dpad = 0;
    int Npad = 0;
    int arows = 0;
    // the same rows as two 16-bit parts (split16 of kind a16_kind; FP16 ones of
    // s mu with s = status->sh_scale) over dpad16 (d padded to 64), for the search
    // of 16-bit operands; a16_err[i] bounds ||mu_i - (p1 + p2) / s||; or null
    uint16_t* a16 = nullptr;
    int64_t dpad16 = 0;
    int a16_kind = 0;
    float* a16_err = nullptr;
    const DevStatus* status = nullptr;
};

cudaError_t launch_sums_from_means(const float* mu, const int32_t* counts, int c, int64_t d, double* sums,
                                   cudaStream_t st);

// One Lloyd update in one launch: centroids from the FP64 sums (previous values
// to mu_old), their norms and drift (the statistics of launch_mu_stats, summed
// in another fixed order), and the TF32 split when sp.hi is set.  part holds
// c x centroids_stats_splits(c, d) float2, done c counters that start at zero
// (the kernel leaves them at zero).
int centroids_stats_splits(int c, int64_t d);
cudaError_t launch_centroids_stats(const double* sums, const int32_t* counts, int c, int64_t d, float* mu,
                                   float* mu_old, double* mu_norm2, float* mu_normf, double* drift,
                                   const MuSplitOut& sp, float4* part, int32_t* done, cudaStream_t st);

cudaError_t launch_flag_bounds(int mode, const float* own_part, const float* dl_part, int nchunks,
                               int64_t n, int c, const int32_t* labels, const int32_t* counts,
                               const double* sep2, double safety, const double* drift, float* ub,
                               float* lb, int32_t* flag_list, DevStatus* status, cudaStream_t st,
                               int32_t* labels_copy = nullptr, const float* ylo_part = nullptr,
                               float* ycol = nullptr, int64_t d = 0);

// FP16 copy fp16(s X) of FP32 columns (16-byte aligned, d % 4 == 0) into Y16
// (column stride ld16), each column's ||x - y~|| and ||y~||^2 into ycol[j] and
// ycol[n + j] (y~ = copy / s), and s into the status (launch_iteration's copy of L,
// for X): the operand of the all-column search over X.
cudaError_t launch_copy16_cols(const float* X, int64_t ldx, int64_t d, int64_t n, float s, void* Y16,
                              int64_t ld16, float* ycol, DevStatus* status, cudaStream_t st);

// The end of a device-run Lloyd pass (its counters and the loop's condition),
// done by the first kernel of the pass's update when on.
struct PassEnd {
    cudaGraphConditionalHandle cond = 0;
    int max_passes = 0;
    int on = 0;
};
cudaError_t launch_moved(const int32_t* now, const int32_t* before, int64_t n, int c, int4* moved,
                         int2* contrib, int32_t* boff, int32_t* counts, DevStatus* status,
                         cudaStream_t st, const PassEnd* pe = nullptr);

cudaError_t launch_mu_norms(const float* mu, int c, int64_t d, double* mu_norm2, float* mu_normf,
                            cudaStream_t st);

cudaError_t launch_separation(const float* mu, const int32_t* counts, int c, int64_t d,
                              float* pair_ss, double* sep2, cudaStream_t st);

cudaError_t launch_iteration(int dtype, int sdtype, const void* X, int64_t ldx, void* L, void* S,
                             void* Th, int64_t lds, const float* mu, const int32_t* perm,
                             const TileDesc* tiles, int max_tiles, DevStatus* status,
                             int64_t d, int64_t n, IterScalars sc, float* Dpart, float* own_part,
                             float* dl_part, double* norm_part, bool vec, cudaStream_t st,
                             void* Lsh = nullptr, int64_t ldsh = 0, float* ylo_part = nullptr);

// part: 64 x 3 doubles of scratch
cudaError_t launch_reduce_norms(const double* norm_part, int max_tiles, int nchunks,
                                DevStatus* status, double* part, cudaStream_t st);

cudaError_t launch_assign(int dtype, const void* Y, int64_t ldy, int64_t d, int64_t n,
                          const int32_t* list, const float* mu, const float* mu_normf,
                          const int32_t* counts, int c, int32_t* labels, DevStatus* status,
                          cudaStream_t st, float* ub = nullptr, float* lb = nullptr);

cudaError_t launch_count_changed(const int32_t* labels, const int32_t* prev, int64_t n,
                                 DevStatus* status, cudaStream_t st);

cudaError_t launch_sum_doubles(const double* part, int64_t count, double* out, cudaStream_t st);

// Closed-form ramp: statistics of X - mu_p, and the state after it.
cudaError_t launch_ramp_stats(int dtype, const void* X, int64_t ldx, int64_t d, int64_t n,
                              const int32_t* labels, const float* mu, const double* sep2,
                              double safety, unsigned int* max_abs_bits,
                              unsigned long long* max_ratio_bits, double* r2_part, cudaStream_t st);
cudaError_t launch_ramp_state(int dtype, const void* X, int64_t ldx, int64_t d, int64_t n,
                              const int32_t* labels, const float* mu, float alpha, float beta,
                              void* L, void* Th, int64_t lds, cudaStream_t st, int sdtype = 0);
// dst (FP32 or BF16 per dst_sdtype, leading dimension ldd) = src (respca_dtype src_dtype)
// The iteration with the l2,1 norm on S: two passes (L and ||B_j||; then S,
// Theta, norms and next D sums).  bn_part: nchunks x n.
cudaError_t launch_iteration_l21(int dtype, const void* X, int64_t ldx, float* L, float* S, float* Th,
                                 int64_t lds, const float* mu, const int32_t* perm,
                                 const TileDesc* tiles, int max_tiles, const DevStatus* status,
                                 int64_t d, int64_t n, IterScalars sc, float* Dpart, float* own_part,
                                 float* dl_part, float* bn_part, double* norm_part, bool vec,
                                 cudaStream_t st);
// Device-run Lloyd loop: start its counters at `passes0` passes.  At the end of
// each pass's search, the update's first kernel (launch_moved with a PassEnd)
// adds the pass's counters and sets the loop's condition (labels changed, fewer
// than max_passes passes, no wait gave up).
cudaError_t launch_lloyd_init(DevStatus* status, int passes0, cudaStream_t st);
cudaError_t launch_column_norms(const float* S, int64_t lds, int64_t d, int64_t n, float* out,
                                cudaStream_t st);
cudaError_t launch_convert(int src_dtype, const void* src, int64_t lds, int dst_sdtype, void* dst,
                           int64_t ldd, int64_t d, int64_t n, cudaStream_t st);

cudaError_t launch_seed_dist(int dtype, const void* X, int64_t ldx, int64_t d, int64_t n,
                             const int32_t* centers, int k, double* D2, cudaStream_t st);

cudaError_t launch_seed_pick(const double* D2, int64_t n, const double* u, int k,
                             int32_t* centers, cudaStream_t st);

cudaError_t launch_gather_centers(int dtype, const void* X, int64_t ldx, int64_t d,
                                  const int32_t* centers, int c, float* mu, int32_t* counts,
                                  cudaStream_t st);

// Tensor-core nearest-centroid search (k_search_tc.cu), used for c <= 256.
constexpr int kTcMaxClusters = 256;

// A column whose best two scores lie within their rounding bounds, queued for
// the FP64 re-decision, with the candidate centroids as a bit mask.
struct RcRec {
    int32_t col;
    uint32_t mask[kTcMaxClusters / 32];
    int32_t done;     // candidate distances of this column computed so far (re-decision)
    int32_t pad[2];
};
// Near-tie queue: the records, and the (record, candidate) pairs of the first
// cap records as record * c + candidate, appended in any order (the
// re-decision spreads exactly these pairs over the CTAs).
struct RcQueue {
    RcRec* rec;
    int32_t* pairs;
    int64_t cap;
};
int tc_npad(int c);
// Raises a kernel's dynamic shared memory cap to the device's opt-in limit,
// once per (kernel, device).  The cap then no longer depends on the launch,
// so launches of one kernel from several host threads, each with its own
// size, cannot see the cap lowered by another thread between setting it and
// launching.
cudaError_t allow_max_dynamic_smem(const void* func);
// With sp16 (its a16 fields; hi, lo, a unused) also the 16-bit split and its
// per-centroid error; part / done: mu_split16_splits(d) floats and one counter
// per row (zero, reset by the kernel).
cudaError_t launch_mu_split(const float* mu, int c, int64_t d, int Npad, int64_t dpad, float* mu_hi,
                            float* mu_lo, cudaStream_t st, float* mu_a = nullptr,
                            const MuSplitOut* sp16 = nullptr, float* part = nullptr, int32_t* done = nullptr);
int mu_split16_splits(int64_t d);
// The 16-bit operand of the all-column tensor-core search (c <= 128): y16 holds
// BF16 or FP16 columns (column j at y16 + j * ld16, ld16 a multiple of 8); when
// ycol is null they are the data themselves, otherwise the FP16 copy fp16(s Y)
// of FP32 data.  a16 / a16_err: the centroids' split (MuSplitOut) of the same type.
struct Search16 {
    const void* y16 = nullptr;
    int64_t ld16 = 0;
    bool fp16 = false;             // FP16 (the copy of L, or FP16 data) rather than BF16
    const float* ycol = nullptr;   // copy of FP32 data: ||Y_j - y16_j / s|| (s = status->sh_scale)
    const uint16_t* a16 = nullptr;
    const float* a16_err = nullptr;
    int64_t dpad16 = 0;
};
// Workspace sizes of the tensor-core search for an n-column, d-row operand.
struct TcPlan {
    int Npad;          // centroids padded to a multiple of 16
    int64_t dpad;      // d padded to a multiple of 32
    size_t gpart;      // floats of partial products
    size_t ynorm;      // floats of partial squared column norms
    int64_t tiles;     // 128-column tiles
    int64_t rc_cap;    // queued near ties whose candidate distances run spread over all SMs
    size_t mu_a;       // floats of the swapped dense kernel's centroid operand (256 x dpad)
    int64_t dpad16;    // d padded to a multiple of 64 (16-bit operands)
    size_t mu_a16;     // BF16 elements of its 16-bit form (256 x dpad16)
};
TcPlan tc_plan(int64_t n, int64_t d, int c);
cudaError_t launch_search_tc(int dtype, const void* Y, int64_t ldy, int64_t d, int64_t n,
                             const int32_t* list, DevStatus* status, const float* mu,
                             const float* mu_hi, const float* mu_lo, int64_t dpad,
                             const float* mu_normf, const int32_t* counts, int c, int32_t* labels,
                             float* ub, float* lb, float* Gpart, float* ynorm_part,
                             int32_t* tile_count, RcRec* rc_list, int32_t* rc_pairs, double* rc_dist, int64_t rc_cap,
                             bool vec, cudaStream_t st, cudaEvent_t ev_dense0 = nullptr,
                             cudaEvent_t ev_dense1 = nullptr, bool* dense_launched = nullptr,
                             const float* mu_a = nullptr, const Search16* s16 = nullptr);
// Queued columns up to which a pass searches its list rather than every column.
int64_t search_list_max(int64_t n, int c, bool op16);

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Element loads of X for the three supported element types.
template <typename T>
struct XLoad;

template <>
struct XLoad<float> {
    static __device__ __forceinline__ float one(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ float4 four(const float* p) {
        return __ldg(reinterpret_cast<const float4*>(p));
    }
};

template <>
struct XLoad<__nv_bfloat16> {
    static __device__ __forceinline__ float one(const __nv_bfloat16* p) {
        return __bfloat162float(p[0]);
    }
    static __device__ __forceinline__ float4 four(const __nv_bfloat16* p) {
        const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
        const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
        const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
        return make_float4(lo.x, lo.y, hi.x, hi.y);
    }
};

template <>
struct XLoad<__half> {
    static __device__ __forceinline__ float one(const __half* p) { return __half2float(p[0]); }
    static __device__ __forceinline__ float4 four(const __half* p) {
        const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
        const float2 lo = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
        const float2 hi = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
        return make_float4(lo.x, lo.y, hi.x, hi.y);
    }
};

// Loads and stores of the iteration state (L, S, Theta) in its storage type:
// FP32, or BF16 in the bf16 phase of the precision=1 schedule.  Streaming
// cache hints (each element is read and written once per pass).  round()
// gives the value that storing and reloading returns.
template <typename TS>
struct StateIO;

template <>
struct StateIO<float> {
    static __device__ __forceinline__ float4 load4(const float* p) {
        return __ldcs(reinterpret_cast<const float4*>(p));
    }
    static __device__ __forceinline__ void store4(float* p, float4 v) {
        __stcs(reinterpret_cast<float4*>(p), v);
    }
    static __device__ __forceinline__ float load1(const float* p) { return *p; }
    static __device__ __forceinline__ void store1(float* p, float v) { *p = v; }
    static __device__ __forceinline__ float round(float v) { return v; }
};

template <>
struct StateIO<__nv_bfloat16> {
    static __device__ __forceinline__ float4 load4(const __nv_bfloat16* p) {
        const uint2 u = __ldcs(reinterpret_cast<const uint2*>(p));
        const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
        const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
        return make_float4(lo.x, lo.y, hi.x, hi.y);
    }
    static __device__ __forceinline__ void store4(__nv_bfloat16* p, float4 v) {
        const __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y);
        const __nv_bfloat162 hi = __floats2bfloat162_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<const uint32_t*>(&lo);
        u.y = *reinterpret_cast<const uint32_t*>(&hi);
        __stcs(reinterpret_cast<uint2*>(p), u);
    }
    static __device__ __forceinline__ float load1(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void store1(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ float round(float v) {
        return __bfloat162float(__float2bfloat16_rn(v));
    }
};

// Dispatch a state storage type (0 f32, 1 bf16).
#define RESPCA_DISPATCH_S(sdtype, TS, ...)  \
    do {                                    \
        if ((sdtype) == 1) {                \
            using TS = __nv_bfloat16;       \
            __VA_ARGS__;                    \
        } else {                            \
            using TS = float;               \
            __VA_ARGS__;                    \
        }                                   \
    } while (0)

__device__ __forceinline__ float f4get(const float4& v, int q) {
    return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
}

__device__ __forceinline__ void f4set(float4& v, int q, float x) {
    if (q == 0) v.x = x;
    else if (q == 1) v.y = x;
    else if (q == 2) v.z = x;
    else v.w = x;
}

// The TF32 part of an FP32 value as the tensor cores read it (mantissa truncated
// to 10 bits).
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// FP16 copy of one value, the square of its error e = l - y~ and of y~ = h / s,
// h = fp16(clamp(s l)) (e exact in FP32 unless clamped or below the normal range).
__device__ __forceinline__ __half copy16(float l, float s, float inv_s, float& e2, float& q2) {
    const __half h = __float2half_rn(fminf(fmaxf(l * s, -65504.f), 65504.f));
    const float y = __half2float(h) * inv_s;
    const float e = l - y;
    e2 = fmaf(e, e, e2);
    q2 = fmaf(y, y, q2);
    return h;
}

// Two-part 16-bit split of a centroid element v for the search of 16-bit
// operands.  kind 1: p1 = bf16(v), p2 = bf16(v - p1); kind 2: the same in FP16
// of w = s v (s a power of two), each part clamped to the FP16 range.  Adds
// the square of the error w - p1 - p2 (units of w; exact in FP32 unless a
// part was clamped or fell below the normal range) to e2.
__device__ __forceinline__ void split16(float v, int kind, float s, uint16_t& p1, uint16_t& p2, float& e2) {
    if (kind == 1) {
        const __nv_bfloat16 h1 = __float2bfloat16_rn(v);
        const float r = v - __bfloat162float(h1);
        const __nv_bfloat16 h2 = __float2bfloat16_rn(r);
        const float e = r - __bfloat162float(h2);
        e2 = fmaf(e, e, e2);
        p1 = __bfloat16_as_ushort(h1);
        p2 = __bfloat16_as_ushort(h2);
    } else {
        const float w = v * s;
        const __half h1 = __float2half_rn(fminf(fmaxf(w, -65504.f), 65504.f));
        const float r = w - __half2float(h1);
        const __half h2 = __float2half_rn(fminf(fmaxf(r, -65504.f), 65504.f));
        const float e = r - __half2float(h2);
        e2 = fmaf(e, e, e2);
        p1 = __half_as_ushort(h1);
        p2 = __half_as_ushort(h2);
    }
}

// Upper bound on a split's error norm from the summed squares e2 (units of s v):
// FP32 sums inflated, plus sqrt(d) 2^-74 for squares that underflowed, over s.
__device__ __forceinline__ float split16_err(float e2, int64_t d, float s) {
    return (sqrtf(e2) * (1.f + 1e-4f) + sqrtf((float)d) * 5.29395592e-23f) / s;
}

// ---------------------------------------------------------------- learned warm start
// Scalars of one unrolled layer (rho_k, tau_k learned; labels fixed).
struct NetScalars {
    float a;             // rho_k / (2 lambda + rho_k)
    float b;             // 2 lambda / (2 lambda + rho_k)
    float rho;           // rho_k
    float inv_rho;       // 1 / rho_k
    float tau;           // soft threshold of the layer's S step
    float inv_rho_next;  // 1 / rho_{k+1}: weight of Theta' in the next layer's D sums
};

int net_row_chunks(int64_t d);
cudaError_t launch_net_layer(const float* X, int64_t ldx, const float* S, const float* Th, float* L,
                             float* Sn, float* Thn, int64_t lds, const float* mu, const int32_t* perm,
                             const TileDesc* tiles, int max_tiles, const DevStatus* status, int64_t d,
                             const NetScalars& sc, float* Dpart, cudaStream_t st);
cudaError_t launch_net_infer(int xdt, int sin, int sout, const void* X, int64_t ldx, const void* S,
                             const void* Th, int64_t ldin, float* L, void* Sn, void* Thn, int64_t ldout,
                             const float* mu, const int32_t* perm, const TileDesc* tiles, int max_tiles,
                             const DevStatus* status, int64_t d, const NetScalars& sc, float* Dpart,
                             cudaStream_t st);
cudaError_t launch_net_back(int pass, const float* X, int64_t ldx, const float* S, const float* Th,
                            int64_t lds, const float* mu, const int32_t* perm, const TileDesc* tiles,
                            int max_tiles, const DevStatus* status, int64_t d, const NetScalars& sc,
                            const float* gLext, float* gS, float* gT, const float* gmean, float* Gpart,
                            double* scal_part, double* scal_out, cudaStream_t st);
cudaError_t launch_net_loss(const float* L, const float* S, int64_t lds, const float* Lt, const float* St,
                            int64_t ldt, int64_t d, int64_t n, float scale, float* gL, float* gS, float* gT,
                            double* part, int parts, double* out, cudaStream_t st);
cudaError_t launch_mlp_forward(const float* P, int nz, int H, int nout, const float* z, float* out,
                               float* hidden, cudaStream_t st);
cudaError_t launch_mlp_backward(const float* P, int nz, int H, int nout, const float* z, const float* hidden,
                                const float* gout, float* G, int accumulate, cudaStream_t st);
cudaError_t launch_adam(float* P, const float* G, float* M, float* V, int64_t count, float lr, float b1,
                        float b2, float eps, float c1, float c2, cudaStream_t st);

// ---------------------------------------------------------------- spectral p step
// G = Y^T Y (n x n, exactly symmetric) on the tensor cores; Y needs 16-byte
// alignment and ldy % 4 == 0 (gram_tc_ok)
bool gram_tc_ok(const float* Y, int64_t ldy);
cudaError_t launch_gram_tc(const float* Y, int64_t ldy, int64_t d, int64_t n, float* G, DevStatus* status,
                           cudaStream_t st);
cudaError_t launch_spec_affinity(const float* Y, int64_t ldy, int64_t d, int64_t n, double scale, float* G,
                                 float* sqn, double* part, int parts, double* colsum, double* sig, double* deg,
                                 float* rinv, DevStatus* status, cudaEvent_t g0, cudaEvent_t g1, cudaStream_t st);
cudaError_t launch_spec_start(float* Y, int64_t n, int b, uint64_t seed, cudaStream_t st);
cudaError_t launch_spec_axpby(float* out, const float* T, const float* Y, const float* Yp, int64_t count,
                              float alpha, float beta, float gamma, cudaStream_t st);
// W = R A R Y (R = diag(r)); P holds spec_symm_chunks(n, b) x n x b partial products
int64_t spec_symm_chunks(int64_t n, int b);
cudaError_t launch_spec_symm(const float* A, const float* r, int64_t n, const float* Y, int b, float* W, float* P,
                             cudaStream_t st);
size_t spec_colsum_doubles(int64_t d);
cudaError_t launch_spec_gram_small(const float* A, const float* B, int64_t n, int b1, int b2, double* out,
                                   cudaStream_t st);
cudaError_t launch_spec_cholqr2(float* Y, float* T, int64_t n, int b, double* G, float* Q, cudaStream_t st);
size_t spec_jacobi_smem(int b);
cudaError_t launch_spec_jacobi(const double* H, int b, float* Q, double* evals, cudaStream_t st);
cudaError_t launch_spec_rotate(const float* Y, const float* Q, float* out, int64_t n, int b, cudaStream_t st);
cudaError_t launch_spec_residual(const float* W, const float* Y, const double* evals, int64_t n, int c,
                                 double* res, cudaStream_t st);
cudaError_t launch_spec_embed(const float* Y, int64_t n, int c, float* E, cudaStream_t st);

// ---------------------------------------------------------------- batched persistent solve
struct BatchedState;
void batched_state_free(BatchedState* s);
respca_status batched_persistent(BatchedState** sp, int device, cudaStream_t st, uint64_t seed, double rho0,
                                 double kappa, int km_max, int32_t batch, const respca_problem* probs,
                                 respca_stats* stats, respca_batch_options* opt, std::string* err);

// Dispatch a runtime dtype (0 f32, 1 bf16, 2 f16) to a template lambda.
#define RESPCA_DISPATCH_X(dtype, TX, ...)                       \
    do {                                                        \
        if ((dtype) == 1) {                                     \
            using TX = __nv_bfloat16;                           \
            __VA_ARGS__;                                        \
        } else if ((dtype) == 2) {                              \
            using TX = __half;                                  \
            __VA_ARGS__;                                        \
        } else {                                                \
            using TX = float;                                   \
            __VA_ARGS__;                                        \
        }                                                       \
    } while (0)

}  // namespace respca
