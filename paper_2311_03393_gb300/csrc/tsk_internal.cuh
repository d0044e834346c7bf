// Internal declarations shared by the translation units of libtsketch.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/tsketch.h"

#define TSK_FULL_MASK 0xffffffffu

// Error-word bits set by kernels (read by tsk_sync).
enum : int { TSK_DEVERR_NONFINITE = 1, TSK_DEVERR_TIMEOUT = 2 };

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------

// Cached device copy of the per-stream bookkeeping mp_selfjoin derives from a
// stream layout (offsets, chunk and tile prefixes).  Rebuilt when the layout,
// m, excl, mask or tile shape changes.
struct tsk_mp_plan {
  std::vector<int32_t> lens;
  std::vector<uint8_t> mask;
  int32_t m = 0, excl = 0, H = 0, D = 0, prec = -1;
  void* dev = nullptr;       // one device blob holding the arrays below
  size_t dev_bytes = 0;
  // device pointers into dev
  int64_t* xoff = nullptr;         // [n+1] sample offsets
  int32_t* len = nullptr;          // [n]
  uint8_t* smask = nullptr;        // [n]
  int64_t* woff = nullptr;         // [n+1] window-array offsets
  int64_t* chunk_prefix = nullptr; // [n+1] window-stat chunks
  int64_t* tile_prefix = nullptr;  // [n+1] float64 path: diagonals before each stream
  int4* tiles = nullptr;           // float32 path work list {stream, d0, r0, r1 | masked << 31}
  // host summaries
  int64_t total_windows = 0;  // sum of (l + pad) over streams
  int64_t total_chunks = 0;
  int64_t total_tiles = 0;
  int64_t total_samples = 0;
};

struct tsk_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int* d_err = nullptr;                 // device error word
  std::string last_error;
  int64_t launches = 0;
  int mp_H = 0;                         // rows per matrix-profile work unit (0 = automatic)
  bool prof = false;                    // record events around the timed kernels
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events[TSK_PROF_COUNT];
};

// Event pair around a timed launch (no-op unless profiling is on and the
// stream is not being captured).
struct tsk_prof_scope {
  tsk_ctx* ctx;
  int kernel;
  cudaEvent_t e1 = nullptr, e2 = nullptr;
  tsk_prof_scope(tsk_ctx* c, int k);
  ~tsk_prof_scope();
};

// ---------------------------------------------------------------------------
// Host helpers (tsk_api.cu)
// ---------------------------------------------------------------------------
tsk_status tsk_fail(tsk_ctx* ctx, tsk_status st, const char* fmt, ...);
tsk_status tsk_cuda_fail(tsk_ctx* ctx, cudaError_t e, const char* where);
// Grow the workspace to `bytes`; fails (without allocating) during stream capture.
tsk_status tsk_ws_require(tsk_ctx* ctx, size_t bytes);

// Bump allocator over the context workspace for one call.
struct tsk_carver {
  char* base;
  size_t off = 0;
  explicit tsk_carver(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
  static size_t bytes_for(size_t count, size_t elt) { return ((count * elt) + 255) & ~size_t(255); }
};

#define TSK_CUDA_TRY(ctx, expr)                                   \
  do {                                                            \
    cudaError_t _e = (expr);                                      \
    if (_e != cudaSuccess) return tsk_cuda_fail((ctx), _e, #expr); \
  } while (0)

#define TSK_LAUNCH_CHECK(ctx, name)                                     \
  do {                                                                  \
    (ctx)->launches++;                                                  \
    cudaError_t _e = cudaGetLastError();                                \
    if (_e != cudaSuccess) return tsk_cuda_fail((ctx), _e, name);       \
  } while (0)

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ double tsk_ld(const T* p, int64_t i) { return static_cast<double>(p[i]); }

// float64 -> bfloat16 bit pattern, round to nearest, ties to even, taken
// directly from the float64 value (no intermediate float32 rounding).
// bfloat16: 1 sign, 8 exponent (bias 127), 7 stored fraction bits.
__device__ __forceinline__ uint16_t tsk_f64_to_bf16_bits(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const uint16_t sign = static_cast<uint16_t>((b >> 48) & 0x8000u);
  const unsigned long long a = b & 0x7fffffffffffffffull;
  if (a > 0x7ff0000000000000ull) return static_cast<uint16_t>(sign | 0x7fc0u);  // NaN
  const int e = static_cast<int>(a >> 52) - 1023;
  if (e >= -126) {
    const unsigned long long frac = a & 0x000fffffffffffffull;
    long long field = (static_cast<long long>(e + 127) << 7) | static_cast<long long>(frac >> 45);
    const unsigned long long rem = frac & ((1ull << 45) - 1ull);
    const unsigned long long half = 1ull << 44;
    if (rem > half || (rem == half && (field & 1))) field += 1;  // carries into the exponent
    if (field >= 0x7f80) field = 0x7f80;                          // overflow to infinity
    return static_cast<uint16_t>(sign | static_cast<uint16_t>(field));
  }
  // below the smallest normal: multiples of 2^-133
  const double q = fabs(x) * 0x1p133;                // exact power-of-two scaling
  const long long r = __double2ll_rn(q);              // nearest, ties to even; r <= 128
  return static_cast<uint16_t>(sign | static_cast<uint16_t>(r));
}

__device__ __forceinline__ float tsk_bf16_bits_to_f32(uint16_t h) {
  return __uint_as_float(static_cast<uint32_t>(h) << 16);
}

// Order-preserving map float -> uint32 (larger float -> larger integer).
__device__ __forceinline__ uint32_t tsk_ordered_u32(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ unsigned long long tsk_ordered_u64(double f) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(f));
  return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double tsk_from_ordered_u64(unsigned long long u) {
  const unsigned long long b = (u & 0x8000000000000000ull) ? (u & 0x7fffffffffffffffull) : ~u;
  return __longlong_as_double(static_cast<long long>(b));
}
// Packed (key, index): atomicMax keeps the largest key, then the lowest index.
__device__ __forceinline__ unsigned long long tsk_pack(float key, int32_t idx) {
  return (static_cast<unsigned long long>(tsk_ordered_u32(key)) << 32) |
         static_cast<unsigned long long>(0xffffffffu - static_cast<uint32_t>(idx));
}
__device__ __forceinline__ int32_t tsk_unpack_idx(unsigned long long p) {
  return static_cast<int32_t>(0xffffffffu - static_cast<uint32_t>(p & 0xffffffffull));
}

// Upper bound search: largest q in [0, n) with a[q] <= v (a non-decreasing, a[0] <= v).
template <typename T>
__device__ __forceinline__ int tsk_find_segment(const T* a, int n, T v) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a[mid] <= v) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Launchers implemented in the other translation units
// ---------------------------------------------------------------------------

// Column statistics (mean, population std) of n_streams streams.
tsk_status tsk_launch_colstats(tsk_ctx* ctx, const void* T, int t_dtype, const int64_t* d_off, const int32_t* d_len,
                               int64_t n_streams, double* stats);
// Sketch S = R^T T_bar over a batch (d_series_off: sample offset of series s / d).
tsk_status tsk_launch_sketch(tsk_ctx* ctx, const void* T, int t_dtype, int32_t n_series, const int64_t* d_cum,
                             const int32_t* d_len, const int64_t* d_blk_prefix, int64_t total_blocks, int32_t d,
                             const float* R, int32_t k, int32_t precision, const double* stats, void* S,
                             int64_t total_samples, char* ws);
// Workspace of tsk_launch_sketch (bfloat16 precision: R in bf16, per-stream constants, partial sums).
size_t tsk_sketch_ws_bytes(int32_t n_series, int32_t d, int32_t k, int64_t total_blocks, int64_t total_samples,
                           int sm_count);
tsk_status tsk_launch_update_dims(tsk_ctx* ctx, void* S, const void* T_dims, int t_dtype, int32_t n_series,
                                  const int64_t* d_cum, const int32_t* d_len, int64_t total_samples, int32_t nd,
                                  const float* d_Rrows, const int8_t* d_op, int32_t k, int32_t precision,
                                  const double* stats);
// Point updates of T and S (distinct points; see tsk_sketch.cu).
tsk_status tsk_launch_point_update(tsk_ctx* ctx, void* S, void* T, int t_dtype, const int4* d_pts, const double* d_delta,
                                   int32_t npts, const int64_t* d_cum, const int32_t* d_len, int32_t d, const float* R,
                                   int32_t k, int32_t precision, const double* stats);
// Matrix profile pipeline (window stats, diagonal kernel, refinement).
tsk_status tsk_run_mp(tsk_ctx* ctx, const void* X, int x_dtype, int32_t n_streams, const tsk_mp_plan& plan,
                      int32_t m, int32_t excl, int32_t precision, void* P, int32_t* I, char* ws);
// AB join: n_pairs test streams (A) against their training partners (B); the
// plan covers the 2 n_pairs streams, test streams first.
tsk_status tsk_run_mp_ab(tsk_ctx* ctx, const void* A, const void* B, int x_dtype, int32_t n_pairs,
                         const tsk_mp_plan& plan, int32_t m, int32_t precision, void* P_a, int32_t* I_a, void* P_b,
                         int32_t* I_b, char* ws);
size_t tsk_mp_ws_bytes(const tsk_mp_plan& plan, int32_t n_streams);
// One bounded device-side wait that runs out (failure-path self-test).
tsk_status tsk_launch_selftest_wait(tsk_ctx* ctx);
// Incremental self-join profile after point updates: `runs` lists the affected
// windows {stream, first, end, 0} (sorted, disjoint); P, I hold the old profile
// on entry, the new one on return.  The plan's mask marks the touched streams.
tsk_status tsk_run_mp_update(tsk_ctx* ctx, const float* X, int32_t n_streams, const int32_t* lens,
                             const tsk_mp_plan& plan, int32_t m, int32_t excl, float* P, int32_t* I,
                             const std::vector<int4>& runs, char* ws);
size_t tsk_mp_update_ws_bytes(const tsk_mp_plan& plan, int32_t n_streams, size_t n_runs, size_t n_tiles_max);
int tsk_mp_band_width();
// Aggregation and ranked discords.
tsk_status tsk_launch_topk(tsk_ctx* ctx, const void* P, int p_dtype, const int32_t* I, int32_t n_series,
                           const int64_t* d_cum, const int32_t* d_len, int32_t group, int32_t m, int32_t K,
                           int32_t topk_excl, int32_t* idx, int32_t* grp, void* score, int32_t* nn, char* ws,
                           int64_t max_l);
// Dimension detection (Alg. 3) and the gather of the chosen streams.
int tsk_dims_window_chunk();
size_t tsk_dims_ws_bytes(int32_t n_series, int32_t K, int32_t d, int32_t m);
tsk_status tsk_launch_dims(tsk_ctx* ctx, const void* T, const void* T_train, int t_dtype, int32_t n_series,
                           const int64_t* d_cum, const int32_t* d_len, const int64_t* d_cum_t, const int32_t* d_len_t,
                           const int64_t* d_item_prefix, int64_t total_items, int64_t total_samples,
                           int64_t total_samples_t, int32_t d, const float* R, int32_t k, int32_t m, int32_t excl,
                           int32_t K, const int32_t* idx, const int32_t* grp, int32_t* dim, double* dim_score,
                           int32_t* dim_nn, double* dim_scores, void* T_sel, void* T_sel_train, char* ws);
// Adjoint.
tsk_status tsk_launch_backward(tsk_ctx* ctx, const float* dscore, const int32_t* idx, const int32_t* grp,
                               const int32_t* nn, int32_t K, const void* T, int t_dtype, const double* stats,
                               const float* R, const float* S, int32_t n_series, const int64_t* d_cum,
                               const int32_t* d_len, int32_t max_len, int32_t d, int32_t k,
                               int32_t m, float* dT, float* dR, char* ws);
