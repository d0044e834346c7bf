// Self-join matrix profile of many streams (Def. 6, Def. 3).
//
// Pipeline per call:
//   1. k_window_stats   per window: mean and centred sum of squares (float64
//                       chunk-local prefix sums), 1/||x - mean|| (float32), and
//                       the two terms of the diagonal update
//                         df_i = (x[i+m] - x[i]) / 2
//                         dg_i = (x[i+m] - mean_{i+1}) + (x[i] - mean_i)
//                       which satisfy, for c(i,j) = sum_t (x[i+t]-mean_i)(x[j+t]-mean_j),
//                         c(i+1, j+1) = c(i, j) + df_i dg_j + df_j dg_i.
//   2. k_next_const     next constant window at or after each index (only for
//                       streams that have constant windows).
//   3. k_mp_diag        persistent, diagonal-banded kernel.  A warp owns a band
//                       of 512 diagonals (two half bands of 256 walked in
//                       lockstep as float2 pairs) and a run of rows; lane t walks
//                       8 diagonals of each half down the rows with the float32
//                       recurrence from an anchor at the first row (float32 from
//                       centred values for float32 series, float64 otherwise).
//                       Each cell's key rho - 1 (rho = c * inv_i * inv_j) updates
//                       the row maximum (reduced over lanes through shared memory)
//                       and the column maximum (carried from lane to lane as the
//                       band's columns slide).  Keys carry the diagonal's offset
//                       within its half band in their 8 low mantissa bits, so a
//                       max also knows its argmax.  Results merge into a packed
//                       (key, index) 64-bit word per window with atomicMax.
//   4. k_mp_refine      for every window: its chosen neighbour's distance,
//                       dist = sqrt(2 m (1 - rho)) with rho re-evaluated exactly
//                       (compensated sums), plus the constant-window rules.
// The float64 variant (k_mp_diag_f64) is exact: one thread per diagonal, a
// first pass takes the float64 maximum per window, a second pass the lowest
// index attaining it.
//
// AB join (Def. 6 with T_test != T_train): the streams are the n test streams
// followed by their n training partners (samples of the two halves in two
// buffers).  The same kernels run with a row side and a column side: rows of
// test stream q against columns of training stream q on diagonals delta >= 0,
// then rows of the training stream against columns of the test stream on
// delta >= 1, with no exclusion zone; row maxima feed the row side's profile
// and column maxima the column side's.
#include "tsk_internal.cuh"
#include "tsk_rho.cuh"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <mutex>
#include <type_traits>

namespace {

constexpr int kVh = 8;                   // diagonals per lane in each half band
constexpr int kHalf = 32 * kVh;          // 256 diagonals per half band
constexpr int kBand = 2 * kHalf;         // 512 diagonals per warp band
constexpr int kChunk = 32;               // rows between row flushes / ring refills
constexpr int kRingEntries = 320;        // column ring entries of (half a, half b) pairs
constexpr int kRingPhys = kRingEntries + kRingEntries / 8;  // with one pad slot per 8 entries
constexpr int kRingInit = 288;           // entries filled before the first row
// During the chunk of steps [S0, S0 + 32) the lanes read ring entries [S0 + 8,
// S0 + 288) while the copies for the next chunk write entries [S0 + 296,
// S0 + 328); with 320 entries those land in slots of entries already consumed
// (S0 + 7 and below), and the next chunk's reads (up to S0 + 319) are covered.
static_assert(kVh + kRingInit >= kHalf + kChunk && kRingEntries >= kRingInit + kChunk && kRingEntries % kVh == 0,
              "column ring too small for the refill distance");
constexpr int kWarps = 4;                // warps per CTA
constexpr int kMaxClaim = 16;            // work units a warp claims at once (at most)
constexpr int kMaxWalk = 8192;           // rows walked from one anchor (at most)
constexpr int kWinChunk = 1024;          // windows per window-stats CTA
constexpr int kWinThreads = 256;
constexpr int kPad = 2048;               // zeroed slack after each stream's window arrays
constexpr float kEmpty = -3.0f;          // below every key (keys are rho - 1 >= -2)
constexpr float kKeyFloor = -2.5f;       // keys above this are real cells
constexpr double kConstRelVar = 1e-12;

struct WinArrays {
  double* mu;
  double* ss;
  float* inv;
  float* df;
  float* dg;
  unsigned long long* best;
  int32_t* nxt;
  int32_t* constcnt;
  double* inv64;   // float64 mode only
  int32_t* bidx;   // float64 mode only
};

// Samples of stream q: streams before `split` live in X, the rest in X2
// (offsets continue across the two buffers).
template <typename TX>
__device__ __forceinline__ const TX* stream_base(const TX* X, const TX* X2, const int64_t* xoff, int split, int q) {
  return q < split ? X + xoff[q] : X2 + (xoff[q] - xoff[split]);
}

// ---------------------------------------------------------------------------
// 1. window statistics
// ---------------------------------------------------------------------------
__device__ __forceinline__ void block_excl_scan2(double& a, double& b, double* sh) {
  // exclusive prefix over the block of (a, b); sh holds 2 * (warps) doubles
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double ia = a, ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double ta = __shfl_up_sync(TSK_FULL_MASK, ia, o);
    const double tb = __shfl_up_sync(TSK_FULL_MASK, ib, o);
    if (lane >= o) { ia += ta; ib += tb; }
  }
  if (lane == 31) { sh[w] = ia; sh[32 + w] = ib; }
  __syncthreads();
  double wa = 0.0, wb = 0.0;
  for (int u = 0; u < w; ++u) { wa += sh[u]; wb += sh[32 + u]; }
  a = wa + ia - a;
  b = wb + ib - b;
  __syncthreads();
}

template <typename TX>
__global__ void __launch_bounds__(kWinThreads) k_window_stats(const TX* __restrict__ X, const TX* __restrict__ X2,
                                                              int split, const int64_t* __restrict__ xoff,
                                                              const int32_t* __restrict__ len,
                                                              const int64_t* __restrict__ woff,
                                                              const int64_t* __restrict__ chunk_prefix, int n_streams,
                                                              int m, int want64, WinArrays wa, int* __restrict__ err) {
  extern __shared__ double sm[];
  __shared__ double scan_sh[64];
  __shared__ int ccount;
  const int q = tsk_find_segment<int64_t>(chunk_prefix, n_streams, static_cast<int64_t>(blockIdx.x));
  const int n = len[q];
  const int l = n - m + 1;
  const int w0 = static_cast<int>(blockIdx.x - chunk_prefix[q]) * kWinChunk;
  const int nw = min(kWinChunk, l - w0);
  const int ns = min(n - w0, nw + m);  // samples w0 .. w0 + ns - 1
  const TX* x = stream_base(X, X2, xoff, split, q);
  const int64_t wb = woff[q];
  double* E1 = sm;             // E1[u] = sum of the first u shifted samples
  double* E2 = sm + (ns + 1);
  if (threadIdx.x == 0) ccount = 0;
  const double xref = static_cast<double>(x[w0]);
  bool bad = false;
  for (int u = threadIdx.x; u < ns; u += kWinThreads) {
    const double xv = static_cast<double>(x[w0 + u]);
    bad |= !isfinite(xv);
    const double y = xv - xref;
    E1[u + 1] = y;
    E2[u + 1] = y * y;
  }
  if (bad) atomicOr(err, TSK_DEVERR_NONFINITE);
  if (threadIdx.x == 0) { E1[0] = 0.0; E2[0] = 0.0; }
  __syncthreads();
  // segmented inclusive scan of E[1..ns]
  const int seg = (ns + kWinThreads - 1) / kWinThreads;
  const int a0 = 1 + threadIdx.x * seg;
  const int a1 = min(ns + 1, a0 + seg);
  double s1 = 0.0, s2 = 0.0;
  for (int u = a0; u < a1; ++u) { s1 += E1[u]; s2 += E2[u]; }
  block_excl_scan2(s1, s2, scan_sh);
  for (int u = a0; u < a1; ++u) {
    s1 += E1[u];
    s2 += E2[u];
    E1[u] = s1;
    E2[u] = s2;
  }
  __syncthreads();
  const double inv_m = 1.0 / m;
  int my_const = 0;
  for (int u = threadIdx.x; u < nw; u += kWinThreads) {
    const int i = w0 + u;
    const double t1 = E1[u + m] - E1[u];
    const double t2 = E2[u + m] - E2[u];
    const double my = t1 * inv_m;
    const double ss = fmax(0.0, t2 - t1 * my);
    const double mu = xref + my;
    const bool cst = ss * inv_m <= kConstRelVar * fmax(1.0, mu * mu);
    my_const += cst ? 1 : 0;
    const double r = cst ? 0.0 : rsqrt(ss);
    float df = 0.f, dg = 0.f;
    if (i < l - 1) {
      const double xa = static_cast<double>(x[i]), xb = static_cast<double>(x[i + m]);
      const double mu1 = xref + (E1[u + 1 + m] - E1[u + 1]) * inv_m;
      df = static_cast<float>((xb - xa) * 0.5);
      dg = static_cast<float>((xb - mu1) + (xa - mu));
    }
    wa.mu[wb + i] = mu;
    wa.ss[wb + i] = ss;
    wa.inv[wb + i] = cst ? 0.f : fmaxf(static_cast<float>(r), FLT_MIN);
    wa.df[wb + i] = df;
    wa.dg[wb + i] = dg;
    if (want64) wa.inv64[wb + i] = r;
  }
  // zero the slack after the last window
  if (w0 + nw == l) {
    for (int u = threadIdx.x; u < kPad; u += kWinThreads) {
      const int64_t e = wb + l + u;
      wa.mu[e] = 0.0;
      wa.ss[e] = 0.0;
      wa.inv[e] = 0.f;
      wa.df[e] = 0.f;
      wa.dg[e] = 0.f;
      if (want64) wa.inv64[e] = 0.0;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_const += __shfl_xor_sync(TSK_FULL_MASK, my_const, o);
  if ((threadIdx.x & 31) == 0 && my_const) atomicAdd(&ccount, my_const);
  __syncthreads();
  if (threadIdx.x == 0 && ccount) atomicAdd(&wa.constcnt[q], ccount);
}

// ---------------------------------------------------------------------------
// 2. next constant window (index of the first window j >= i with inv_j == 0)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kWinThreads) k_next_const(const int32_t* __restrict__ len, const uint8_t* __restrict__ smask,
                                                            const int64_t* __restrict__ woff, int m, WinArrays wa) {
  const int q = blockIdx.x;
  if (!smask[q] || wa.constcnt[q] == 0) return;
  const int l = len[q] - m + 1;
  const int64_t wb = woff[q];
  const int seg = (l + kWinThreads - 1) / kWinThreads;
  const int a0 = threadIdx.x * seg, a1 = min(l, a0 + seg);
  int first = INT_MAX;
  for (int i = a1 - 1; i >= a0; --i)
    if (wa.inv[wb + i] == 0.f) first = i;
  __shared__ int sfirst[kWinThreads];
  sfirst[threadIdx.x] = first;
  __syncthreads();
  int carry = INT_MAX;
  for (int u = threadIdx.x + 1; u < kWinThreads; ++u) carry = min(carry, sfirst[u]);
  for (int i = a1 - 1; i >= a0; --i) {
    if (wa.inv[wb + i] == 0.f) carry = i;
    wa.nxt[wb + i] = carry;
  }
}

// ---------------------------------------------------------------------------
// 3. the diagonal kernel (float32 recurrence)
//
// A warp owns a band of 512 diagonals d0 .. d0+511 and a block of rows.  Lane
// t walks two groups of 8 diagonals, d0 + 8t + v (half a) and the same + 256
// (half b); the two halves advance in lockstep, so every quantity of a cell
// comes as a float2 pair (half a, half b) and the arithmetic runs as paired
// float32 FMA/MUL.  Per row the lane's 8 + 8 cells update
//   - the row maximum (one key per half, reduced over lanes in shared memory
//     every 32 rows), and
//   - 8 + 8 column maxima held in registers; as the rows advance the band's
//     columns slide, the column leaving lane t passes to lane t-1 and the one
//     leaving lane 0 is complete for this band.
// A key is rho - 1 (one FMA: t * inv_i - 1, exact to float32 relative
// precision near rho = 1, where close matches are told apart) with its 8 low
// mantissa bits replaced by the diagonal's offset within its half (8t + v), so
// maxima carry their argmax; the tag then costs at most 2^-16 of 1 - rho.
// Column data (df, dg, 1/norm) stream through a padded shared-memory ring
// refilled 32 rows ahead; row data through a 32-row buffer of broadcast pairs.
// Every per-row shared-memory access is a fixed offset from a per-block base.
// ---------------------------------------------------------------------------
struct MpArgs {
  const void* X;
  const void* X2;              // AB join: samples of the training streams (streams >= split)
  int split;                   // AB join: number of test streams (self-join: n_streams)
  const int64_t* xoff;
  const int32_t* len;
  const int64_t* woff;
  const int64_t* tile_prefix;  // float64 path: diagonals before stream q
  const int4* tiles;           // float32 path: {stream, d0, r0, r1 | masked << 31}
  unsigned long long* counter;
  WinArrays wa;
  int64_t total_tiles;
  int n_streams, m, excl, H;
  int total_warps;
};

struct __align__(16) MpWarpSmem {
  float2 ring[3][kRingPhys];      // column pairs (half a, half b), slot ring_phys(entry)
  float4 rrow[2][3][kChunk / 2];  // row broadcast pairs (v_s, v_s, v_s+1, v_s+1), double buffered
  float2 rowbuf[32][kChunk + 1];  // (row key half a, half b): [lane][step], rows padded by one slot
  float2 colbuf[kChunk];          // keys of the columns leaving lane 0, per step
};

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ float tag_key(float rho, unsigned tag) {
  return __uint_as_float((__float_as_uint(rho) & 0xffffff00u) | tag);
}
__device__ __forceinline__ float untag_key(float key) { return __uint_as_float(__float_as_uint(key) & 0xffffff00u); }
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
// ring entry (0 <= e < kRingEntries) -> physical 8-byte slot: one pad slot after
// every 8 entries.  A lane reads the 8 entries of an aligned block (one base plus
// fixed offsets).  At a step the lanes read entries e0 + 8t, whose blocks start 9
// slots apart, so the 16 lanes of a half warp fall on 16 distinct 8-byte bank
// pairs unless their range wraps around the ring.
__device__ __forceinline__ int ring_phys(int e) { return e + (e >> 3); }

template <typename TX>
__device__ __forceinline__ double ld_guard(const TX* __restrict__ x, int idx, int n) {
  return idx < n ? static_cast<double>(x[idx]) : 0.0;
}

// Merge the 32 (or `count`) buffered rows and lane-0 column exits into the profile.
// Buffer step u belongs to row base + u and to columns base + u + d0 (+ 256).
__device__ __forceinline__ void flush_chunk(MpWarpSmem& w, int count, int base, int d0, int l,
                                            unsigned long long* __restrict__ best,
                                            unsigned long long* __restrict__ bestc, int lane) {
  __syncwarp();
  if (lane < count) {
    const int ir = base + lane;
    float ma = kEmpty, mb = kEmpty;
#pragma unroll
    for (int u = 0; u < 32; u += 2) {  // row `lane` of the chunk, from every source lane u
      const float2 q0 = w.rowbuf[u][lane], q1 = w.rowbuf[u + 1][lane];
      ma = max3f(ma, q0.x, q1.x);
      mb = max3f(mb, q0.y, q1.y);
    }
    const bool useb = mb > ma;
    const float bk = useb ? mb : ma;
    if (bk > kKeyFloor) {
      const int col = ir + d0 + (useb ? kHalf : 0) + static_cast<int>(__float_as_uint(bk) & 0xffu);
      atomicMax(&best[ir], tsk_pack(untag_key(bk), col));
    }
    const float2 ck = w.colbuf[lane];
    const int ja = ir + d0;
    if (ck.x > kKeyFloor && ja < l)
      atomicMax(&bestc[ja], tsk_pack(untag_key(ck.x), ir - static_cast<int>(__float_as_uint(ck.x) & 0xffu)));
    if (ck.y > kKeyFloor && ja + kHalf < l)
      atomicMax(&bestc[ja + kHalf], tsk_pack(untag_key(ck.y), ir - static_cast<int>(__float_as_uint(ck.y) & 0xffu)));
  }
  __syncwarp();
}

// Row side: stream x (n samples, window arrays at wb); column side: stream xc
// (nc samples, lc windows, window arrays at wbc).  The self-join passes the
// same stream twice (AB = false: the column pointers are the row pointers).
template <bool MASKED, bool AB, typename TX>
__device__ __forceinline__ void mp_tile(const MpArgs& a, const TX* __restrict__ x, int64_t wb,
                                        const TX* __restrict__ xc, int nc, int l, int64_t wbc, int d0, int r0,
                                        int rEnd, MpWarpSmem& w, int lane) {
  const float* __restrict__ inv = a.wa.inv + wb;
  const float* __restrict__ df = a.wa.df + wb;
  const float* __restrict__ dg = a.wa.dg + wb;
  unsigned long long* __restrict__ best = a.wa.best + wb;
  const float* __restrict__ invc = AB ? a.wa.inv + wbc : inv;
  const float* __restrict__ dfc = AB ? a.wa.df + wbc : df;
  const float* __restrict__ dgc = AB ? a.wa.dg + wbc : dg;
  unsigned long long* __restrict__ bestc = AB ? a.wa.best + wbc : best;
  const int m = a.m;
  const int dA = d0 + lane * kVh;  // first diagonal of half a (half b: + kHalf)
  const float2 kMinusOne2 = make_float2(-1.f, -1.f);

  // ---- anchors c(r0, r0 + dA + v) and c(r0, r0 + dA + 256 + v) at the first row
  float2 cov2[kVh];
  if constexpr (std::is_same<TX, float>::value) {
    // float32, from centred values: the row window a_t = x[r0+t] - mean_r0 (two-term
    // mean), the column samples shifted by a nearby sample ref (one subtraction per
    // loaded sample), then c = sum_t a_t (x[c+t] - ref) - (mean_c - ref) sum_t a_t,
    // exact algebra on the rounded a_t.  Every term is of the size of the windows'
    // spread, so the float32 sums carry ~1e-7 relative error per term and no
    // cancellation of the series' offset.
    const int baseA = r0 + dA, baseB = baseA + kHalf;
    const double mr = a.wa.mu[wb + r0];
    const float mrh = static_cast<float>(mr), mrl = static_cast<float>(mr - static_cast<double>(mrh));
    const float refA = baseA < nc ? xc[baseA] : 0.f;
    const float refB = baseB < nc ? xc[baseB] : 0.f;
    float accA[kVh], accB[kVh], wa_[kVh], wbv[kVh];
#pragma unroll
    for (int v = 0; v < kVh; ++v) {
      accA[v] = 0.f;
      accB[v] = 0.f;
      wa_[v] = (baseA + v < nc) ? __fsub_rn(xc[baseA + v], refA) : 0.f;
      wbv[v] = (baseB + v < nc) ? __fsub_rn(xc[baseB + v], refB) : 0.f;
    }
    float sa = 0.f;
    int t0 = 0;
    for (; t0 + kVh <= m; t0 += kVh) {
#pragma unroll
      for (int u = 0; u < kVh; ++u) {
        const float at = __fsub_rn(__fsub_rn(x[r0 + t0 + u], mrh), mrl);
        sa = __fadd_rn(sa, at);
#pragma unroll
        for (int v = 0; v < kVh; ++v) {
          accA[v] = __fmaf_rn(at, wa_[(v + u) & (kVh - 1)], accA[v]);
          accB[v] = __fmaf_rn(at, wbv[(v + u) & (kVh - 1)], accB[v]);
        }
        const int ia = baseA + t0 + u + kVh, ib = baseB + t0 + u + kVh;
        wa_[u] = ia < nc ? __fsub_rn(xc[ia], refA) : 0.f;
        wbv[u] = ib < nc ? __fsub_rn(xc[ib], refB) : 0.f;
      }
    }
    for (int t = t0; t < m; ++t) {
      const float at = __fsub_rn(__fsub_rn(x[r0 + t], mrh), mrl);
      sa = __fadd_rn(sa, at);
#pragma unroll
      for (int v = 0; v < kVh; ++v) {
        const int ia = baseA + v + t, ib = baseB + v + t;
        accA[v] = __fmaf_rn(at, ia < nc ? __fsub_rn(xc[ia], refA) : 0.f, accA[v]);
        accB[v] = __fmaf_rn(at, ib < nc ? __fsub_rn(xc[ib], refB) : 0.f, accB[v]);
      }
    }
    const double* muc = a.wa.mu + wbc;
#pragma unroll
    for (int v = 0; v < kVh; ++v) {
      const float ca = static_cast<float>(static_cast<double>(accA[v]) -
                                         (muc[baseA + v] - static_cast<double>(refA)) * static_cast<double>(sa));
      const float cb = static_cast<float>(static_cast<double>(accB[v]) -
                                         (muc[baseB + v] - static_cast<double>(refB)) * static_cast<double>(sa));
      cov2[v] = make_float2(ca, cb);
    }
  } else {
    // float64 samples: the anchors in float64, sum_t (x[r0+t] - mean_r0) * x[c + t]
    double accA[kVh], accB[kVh], wa_[kVh], wbv[kVh];
    const int baseA = r0 + dA, baseB = baseA + kHalf;
#pragma unroll
    for (int v = 0; v < kVh; ++v) {
      accA[v] = 0.0;
      accB[v] = 0.0;
      wa_[v] = ld_guard(xc, baseA + v, nc);
      wbv[v] = ld_guard(xc, baseB + v, nc);
    }
    const double mr = a.wa.mu[wb + r0];
    int t0 = 0;
    for (; t0 + kVh <= m; t0 += kVh) {
#pragma unroll
      for (int u = 0; u < kVh; ++u) {
        const double at = static_cast<double>(x[r0 + t0 + u]) - mr;
#pragma unroll
        for (int v = 0; v < kVh; ++v) {
          accA[v] = fma(at, wa_[(v + u) & (kVh - 1)], accA[v]);
          accB[v] = fma(at, wbv[(v + u) & (kVh - 1)], accB[v]);
        }
        wa_[u] = ld_guard(xc, baseA + t0 + u + kVh, nc);
        wbv[u] = ld_guard(xc, baseB + t0 + u + kVh, nc);
      }
    }
    for (int t = t0; t < m; ++t) {
      const double at = static_cast<double>(x[r0 + t]) - mr;
#pragma unroll
      for (int v = 0; v < kVh; ++v) {
        accA[v] = fma(at, ld_guard(xc, baseA + v + t, nc), accA[v]);
        accB[v] = fma(at, ld_guard(xc, baseB + v + t, nc), accB[v]);
      }
    }
#pragma unroll
    for (int v = 0; v < kVh; ++v) cov2[v] = make_float2(static_cast<float>(accA[v]), static_cast<float>(accB[v]));
  }

  // ---- column state for the first row: slot v <-> columns r0 + dA + v (a) and + 256 (b)
  float2 cdf2[kVh], cdg2[kVh], cinv2[kVh];
  float ckA[kVh], ckB[kVh];
  unsigned tagv[kVh];
#pragma unroll
  for (int v = 0; v < kVh; ++v) {
    const int j = r0 + dA + v;
    cdf2[v] = make_float2(dfc[j], dfc[j + kHalf]);
    cdg2[v] = make_float2(dgc[j], dgc[j + kHalf]);
    cinv2[v] = make_float2(invc[j], invc[j + kHalf]);
    ckA[v] = kEmpty;
    ckB[v] = kEmpty;
    tagv[v] = static_cast<unsigned>(lane * kVh + v);
  }

  // ---- column ring: entry e <-> columns r0 + d0 + e (a) and + 256 (b)
  const int colbase = r0 + d0;
  auto ring_store = [&](int e, float vdf_a, float vdf_b, float vdg_a, float vdg_b, float vin_a, float vin_b) {
    const int p = ring_phys(e % kRingEntries);
    w.ring[0][p] = make_float2(vdf_a, vdf_b);
    w.ring[1][p] = make_float2(vdg_a, vdg_b);
    w.ring[2][p] = make_float2(vin_a, vin_b);
  };
  // initial fill: ring entries [8, 8 + kRingInit) and the rows of the first chunk
  for (int e = kVh + lane; e < kVh + kRingInit; e += 32) {
    const int j = colbase + e;
    ring_store(e, dfc[j], dfc[j + kHalf], dgc[j], dgc[j + kHalf], invc[j], invc[j + kHalf]);
  }
  {
    float2* rr = reinterpret_cast<float2*>(&w.rrow[0][0][0]);
    const int i = r0 + lane;
    rr[lane] = make_float2(df[i], df[i]);
    rr[kChunk + lane] = make_float2(dg[i], dg[i]);
    rr[2 * kChunk + lane] = make_float2(inv[i], inv[i]);
  }

  const int nsteps = MASKED ? ((rEnd - r0 + kChunk - 1) / kChunk) * kChunk : (rEnd - r0);
  int ering = (kVh * (lane + 1)) % kRingEntries;  // ring entry of the column entering at step 0
  for (int S0 = 0; S0 < nsteps; S0 += kChunk) {
    const int buf = (S0 / kChunk) & 1;
    // copies issued one chunk ago have landed; start those for the next chunk:
    // ring entries kVh + kRingInit + S0 + lane and the rows of the next chunk
    cp_async_wait_all();
    __syncwarp();
    {
      const int e = kVh + kRingInit + S0 + lane;
      const int j = colbase + e;
      float* d0p = reinterpret_cast<float*>(&w.ring[0][ring_phys(e % kRingEntries)]);
      float* d1p = reinterpret_cast<float*>(&w.ring[1][ring_phys(e % kRingEntries)]);
      float* d2p = reinterpret_cast<float*>(&w.ring[2][ring_phys(e % kRingEntries)]);
      cp_async4(d0p, dfc + j);
      cp_async4(d0p + 1, dfc + j + kHalf);
      cp_async4(d1p, dgc + j);
      cp_async4(d1p + 1, dgc + j + kHalf);
      cp_async4(d2p, invc + j);
      cp_async4(d2p + 1, invc + j + kHalf);
      float* rr = reinterpret_cast<float*>(&w.rrow[buf ^ 1][0][0]);
      const int i = r0 + S0 + kChunk + lane;
      cp_async4(rr + 2 * lane, df + i);
      cp_async4(rr + 2 * lane + 1, df + i);
      cp_async4(rr + 2 * kChunk + 2 * lane, dg + i);
      cp_async4(rr + 2 * kChunk + 2 * lane + 1, dg + i);
      cp_async4(rr + 4 * kChunk + 2 * lane, inv + i);
      cp_async4(rr + 4 * kChunk + 2 * lane + 1, inv + i);
      cp_async_commit();
    }
#pragma unroll 1
    for (int sb = 0; sb < kChunk; sb += kVh) {  // 8-row blocks: one period of the slot rotation
    // in a block the entering columns are ring entries ering .. ering + 7 (ering is
    // a multiple of 8): consecutive slots from ring_phys(ering)
    const float2* ringb = &w.ring[0][ring_phys(ering)];
    ering = (ering + kVh == kRingEntries) ? 0 : ering + kVh;
    float2* rowp = &w.rowbuf[lane][sb];
    // keys of one row (slot c = (v + sr) % 8 holds the column of diagonal v), with
    // the covariance advanced to the next row
    auto row_keys = [&](int sr, int i, float2 rdf2, float2 rdg2, float2 rinv2, float (&kA)[kVh],
                        float (&kB)[kVh]) {
#pragma unroll
      for (int v = 0; v < kVh; ++v) {
        const int c = (v + sr) & (kVh - 1);
        const float2 t = __fmul2_rn(cov2[v], cinv2[c]);
        const float2 r = __ffma2_rn(t, rinv2, kMinusOne2);  // rho - 1: full relative precision near rho = 1
        float ka = tag_key(r.x, tagv[v]);
        float kb = tag_key(r.y, tagv[v]);
        if (MASKED) {
          const bool rowok = i < rEnd;
          ka = (rowok && i + dA + v < l) ? ka : kEmpty;
          kb = (rowok && i + dA + kHalf + v < l) ? kb : kEmpty;
        }
        kA[v] = ka;
        kB[v] = kb;
        cov2[v] = __ffma2_rn(rdf2, cdg2[c], cov2[v]);
        cov2[v] = __ffma2_rn(cdf2[c], rdg2, cov2[v]);
      }
      const float rka = fmaxf(max3f(max3f(max3f(kA[0], kA[1], kA[2]), kA[3], kA[4]), kA[5], kA[6]), kA[7]);
      const float rkb = fmaxf(max3f(max3f(max3f(kB[0], kB[1], kB[2]), kB[3], kB[4]), kB[5], kB[6]), kB[7]);
      rowp[sr] = make_float2(rka, rkb);
    };
    // the column in slot c0 leaves the lane (to lane - 1; lane 0's is complete for
    // this band) and the column entering from the ring takes its place
    auto exit_column = [&](int sr, int s, float la, float lb) {
      const float ia = __shfl_down_sync(TSK_FULL_MASK, la, 1);
      const float ib = __shfl_down_sync(TSK_FULL_MASK, lb, 1);
      if (lane == 0) w.colbuf[s] = make_float2(la, lb);
      ckA[sr] = (lane == 31) ? kEmpty : ia;
      ckB[sr] = (lane == 31) ? kEmpty : ib;
      cdf2[sr] = ringb[sr];
      cdg2[sr] = ringb[kRingPhys + sr];
      cinv2[sr] = ringb[2 * kRingPhys + sr];
    };
#pragma unroll
    for (int gg = 0; gg < kVh / 2; ++gg) {
      const int g = sb / 2 + gg;
      const float4 rf4 = w.rrow[buf][0][g], rg4 = w.rrow[buf][1][g], ri4 = w.rrow[buf][2][g];
      // rows s0 = 2gg and s0 + 1 of the 8-row block; column maxima are folded over
      // the two rows with 3-input max: slot c takes the key of diagonal (c - s0) % 8
      // of row s0 and of diagonal (c - s0 - 1) % 8 of row s0 + 1
      const int s0 = 2 * gg;
      const int i0 = r0 + S0 + sb + s0;
      float k0A[kVh], k0B[kVh], k1A[kVh], k1B[kVh];
      row_keys(s0, i0, make_float2(rf4.x, rf4.y), make_float2(rg4.x, rg4.y), make_float2(ri4.x, ri4.y), k0A, k0B);
      // slot s0 leaves after row s0: its last key is diagonal 0 of row s0
      exit_column(s0, sb + s0, fmaxf(ckA[s0], k0A[0]), fmaxf(ckB[s0], k0B[0]));
      row_keys(s0 + 1, i0 + 1, make_float2(rf4.z, rf4.w), make_float2(rg4.z, rg4.w), make_float2(ri4.z, ri4.w),
               k1A, k1B);
#pragma unroll
      for (int c = 0; c < kVh; ++c) {
        if (c == s0) {  // the column that entered after row s0 has only row s0 + 1's key (diagonal 7)
          ckA[c] = fmaxf(ckA[c], k1A[kVh - 1]);
          ckB[c] = fmaxf(ckB[c], k1B[kVh - 1]);
        } else {
          ckA[c] = max3f(ckA[c], k0A[(c - s0) & (kVh - 1)], k1A[(c - s0 - 1) & (kVh - 1)]);
          ckB[c] = max3f(ckB[c], k0B[(c - s0) & (kVh - 1)], k1B[(c - s0 - 1) & (kVh - 1)]);
        }
      }
      exit_column(s0 + 1, sb + s0 + 1, ckA[s0 + 1], ckB[s0 + 1]);
    }
    }
    flush_chunk(w, kChunk, r0 + S0, d0, l, best, bestc, lane);
  }
  cp_async_wait_all();
  __syncwarp();
  // columns still inside the band: slot v <-> columns r0 + nsteps + dA + v (+ 256)
#pragma unroll
  for (int v = 0; v < kVh; ++v) {
    const int j = r0 + nsteps + dA + v;
    const int row0 = r0 + nsteps + lane * kVh + v;  // = j - d0
    if (ckA[v] > kKeyFloor && j < l)
      atomicMax(&bestc[j], tsk_pack(untag_key(ckA[v]), row0 - static_cast<int>(__float_as_uint(ckA[v]) & 0xffu)));
    if (ckB[v] > kKeyFloor && j + kHalf < l)
      atomicMax(&bestc[j + kHalf], tsk_pack(untag_key(ckB[v]), row0 - static_cast<int>(__float_as_uint(ckB[v]) & 0xffu)));
  }
}

template <typename TX, bool AB>
__global__ void __launch_bounds__(kWarps * 32, 3) k_mp_diag(MpArgs a) {
  extern __shared__ __align__(16) unsigned char mp_smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  MpWarpSmem& w = reinterpret_cast<MpWarpSmem*>(mp_smem)[wid];
  for (;;) {
    // guided claim: a run of consecutive work units, long while much work
    // remains (contiguous units of a band then share one anchor),
    // single units at the end (balance)
    int w0 = 0, wend = 0;
    if (lane == 0) {
      const long long cur = static_cast<long long>(*reinterpret_cast<volatile unsigned long long*>(a.counter));
      const long long remaining = a.total_tiles - cur;
      const long long c = min(static_cast<long long>(kMaxClaim), max(1LL, remaining / (2LL * a.total_warps)));
      const long long s0 = static_cast<long long>(atomicAdd(a.counter, static_cast<unsigned long long>(c)));
      w0 = static_cast<int>(min(s0, static_cast<long long>(a.total_tiles)));
      wend = static_cast<int>(min(s0 + c, static_cast<long long>(a.total_tiles)));
    }
    w0 = __shfl_sync(TSK_FULL_MASK, w0, 0);
    wend = __shfl_sync(TSK_FULL_MASK, wend, 0);
    if (w0 >= wend) break;
    for (int wk = w0; wk < wend;) {
      const int4 td = a.tiles[wk];
      const int q = td.x, d0 = td.y, r0 = td.z;
      int rEnd = td.w & 0x7fffffff;
      const bool masked = td.w < 0;
      ++wk;
      if (!masked) {
        // merge the following units that continue this band
        while (wk < wend) {
          const int4 nx = a.tiles[wk];
          if (nx.w < 0 || nx.x != q || nx.y != d0 || nx.z != rEnd || nx.w - r0 > kMaxWalk) break;
          rEnd = nx.w;
          ++wk;
        }
      }
      const TX* X = static_cast<const TX*>(a.X);
      const TX* x;
      const TX* xc;
      int nc;
      int64_t wb, wbc;
      if (AB) {
        const TX* X2 = static_cast<const TX*>(a.X2);
        const int p = q < a.split ? q + a.split : q - a.split;  // the partner stream
        x = stream_base(X, X2, a.xoff, a.split, q);
        xc = stream_base(X, X2, a.xoff, a.split, p);
        nc = a.len[p];
        wb = a.woff[q];
        wbc = a.woff[p];
      } else {
        x = X + a.xoff[q];
        xc = x;
        nc = a.len[q];
        wb = a.woff[q];
        wbc = wb;
      }
      const int lc = nc - a.m + 1;
      if (!masked)
        mp_tile<false, AB, TX>(a, x, wb, xc, nc, lc, wbc, d0, r0, rEnd, w, lane);
      else
        mp_tile<true, AB, TX>(a, x, wb, xc, nc, lc, wbc, d0, r0, rEnd, w, lane);
    }
  }
}

// ---------------------------------------------------------------------------
// 3'. exact float64 variant: one thread per (stream, diagonal)
// ---------------------------------------------------------------------------
template <typename TX>
__device__ __forceinline__ double f64_cell_rho(double cov, const double* inv64, int i, int j) {
  return cov * inv64[i] * inv64[j];
}

template <typename TX, bool AB>
__global__ void __launch_bounds__(128) k_mp_diag_f64(MpArgs a, int pass) {
  const int64_t w = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (w >= a.total_tiles) return;
  const int q = tsk_find_segment<int64_t>(a.tile_prefix, a.n_streams, w);
  const int p = AB ? (q < a.split ? q + a.split : q - a.split) : q;  // the column side
  const int m = a.m;
  const int l = a.len[q] - m + 1, lp = a.len[p] - m + 1;
  const int dmin = AB ? (q < a.split ? 0 : 1) : a.excl;
  const int delta = dmin + static_cast<int>(w - a.tile_prefix[q]);
  const TX* X = static_cast<const TX*>(a.X);
  const TX* x = AB ? stream_base(X, static_cast<const TX*>(a.X2), a.xoff, a.split, q) : X + a.xoff[q];
  const TX* xp = AB ? stream_base(X, static_cast<const TX*>(a.X2), a.xoff, a.split, p) : x;
  const int64_t wb = a.woff[q], wbp = a.woff[p];
  const double* mu = a.wa.mu + wb;
  const double* mup = a.wa.mu + wbp;
  const double* inv64 = a.wa.inv64 + wb;
  const double* inv64p = a.wa.inv64 + wbp;
  unsigned long long* best = a.wa.best + wb;
  unsigned long long* bestp = a.wa.best + wbp;
  int32_t* bidx = a.wa.bidx + wb;
  int32_t* bidxp = a.wa.bidx + wbp;
  double cov = 0.0;
  const double m0 = mu[0];
  for (int t = 0; t < m; ++t) cov = fma(static_cast<double>(x[t]) - m0, static_cast<double>(xp[delta + t]), cov);
  for (int i = 0; i < l && i + delta < lp; ++i) {
    const int j = i + delta;
    const double rho = cov * inv64[i] * inv64p[j];
    const unsigned long long key = tsk_ordered_u64(rho);
    if (pass == 0) {
      atomicMax(&best[i], key);
      atomicMax(&bestp[j], key);
    } else {
      if (key == best[i]) atomicMin(&bidx[i], j);
      if (key == bestp[j]) atomicMin(&bidxp[j], i);
    }
    if (i + 1 < l && j + 1 < lp) {
      const double xa = static_cast<double>(x[i]), xb = static_cast<double>(x[i + m]);
      const double ya = static_cast<double>(xp[j]), yb = static_cast<double>(xp[j + m]);
      const double dfi = (xb - xa) * 0.5, dfj = (yb - ya) * 0.5;
      const double dgi = (xb - mu[i + 1]) + (xa - mu[i]);
      const double dgj = (yb - mup[j + 1]) + (ya - mup[j]);
      cov = fma(dfi, dgj, cov);
      cov = fma(dfj, dgi, cov);
    }
  }
}

// ---------------------------------------------------------------------------
// 4. refinement: exact distance to each window's chosen neighbour
// ---------------------------------------------------------------------------
template <typename TX, typename TP, bool AB>
__global__ void __launch_bounds__(256) k_mp_refine(const TX* __restrict__ X, const TX* __restrict__ X2, int split,
                                                   const int64_t* __restrict__ xoff,
                                                   const int32_t* __restrict__ len, const uint8_t* __restrict__ smask,
                                                   const int64_t* __restrict__ woff, int n_streams, int64_t total, int m,
                                                   int excl, int exact64, WinArrays wa, TP* __restrict__ P,
                                                   int32_t* __restrict__ I, TP* __restrict__ P2,
                                                   int32_t* __restrict__ I2) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int q = tsk_find_segment<int64_t>(xoff, n_streams, e);
  if (!smask[q]) return;
  // output slot: the AB join writes the training side's profile to P2 / I2
  TP* Pout = P;
  int32_t* Iout = I;
  int64_t eo = e;
  if (AB && q >= split) {
    if (!P2) return;
    Pout = P2;
    Iout = I2;
    eo = e - xoff[split];
  }
  const int n = len[q];
  const int l = n - m + 1;
  const int i = static_cast<int>(e - xoff[q]);
  if (i >= l) {
    Pout[eo] = static_cast<TP>(NAN);
    Iout[eo] = -1;
    return;
  }
  const int p = AB ? (q < split ? q + split : q - split) : q;  // stream holding the candidates
  const int lp = len[p] - m + 1;
  const int64_t wb = woff[q], wbp = woff[p];
  const TX* x = AB ? stream_base(X, X2, xoff, split, q) : X + xoff[q];
  const TX* xp = AB ? stream_base(X, X2, xoff, split, p) : x;
  // lowest admissible constant window
  int jc = -1;
  if (wa.constcnt[p] > 0) {
    const int f = wa.nxt[wbp];
    if (AB) {
      if (f < lp) jc = f;
    } else if (f <= i - excl) {
      jc = f;
    } else if (i + excl < l) {
      const int g = wa.nxt[wb + i + excl];
      if (g < l) jc = g;
    }
  }
  const double sqm = sqrt(static_cast<double>(m));
  if (wa.inv[wb + i] == 0.f) {
    if (jc >= 0) { Pout[eo] = static_cast<TP>(0); Iout[eo] = jc; return; }
    const int jl = AB ? 0 : ((i >= excl) ? 0 : ((i + excl < l) ? i + excl : -1));
    Pout[eo] = static_cast<TP>(jl >= 0 ? sqm : INFINITY);
    Iout[eo] = jl;
    return;
  }
  int j = -1;
  if (exact64) {
    const int b = wa.bidx[wb + i];  // initialised to 0x7f7f7f7f (no neighbour)
    j = (b >= lp) ? -1 : b;
  } else {
    const unsigned long long pk = wa.best[wb + i];
    j = pk ? tsk_unpack_idx(pk) : -1;
  }
  double dist = INFINITY;
  if (j >= 0) {
    if (wa.inv[wbp + j] == 0.f) {
      dist = sqm;
    } else {
      const double rho = tsk::window_rho(x, i, xp, j, m, wa.mu[wb + i], wa.mu[wbp + j]);
      dist = sqrt(fmax(0.0, 2.0 * m * (1.0 - rho)));
    }
  }
  if (jc >= 0 && (sqm < dist || (sqm == dist && jc < j))) { dist = sqm; j = jc; }
  Pout[eo] = static_cast<TP>(dist);
  Iout[eo] = j;
}

// Raise a kernel's dynamic shared-memory limit once per (device, kernel), and
// only when a larger size is needed, so calls captured in a CUDA graph issue
// no attribute changes.
template <typename K>
cudaError_t set_smem_limit(K kernel, int device, int bytes, int /*slot*/) {
  struct Entry {
    int device;
    const void* fn;
    int bytes;
  };
  static std::mutex mu;
  static std::vector<Entry> done;
  std::lock_guard<std::mutex> lock(mu);
  const void* fn = reinterpret_cast<const void*>(kernel);
  for (auto& e : done)
    if (e.device == device && e.fn == fn) {
      if (bytes <= e.bytes) return cudaSuccess;
      const cudaError_t r = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
      if (r == cudaSuccess) e.bytes = bytes;
      return r;
    }
  const cudaError_t r = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (r == cudaSuccess) done.push_back({device, fn, bytes});
  return r;
}

template <typename TX>
tsk_status run_typed(tsk_ctx* ctx, const TX* X, const TX* X2, int32_t split, bool ab, int32_t n_streams,
                     const tsk_mp_plan& plan, int32_t m, int32_t excl, int32_t precision, void* P, int32_t* I,
                     void* P2, int32_t* I2, char* ws) {
  tsk_carver cv(ws);
  const int64_t W = plan.total_windows;
  const bool f64 = precision == TSK_MP_FP64;
  WinArrays wa{};
  wa.mu = cv.take<double>(W);
  wa.ss = cv.take<double>(W);
  wa.inv = cv.take<float>(W);
  wa.df = cv.take<float>(W);
  wa.dg = cv.take<float>(W);
  wa.best = cv.take<unsigned long long>(W);
  wa.nxt = cv.take<int32_t>(W);
  wa.constcnt = cv.take<int32_t>(n_streams);
  unsigned long long* counter = cv.take<unsigned long long>(1);
  if (f64) {
    wa.inv64 = cv.take<double>(W);
    wa.bidx = cv.take<int32_t>(W);
  }
  cudaStream_t st = ctx->stream;
  TSK_CUDA_TRY(ctx, cudaMemsetAsync(wa.best, 0, sizeof(unsigned long long) * W, st));
  TSK_CUDA_TRY(ctx, cudaMemsetAsync(wa.constcnt, 0, sizeof(int32_t) * n_streams, st));
  TSK_CUDA_TRY(ctx, cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
  if (f64) TSK_CUDA_TRY(ctx, cudaMemsetAsync(wa.bidx, 0x7f, sizeof(int32_t) * W, st));  // ~INT_MAX
  if (plan.total_chunks > 0) {
    const size_t smem = sizeof(double) * 2 * (kWinChunk + m + 2);
    TSK_CUDA_TRY(ctx, set_smem_limit(k_window_stats<TX>, ctx->device, static_cast<int>(smem), 0));
    k_window_stats<TX><<<static_cast<unsigned>(plan.total_chunks), kWinThreads, smem, st>>>(
        X, X2, split, plan.xoff, plan.len, plan.woff, plan.chunk_prefix, n_streams, m, f64 ? 1 : 0, wa, ctx->d_err);
    TSK_LAUNCH_CHECK(ctx, "k_window_stats");
    k_next_const<<<n_streams, kWinThreads, 0, st>>>(plan.len, plan.smask, plan.woff, m, wa);
    TSK_LAUNCH_CHECK(ctx, "k_next_const");
  }
  MpArgs a{};
  a.X = X;
  a.X2 = X2;
  a.split = split;
  a.xoff = plan.xoff;
  a.len = plan.len;
  a.woff = plan.woff;
  a.tile_prefix = plan.tile_prefix;
  a.tiles = plan.tiles;
  a.counter = counter;
  a.wa = wa;
  a.total_tiles = plan.total_tiles;
  a.n_streams = n_streams;
  a.m = m;
  a.excl = excl;
  a.H = plan.H;
  if (plan.total_tiles > 0) {
    if (f64) {
      const int64_t blocks = (plan.total_tiles + 127) / 128;
      for (int pass = 0; pass < 2; ++pass) {
        if (ab)
          k_mp_diag_f64<TX, true><<<static_cast<unsigned>(blocks), 128, 0, st>>>(a, pass);
        else
          k_mp_diag_f64<TX, false><<<static_cast<unsigned>(blocks), 128, 0, st>>>(a, pass);
        TSK_LAUNCH_CHECK(ctx, "k_mp_diag_f64");
      }
    } else {
      const size_t smem = sizeof(MpWarpSmem) * kWarps;
      auto kern = ab ? k_mp_diag<TX, true> : k_mp_diag<TX, false>;
      TSK_CUDA_TRY(ctx, set_smem_limit(kern, ctx->device, static_cast<int>(smem), 1));
      int per_sm = 0;
      TSK_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarps * 32, smem));
      per_sm = std::max(per_sm, 1);
      const int64_t want = (plan.total_tiles + kWarps - 1) / kWarps;
      const int64_t grid = std::min<int64_t>(want, static_cast<int64_t>(per_sm) * ctx->sm_count);
      a.total_warps = static_cast<int>(grid) * kWarps;
      {
        tsk_prof_scope ps(ctx, TSK_PROF_MP_DIAG);
        kern<<<static_cast<unsigned>(grid), kWarps * 32, smem, st>>>(a);
      }
      TSK_LAUNCH_CHECK(ctx, "k_mp_diag");
    }
  }
  const int64_t total = plan.total_samples;
  if (total > 0) {
    const int64_t blocks = (total + 255) / 256;
    const unsigned g = static_cast<unsigned>(blocks);
    if (f64 && ab)
      k_mp_refine<TX, double, true><<<g, 256, 0, st>>>(X, X2, split, plan.xoff, plan.len, plan.smask, plan.woff,
                                                       n_streams, total, m, 0, 1, wa, static_cast<double*>(P), I,
                                                       static_cast<double*>(P2), I2);
    else if (f64)
      k_mp_refine<TX, double, false><<<g, 256, 0, st>>>(X, X2, split, plan.xoff, plan.len, plan.smask, plan.woff,
                                                        n_streams, total, m, excl, 1, wa, static_cast<double*>(P), I,
                                                        nullptr, nullptr);
    else if (ab)
      k_mp_refine<TX, float, true><<<g, 256, 0, st>>>(X, X2, split, plan.xoff, plan.len, plan.smask, plan.woff,
                                                      n_streams, total, m, 0, 0, wa, static_cast<float*>(P), I,
                                                      static_cast<float*>(P2), I2);
    else
      k_mp_refine<TX, float, false><<<g, 256, 0, st>>>(X, X2, split, plan.xoff, plan.len, plan.smask, plan.woff,
                                                       n_streams, total, m, excl, 0, wa, static_cast<float*>(P), I,
                                                       nullptr, nullptr);
    TSK_LAUNCH_CHECK(ctx, "k_mp_refine");
  }
  return TSK_OK;
}

}  // namespace

int tsk_mp_band_width() { return kBand; }
int tsk_mp_chunk_rows() { return kChunk; }
int tsk_mp_pad() { return kPad; }
int tsk_mp_chunk() { return kWinChunk; }

size_t tsk_mp_ws_bytes(const tsk_mp_plan& plan, int32_t n_streams) {
  const size_t W = static_cast<size_t>(plan.total_windows);
  size_t b = 0;
  b += tsk_carver::bytes_for(W, 8) * 2 + tsk_carver::bytes_for(W, 4) * 3 + tsk_carver::bytes_for(W, 8) +
       tsk_carver::bytes_for(W, 4) + tsk_carver::bytes_for(n_streams, 4) + tsk_carver::bytes_for(1, 8);
  if (plan.prec == TSK_MP_FP64) b += tsk_carver::bytes_for(W, 8) + tsk_carver::bytes_for(W, 4);
  return b + 4096;
}

tsk_status tsk_run_mp(tsk_ctx* ctx, const void* X, int x_dtype, int32_t n_streams, const tsk_mp_plan& plan, int32_t m,
                      int32_t excl, int32_t precision, void* P, int32_t* I, char* ws) {
  if (x_dtype == TSK_F64)
    return run_typed<double>(ctx, static_cast<const double*>(X), static_cast<const double*>(X), n_streams, false,
                             n_streams, plan, m, excl, precision, P, I, nullptr, nullptr, ws);
  return run_typed<float>(ctx, static_cast<const float*>(X), static_cast<const float*>(X), n_streams, false, n_streams,
                          plan, m, excl, precision, P, I, nullptr, nullptr, ws);
}

tsk_status tsk_run_mp_ab(tsk_ctx* ctx, const void* A, const void* B, int x_dtype, int32_t n_pairs,
                         const tsk_mp_plan& plan, int32_t m, int32_t precision, void* P_a, int32_t* I_a, void* P_b,
                         int32_t* I_b, char* ws) {
  if (x_dtype == TSK_F64)
    return run_typed<double>(ctx, static_cast<const double*>(A), static_cast<const double*>(B), n_pairs, true,
                             2 * n_pairs, plan, m, 0, precision, P_a, I_a, P_b, I_b, ws);
  return run_typed<float>(ctx, static_cast<const float*>(A), static_cast<const float*>(B), n_pairs, true, 2 * n_pairs,
                          plan, m, 0, precision, P_a, I_a, P_b, I_b, ws);
}

// ---------------------------------------------------------------------------
// Allocation-free variant for one stream.
//
// All device scratch of the matrix-profile pipeline (window statistics, the
// packed per-window maxima, the work list, counters) lives in one file-scope
// __device__ array.  Host code never uses the array's name as an address: its
// device address comes from cudaGetSymbolAddress, once per device.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchBytes = size_t(3) << 20;  // 3 MiB on every device that loads the library
constexpr int kStaticMaxWindows = 65536;                   // l = n - m + 1 at most
constexpr int kStaticMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_addr[kStaticMaxDevices] = {};

// Per-device set-up: the scratch array's device address and the kernels'
// shared-memory limits.  Runs on the first call on each device.
tsk_status static_setup(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return TSK_ERR_CUDA;
    }
    const int win_smem = static_cast<int>(sizeof(double) * 2 * (kWinChunk + 4096 + 2));
    if (cudaFuncSetAttribute(k_window_stats<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, win_smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_mp_diag<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sizeof(MpWarpSmem) * kWarps)) != cudaSuccess) {
      cudaGetLastError();
      return TSK_ERR_CUDA;
    }
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return TSK_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" TSK_API tsk_status mp_selfjoin_static(const float* X, int32_t n, int32_t m, int32_t excl, float* P,
                                                 int32_t* I, void* cuda_stream) {
  if (!X || !P || !I || m < 2 || m > 4096 || n < m || excl < 1) return TSK_ERR_INVALID_ARG;
  const int64_t l = static_cast<int64_t>(n) - m + 1;
  if (l > kStaticMaxWindows) return TSK_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) return TSK_ERR_CUDA;
  void* base = nullptr;
  tsk_status st = static_setup(dev, &base);
  if (st) return st;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TSK_ERR_CUDA;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

  // work list of the one stream: interior units of every band, then the band ends
  const int64_t e = l - excl;
  const double cells = e > 0 ? static_cast<double>(e) * (e + 1) / 2 : 0.0;
  int32_t H = static_cast<int32_t>(std::min(8192.0, std::max(2048.0, cells / (sms * 12.0 * 64.0 * kBand))));
  H = (H + kChunk - 1) / kChunk * kChunk;
  std::vector<int4> tiles, tri;
  for (int64_t d0 = excl; d0 < l; d0 += kBand) {
    const int64_t rows = l - d0;
    int64_t rint = std::max<int64_t>(0, rows - (kBand - 1));
    rint -= rint % kChunk;
    for (int64_t r0 = 0; r0 < rint; r0 += H)
      tiles.push_back(make_int4(0, static_cast<int>(d0), static_cast<int>(r0), static_cast<int>(std::min<int64_t>(r0 + H, rint))));
    if (rows > rint)
      tri.push_back(make_int4(0, static_cast<int>(d0), static_cast<int>(rint),
                              static_cast<int>(static_cast<uint32_t>(rows) | 0x80000000u)));
  }
  tiles.insert(tiles.end(), tri.begin(), tri.end());

  // carve the scratch array
  const int64_t W = (l + kPad + 3) & ~int64_t(3);
  struct Head {
    int64_t xoff[2], woff[2], chunk_prefix[2];
    int32_t len[1];
    uint8_t smask[4];
  };
  size_t off = 0;
  const size_t o_head = off; off = align256(off + sizeof(Head));
  const size_t o_mu = off; off = align256(off + 8 * W);
  const size_t o_ss = off; off = align256(off + 8 * W);
  const size_t o_inv = off; off = align256(off + 4 * W);
  const size_t o_df = off; off = align256(off + 4 * W);
  const size_t o_dg = off; off = align256(off + 4 * W);
  const size_t o_best = off; off = align256(off + 8 * W);
  const size_t o_nxt = off; off = align256(off + 4 * W);
  const size_t o_small = off; off = align256(off + 64);  // constcnt, counter, error word
  const size_t o_tiles = off; off = align256(off + sizeof(int4) * tiles.size());
  if (off > kStaticScratchBytes) return TSK_ERR_INVALID_ARG;
  char* sb = static_cast<char*>(base);
  Head h{};
  h.xoff[1] = n;
  h.woff[1] = W;
  h.chunk_prefix[1] = (l + kWinChunk - 1) / kWinChunk;
  h.len[0] = n;
  h.smask[0] = 1;
  if (cudaMemcpyAsync(sb + o_head, &h, sizeof(Head), cudaMemcpyHostToDevice, stream) != cudaSuccess ||
      (!tiles.empty() && cudaMemcpyAsync(sb + o_tiles, tiles.data(), sizeof(int4) * tiles.size(),
                                         cudaMemcpyHostToDevice, stream) != cudaSuccess) ||
      cudaMemsetAsync(sb + o_best, 0, 8 * W, stream) != cudaSuccess ||
      cudaMemsetAsync(sb + o_small, 0, 64, stream) != cudaSuccess) {
    cudaGetLastError();
    return TSK_ERR_CUDA;
  }
  const Head* dh = reinterpret_cast<const Head*>(sb + o_head);
  WinArrays wa{};
  wa.mu = reinterpret_cast<double*>(sb + o_mu);
  wa.ss = reinterpret_cast<double*>(sb + o_ss);
  wa.inv = reinterpret_cast<float*>(sb + o_inv);
  wa.df = reinterpret_cast<float*>(sb + o_df);
  wa.dg = reinterpret_cast<float*>(sb + o_dg);
  wa.best = reinterpret_cast<unsigned long long*>(sb + o_best);
  wa.nxt = reinterpret_cast<int32_t*>(sb + o_nxt);
  wa.constcnt = reinterpret_cast<int32_t*>(sb + o_small);
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(sb + o_small + 8);
  int* err = reinterpret_cast<int*>(sb + o_small + 16);

  const size_t win_smem = sizeof(double) * 2 * (kWinChunk + m + 2);
  k_window_stats<float><<<static_cast<unsigned>(h.chunk_prefix[1]), kWinThreads, win_smem, stream>>>(
      X, X, 1, dh->xoff, dh->len, dh->woff, dh->chunk_prefix, 1, m, 0, wa, err);
  k_next_const<<<1, kWinThreads, 0, stream>>>(dh->len, dh->smask, dh->woff, m, wa);
  if (!tiles.empty()) {
    MpArgs a{};
    a.X = X;
    a.X2 = X;
    a.split = 1;
    a.xoff = dh->xoff;
    a.len = dh->len;
    a.woff = dh->woff;
    a.tiles = reinterpret_cast<const int4*>(sb + o_tiles);
    a.counter = counter;
    a.wa = wa;
    a.total_tiles = static_cast<int64_t>(tiles.size());
    a.n_streams = 1;
    a.m = m;
    a.excl = excl;
    a.H = H;
    const size_t smem = sizeof(MpWarpSmem) * kWarps;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mp_diag<float, false>, kWarps * 32, smem) != cudaSuccess) {
      cudaGetLastError();
      return TSK_ERR_CUDA;
    }
    per_sm = std::max(per_sm, 1);
    const int64_t grid = std::min<int64_t>((a.total_tiles + kWarps - 1) / kWarps, static_cast<int64_t>(per_sm) * sms);
    a.total_warps = static_cast<int>(grid) * kWarps;
    k_mp_diag<float, false><<<static_cast<unsigned>(grid), kWarps * 32, smem, stream>>>(a);
  }
  k_mp_refine<float, float, false><<<static_cast<unsigned>((n + 255) / 256), 256, 0, stream>>>(
      X, X, 1, dh->xoff, dh->len, dh->smask, dh->woff, 1, n, m, excl, 0, wa, P, I, nullptr, nullptr);
  if (cudaGetLastError() != cudaSuccess) return TSK_ERR_CUDA;
  return TSK_OK;
}
