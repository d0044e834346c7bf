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
//                       band's columns slide).  Maxima are tagged once per lane
//                       (8 low mantissa bits), so a maximum names a group of 8
//                       candidate windows.  Results merge into a packed (key,
//                       first window of the group) 64-bit word per window with
//                       atomicMax; groups within kNearTie of a window's maximum
//                       are kept as near-tie candidates.
//   4. k_mp_refine      for every window: its candidate groups scored in float32,
//                       the best re-scored exactly (compensated sums) where the
//                       match is close, dist = sqrt(2 m (1 - rho)), plus the
//                       constant-window rules.
//   5. k_mp_rescan      windows with a near-exact match (1 - rho < 1e-4) or an
//                       overflowed near-tie list: the whole row swept in
//                       float32, every window within float32 resolution of its
//                       best re-scored exactly.
// After point updates (section 6 below) only the windows covering changed
// samples, and those whose nearest neighbour was among them, are re-profiled.
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
#include "tsk_tc.cuh"

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
constexpr int kCand = 4;                 // near-tie candidate groups kept per window
// Two groups whose float32 keys differ by at most this much (in rho) are near
// ties: the recurrence's rounding (~1e-6 over the longest walks) may order them
// either way, so both are re-scored exactly.
constexpr float kNearTie = 3e-5f;
// Near ties only matter for close matches: with keys within 1e-6 of each other
// the 1e-3 bar on the distance binds once 1 - rho is below ~5e-3.  Groups with
// keys below -kCloseKey go straight to the maximum (no candidate list).
constexpr float kCloseKey = 0.02f;
// The refinement re-scores candidates exactly only where some float32
// correlation reaches this; below it float32 (~1e-6 in rho) gives the distance
// to ~1e-4 relative (dist error ~ drho / (2 (1 - rho))), a tenth of the 1e-3 bar.
constexpr float kExactRho = 0.99f;
// A window whose nearest neighbour is within this of rho = 1, or a close match
// (1 - rho < 5e-3) whose near-tie list overflowed, is re-scanned whole: every
// window within kRescanTol (in rho) of the best float32 score is re-scored
// exactly.  Choosing a neighbour d_rho worse moves the distance by about
// d_rho / (2 (1 - rho)) of itself, so near ties that float32 orders only to
// ~1e-6 (up to ~2e-6 over the longest walks) can break the 1e-3 bar wherever
// 1 - rho < 1e-3; those rows do not rely on the near-tie lists, whose content
// depends on the order of the merges.  Not when the chosen neighbour's exact
// 1 - rho is at most kRescanExact: its distance, sqrt(2m (1 - rho)) <=
// 1e-5 sqrt(2m), is already within the bar's absolute floor of any better one
// (exact repeats, e.g. periodic square waves).
constexpr double kRescanGap = 1e-3;
constexpr double kRescanExact = 1e-10;
// A window whose norm ||x - mean|| is below this fraction of the largest in
// its stream or its partner's is re-scanned too.  The float32 recurrence keeps
// an absolute error set by the loud windows of a walk (~2^-24 of their
// covariances); relative to a window a thousand times quieter (a flat stretch
// with sensor noise between steps or spikes) that error reorders its
// candidates.  The re-scan's float32 scores come from centred values, not the
// recurrence, so they resolve such windows.
constexpr float kQuietNorm = 1e-2f;
constexpr int kRescanThreads = 512;  // one block per listed window: a row's latency is spread over 16 warps
constexpr float kRescanTol = 4e-6f;

struct WinArrays {
  double* mu;
  double* ss;
  float* inv;
  float* df;
  float* dg;
  unsigned long long* best;   // packed (key, first window of the best candidate group)
  int32_t* nxt;
  int32_t* constcnt;
  unsigned int* nmax;         // per stream: the largest window norm ||x - mean|| (float bits)
  int32_t* ncnt;              // near-tie groups offered per window (may exceed kCand)
  unsigned long long* near;   // [window][kCand] near-tie groups, packed like best
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
  __shared__ unsigned int bnmax;
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
  if (threadIdx.x == 0) {
    ccount = 0;
    bnmax = 0u;
  }
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
  float my_nmax = 0.f;
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
    if (!cst) my_nmax = fmaxf(my_nmax, static_cast<float>(ss * r));  // ||x - mean|| = ss / sqrt(ss)
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
  for (int o = 16; o > 0; o >>= 1) {
    my_const += __shfl_xor_sync(TSK_FULL_MASK, my_const, o);
    my_nmax = fmaxf(my_nmax, __shfl_xor_sync(TSK_FULL_MASK, my_nmax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (my_const) atomicAdd(&ccount, my_const);
    atomicMax(&bnmax, __float_as_uint(my_nmax));  // non-negative floats order as their bits
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (ccount) atomicAdd(&wa.constcnt[q], ccount);
    atomicMax(&wa.nmax[q], bnmax);
  }
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
// float32 FMA/MUL.  A cell's key is rho - 1 (one FMA: t * inv_i - 1, exact to
// float32 relative precision near rho = 1, where close matches are told apart).
// Per row the lane's 8 + 8 cells update
//   - the row maximum: the maximum of each half's 8 keys, tagged with the lane
//     (its 8 low mantissa bits), reduced over lanes in shared memory every 32
//     rows, and
//   - 8 + 8 column maxima held in registers: a column spends 8 rows in a lane
//     (one slot); its maximum there is tagged with the lane when it leaves for
//     lane t-1 and merged with the maximum it brought from the lanes above;
//     lane 0's is complete for this band.
// A maximum therefore names a group of 8 candidate windows (one lane's 8
// diagonals, or the 8 rows a column spends in one lane), not one cell: tags
// cost one operation per reduced maximum instead of one per cell.  Results
// merge into a packed (key, first window of the group) 64-bit word per window
// with atomicMax; a group that loses by at most kNearTie (or is displaced by
// one at most kNearTie better) is kept as a near-tie candidate.  The
// refinement re-scores the groups exactly.
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
  float rowbuf[32][kChunk + 1];   // row maximum of both halves (tag: lane + 32 half): [lane][step]
  float2 colbuf[kChunk];          // keys of the columns leaving lane 0, per step
  float2 inbuf[kVh][32];          // [slot][lane]: the slot's column maximum over the lanes above
                                  // (each lane reads and writes only its own entries)
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
__device__ __forceinline__ int key_lane(float key) { return static_cast<int>(__float_as_uint(key) & 0x1fu); }
// the float key of a packed (key, index) word
__device__ __forceinline__ float packed_key(unsigned long long pk) {
  const uint32_t u = static_cast<uint32_t>(pk >> 32);
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Per-window results of one side (row or column) of a tile.
struct GroupOut {
  unsigned long long* best;
  int32_t* ncnt;
  unsigned long long* near;
};
__device__ __forceinline__ GroupOut group_out(const WinArrays& wa, int64_t wb) {
  return GroupOut{wa.best + wb, wa.ncnt + wb, wa.near + wb * kCand};
}
// Merge candidate group pk into window w's maximum (returns the previous one).
__device__ __forceinline__ unsigned long long offer_max(const GroupOut& o, int w, unsigned long long pk) {
  return atomicMax(&o.best[w], pk);
}
// Whichever of pk and the previous maximum `old` lost is kept as a near-tie
// candidate when its key is within kNearTie of the winner's: every group within
// kNearTie of the final maximum is then either the maximum or was offered to
// the list.  A full list keeps its kCand largest entries.
__device__ __noinline__ void offer_near(const GroupOut& o, int w, unsigned long long pk, unsigned long long old) {
  const unsigned long long lo = old < pk ? old : pk;
  if (lo == 0ull) return;
  const unsigned long long hi = old < pk ? pk : old;
  if (packed_key(lo) < packed_key(hi) - kNearTie) return;
  unsigned long long* slot = o.near + static_cast<int64_t>(w) * kCand;
  const int s = atomicAdd(&o.ncnt[w], 1);
  if (s < kCand) {
    slot[s] = lo;
    return;
  }
  // full: replace the smallest entry if lo is larger (a few tries under contention)
  for (int tries = 0; tries < kCand; ++tries) {
    int at = 0;
    unsigned long long mn = ~0ull;
    for (int c = 0; c < kCand; ++c) {
      const unsigned long long v = *reinterpret_cast<volatile unsigned long long*>(slot + c);
      if (v < mn) {
        mn = v;
        at = c;
      }
    }
    if (mn >= lo || atomicCAS(slot + at, mn, lo) == mn) return;
  }
}
__device__ __forceinline__ unsigned long long umax64_mp(unsigned long long a, unsigned long long b) { return a > b ? a : b; }
__device__ __forceinline__ void offer(const GroupOut& o, int w, unsigned long long pk) {
  offer_near(o, w, pk, offer_max(o, w, pk));
}

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

// Merge the 32 buffered rows and lane-0 column exits into the profile.  Buffer
// step u belongs to row base + u and to columns base + u + d0 (+ 256).  A row
// maximum from lane t' names the group of columns row + d0 (+ 256) + 8 t' + v;
// a column maximum from lane t' the group of rows base + u - 8 t' - 7 + v
// (v = 0 .. 7, either half).
__device__ __forceinline__ void flush_chunk(MpWarpSmem& w, int base, int d0, int l, const GroupOut& rows,
                                            const GroupOut& cols, int lane) {
  __syncwarp();
  const int ir = base + lane;
  float bk = kEmpty;
#pragma unroll
  for (int u = 0; u < 32; u += 2) bk = max3f(bk, w.rowbuf[u][lane], w.rowbuf[u + 1][lane]);  // row `lane`, every source lane u
  const float2 ck = w.colbuf[lane];
  const int ja = ir + d0;
  // the three merges are issued before any result is used (one round trip)
  const int tg = static_cast<int>(__float_as_uint(bk) & 0x3fu);  // source lane + 32 half
  const bool vr = bk > kKeyFloor, va = ck.x > kKeyFloor && ja < l, vb = ck.y > kKeyFloor && ja + kHalf < l;
  const unsigned long long pr = tsk_pack(untag_key(bk), ir + d0 + (tg >> 5) * kHalf + kVh * (tg & 31));
  const unsigned long long pa = tsk_pack(untag_key(ck.x), ir - kVh * key_lane(ck.x) - (kVh - 1));
  const unsigned long long pb = tsk_pack(untag_key(ck.y), ir - kVh * key_lane(ck.y) - (kVh - 1));
  const bool cr = vr && bk > -kCloseKey, ca = va && ck.x > -kCloseKey, cb = vb && ck.y > -kCloseKey;
  if (cr || ca || cb) {
    const unsigned long long orr = vr ? offer_max(rows, ir, pr) : 0ull;
    const unsigned long long oa = va ? offer_max(cols, ja, pa) : 0ull;
    const unsigned long long ob = vb ? offer_max(cols, ja + kHalf, pb) : 0ull;
    if (cr) offer_near(rows, ir, pr, orr);
    if (ca) offer_near(cols, ja, pa, oa);
    if (cb) offer_near(cols, ja + kHalf, pb, ob);
  } else {  // no close match: the results are not needed (fire and forget)
    if (vr) atomicMax(&rows.best[ir], pr);
    if (va) atomicMax(&cols.best[ja], pa);
    if (vb) atomicMax(&cols.best[ja + kHalf], pb);
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
  const float* __restrict__ invc = AB ? a.wa.inv + wbc : inv;
  const float* __restrict__ dfc = AB ? a.wa.df + wbc : df;
  const float* __restrict__ dgc = AB ? a.wa.dg + wbc : dg;
  const GroupOut rows = group_out(a.wa, wb), cols = group_out(a.wa, AB ? wbc : wb);
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

  // ---- column state for the first row: slot v <-> columns r0 + dA + v (a) and + 256 (b);
  // ck: the column's maximum over this lane's rows so far (untagged), in: its
  // maximum over the lanes above (tagged with the lane it came from)
  float2 cdf2[kVh], cdg2[kVh], cinv2[kVh];
  float ckA[kVh], ckB[kVh];
  const unsigned ltag = static_cast<unsigned>(lane), ltagb = ltag | 32u;
#pragma unroll
  for (int v = 0; v < kVh; ++v) {
    const int j = r0 + dA + v;
    cdf2[v] = make_float2(dfc[j], dfc[j + kHalf]);
    cdg2[v] = make_float2(dgc[j], dgc[j + kHalf]);
    cinv2[v] = make_float2(invc[j], invc[j + kHalf]);
    ckA[v] = kEmpty;
    ckB[v] = kEmpty;
    w.inbuf[v][lane] = make_float2(kEmpty, kEmpty);
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
    float* rowp = &w.rowbuf[lane][sb];
    // keys of one row (slot c = (v + sr) % 8 holds the column of diagonal v), with
    // the covariance advanced to the next row
    auto row_keys = [&](int sr, int i, float2 rdf2, float2 rdg2, float2 rinv2, float (&kA)[kVh],
                        float (&kB)[kVh]) {
#pragma unroll
      for (int v = 0; v < kVh; ++v) {
        const int c = (v + sr) & (kVh - 1);
        const float2 t = __fmul2_rn(cov2[v], cinv2[c]);
        const float2 r = __ffma2_rn(t, rinv2, kMinusOne2);  // rho - 1: full relative precision near rho = 1
        float ka = r.x;
        float kb = r.y;
        if (MASKED) {
          const bool rowok = i < rEnd;
          ka = (rowok && i + dA + v < l) ? ka : kEmpty;
          kb = (rowok && i + dA + kHalf + v < l) ? kb : kEmpty;
        }
        kA[v] = ka;
        kB[v] = kb;
        cov2[v] = __ffma2_rn(cdg2[c], rdf2, cov2[v]);
        cov2[v] = __ffma2_rn(cdf2[c], rdg2, cov2[v]);
      }
      const float rka = fmaxf(max3f(max3f(max3f(kA[0], kA[1], kA[2]), kA[3], kA[4]), kA[5], kA[6]), kA[7]);
      const float rkb = fmaxf(max3f(max3f(max3f(kB[0], kB[1], kB[2]), kB[3], kB[4]), kB[5], kB[6]), kB[7]);
      rowp[sr] = fmaxf(tag_key(rka, ltag), tag_key(rkb, ltagb));
    };
    // the column in slot sr leaves the lane with its maximum over this lane's
    // rows (la, lb; tagged here) merged with the one it brought from above; it
    // goes to lane - 1 (lane 0's is complete for this band) and the column
    // entering from the ring takes the slot
    auto exit_column = [&](int sr, int s, float la, float lb, float2 in) {
      const float oa = fmaxf(in.x, tag_key(la, ltag));
      const float ob = fmaxf(in.y, tag_key(lb, ltag));
      const float ia = __shfl_down_sync(TSK_FULL_MASK, oa, 1);
      const float ib = __shfl_down_sync(TSK_FULL_MASK, ob, 1);
      if (lane == 0) w.colbuf[s] = make_float2(oa, ob);
      w.inbuf[sr][lane] = make_float2((lane == 31) ? kEmpty : ia, (lane == 31) ? kEmpty : ib);
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
      // maxima over the lanes above of the two columns leaving this group's rows
      // (stored by this lane when they arrived, 8 rows ago), read ahead of use
      const float2 inS0 = w.inbuf[s0][lane], inS1 = w.inbuf[s0 + 1][lane];
      float k0A[kVh], k0B[kVh], k1A[kVh], k1B[kVh];
      row_keys(s0, i0, make_float2(rf4.x, rf4.y), make_float2(rg4.x, rg4.y), make_float2(ri4.x, ri4.y), k0A, k0B);
      // slot s0 leaves after row s0: its last key is diagonal 0 of row s0
      exit_column(s0, sb + s0, fmaxf(ckA[s0], k0A[0]), fmaxf(ckB[s0], k0B[0]), inS0);
      row_keys(s0 + 1, i0 + 1, make_float2(rf4.z, rf4.w), make_float2(rg4.z, rg4.w), make_float2(ri4.z, ri4.w),
               k1A, k1B);
#pragma unroll
      for (int c = 0; c < kVh; ++c) {
        if (c == s0) {  // the column that entered after row s0 has only row s0 + 1's key (diagonal 7)
          ckA[c] = k1A[kVh - 1];
          ckB[c] = k1B[kVh - 1];
        } else if (c == ((s0 + kVh - 1) & (kVh - 1))) {  // entered after row s0 - 1: diagonals 7, 6
          ckA[c] = fmaxf(k0A[kVh - 1], k1A[kVh - 2]);
          ckB[c] = fmaxf(k0B[kVh - 1], k1B[kVh - 2]);
        } else {
          ckA[c] = max3f(ckA[c], k0A[(c - s0) & (kVh - 1)], k1A[(c - s0 - 1) & (kVh - 1)]);
          ckB[c] = max3f(ckB[c], k0B[(c - s0) & (kVh - 1)], k1B[(c - s0 - 1) & (kVh - 1)]);
        }
      }
      exit_column(s0 + 1, sb + s0 + 1, ckA[s0 + 1], ckB[s0 + 1], inS1);
    }
    }
    flush_chunk(w, r0 + S0, d0, l, rows, cols, lane);
  }
  cp_async_wait_all();
  __syncwarp();
  // columns still inside the band: slot v <-> columns r0 + nsteps + dA + v (+ 256).
  // The walk ends after an 8-row block, whose last row sent slot 7's column on:
  // the column now in slot 7 has no rows in this lane yet.
  ckA[kVh - 1] = kEmpty;
  ckB[kVh - 1] = kEmpty;
#pragma unroll
  for (int v = 0; v < kVh; ++v) {
    const int j = r0 + nsteps + dA + v;
    const int row0 = r0 + nsteps + lane * kVh + v - (kVh - 1);  // = j - d0 - 7
    const float2 in = w.inbuf[v][lane];
    const float fa = fmaxf(in.x, tag_key(ckA[v], ltag));
    const float fb = fmaxf(in.y, tag_key(ckB[v], ltag));
    if (fa > kKeyFloor && j < l) {
      const unsigned long long pk = tsk_pack(untag_key(fa), row0 - kVh * key_lane(fa));
      if (fa > -kCloseKey) offer(cols, j, pk); else atomicMax(&cols.best[j], pk);
    }
    if (fb > kKeyFloor && j + kHalf < l) {
      const unsigned long long pk = tsk_pack(untag_key(fb), row0 - kVh * key_lane(fb));
      if (fb > -kCloseKey) offer(cols, j + kHalf, pk); else atomicMax(&cols.best[j + kHalf], pk);
    }
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
// 4. refinement: exact distance to each window's nearest candidate
//
// The diagonal kernel names groups of 8 consecutive candidate windows of the
// partner stream: the window's maximum's group and its near-tie groups.  Each
// group's windows are scored with float32 sliding dot products of the centred
// query window (c = sum_t a_t (y_t - ref) - (mean_j - ref) sum_t a_t, the
// anchors' algebra), the group's best is re-scored exactly
// (compensated sums), and the exact best over the groups is the neighbour
// (lowest index on ties).  Constant candidates are left to the
// constant-window rule.
// ---------------------------------------------------------------------------
template <typename TX>
struct GroupScan;

template <>
struct GroupScan<float> {
  // scores k[v] = rho(i, p + v) * ||x_i - mean|| of group [p, p + 8) for window
  // i; -FLT_MAX for windows that are not admissible (outside the stream, inside
  // the exclusion zone, constant)
  static __device__ void scores(const float* __restrict__ x, int i, const float* __restrict__ xp, int p, int m,
                                double mu_i, const double* __restrict__ mup, const float* __restrict__ invp, int lp,
                                int excl, bool ab, float (&ks)[kVh]) {
    const float mih = static_cast<float>(mu_i), mil = static_cast<float>(mu_i - static_cast<double>(mih));
    const int pc = max(p, 0);
    const float ref = xp[pc];
    float acc[kVh], win[kVh];
#pragma unroll
    for (int v = 0; v < kVh; ++v) {
      acc[v] = 0.f;
      const int q = p + v;
      win[v] = (q >= 0 && q < lp + m - 1) ? __fsub_rn(xp[q], ref) : 0.f;
    }
    // win[s & 7] holds sample p + s (shifted by ref) for the 8 samples in use
    const int np = lp + m - 1;
    float sa = 0.f;
    int t0 = 0;
    for (; t0 + kVh <= m; t0 += kVh) {
#pragma unroll
      for (int u = 0; u < kVh; ++u) {
        const float at = __fsub_rn(__fsub_rn(x[i + t0 + u], mih), mil);
        sa = __fadd_rn(sa, at);
#pragma unroll
        for (int v = 0; v < kVh; ++v) acc[v] = __fmaf_rn(at, win[(v + u) & (kVh - 1)], acc[v]);
        const int q = p + t0 + u + kVh;  // replaces sample p + t0 + u, no longer used
        win[u] = (q >= 0 && q < np) ? __fsub_rn(xp[q], ref) : 0.f;
      }
    }
    for (int t = t0; t < m; ++t) {
      const float at = __fsub_rn(__fsub_rn(x[i + t], mih), mil);
      sa = __fadd_rn(sa, at);
#pragma unroll
      for (int v = 0; v < kVh; ++v) {
        const int q = p + v + t;
        acc[v] = __fmaf_rn(at, (q >= 0 && q < np) ? __fsub_rn(xp[q], ref) : 0.f, acc[v]);
      }
    }
#pragma unroll
    for (int v = 0; v < kVh; ++v) {
      const int j = p + v;
      ks[v] = -FLT_MAX;
      if (j < 0 || j >= lp || (!ab && abs(i - j) < excl) || invp[j] == 0.f) continue;
      const float c = acc[v] - static_cast<float>(mup[j] - static_cast<double>(ref)) * sa;
      ks[v] = c * invp[j];  // rho * norm_i: same scale for every candidate of window i
    }
  }
  // best admissible window of the group (-1 if none), lowest index on ties
  static __device__ int best(const float* __restrict__ x, int i, const float* __restrict__ xp, int p, int m,
                             double mu_i, const double* __restrict__ mup, const float* __restrict__ invp, int lp,
                             int excl, bool ab, float* key = nullptr) {
    float ks[kVh];
    scores(x, i, xp, p, m, mu_i, mup, invp, lp, excl, ab, ks);
    int bj = -1;
    float bk = 0.f;
#pragma unroll
    for (int v = 0; v < kVh; ++v)
      if (ks[v] > -FLT_MAX && (bj < 0 || ks[v] > bk)) {
        bj = p + v;
        bk = ks[v];
      }
    if (key) *key = bk;
    return bj;
  }
};

template <>
struct GroupScan<double> {
  static __device__ int best(const double* __restrict__ x, int i, const double* __restrict__ xp, int p, int m,
                             double mu_i, const double* __restrict__ mup, const float* __restrict__ invp, int lp,
                             int excl, bool ab, float* key = nullptr) {
    int bj = -1;
    double bk = 0.0;
    for (int v = 0; v < kVh; ++v) {
      const int j = p + v;
      if (j < 0 || j >= lp || (!ab && abs(i - j) < excl) || invp[j] == 0.f) continue;
      double c = 0.0;
      for (int t = 0; t < m; ++t) c = fma(x[i + t] - mu_i, xp[j + t], c);
      const double k = c * static_cast<double>(invp[j]);
      if (bj < 0 || k > bk) {
        bj = j;
        bk = k;
      }
    }
    if (key) *key = static_cast<float>(bk);
    return bj;
  }
};

template <typename TX, typename TP, bool AB>
__global__ void __launch_bounds__(256) k_mp_refine(const TX* __restrict__ X, const TX* __restrict__ X2, int split,
                                                   const int64_t* __restrict__ xoff,
                                                   const int32_t* __restrict__ len, const uint8_t* __restrict__ smask,
                                                   const int64_t* __restrict__ woff, int n_streams, int64_t total, int m,
                                                   int excl, int exact64, WinArrays wa, TP* __restrict__ P,
                                                   int32_t* __restrict__ I, TP* __restrict__ P2,
                                                   int32_t* __restrict__ I2, int keep_old = 0,
                                                   int64_t* __restrict__ rescan = nullptr,
                                                   unsigned int* __restrict__ rescan_n = nullptr) {
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
  double dist = INFINITY;
  if (exact64) {
    const int b = wa.bidx[wb + i];  // initialised to 0x7f7f7f7f (no neighbour)
    j = (b >= lp) ? -1 : b;
    if (j >= 0) {
      if (wa.inv[wbp + j] == 0.f) {
        dist = sqm;
      } else {
        const double rho = tsk::window_rho(x, i, xp, j, m, wa.mu[wb + i], wa.mu[wbp + j]);
        dist = sqrt(fmax(0.0, 2.0 * m * (1.0 - rho)));
      }
    }
  } else {
    const int64_t wi = wb + i;
    const unsigned long long pk = wa.best[wi];
    if (keep_old && pk && wa.ncnt[wi] == 0) {
      // incremental update: a maximum still at the old value it started from (no
      // group beat it or came near) keeps the old result, unless the
      // constant-window rule now gives a nearer window
      const int jo = Iout[eo];
      const float po = static_cast<float>(Pout[eo]);
      if (jo >= 0 && jo < lp) {
        const float key = wa.inv[wbp + jo] == 0.f ? -1.f : static_cast<float>(-(static_cast<double>(po) * po) / (2.0 * m));
        if (tsk_pack(key, jo) == pk && !(jc >= 0 && (sqm < po || (sqm == po && jc < jo)))) return;
      }
    }
    if (pk) {
      // the maximum's group and the near-tie groups within kNearTie of it
      int grp[1 + kCand];
      int ng = 0;
      grp[ng++] = tsk_unpack_idx(pk);
      const float k0 = packed_key(pk);
      const int nc = min(wa.ncnt[wi], kCand);
      for (int c = 0; c < nc; ++c) {
        const unsigned long long q = wa.near[wi * kCand + c];
        const int g = tsk_unpack_idx(q);
        bool dup = packed_key(q) < k0 - kNearTie;
        for (int e = 0; e < ng; ++e) dup |= grp[e] == g;
        if (!dup) grp[ng++] = g;
      }
      const double* mup = wa.mu + wbp;
      const float* invp = wa.inv + wbp;
      // each group's best by float32 sliding dot products; correlations rho ~ key / ||x_i - mean||
      int gj[1 + kCand];
      float gr[1 + kCand];
      int nv = 0;
      float rmax = -2.f;
      const float inv_i = wa.inv[wb + i];
      for (int c = 0; c < ng; ++c) {
        float kg = 0.f;
        const int jg = GroupScan<TX>::best(x, i, xp, grp[c], m, wa.mu[wb + i], mup, invp, lp, excl, AB, &kg);
        if (jg < 0) continue;
        gj[nv] = jg;
        gr[nv] = kg * inv_i;
        rmax = fmaxf(rmax, gr[nv]);
        ++nv;
      }
      double best_rho = -2.0;
      if (rmax < kExactRho) {
        // no close match: float32 resolves rho to ~1e-6, 1e-5 of the distance
        for (int c = 0; c < nv; ++c)
          if (gr[c] > best_rho || (gr[c] == best_rho && gj[c] < j)) {
            best_rho = gr[c];
            j = gj[c];
          }
      } else {
        for (int c = 0; c < nv; ++c) {
          const double rho = tsk::window_rho(x, i, xp, gj[c], m, wa.mu[wb + i], mup[gj[c]]);
          if (rho > best_rho || (rho == best_rho && gj[c] < j)) {
            best_rho = rho;
            j = gj[c];
          }
        }
      }
      if (j >= 0) dist = sqrt(fmax(0.0, 2.0 * m * (1.0 - fmin(1.0, best_rho))));
      // near ties decide the bar only for close matches (error ~ 1e-6 / (1 - rho));
      // a quiet window's keys carry the recurrence's error of the loud ones
      const double gap = 1.0 - best_rho;
      const float nloud = fmaxf(__uint_as_float(wa.nmax[q]), __uint_as_float(wa.nmax[p]));
      const bool quiet = wa.inv[wi] > 0.f && kQuietNorm * nloud * wa.inv[wi] > 1.f;
      if (rescan && j >= 0 && gap > kRescanExact &&
          (gap < kRescanGap || (wa.ncnt[wi] > kCand && gap < 5e-3) || quiet))
        rescan[atomicAdd(rescan_n, 1u)] = e;
    }
  }
  if (jc >= 0 && (sqm < dist || (sqm == dist && jc < j))) { dist = sqm; j = jc; }
  Pout[eo] = static_cast<TP>(dist);
  Iout[eo] = j;
}

// ---------------------------------------------------------------------------
// 5. whole-row rescan of the windows the refinement listed: near-exact matches
// (distance below the bar's floor) and windows whose near-tie list overflowed.
// One block per window: a first float32 sweep over every admissible partner
// window (groups of 8, sliding dot products) finds the best score, a second
// sweep re-scores exactly (compensated sums) every window within kRescanTol of
// it.  The exact best, lowest index on ties, replaces the refinement's result;
// the constant-window rule applies as there.  float32 series only.
// ---------------------------------------------------------------------------
template <bool AB>
__global__ void __launch_bounds__(kRescanThreads) k_mp_rescan(const float* __restrict__ X, const float* __restrict__ X2, int split,
                                                   const int64_t* __restrict__ xoff, const int32_t* __restrict__ len,
                                                   const int64_t* __restrict__ woff, int n_streams, int m, int excl,
                                                   WinArrays wa, float* __restrict__ P, int32_t* __restrict__ I,
                                                   float* __restrict__ P2, int32_t* __restrict__ I2,
                                                   const int64_t* __restrict__ rescan,
                                                   const unsigned int* __restrict__ rescan_n) {
  constexpr int kW = kRescanThreads / 32;
  __shared__ float skmax[kW];
  __shared__ double srho[kW];
  __shared__ int sj[kW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long n = static_cast<long long>(*rescan_n);
  for (long long r = blockIdx.x; r < n; r += gridDim.x) {
    const int64_t e = rescan[r];
    const int q = tsk_find_segment<int64_t>(xoff, n_streams, e);
    float* Pout = P;
    int32_t* Iout = I;
    int64_t eo = e;
    if (AB && q >= split) {
      Pout = P2;
      Iout = I2;
      eo = e - xoff[split];
    }
    const int i = static_cast<int>(e - xoff[q]);
    const int l = len[q] - m + 1;
    const int p = AB ? (q < split ? q + split : q - split) : q;
    const int lp = len[p] - m + 1;
    const int64_t wb = woff[q], wbp = woff[p];
    const float* x = AB ? stream_base(X, X2, xoff, split, q) : X + xoff[q];
    const float* xp = AB ? stream_base(X, X2, xoff, split, p) : x;
    const double mu_i = wa.mu[wb + i];
    const double* mup = wa.mu + wbp;
    const float* invp = wa.inv + wbp;
    const int ex = AB ? 0 : excl;
    // sweep 1: the best float32 score (the block's threads take groups of 8 windows in turn)
    float kmax = -FLT_MAX;
    for (int g = tid * kVh; g < lp; g += kRescanThreads * kVh) {
      float ks[kVh];
      GroupScan<float>::scores(x, i, xp, g, m, mu_i, mup, invp, lp, ex, AB, ks);
#pragma unroll
      for (int v = 0; v < kVh; ++v) kmax = fmaxf(kmax, ks[v]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kmax = fmaxf(kmax, __shfl_xor_sync(TSK_FULL_MASK, kmax, o));
    if (lane == 0) skmax[warp] = kmax;
    __syncthreads();
    kmax = skmax[0];
#pragma unroll
    for (int w = 1; w < kW; ++w) kmax = fmaxf(kmax, skmax[w]);
    if (kmax == -FLT_MAX) {  // no non-constant partner: the refinement's result stands
      __syncthreads();       // skmax is rewritten by the next row
      continue;
    }
    const float thr = kmax - kRescanTol / fmaxf(wa.inv[wb + i], FLT_MIN);
    // sweep 2: exact scores of every window within the tolerance
    double brho = -2.0;
    int bj = INT_MAX;
    for (int g = tid * kVh; g < lp; g += kRescanThreads * kVh) {
      float ks[kVh];
      GroupScan<float>::scores(x, i, xp, g, m, mu_i, mup, invp, lp, ex, AB, ks);
#pragma unroll
      for (int v = 0; v < kVh; ++v) {
        if (ks[v] < thr) continue;
        const int j = g + v;
        const double rho = tsk::window_rho(x, i, xp, j, m, mu_i, mup[j]);
        if (rho > brho || (rho == brho && j < bj)) {
          brho = rho;
          bj = j;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double orho = __shfl_xor_sync(TSK_FULL_MASK, brho, o);
      const int oj = __shfl_xor_sync(TSK_FULL_MASK, bj, o);
      if (orho > brho || (orho == brho && oj < bj)) {
        brho = orho;
        bj = oj;
      }
    }
    if (lane == 0) {
      srho[warp] = brho;
      sj[warp] = bj;
    }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < kW; ++w)
        if (srho[w] > brho || (srho[w] == brho && sj[w] < bj)) {
          brho = srho[w];
          bj = sj[w];
        }
      {  // the refinement's own neighbour stays a candidate (never a worse result)
        const int j0 = Iout[eo];
        if (j0 >= 0 && j0 < lp && (AB || abs(i - j0) >= excl) && invp[j0] != 0.f) {
          const double rho0 = tsk::window_rho(x, i, xp, j0, m, mu_i, mup[j0]);
          if (rho0 > brho || (rho0 == brho && j0 < bj)) {
            brho = rho0;
            bj = j0;
          }
        }
      }
      if (bj != INT_MAX) {
        double dist = sqrt(fmax(0.0, 2.0 * m * (1.0 - fmin(1.0, brho))));
        int j = bj;
        // the constant-window rule (lowest admissible constant window at sqrt(m))
        int jc = -1;
        if (wa.constcnt[p] > 0) {
          const int f = wa.nxt[wbp];
          if (AB) {
            if (f < lp) jc = f;
          } else if (f <= i - excl) {
            jc = f;
          } else if (i + excl < l) {
            const int gg = wa.nxt[wb + i + excl];
            if (gg < l) jc = gg;
          }
        }
        const double sqm = sqrt(static_cast<double>(m));
        if (jc >= 0 && (sqm < dist || (sqm == dist && jc < j))) {
          dist = sqm;
          j = jc;
        }
        Pout[eo] = static_cast<float>(dist);
        Iout[eo] = j;
      }
    }
    __syncthreads();  // skmax, srho and sj are rewritten by the next row
  }
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
  wa.nmax = cv.take<unsigned int>(n_streams);
  if (!f64) {
    wa.ncnt = cv.take<int32_t>(W);
    wa.near = cv.take<unsigned long long>(W * kCand);
  }
  unsigned long long* counter = cv.take<unsigned long long>(1);
  if (f64) {
    wa.inv64 = cv.take<double>(W);
    wa.bidx = cv.take<int32_t>(W);
  }
  // windows listed for a whole-row rescan (float32 series)
  int64_t* rescan = nullptr;
  unsigned int* rescan_n = nullptr;
  if (!f64 && std::is_same<TX, float>::value) {
    rescan = cv.take<int64_t>(W);
    rescan_n = cv.take<unsigned int>(1);
  }
  cudaStream_t st = ctx->stream;
  if (rescan_n) TSK_CUDA_TRY(ctx, cudaMemsetAsync(rescan_n, 0, sizeof(unsigned int), st));
  TSK_CUDA_TRY(ctx, cudaMemsetAsync(wa.best, 0, sizeof(unsigned long long) * W, st));
  TSK_CUDA_TRY(ctx, cudaMemsetAsync(wa.constcnt, 0, sizeof(int32_t) * n_streams, st));
  TSK_CUDA_TRY(ctx, cudaMemsetAsync(wa.nmax, 0, sizeof(unsigned int) * n_streams, st));
  if (!f64) TSK_CUDA_TRY(ctx, cudaMemsetAsync(wa.ncnt, 0, sizeof(int32_t) * W, st));
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
                                                      static_cast<float*>(P2), I2, 0, rescan, rescan_n);
    else
      k_mp_refine<TX, float, false><<<g, 256, 0, st>>>(X, X2, split, plan.xoff, plan.len, plan.smask, plan.woff,
                                                       n_streams, total, m, excl, 0, wa, static_cast<float*>(P), I,
                                                       nullptr, nullptr, 0, rescan, rescan_n);
    TSK_LAUNCH_CHECK(ctx, "k_mp_refine");
    if constexpr (std::is_same<TX, float>::value) {
      if (rescan) {
        const unsigned gr = static_cast<unsigned>(ctx->sm_count * 2);  // two resident blocks per SM
        if (ab)
          k_mp_rescan<true><<<gr, kRescanThreads, 0, st>>>(X, X2, split, plan.xoff, plan.len, plan.woff, n_streams, m, excl, wa,
                                                static_cast<float*>(P), I, static_cast<float*>(P2), I2, rescan,
                                                rescan_n);
        else
          k_mp_rescan<false><<<gr, kRescanThreads, 0, st>>>(X, X2, split, plan.xoff, plan.len, plan.woff, n_streams, m, excl,
                                                 wa, static_cast<float*>(P), I, nullptr, nullptr, rescan, rescan_n);
        TSK_LAUNCH_CHECK(ctx, "k_mp_rescan");
      }
    }
  }
  return TSK_OK;
}

// ---------------------------------------------------------------------------
// 6. incremental profile after point updates (Sec. III-C point updates; the
//    streaming use of Sec. III-B)
//
// A sample t that changes moves the windows t-m+1 .. t (the affected set A).
// The distance of two windows outside A is unchanged, so for such a window i
// whose old neighbour is also outside A the new profile value is
//   min(old value, min over a in A of dist(i, a)),
// a window of A needs its whole row, and a window outside A whose old
// neighbour was in A (the set R) needs its whole row too.  The cells with a
// window of A on either side come from the diagonal kernel on work units that
// cover only those rows and columns (per band: the rows of A, and the rows
// whose columns in that band meet A); R's rows from a direct scan in groups
// of 8 windows.  The maxima start from the old values (or nothing, for A and
// R), and the refinement re-scores the winning groups exactly.
// ---------------------------------------------------------------------------
__global__ void k_upd_mark(const int4* __restrict__ runs, int n_runs, const int64_t* __restrict__ woff,
                           uint8_t* __restrict__ aflag) {
  const int r = blockIdx.x;
  if (r >= n_runs) return;
  const int4 u = runs[r];  // {stream, first window, end window, 0}
  for (int i = u.y + threadIdx.x; i < u.z; i += blockDim.x) aflag[woff[u.x] + i] = 1;
}

// Start each touched window's maximum from its old profile value, or empty
// for A and R; R's windows are listed for the row scan.
__global__ void k_upd_init(const int64_t* __restrict__ xoff, const int32_t* __restrict__ len,
                           const uint8_t* __restrict__ smask, const int64_t* __restrict__ woff, int n_streams,
                           int64_t total, int m, const float* __restrict__ P, const int32_t* __restrict__ I,
                           const uint8_t* __restrict__ aflag, WinArrays wa, int32_t* __restrict__ rlist,
                           int32_t* __restrict__ rcount) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int q = tsk_find_segment<int64_t>(xoff, n_streams, e);
  if (!smask[q]) return;
  const int l = len[q] - m + 1;
  const int i = static_cast<int>(e - xoff[q]);
  if (i >= l) return;
  const int64_t w = woff[q] + i;
  wa.ncnt[w] = 0;
  unsigned long long pk = 0ull;
  if (!aflag[w]) {
    const int j = I[e];
    if (j >= 0 && j < l && aflag[woff[q] + j]) {
      const int at = atomicAdd(&rcount[q], 1);  // R of stream q: rlist[woff[q] + k]
      rlist[woff[q] + at] = i;
    } else if (j >= 0 && j < l) {
      // the old value as a key: rho - 1 = -P^2 / (2m); a constant neighbour as the
      // diagonal kernel sees it (rho = 0), the constant-window rule restores it
      const float p = P[e];
      const float key = wa.inv[woff[q] + j] == 0.f ? -1.f : static_cast<float>(-(static_cast<double>(p) * p) / (2.0 * m));
      pk = tsk_pack(key, j);
    }
  }
  wa.best[w] = pk;
}

// Whole rows of the windows in R on the FP32 pipe (m > 512): one warp per
// window, lanes over groups of 8 candidates, every group's best offered (near
// ties kept).
__global__ void __launch_bounds__(256) k_upd_rowscan(const float* __restrict__ X, const int64_t* __restrict__ xoff,
                                                     const int32_t* __restrict__ len, const int64_t* __restrict__ woff,
                                                     int n_streams, int m, int excl, WinArrays wa,
                                                     const int32_t* __restrict__ rlist,
                                                     const int32_t* __restrict__ rcount) {
  const int lane = threadIdx.x & 31;
  const int nwarps = static_cast<int>(gridDim.x) * (blockDim.x >> 5);
  const int wg = static_cast<int>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  for (int q = 0; q < n_streams; ++q) {
    const int nr = rcount[q];
    const int l = len[q] - m + 1;
    const float* x = X + xoff[q];
    const int64_t wb = woff[q];
    const GroupOut o = group_out(wa, wb);
    for (int k = wg; k < nr; k += nwarps) {
      const int i = rlist[wb + k];
      const float inv_i = wa.inv[wb + i];
      for (int p = lane * kVh; p < l; p += 32 * kVh) {
        float key = 0.f;
        const int j = GroupScan<float>::best(x, i, x, p, m, wa.mu[wb + i], wa.mu + wb, wa.inv + wb, l, excl, false, &key);
        if (j >= 0) offer(o, i, tsk_pack(key * inv_i - 1.f, p));
      }
    }
  }
}

// Whole rows of the windows in R on the tensor cores (m <= 512): one CTA per
// (stream, chunk of 1024 windows), the stream's R windows as queries in batches
// of 16 against the chunk's Hankel matrix (tsk_tc.cuh); each query's best
// window of the chunk is offered (near ties kept).
constexpr int kUpdPairs = kWinChunk + tsk::kTcMaxKT * 16 + 32;

size_t upd_tc_smem_bytes() {
  return 2 * static_cast<size_t>(kUpdPairs) * sizeof(uint32_t) + 2 * static_cast<size_t>(kWinChunk) * sizeof(float) +
         static_cast<size_t>(tsk::kTcMaxKT) * 2 * 32 * sizeof(uint4);
}

__global__ void __launch_bounds__(256, 2) k_upd_rowscan_tc(const float* __restrict__ X, const int64_t* __restrict__ xoff,
                                                           const int32_t* __restrict__ len,
                                                           const int64_t* __restrict__ woff,
                                                           const int64_t* __restrict__ chunk_prefix, int n_streams,
                                                           int64_t total_chunks, int m, int excl, WinArrays wa,
                                                           const int32_t* __restrict__ rlist,
                                                           const int32_t* __restrict__ rcount) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t* Hp = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* Lp = Hp + kUpdPairs;
  float* wmean = reinterpret_cast<float*>(Lp + kUpdPairs);  // window mean - x_ref
  float* winv = wmean + kWinChunk;
  uint4* Bs = reinterpret_cast<uint4*>(winv + kWinChunk);
  __shared__ float red[8];
  __shared__ int qidx[16];
  __shared__ float qscale[16], qsum[16], qinv[16], qmh[16], qml[16];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, tq = lane & 3;
  const int KT = (m + 15) >> 4;
  for (int64_t item = blockIdx.x; item < total_chunks; item += gridDim.x) {
    const int q = tsk_find_segment<int64_t>(chunk_prefix, n_streams, item);
    const int nr = rcount[q];
    if (nr == 0) continue;
    const int l = len[q] - m + 1;
    const int t0 = static_cast<int>(item - chunk_prefix[q]) * kWinChunk;
    const int nw = min(kWinChunk, l - t0);
    const float* xs = X + xoff[q];
    const float* x = xs + t0;
    const int64_t wb = woff[q];
    const float x_ref = x[0];
    const int ns = nw + m - 1;
    // ---- stage the chunk: scale, (hi, lo) pairs, window means and inverse norms
    float amax = 0.f;
    for (int p = tid; p < ns; p += blockDim.x) amax = fmaxf(amax, fabsf(x[p] - x_ref));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(TSK_FULL_MASK, amax, o));
    if (lane == 0) red[warp] = amax;
    __syncthreads();
    amax = 0.f;
    for (int u = 0; u < 8; ++u) amax = fmaxf(amax, red[u]);
    const float sx = tsk::pow2_scale(amax);
    for (int p = tid; p < kUpdPairs; p += blockDim.x) {
      __half h0 = __float2half_rn(0.f), l0 = h0, h1 = h0, l1 = h0;
      if (p < ns) tsk::split_h((x[p] - x_ref) * sx, h0, l0);
      if (p + 1 < ns) tsk::split_h((x[p + 1] - x_ref) * sx, h1, l1);
      Hp[p] = tsk::h2_bits(h0, h1);
      Lp[p] = tsk::h2_bits(l0, l1);
    }
    for (int w = tid; w < kWinChunk; w += blockDim.x) {
      wmean[w] = w < nw ? static_cast<float>(wa.mu[wb + t0 + w] - static_cast<double>(x_ref)) : 0.f;
      winv[w] = w < nw ? wa.inv[wb + t0 + w] : 0.f;
    }
    for (int b0 = 0; b0 < nr; b0 += 16) {
      const int nb = min(16, nr - b0);
      __syncthreads();  // staging done / the previous batch's fragments no longer read
      // ---- the batch's queries: centred in float32 (two-term mean), their sum and scale
      for (int r = warp; r < nb; r += 8) {
        const int i = rlist[wb + b0 + r];
        const double mu = wa.mu[wb + i];
        const float mh = static_cast<float>(mu), ml = static_cast<float>(mu - static_cast<double>(mh));
        float sum = 0.f;
        for (int t = lane; t < m; t += 32) sum += __fsub_rn(__fsub_rn(xs[i + t], mh), ml);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(TSK_FULL_MASK, sum, o);
        if (lane == 0) {
          const float inv = wa.inv[wb + i];
          qidx[r] = i;
          qsum[r] = sum;
          qinv[r] = inv;
          qscale[r] = inv > 0.f ? 1.f / tsk::pow2_scale(1.f / inv) : 1.f;  // max |q| <= ||q|| < qscale
          qmh[r] = mh;
          qml[r] = ml;
        }
      }
      __syncthreads();
      const int NT = (nb + 7) >> 3;
      for (int e = tid; e < KT * NT * 32; e += blockDim.x) {
        const tsk::BEntry be = tsk::b_entry(e, NT);
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        if (be.slot < nb) {
          const int i = qidx[be.slot];
          const float sc = 1.f / qscale[be.slot];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int t = tsk::b_tap(be, u);
            v[u] = t < m ? __fsub_rn(__fsub_rn(xs[i + t], qmh[be.slot]), qml[be.slot]) * sc : 0.f;
          }
        }
        Bs[(be.kt * 2 + be.nt) * 32 + be.lane] = tsk::b_pack(v);
      }
      __syncthreads();
      unsigned long long best[2][2] = {{0ull, 0ull}, {0ull, 0ull}};
      for (int mt = warp; mt * 16 < nw; mt += 8) {
        float c1[2][4], c2[2][4];
        tsk::hankel_tile(Hp, Lp, Bs, mt * 16, KT, NT, lane, c1, c2);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int cc = 0; cc < 2; ++cc) {
            const int slot = nt * 8 + 2 * tq + cc;
            if (nt >= NT || slot >= nb || qinv[slot] == 0.f) continue;
            const int i = qidx[slot];
            const float back = qscale[slot] / sx;
#pragma unroll
            for (int rh = 0; rh < 2; ++rh) {
              const int w = mt * 16 + g + 8 * rh;
              const int t = t0 + w;
              if (w >= nw || abs(t - i) < excl || winv[w] == 0.f) continue;
              const float acc = __fmaf_rn(c2[nt][2 * rh + cc], 0x1p-11f, c1[nt][2 * rh + cc]) * back;
              const float cov = __fmaf_rn(-wmean[w], qsum[slot], acc);
              const float key = fminf(0.f, fmaxf(-2.f, __fmaf_rn(cov * qinv[slot], winv[w], -1.f)));
              best[nt][cc] = umax64_mp(best[nt][cc], tsk_pack(key, t));
            }
          }
      }
      const GroupOut o = group_out(wa, wb);
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          unsigned long long bb = best[nt][cc];
#pragma unroll
          for (int sh = 4; sh < 32; sh <<= 1) bb = umax64_mp(bb, __shfl_xor_sync(TSK_FULL_MASK, bb, sh));
          const int slot = nt * 8 + 2 * tq + cc;
          if (g == 0 && slot < nb && bb) offer(o, qidx[slot], bb);
        }
    }
    __syncthreads();  // shared buffers are reused by the next item
  }
}

tsk_status run_update(tsk_ctx* ctx, const float* X, int32_t n_streams, const int32_t* lens, const tsk_mp_plan& plan,
                      int32_t m, int32_t excl, float* P, int32_t* I, const std::vector<int4>& runs, char* ws) {
  // work units of the diagonal kernel, all masked: per band, the rows of each
  // affected run and the rows whose columns in that band meet it (one unit
  // when the two overlap)
  std::vector<int4> tiles;
  for (const int4& u : runs) {
    const int64_t l = static_cast<int64_t>(lens[u.x]) - m + 1;
    for (int64_t d0 = excl; d0 < l; d0 += kBand) {
      const int64_t top = l - d0;  // rows with a cell in this band
      int64_t r0 = u.y, r1 = std::min<int64_t>(u.z, top);                                   // rows in the run
      int64_t c0 = std::max<int64_t>(0, u.y - d0 - (kBand - 1)), c1 = std::min<int64_t>(u.z - d0, top);  // rows meeting it
      auto add = [&](int64_t a, int64_t b) {
        if (a < b)
          tiles.push_back(make_int4(u.x, static_cast<int>(d0), static_cast<int>(a),
                                    static_cast<int>(static_cast<uint32_t>(b) | 0x80000000u)));
      };
      if (r0 < r1 && c0 < c1 && c1 >= r0 && r1 >= c0) {
        add(std::min(r0, c0), std::max(r1, c1));
      } else {
        add(c0, c1);
        add(r0, r1);
      }
    }
  }
  tsk_carver cv(ws);
  const int64_t W = plan.total_windows;
  WinArrays wa{};
  wa.mu = cv.take<double>(W);
  wa.ss = cv.take<double>(W);
  wa.inv = cv.take<float>(W);
  wa.df = cv.take<float>(W);
  wa.dg = cv.take<float>(W);
  wa.best = cv.take<unsigned long long>(W);
  wa.nxt = cv.take<int32_t>(W);
  wa.constcnt = cv.take<int32_t>(n_streams);
  wa.nmax = cv.take<unsigned int>(n_streams);
  wa.ncnt = cv.take<int32_t>(W);
  wa.near = cv.take<unsigned long long>(W * kCand);
  unsigned long long* counter = cv.take<unsigned long long>(1);  // diagonal-kernel claims
  int32_t* rcount = cv.take<int32_t>(n_streams);                 // |R| per stream
  uint8_t* aflag = cv.take<uint8_t>(W);
  int32_t* rlist = cv.take<int32_t>(W);                          // R of stream q at woff[q]
  int64_t* rescan = cv.take<int64_t>(W);                         // windows for a whole-row rescan
  unsigned int* rescan_n = cv.take<unsigned int>(1);
  int4* d_runs = cv.take<int4>(runs.size());
  int4* d_tiles = cv.take<int4>(std::max<size_t>(tiles.size(), 1));
  cudaStream_t st = ctx->stream;
  TSK_CUDA_TRY(ctx, cudaMemsetAsync(aflag, 0, static_cast<size_t>(W), st));
  TSK_CUDA_TRY(ctx, cudaMemsetAsync(wa.constcnt, 0, sizeof(int32_t) * n_streams, st));
  TSK_CUDA_TRY(ctx, cudaMemsetAsync(wa.nmax, 0, sizeof(unsigned int) * n_streams, st));
  TSK_CUDA_TRY(ctx, cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
  TSK_CUDA_TRY(ctx, cudaMemsetAsync(rcount, 0, sizeof(int32_t) * n_streams, st));
  TSK_CUDA_TRY(ctx, cudaMemsetAsync(rescan_n, 0, sizeof(unsigned int), st));
  // (copies from pageable memory return once staged, so the vectors may go out of scope)
  TSK_CUDA_TRY(ctx, cudaMemcpyAsync(d_runs, runs.data(), sizeof(int4) * runs.size(), cudaMemcpyHostToDevice, st));
  if (!tiles.empty())
    TSK_CUDA_TRY(ctx, cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice, st));
  if (plan.total_chunks > 0) {
    const size_t smem = sizeof(double) * 2 * (kWinChunk + m + 2);
    TSK_CUDA_TRY(ctx, set_smem_limit(k_window_stats<float>, ctx->device, static_cast<int>(smem), 0));
    k_window_stats<float><<<static_cast<unsigned>(plan.total_chunks), kWinThreads, smem, st>>>(
        X, X, n_streams, plan.xoff, plan.len, plan.woff, plan.chunk_prefix, n_streams, m, 0, wa, ctx->d_err);
    TSK_LAUNCH_CHECK(ctx, "k_window_stats");
    k_next_const<<<n_streams, kWinThreads, 0, st>>>(plan.len, plan.smask, plan.woff, m, wa);
    TSK_LAUNCH_CHECK(ctx, "k_next_const");
  }
  k_upd_mark<<<static_cast<unsigned>(runs.size()), 256, 0, st>>>(d_runs, static_cast<int>(runs.size()), plan.woff, aflag);
  TSK_LAUNCH_CHECK(ctx, "k_upd_mark");
  const int64_t total = plan.total_samples;
  const unsigned gs = static_cast<unsigned>((total + 255) / 256);
  k_upd_init<<<gs, 256, 0, st>>>(plan.xoff, plan.len, plan.smask, plan.woff, n_streams, total, m, P, I, aflag, wa,
                                 rlist, rcount);
  TSK_LAUNCH_CHECK(ctx, "k_upd_init");
  if (!tiles.empty()) {
    MpArgs a{};
    a.X = X;
    a.X2 = X;
    a.split = n_streams;
    a.xoff = plan.xoff;
    a.len = plan.len;
    a.woff = plan.woff;
    a.tiles = d_tiles;
    a.counter = counter;
    a.wa = wa;
    a.total_tiles = static_cast<int64_t>(tiles.size());
    a.n_streams = n_streams;
    a.m = m;
    a.excl = excl;
    a.H = 0;
    const size_t smem = sizeof(MpWarpSmem) * kWarps;
    TSK_CUDA_TRY(ctx, set_smem_limit(k_mp_diag<float, false>, ctx->device, static_cast<int>(smem), 1));
    int per_sm = 0;
    TSK_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mp_diag<float, false>, kWarps * 32, smem));
    per_sm = std::max(per_sm, 1);
    const int64_t grid = std::min<int64_t>((a.total_tiles + kWarps - 1) / kWarps, static_cast<int64_t>(per_sm) * ctx->sm_count);
    a.total_warps = static_cast<int>(grid) * kWarps;
    k_mp_diag<float, false><<<static_cast<unsigned>(grid), kWarps * 32, smem, st>>>(a);
    TSK_LAUNCH_CHECK(ctx, "k_mp_diag");
  }
  if (m <= tsk::kTcMaxKT * 16) {
    const size_t smem = upd_tc_smem_bytes();
    TSK_CUDA_TRY(ctx, set_smem_limit(k_upd_rowscan_tc, ctx->device, static_cast<int>(smem), 2));
    int per_sm = 0;
    TSK_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_upd_rowscan_tc, 256, smem));
    const int64_t grid = std::min<int64_t>(std::max<int64_t>(plan.total_chunks, 1),
                                           static_cast<int64_t>(std::max(per_sm, 1)) * ctx->sm_count);
    k_upd_rowscan_tc<<<static_cast<unsigned>(grid), 256, smem, st>>>(X, plan.xoff, plan.len, plan.woff,
                                                                      plan.chunk_prefix, n_streams, plan.total_chunks,
                                                                      m, excl, wa, rlist, rcount);
  } else {
    k_upd_rowscan<<<static_cast<unsigned>(ctx->sm_count * 4), 256, 0, st>>>(X, plan.xoff, plan.len, plan.woff,
                                                                             n_streams, m, excl, wa, rlist, rcount);
  }
  TSK_LAUNCH_CHECK(ctx, "k_upd_rowscan");
  k_mp_refine<float, float, false><<<gs, 256, 0, st>>>(X, X, n_streams, plan.xoff, plan.len, plan.smask, plan.woff,
                                                       n_streams, total, m, excl, 0, wa, P, I, nullptr, nullptr, 1,
                                                       rescan, rescan_n);
  TSK_LAUNCH_CHECK(ctx, "k_mp_refine");
  k_mp_rescan<false><<<static_cast<unsigned>(ctx->sm_count * 2), kRescanThreads, 0, st>>>(
      X, X, n_streams, plan.xoff, plan.len, plan.woff, n_streams, m, excl, wa, P, I, nullptr, nullptr, rescan, rescan_n);
  TSK_LAUNCH_CHECK(ctx, "k_mp_rescan");
  return TSK_OK;
}

size_t update_ws_bytes(const tsk_mp_plan& plan, int32_t n_streams, size_t n_runs, size_t n_tiles_max) {
  const size_t W = static_cast<size_t>(plan.total_windows);
  return tsk_carver::bytes_for(W, 8) * 2 + tsk_carver::bytes_for(W, 4) * 3 + tsk_carver::bytes_for(W, 8) +
         tsk_carver::bytes_for(W, 4) + tsk_carver::bytes_for(n_streams, 4) + tsk_carver::bytes_for(W, 4) +
         tsk_carver::bytes_for(W * kCand, 8) + tsk_carver::bytes_for(1, 8) + tsk_carver::bytes_for(n_streams, 4) +
         tsk_carver::bytes_for(W, 1) + tsk_carver::bytes_for(W, 4) + tsk_carver::bytes_for(W, 8) +
         tsk_carver::bytes_for(1, 4) + tsk_carver::bytes_for(n_runs, 16) + tsk_carver::bytes_for(n_tiles_max, 16) +
         tsk_carver::bytes_for(n_streams, 4) + 4096;
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
       tsk_carver::bytes_for(W, 4) + tsk_carver::bytes_for(n_streams, 4) * 2 + tsk_carver::bytes_for(1, 8);
  if (plan.prec == TSK_MP_FP64)
    b += tsk_carver::bytes_for(W, 8) + tsk_carver::bytes_for(W, 4);
  else
    b += tsk_carver::bytes_for(W, 4) + tsk_carver::bytes_for(W * kCand, 8) + tsk_carver::bytes_for(W, 8) +
         tsk_carver::bytes_for(1, 4);
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

tsk_status tsk_run_mp_update(tsk_ctx* ctx, const float* X, int32_t n_streams, const int32_t* lens,
                             const tsk_mp_plan& plan, int32_t m, int32_t excl, float* P, int32_t* I,
                             const std::vector<int4>& runs, char* ws) {
  return run_update(ctx, X, n_streams, lens, plan, m, excl, P, I, runs, ws);
}

size_t tsk_mp_update_ws_bytes(const tsk_mp_plan& plan, int32_t n_streams, size_t n_runs, size_t n_tiles_max) {
  return update_ws_bytes(plan, n_streams, n_runs, n_tiles_max);
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

constexpr size_t kStaticScratchBytes = size_t(6) << 20;  // 6 MiB on every device that loads the library
constexpr int kStaticMaxWindows = 65536;                   // l = n - m + 1 at most
constexpr int kStaticMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_addr[kStaticMaxDevices] = {};

// Per-device set-up: the scratch array's device address and the kernels'
// shared-memory limits (raised to the largest size this entry point uses,
// through the same per-device cache as the context path, so neither path can
// lower a limit the other relies on).  Runs on the first call on each device.
tsk_status static_setup(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return TSK_ERR_CUDA;
    }
    const int win_smem = static_cast<int>(sizeof(double) * 2 * (kWinChunk + 4096 + 2));
    if (set_smem_limit(k_window_stats<float>, dev, win_smem, 0) != cudaSuccess ||
        set_smem_limit(k_mp_diag<float, false>, dev, static_cast<int>(sizeof(MpWarpSmem) * kWarps), 1) !=
            cudaSuccess) {
      cudaGetLastError();
      return TSK_ERR_CUDA;
    }
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return TSK_OK;
}

// Layout words of the one stream, written by the device (no host copy).
struct StaticHead {
  int64_t xoff[2], woff[2], chunk_prefix[2];
  int32_t len[1];
  uint8_t smask[4];
};

// Interior work units of band b (diagonals excl + 512 b ..): rows [0, rint) in
// runs of H; the band's triangular end is one masked unit.
__host__ __device__ inline int64_t static_band_rint(int64_t l, int64_t d0) {
  int64_t rint = l - d0 - (kBand - 1);
  if (rint < 0) rint = 0;
  return rint - rint % kChunk;
}

// One warp writes the layout words and the work list: the interior units of
// every band in band order, then one band-end unit per band.
__global__ void k_static_plan(StaticHead h, StaticHead* __restrict__ dh, int4* __restrict__ tiles, int l, int excl,
                              int H, int bands) {
  if (threadIdx.x == 0) *dh = h;
  int64_t interior = 0;
  for (int b = 0; b < bands; ++b) interior += (static_band_rint(l, excl + static_cast<int64_t>(b) * kBand) + H - 1) / H;
  for (int b = threadIdx.x; b < bands; b += blockDim.x) {
    int64_t at = 0;
    for (int c = 0; c < b; ++c) at += (static_band_rint(l, excl + static_cast<int64_t>(c) * kBand) + H - 1) / H;
    const int d0 = excl + b * kBand;
    const int64_t rint = static_band_rint(l, d0);
    for (int64_t r0 = 0; r0 < rint; r0 += H)
      tiles[at++] = make_int4(0, d0, static_cast<int>(r0), static_cast<int>(r0 + H < rint ? r0 + H : rint));
    tiles[interior + b] =
        make_int4(0, d0, static_cast<int>(rint), static_cast<int>(static_cast<uint32_t>(l - d0) | 0x80000000u));
  }
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

  // work list of the one stream (built on the device): interior units of every
  // band, then the band ends
  const int64_t e = l - excl;
  const double cells = e > 0 ? static_cast<double>(e) * (e + 1) / 2 : 0.0;
  int32_t H = static_cast<int32_t>(std::min(8192.0, std::max(2048.0, cells / (sms * 12.0 * 64.0 * kBand))));
  H = (H + kChunk - 1) / kChunk * kChunk;
  const int bands = l > excl ? static_cast<int>((l - excl + kBand - 1) / kBand) : 0;
  int64_t n_tiles = bands;
  for (int b = 0; b < bands; ++b) n_tiles += (static_band_rint(l, excl + static_cast<int64_t>(b) * kBand) + H - 1) / H;

  // carve the scratch array
  const int64_t W = (l + kPad + 3) & ~int64_t(3);
  size_t off = 0;
  const size_t o_head = off; off = align256(off + sizeof(StaticHead));
  const size_t o_mu = off; off = align256(off + 8 * W);
  const size_t o_ss = off; off = align256(off + 8 * W);
  const size_t o_inv = off; off = align256(off + 4 * W);
  const size_t o_df = off; off = align256(off + 4 * W);
  const size_t o_dg = off; off = align256(off + 4 * W);
  const size_t o_best = off; off = align256(off + 8 * W);
  const size_t o_nxt = off; off = align256(off + 4 * W);
  const size_t o_ncnt = off; off = align256(off + 4 * W);
  const size_t o_near = off; off = align256(off + 8 * kCand * W);
  const size_t o_rescan = off; off = align256(off + 8 * W);
  const size_t o_small = off; off = align256(off + 64);  // constcnt, counter, error word, rescan count, nmax
  const size_t o_tiles = off; off = align256(off + sizeof(int4) * n_tiles);
  if (off > kStaticScratchBytes) return TSK_ERR_INVALID_ARG;
  char* sb = static_cast<char*>(base);
  StaticHead h{};
  h.xoff[1] = n;
  h.woff[1] = W;
  h.chunk_prefix[1] = (l + kWinChunk - 1) / kWinChunk;
  h.len[0] = n;
  h.smask[0] = 1;
  StaticHead* dh = reinterpret_cast<StaticHead*>(sb + o_head);
  int4* tiles = reinterpret_cast<int4*>(sb + o_tiles);
  // every launch is checked before the next is issued: a failed one ends the call
  auto launched = []() { return cudaGetLastError() == cudaSuccess; };
  if (cudaMemsetAsync(sb + o_best, 0, 8 * W, stream) != cudaSuccess ||
      cudaMemsetAsync(sb + o_ncnt, 0, 4 * W, stream) != cudaSuccess ||
      cudaMemsetAsync(sb + o_small, 0, 64, stream) != cudaSuccess) {
    cudaGetLastError();
    return TSK_ERR_CUDA;
  }
  k_static_plan<<<1, 32, 0, stream>>>(h, dh, tiles, static_cast<int>(l), excl, H, bands);
  if (!launched()) return TSK_ERR_CUDA;
  WinArrays wa{};
  wa.mu = reinterpret_cast<double*>(sb + o_mu);
  wa.ss = reinterpret_cast<double*>(sb + o_ss);
  wa.inv = reinterpret_cast<float*>(sb + o_inv);
  wa.df = reinterpret_cast<float*>(sb + o_df);
  wa.dg = reinterpret_cast<float*>(sb + o_dg);
  wa.best = reinterpret_cast<unsigned long long*>(sb + o_best);
  wa.nxt = reinterpret_cast<int32_t*>(sb + o_nxt);
  wa.ncnt = reinterpret_cast<int32_t*>(sb + o_ncnt);
  wa.near = reinterpret_cast<unsigned long long*>(sb + o_near);
  wa.constcnt = reinterpret_cast<int32_t*>(sb + o_small);
  wa.nmax = reinterpret_cast<unsigned int*>(sb + o_small + 28);
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(sb + o_small + 8);
  int* err = reinterpret_cast<int*>(sb + o_small + 16);

  const size_t win_smem = sizeof(double) * 2 * (kWinChunk + m + 2);
  k_window_stats<float><<<static_cast<unsigned>(h.chunk_prefix[1]), kWinThreads, win_smem, stream>>>(
      X, X, 1, dh->xoff, dh->len, dh->woff, dh->chunk_prefix, 1, m, 0, wa, err);
  if (!launched()) return TSK_ERR_CUDA;
  k_next_const<<<1, kWinThreads, 0, stream>>>(dh->len, dh->smask, dh->woff, m, wa);
  if (!launched()) return TSK_ERR_CUDA;
  if (n_tiles > 0) {
    MpArgs a{};
    a.X = X;
    a.X2 = X;
    a.split = 1;
    a.xoff = dh->xoff;
    a.len = dh->len;
    a.woff = dh->woff;
    a.tiles = tiles;
    a.counter = counter;
    a.wa = wa;
    a.total_tiles = n_tiles;
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
    if (!launched()) return TSK_ERR_CUDA;
  }
  int64_t* rescan = reinterpret_cast<int64_t*>(sb + o_rescan);
  unsigned int* rescan_n = reinterpret_cast<unsigned int*>(sb + o_small + 24);
  k_mp_refine<float, float, false><<<static_cast<unsigned>((n + 255) / 256), 256, 0, stream>>>(
      X, X, 1, dh->xoff, dh->len, dh->smask, dh->woff, 1, n, m, excl, 0, wa, P, I, nullptr, nullptr, 0, rescan,
      rescan_n);
  if (!launched()) return TSK_ERR_CUDA;
  k_mp_rescan<false><<<static_cast<unsigned>(sms * 2), kRescanThreads, 0, stream>>>(X, X, 1, dh->xoff, dh->len, dh->woff, 1, m,
                                                                         excl, wa, P, I, nullptr, nullptr, rescan,
                                                                         rescan_n);
  if (!launched()) return TSK_ERR_CUDA;
  return TSK_OK;
}
