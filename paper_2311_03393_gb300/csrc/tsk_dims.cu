// Discord dimension detection (Alg. 3) for the discords of the time-detection
// phase, and the gather of each chosen raw stream for the optional refinement.
//
// For discord r of series s at window i* in sketch stream g*, every raw stream
// j of the group J_g* = {j : R[j, g*] != 0} is scored by the 1NN distance of
// its own window i* (Def. 6 at a single row: self-join exclusion |t - i*| <
// excl, or, in the train/test form, against every window of the training
// series' stream j), and j* is the first j (ascending) whose score exceeds
// every earlier one, starting from 0.
//
// Pipeline per call:
//   1. k_dd_query   one warp per (series, discord, stream of its group): the
//                   discord window centred in float64, stored in float32, with
//                   its norm, sum and constant flag.
//   2. k_dd_scan    one CTA per (series, stream, chunk of 2048 windows), for every
//                   discord whose group holds the stream.  The chunk is staged in
//                   shared memory shifted by its first sample; window means and
//                   norms come from float-float prefix sums (no float64 on the
//                   hot path: the FP64 pipe runs at 1/64 of FP32); each thread
//                   forms 8 consecutive sliding dot products with four centred
//                   queries at a time in paired float32 FMAs (128 FMAs in 64
//                   issue slots per vector load of samples; swizzled staging so
//                   the loads are free of bank conflicts).  The active
//                   discords of an item are found once (one per thread, then
//                   compacted).  Each thread keeps its best window per
//                   discord; the largest key rho - 1 and lowest window index
//                   merge per (series, discord, stream) in a packed 64-bit word
//                   with atomicMax.
//   3. k_dd_exact   one warp per (series, discord, stream): the chosen window
//                   re-evaluated exactly (compensated sums).
//   4. k_dd_select  one CTA per (series, discord): the strict running maximum
//                   over ascending j, as a reduction.
//   5. k_dd_gather  (optional) copies stream j* of every discord into a
//                   contiguous buffer for a self-join refinement profile.
#include "tsk_internal.cuh"
#include "tsk_ff.cuh"
#include "tsk_rho.cuh"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <type_traits>

namespace {

constexpr int kScanThreads = 256;
constexpr int kWinPerThread = 8;                      // consecutive windows per thread
constexpr int kTW = kScanThreads * kWinPerThread;     // 2048 windows per scan item
constexpr int kQB = 16;                               // discords staged per batch (at most)
constexpr int kQBudget = 8192;                        // floats of staged queries (32 KB)

// discords staged per batch for subsequence length m (a multiple of 4 up to kQB, else 2)
__host__ __device__ inline int query_batch(int m) {
  const int m4 = (m + 3) & ~3;
  const int q = kQBudget / m4;
  return q >= kQB ? kQB : (q < 4 ? 2 : (q & ~3));
}
constexpr double kConstRelVar = 1e-12;

struct DimArgs {
  const int64_t* cum;          // [n_series + 1] sample offsets of series (per stream): the queried series
  const int32_t* len;          // [n_series]
  const int64_t* cum_t;        // scanned series (the training series in the AB form; else = cum)
  const int32_t* len_t;
  const int64_t* item_prefix;  // [n_series + 1] scan items before each series
  const float* R;              // d x k
  const int32_t* idx;          // n_series x K
  const int32_t* grp;          // n_series x K
  unsigned long long* best;    // n_series x K x d
  float* Q;                    // n_series x K x d x m4: centred queries
  float4* qinfo;               // n_series x K x d: {1/||q||, sum(q), active, constant}
  double* sc;                  // n_series x K x d: exact score of each stream's chosen window
  int32_t* nn;                 // n_series x K x d: that window
  int n_series, d, k, m, m4, excl, K;
};

// x - x_ref as float-float: exact for float samples (two-sum), rounded to ~2^-48 for double samples
__device__ __forceinline__ FF ff_shift(float x, float xr) { return ff_two_sum(x, -xr); }
__device__ __forceinline__ FF ff_shift(double x, double xr) {
  const double y = x - xr;
  const float h = static_cast<float>(y);
  return {h, static_cast<float>(y - static_cast<double>(h))};
}
__device__ __forceinline__ FF ff_shfl_up(FF v, int o) {
  return {__shfl_up_sync(TSK_FULL_MASK, v.h, o), __shfl_up_sync(TSK_FULL_MASK, v.l, o)};
}
__device__ __forceinline__ FF ff_shfl(FF v, int lane) {
  return {__shfl_sync(TSK_FULL_MASK, v.h, lane), __shfl_sync(TSK_FULL_MASK, v.l, lane)};
}

// staging index: 16-byte granule g goes to g ^ ((g >> 3) & 1), so that the 8
// lanes of a quarter warp reading float4s 32 bytes apart (samples 8 l + c, any
// c = 0 mod 4) fall in 8 distinct bank groups, and 32 consecutive scalar stores
// stay a permutation of one 128-byte row
__device__ __forceinline__ int xs_phys(int p) { return p ^ (((p >> 5) & 1) << 2); }

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) { return a > b ? a : b; }

// One warp per (series, discord, stream): the discord window of the stream,
// centred in float64 and stored as float32, with its norm, sum and constant flag.
template <typename TX>
__global__ void __launch_bounds__(256) k_dd_query(const TX* __restrict__ T, DimArgs a) {
  const int64_t wid = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t total = static_cast<int64_t>(a.n_series) * a.K * a.d;
  if (wid >= total) return;
  const int j = static_cast<int>(wid % a.d);
  const int64_t sr = wid / a.d;
  const int s = static_cast<int>(sr / a.K);
  const int n = a.len[s];
  const int l = n - a.m + 1;
  const int i_star = a.idx[sr];
  const int g_star = a.grp[sr];
  const bool active = i_star >= 0 && i_star < l && g_star >= 0 && g_star < a.k &&
                      a.R[static_cast<int64_t>(j) * a.k + g_star] != 0.f;
  if (!active) {
    if (lane == 0) a.qinfo[wid] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const TX* x = T + a.cum[s] * static_cast<int64_t>(a.d) + static_cast<int64_t>(j) * n + i_star;
  double sum = 0.0;
  for (int t = lane; t < a.m; t += 32) sum += static_cast<double>(x[t]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(TSK_FULL_MASK, sum, o);
  const double mu = sum / a.m;
  double var = 0.0, sq = 0.0, nq = 0.0;
  float* q = a.Q + wid * a.m4;
  for (int t = lane; t < a.m4; t += 32) {
    float v = 0.f;
    if (t < a.m) {
      const double dv = static_cast<double>(x[t]) - mu;
      var += dv * dv;
      v = static_cast<float>(dv);
    }
    q[t] = v;
    sq += static_cast<double>(v);
    nq += static_cast<double>(v) * static_cast<double>(v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    var += __shfl_xor_sync(TSK_FULL_MASK, var, o);
    sq += __shfl_xor_sync(TSK_FULL_MASK, sq, o);
    nq += __shfl_xor_sync(TSK_FULL_MASK, nq, o);
  }
  const bool q_const = (var / a.m) <= kConstRelVar * fmax(1.0, mu * mu);
  if (lane == 0)
    a.qinfo[wid] = make_float4(nq > 0.0 ? static_cast<float>(1.0 / sqrt(nq)) : 0.f, static_cast<float>(sq), 1.f,
                               q_const ? 1.f : 0.f);
}

// Sliding dot products of the centred queries with the 8 consecutive windows
// starting at staged sample w0.  One query (qs contiguous): 32 FMAs per 16-byte
// load of samples.  Two queries (qs interleaved, qs[2k + q]): paired FFMA2 with
// (sample, sample) x (q0_k, q1_k), 64 FMAs in 32 issue slots per load.  Four
// queries (qs[4k + q]): each (sample, sample) pair feeds two FFMA2s, 128 FMAs
// per load of samples.
template <int NQ>
__device__ __forceinline__ void dot_windows(const float* __restrict__ xs, const float* __restrict__ qs, int m4,
                                            int w0, float (&acc)[4][kWinPerThread]) {
  float4 A = *reinterpret_cast<const float4*>(xs + xs_phys(w0));
  float4 B = *reinterpret_cast<const float4*>(xs + xs_phys(w0 + 4));
  if constexpr (NQ == 1) {
#pragma unroll
    for (int u = 0; u < kWinPerThread; ++u) acc[0][u] = 0.f;
    for (int kk = 0; kk < m4; kk += 4) {
      const float4 C = *reinterpret_cast<const float4*>(xs + xs_phys(w0 + kk + 8));
      const float v[12] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w, C.x, C.y, C.z, C.w};
      const float4 qv = *reinterpret_cast<const float4*>(qs + kk);
#pragma unroll
      for (int u = 0; u < kWinPerThread; ++u) {
        acc[0][u] = __fmaf_rn(qv.x, v[u + 0], acc[0][u]);
        acc[0][u] = __fmaf_rn(qv.y, v[u + 1], acc[0][u]);
        acc[0][u] = __fmaf_rn(qv.z, v[u + 2], acc[0][u]);
        acc[0][u] = __fmaf_rn(qv.w, v[u + 3], acc[0][u]);
      }
      A = B;
      B = C;
    }
  } else if constexpr (NQ == 4) {
    float2 acc2[kWinPerThread][2];
#pragma unroll
    for (int u = 0; u < kWinPerThread; ++u) acc2[u][0] = acc2[u][1] = make_float2(0.f, 0.f);
    for (int kk = 0; kk < m4; kk += 4) {
      const float4 C = *reinterpret_cast<const float4*>(xs + xs_phys(w0 + kk + 8));
      const float v[12] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w, C.x, C.y, C.z, C.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float4 q = *reinterpret_cast<const float4*>(qs + 4 * (kk + k));  // (q0, q1, q2, q3) at tap kk + k
        const float2 q01 = make_float2(q.x, q.y), q23 = make_float2(q.z, q.w);
#pragma unroll
        for (int u = 0; u < kWinPerThread; ++u) {
          const float2 vv = make_float2(v[u + k], v[u + k]);
          acc2[u][0] = __ffma2_rn(vv, q01, acc2[u][0]);
          acc2[u][1] = __ffma2_rn(vv, q23, acc2[u][1]);
        }
      }
      A = B;
      B = C;
    }
#pragma unroll
    for (int u = 0; u < kWinPerThread; ++u) {
      acc[0][u] = acc2[u][0].x;
      acc[1][u] = acc2[u][0].y;
      acc[2][u] = acc2[u][1].x;
      acc[3][u] = acc2[u][1].y;
    }
  } else {
    float2 acc2[kWinPerThread];
#pragma unroll
    for (int u = 0; u < kWinPerThread; ++u) acc2[u] = make_float2(0.f, 0.f);
    for (int kk = 0; kk < m4; kk += 4) {
      const float4 C = *reinterpret_cast<const float4*>(xs + xs_phys(w0 + kk + 8));
      const float v[12] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w, C.x, C.y, C.z, C.w};
      const float4 q01 = *reinterpret_cast<const float4*>(qs + 2 * kk);      // (q0, q1) at kk, kk + 1
      const float4 q23 = *reinterpret_cast<const float4*>(qs + 2 * kk + 4);  // (q0, q1) at kk + 2, kk + 3
      const float2 qk[4] = {make_float2(q01.x, q01.y), make_float2(q01.z, q01.w), make_float2(q23.x, q23.y),
                            make_float2(q23.z, q23.w)};
#pragma unroll
      for (int u = 0; u < kWinPerThread; ++u)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc2[u] = __ffma2_rn(make_float2(v[u + k], v[u + k]), qk[k], acc2[u]);
      A = B;
      B = C;
    }
#pragma unroll
    for (int u = 0; u < kWinPerThread; ++u) {
      acc[0][u] = acc2[u].x;
      acc[1][u] = acc2[u].y;
    }
  }
}

// One CTA per (series, stream, chunk of 2048 windows), for every discord whose
// group holds the stream.  See the file comment.
template <typename TX>
__global__ void __launch_bounds__(kScanThreads, 3) k_dd_scan(const TX* __restrict__ T, DimArgs a, int64_t total_items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = a.m;
  const int m4 = a.m4;
  const int ns_max = kTW + m4 + 8;                             // staged samples (zero padded)
  float* xs = reinterpret_cast<float*>(smem_raw);              // [xs_phys(ns_max)]
  const int xs_words = ns_max + 8;
  const int qb = query_batch(m);
  float* qbuf = xs + xs_words;                                 // [qb * m4] staged queries (fours, pairs, taps interleaved)
  float* w_inv = qbuf + qb * m4;                               // [kTW] 1/||window - mean|| (0: constant)
  float* w_mean = w_inv + kTW;                                 // [kTW] window mean of the shifted samples
  float* p1h = w_mean + kTW;                                   // [kTW + m] prefix of shifted samples (float-float)
  float* p1l = p1h + (kTW + m);
  float* p2h = p1l + (kTW + m);                                // [kTW + m] prefix of their squares
  float* p2l = p2h + (kTW + m);
  __shared__ float segs[4][kScanThreads / 32];  // per-warp totals of the prefix scan
  __shared__ int act[kScanThreads];  // active discords r of the item (ascending), up to 256 at a time
  __shared__ int wcnt[kScanThreads / 32];
  __shared__ float4 qinf[kQB];
  __shared__ int qstar[kQB];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (int64_t item = blockIdx.x; item < total_items; item += gridDim.x) {
    const int s = tsk_find_segment<int64_t>(a.item_prefix, a.n_series, item);
    const int n = a.len_t[s];
    const int l = n - m + 1;
    const int chunks = (l + kTW - 1) / kTW;
    const int64_t rem = item - a.item_prefix[s];
    const int c = static_cast<int>(rem % chunks);
    const int j = static_cast<int>(rem / chunks);
    const int t0 = c * kTW;
    const int nw = min(kTW, l - t0);
    const int w0 = tid * kWinPerThread;  // this thread's 8 windows
    if (item + gridDim.x < total_items) {  // the next item's samples into L2 while this one runs
      const int64_t nx = item + gridDim.x;
      const int s2 = tsk_find_segment<int64_t>(a.item_prefix, a.n_series, nx);
      const int n2 = a.len_t[s2];
      const int ch2 = (n2 - m + 1 + kTW - 1) / kTW;
      const int64_t rem2 = nx - a.item_prefix[s2];
      const int t02 = static_cast<int>(rem2 % ch2) * kTW;
      const int nw2 = min(kTW, n2 - m + 1 - t02);
      const char* px = reinterpret_cast<const char*>(T + a.cum_t[s2] * static_cast<int64_t>(a.d) +
                                                     static_cast<int64_t>(rem2 / ch2) * n2 + t02);
      const int bytes = (nw2 + m - 1) * static_cast<int>(sizeof(TX));
      for (int o = tid * 128; o < bytes; o += kScanThreads * 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(px + o));
    }
    bool staged = false;
    for (int r0 = 0; r0 < a.K; r0 += kScanThreads) {
      // discords r0 .. r0 + 255 whose group holds stream j and whose exclusion zone
      // leaves a window in this chunk, compacted in ascending r (one per thread)
      const int r = r0 + tid;
      bool on = false;
      if (r < a.K) {
        const int64_t sr = static_cast<int64_t>(s) * a.K + r;
        if (a.qinfo[sr * a.d + j].z != 0.f) {
          const int i_star = a.idx[sr];
          on = !(t0 > i_star - a.excl && t0 + nw - 1 < i_star + a.excl);
        }
      }
      const unsigned bal = __ballot_sync(TSK_FULL_MASK, on);
      if (lane == 0) wcnt[warp] = __popc(bal);
      __syncthreads();
      int base = 0, total = 0;
#pragma unroll
      for (int u = 0; u < kScanThreads / 32; ++u) {
        base += (u < warp) ? wcnt[u] : 0;
        total += wcnt[u];
      }
      if (on) act[base + __popc(bal & ((1u << lane) - 1u))] = r;
      __syncthreads();  // act written; wcnt read (the next chunk rewrites it)
      if (total == 0) continue;
      if (!staged) {
        staged = true;
        const TX* x = T + a.cum_t[s] * static_cast<int64_t>(a.d) + static_cast<int64_t>(j) * n + t0;

        // ---- stage the chunk shifted by its first sample; float-float prefix sums ----
        const TX x_ref = x[0];
        const int ns = nw + m - 1;
        // loads issued four at a time before their stores (memory-level parallelism)
        for (int p0 = tid; p0 < ns_max; p0 += 4 * kScanThreads) {
          TX v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int p = p0 + u * kScanThreads;
            v[u] = (p < ns) ? x[p] : x_ref;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int p = p0 + u * kScanThreads;
            if (p < ns_max) xs[xs_phys(p)] = (p < ns) ? ff_shift(v[u], x_ref).h : 0.f;
          }
        }
        const int seg = (ns + kScanThreads - 1) / kScanThreads;
        const int lo = tid * seg, hi = min(ns, lo + seg);
        FF a1{0.f, 0.f}, a2{0.f, 0.f};
        for (int p = lo; p < hi; ++p) {
          const FF y = ff_shift(x[p], x_ref);
          a1 = ff_add(a1, y);
          a2 = ff_add(a2, ff_sqr(y));
          p1h[p + 1] = a1.h; p1l[p + 1] = a1.l;
          p2h[p + 1] = a2.h; p2l[p + 1] = a2.l;
        }
        // exclusive scan of the 256 segment totals (float-float): each warp scans its
        // 32 in registers, then adds the totals of the warps before it
        FF i1 = a1, i2 = a2;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const FF t1 = ff_shfl_up(i1, o), t2 = ff_shfl_up(i2, o);
          if (lane >= o) { i1 = ff_add(i1, t1); i2 = ff_add(i2, t2); }
        }
        if (lane == 31) { segs[0][warp] = i1.h; segs[1][warp] = i1.l; segs[2][warp] = i2.h; segs[3][warp] = i2.l; }
        FF o1 = ff_shfl_up(i1, 1), o2 = ff_shfl_up(i2, 1);  // exclusive within the warp
        if (lane == 0) { o1 = FF{0.f, 0.f}; o2 = FF{0.f, 0.f}; }
        __syncthreads();
        for (int v = 0; v < warp; ++v) {
          o1 = ff_add(o1, FF{segs[0][v], segs[1][v]});
          o2 = ff_add(o2, FF{segs[2][v], segs[3][v]});
        }
        if (tid == 0) { p1h[0] = 0.f; p1l[0] = 0.f; p2h[0] = 0.f; p2l[0] = 0.f; }
        for (int p = lo; p < hi; ++p) {
          const FF v1 = ff_add(o1, FF{p1h[p + 1], p1l[p + 1]});
          const FF v2 = ff_add(o2, FF{p2h[p + 1], p2l[p + 1]});
          p1h[p + 1] = v1.h; p1l[p + 1] = v1.l;
          p2h[p + 1] = v2.h; p2l[p + 1] = v2.l;
        }
        __syncthreads();
        // ---- window statistics: D = m * sum(y^2) - sum(y)^2 = m^2 var ----
        // A window whose D is within the prefix sums' rounding of the constant
        // threshold is decided from its samples: all equal (constant), else the
        // float64 two-pass variance.
        const float fm = static_cast<float>(m);
        const float m_ref = fm * static_cast<float>(x_ref);
        const float sqrt_m = sqrtf(fm);
        for (int w = tid; w < nw; w += kScanThreads) {
          const FF s1 = ff_add(FF{p1h[w + m], p1l[w + m]}, ff_neg(FF{p1h[w], p1l[w]}));
          const FF s2 = ff_add(FF{p2h[w + m], p2l[w + m]}, ff_neg(FF{p2h[w], p2l[w]}));
          const FF D = ff_add(ff_mul(s2, fm), ff_neg(ff_sqr(s1)));
          const float Df = D.h + D.l;
          const float mmu = m_ref + s1.h;                         // m * window mean
          const float thr = static_cast<float>(kConstRelVar) * fmaxf(fm * fm, mmu * mmu);
          const float slack = 0x1p-30f * fm * (p2h[w + m] + p2h[w]);
          float inv;
          if (Df > thr + slack) {
            inv = sqrt_m * rsqrtf(Df);
          } else {
            bool equal = true;
            for (int t = 1; t < m && equal; ++t) equal = (x[w + t] == x[w]);
            if (equal) {
              inv = 0.f;
            } else {
              double mu = 0.0;
              for (int t = 0; t < m; ++t) mu += static_cast<double>(x[w + t]);
              mu /= m;
              double v = 0.0;
              for (int t = 0; t < m; ++t) {
                const double dv = static_cast<double>(x[w + t]) - mu;
                v += dv * dv;
              }
              inv = (v / m <= kConstRelVar * fmax(1.0, mu * mu)) ? 0.f : static_cast<float>(1.0 / sqrt(v));
            }
          }
          w_inv[w] = inv;
          w_mean[w] = s1.h / fm;
        }
        __syncthreads();

      }

      // batches of up to qb discords: staged in groups of four (taps interleaved,
      // four per 16 bytes), a pair or one; every warp then runs its 256 windows
      // through each group and merges with one atomic per discord
      for (int b0 = 0; b0 < total; b0 += qb) {
        const int nb = min(qb, total - b0);
        for (int b = 0; b < nb;) {
          const int nq = (nb - b >= 3) ? 4 : nb - b;
          float* qs = qbuf + b * m4;
          auto qsrc = [&](int q) {  // discord b + q's centred query of stream j
            return a.Q + ((static_cast<int64_t>(s) * a.K + act[b0 + b + q]) * a.d + j) * m4;
          };
          if (nq == 4) {
            const float *q0 = qsrc(0), *q1 = qsrc(1), *q2 = qsrc(2), *q3 = (b + 3 < nb) ? qsrc(3) : nullptr;
            for (int t = tid; t < m4; t += kScanThreads)
              *reinterpret_cast<float4*>(qs + 4 * t) = make_float4(q0[t], q1[t], q2[t], q3 ? q3[t] : 0.f);
          } else if (nq == 2) {
            const float *q0 = qsrc(0), *q1 = qsrc(1);
            for (int t = tid; t < m4; t += kScanThreads) *reinterpret_cast<float2*>(qs + 2 * t) = make_float2(q0[t], q1[t]);
          } else {
            const float* q0 = qsrc(0);
            for (int t = tid; t < m4; t += kScanThreads) qs[t] = q0[t];
          }
          b += nq;
        }
        if (tid < nb) {
          const int64_t sr = static_cast<int64_t>(s) * a.K + act[b0 + tid];
          qinf[tid] = a.qinfo[sr * a.d + j];
          qstar[tid] = a.idx[sr];
        }
        __syncthreads();
        for (int b = 0; b < nb;) {
          const int nq = (nb - b >= 3) ? 4 : nb - b;
          float acc[4][kWinPerThread];
          if (nq == 4)
            dot_windows<4>(xs, qbuf + b * m4, m4, w0, acc);
          else if (nq == 2)
            dot_windows<2>(xs, qbuf + b * m4, m4, w0, acc);
          else
            dot_windows<1>(xs, qbuf + b * m4, m4, w0, acc);
          // this thread's window statistics (read after the products: fewer live registers)
          float winv[kWinPerThread], wmean[kWinPerThread];
          {
            const float4 i0 = *reinterpret_cast<const float4*>(w_inv + w0);
            const float4 i1 = *reinterpret_cast<const float4*>(w_inv + w0 + 4);
            const float4 m0 = *reinterpret_cast<const float4*>(w_mean + w0);
            const float4 m1 = *reinterpret_cast<const float4*>(w_mean + w0 + 4);
            winv[0] = i0.x; winv[1] = i0.y; winv[2] = i0.z; winv[3] = i0.w;
            winv[4] = i1.x; winv[5] = i1.y; winv[6] = i1.z; winv[7] = i1.w;
            wmean[0] = m0.x; wmean[1] = m0.y; wmean[2] = m0.z; wmean[3] = m0.w;
            wmean[4] = m1.x; wmean[5] = m1.y; wmean[6] = m1.z; wmean[7] = m1.w;
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (q < nq && b + q < nb) {
              const float4 qi = qinf[b + q];
              const int i_star = qstar[b + q];
              // this thread's best window for the discord (the first of equal keys), packed once
              float bk = -FLT_MAX;
              int bu = -1;
#pragma unroll
              for (int u = 0; u < kWinPerThread; ++u) {
                const int w = w0 + u;
                const int t = t0 + w;
                const float inv_t = winv[u];
                float key;
                if (qi.w != 0.f) key = (inv_t == 0.f) ? 0.0f : -0.5f;  // rho 1 (dist 0) to a constant window, else 1/2
                else if (inv_t == 0.f) key = -0.5f;                     // rho 1/2: 2m(1 - 1/2) = m
                else {
                  const float cov = __fmaf_rn(-wmean[u], qi.y, acc[q][u]);
                  key = fminf(0.0f, fmaxf(-2.0f, __fmaf_rn(cov * qi.x, inv_t, -1.0f)));  // rho - 1
                }
                const bool ok = w < nw && !(t > i_star - a.excl && t < i_star + a.excl);
                if (ok && key > bk) {
                  bk = key;
                  bu = u;
                }
              }
              unsigned long long best = bu >= 0 ? tsk_pack(bk, t0 + w0 + bu) : 0ull;
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) best = umax64(best, __shfl_xor_sync(TSK_FULL_MASK, best, o));
              if (lane == 0 && best)
                atomicMax(&a.best[(static_cast<int64_t>(s) * a.K + act[b0 + b + q]) * a.d + j], best);
            }
          }
          b += nq;
        }
        __syncthreads();  // the staged batch is rewritten by the next one
      }
    }
    __syncthreads();  // shared buffers are reused by the next item
  }
}

// Exact re-evaluation of one chosen window by a whole warp: lanes take every
// 32nd sample, float64 window means and the constant test, then the window
// correlation with compensated float32 sums (products split exactly, running
// sums as (hi, lo) pairs, the same arithmetic as the refinement kernel), the
// lane partials added in float64.  Returns the distance; the whole warp calls it.
template <typename TX>
__device__ double warp_window_dist(const TX* xq, int i, const TX* x, int t, int m) {
  const int lane = threadIdx.x & 31;
  double sq = 0.0, st = 0.0;
  for (int u = lane; u < m; u += 32) {
    sq += static_cast<double>(xq[i + u]);
    st += static_cast<double>(x[t + u]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sq += __shfl_xor_sync(TSK_FULL_MASK, sq, o);
    st += __shfl_xor_sync(TSK_FULL_MASK, st, o);
  }
  const double mq = sq / m, mt = st / m;
  double vq = 0.0, vt = 0.0;
  [[maybe_unused]] const float mqh = static_cast<float>(mq), mql = static_cast<float>(mq - static_cast<double>(mqh));
  [[maybe_unused]] const float mth = static_cast<float>(mt), mtl = static_cast<float>(mt - static_cast<double>(mth));
  double ab = 0.0, aa = 0.0, bb = 0.0;
  if constexpr (std::is_same<TX, float>::value) {
    tsk::DSum sab, saa, sbb;
    for (int u = lane; u < m; u += 32) {
      const double dq = static_cast<double>(xq[i + u]) - mq, dt = static_cast<double>(x[t + u]) - mt;
      vq += dq * dq;
      vt += dt * dt;
      const float fa = __fsub_rn(__fsub_rn(xq[i + u], mqh), mql);
      const float fb = __fsub_rn(__fsub_rn(x[t + u], mth), mtl);
      sab.add_prod(fa, fb);
      saa.add_prod(fa, fa);
      sbb.add_prod(fb, fb);
    }
    ab = sab.value();
    aa = saa.value();
    bb = sbb.value();
  } else {  // float64 series: float64 sums
    for (int u = lane; u < m; u += 32) {
      const double dq = static_cast<double>(xq[i + u]) - mq, dt = static_cast<double>(x[t + u]) - mt;
      vq += dq * dq;
      vt += dt * dt;
      ab = fma(dq, dt, ab);
      aa = fma(dq, dq, aa);
      bb = fma(dt, dt, bb);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    vq += __shfl_xor_sync(TSK_FULL_MASK, vq, o);
    vt += __shfl_xor_sync(TSK_FULL_MASK, vt, o);
    ab += __shfl_xor_sync(TSK_FULL_MASK, ab, o);
    aa += __shfl_xor_sync(TSK_FULL_MASK, aa, o);
    bb += __shfl_xor_sync(TSK_FULL_MASK, bb, o);
  }
  const bool cq = (vq / m) <= kConstRelVar * fmax(1.0, mq * mq);
  const bool ct = (vt / m) <= kConstRelVar * fmax(1.0, mt * mt);
  const double sqm = sqrt(static_cast<double>(m));
  if (cq) return ct ? 0.0 : sqm;
  if (ct) return sqm;
  const double rho = ab / sqrt(aa * bb);
  return sqrt(fmax(0.0, 2.0 * m * (1.0 - rho)));
}

// One warp per (series, discord, stream): the stream's chosen window
// re-evaluated exactly.  NaN: the stream is not in the discord's group; +inf:
// no admissible neighbour.
template <typename TX>
__global__ void __launch_bounds__(256) k_dd_exact(const TX* __restrict__ Tq, const TX* __restrict__ T, DimArgs a,
                                                  double* __restrict__ sc_out, int32_t* __restrict__ nn_out,
                                                  double* __restrict__ dim_scores) {
  const int64_t wid = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= static_cast<int64_t>(a.n_series) * a.K * a.d) return;
  const int j = static_cast<int>(wid % a.d);
  const int64_t sr = wid / a.d;
  const int s = static_cast<int>(sr / a.K);
  const int n = a.len[s];
  const int l = n - a.m + 1;
  const int i_star = a.idx[sr];
  const int g_star = a.grp[sr];
  const bool valid = i_star >= 0 && i_star < l && g_star >= 0 && g_star < a.k;
  double sc = NAN;
  int nn = -1;
  if (valid && a.R[static_cast<int64_t>(j) * a.k + g_star] != 0.f) {
    const unsigned long long p = a.best[wid];
    if (p == 0ull) {
      sc = INFINITY;
    } else {
      nn = tsk_unpack_idx(p);
      const TX* xq = Tq + a.cum[s] * static_cast<int64_t>(a.d) + static_cast<int64_t>(j) * n;
      const TX* x = T + a.cum_t[s] * static_cast<int64_t>(a.d) + static_cast<int64_t>(j) * a.len_t[s];
      sc = warp_window_dist(xq, i_star, x, nn, a.m);
    }
  }
  if (lane == 0) {
    sc_out[wid] = sc;
    nn_out[wid] = nn;
    if (dim_scores) dim_scores[wid] = sc;
  }
}

// One CTA per (series, discord): Alg. 3's strict running maximum from 0 over
// ascending j, i.e. the largest score above 0 (the lowest j among equal ones),
// else the group's first stream; -1 for an empty group or an invalid discord.
__global__ void __launch_bounds__(256) k_dd_select(DimArgs a, const double* __restrict__ sc, const int32_t* __restrict__ nn,
                                                   int32_t* __restrict__ dim, double* __restrict__ dim_score,
                                                   int32_t* __restrict__ dim_nn) {
  const int64_t sr = blockIdx.x;
  const double* v = sc + sr * a.d;
  double bs = 0.0;
  int bj = -1, first = a.d;
  for (int j = threadIdx.x; j < a.d; j += blockDim.x) {  // ascending j per thread: ties keep the lower j
    const double x = v[j];
    if (isnan(x)) continue;  // not in the group
    first = min(first, j);
    if (x > bs) {
      bs = x;
      bj = j;
    }
  }
  auto better = [](double s1, int j1, double s2, int j2) {  // (s2, j2) replaces (s1, j1)
    return j2 >= 0 && (j1 < 0 || s2 > s1 || (s2 == s1 && j2 < j1));
  };
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double s2 = __shfl_xor_sync(TSK_FULL_MASK, bs, o);
    const int j2 = __shfl_xor_sync(TSK_FULL_MASK, bj, o);
    const int f2 = __shfl_xor_sync(TSK_FULL_MASK, first, o);
    if (better(bs, bj, s2, j2)) {
      bs = s2;
      bj = j2;
    }
    first = min(first, f2);
  }
  __shared__ double wbs[8];
  __shared__ int wbj[8], wf[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    wbs[warp] = bs;
    wbj[warp] = bj;
    wf[warp] = first;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w) {
      if (better(bs, bj, wbs[w], wbj[w])) {
        bs = wbs[w];
        bj = wbj[w];
      }
      first = min(first, wf[w]);
    }
    if (bj >= 0) {
      dim[sr] = bj;
      dim_score[sr] = bs;
      dim_nn[sr] = nn[sr * a.d + bj];
    } else if (first < a.d) {
      dim[sr] = first;
      dim_score[sr] = v[first];
      dim_nn[sr] = nn[sr * a.d + first];
    } else {
      dim[sr] = -1;
      dim_score[sr] = NAN;
      dim_nn[sr] = -1;
    }
  }
}

template <typename TX>
__global__ void k_dd_gather(const TX* __restrict__ T, const int64_t* __restrict__ cum, const int32_t* __restrict__ len,
                            const int32_t* __restrict__ dim, int n_series, int d, int K, int64_t total,
                            TX* __restrict__ out) {
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    // out holds, per series s, K streams of len[s] samples starting at K * cum[s]
    const int64_t base_scaled = e;  // K * cum is non-decreasing: search on cum with e / K bounds
    int lo = 0, hi = n_series - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (static_cast<int64_t>(K) * cum[mid] <= base_scaled) lo = mid; else hi = mid - 1;
    }
    const int s = lo;
    const int n = len[s];
    const int64_t off = e - static_cast<int64_t>(K) * cum[s];
    const int r = static_cast<int>(off / n);
    const int t = static_cast<int>(off - static_cast<int64_t>(r) * n);
    const int j = dim[static_cast<int64_t>(s) * K + r];
    out[e] = (j >= 0) ? T[cum[s] * static_cast<int64_t>(d) + static_cast<int64_t>(j) * n + t] : static_cast<TX>(0);
  }
}

size_t scan_smem_bytes(int m) {
  const int m4 = (m + 3) & ~3;
  const int ns_max = kTW + m4 + 8;
  const size_t xs_words = static_cast<size_t>(ns_max) + 8;
  return (xs_words + static_cast<size_t>(query_batch(m)) * m4 + 2 * static_cast<size_t>(kTW) +
          4 * static_cast<size_t>(kTW + m)) *
         sizeof(float);
}

template <typename TX>
tsk_status run_dims(tsk_ctx* ctx, const TX* T, const TX* Tt, const DimArgs& a, int64_t total_items, int32_t* dim,
                    double* dim_score, int32_t* dim_nn, double* dim_scores, TX* T_sel, TX* T_sel_t,
                    int64_t total_samples, int64_t total_samples_t) {
  cudaStream_t st = ctx->stream;
  const int64_t triples = static_cast<int64_t>(a.n_series) * a.K * a.d;
  TSK_CUDA_TRY(ctx, cudaMemsetAsync(a.best, 0, sizeof(unsigned long long) * static_cast<size_t>(triples), st));
  k_dd_query<TX><<<static_cast<unsigned>((triples * 32 + 255) / 256), 256, 0, st>>>(T, a);
  TSK_LAUNCH_CHECK(ctx, "k_dd_query");
  const size_t smem = scan_smem_bytes(a.m);
  TSK_CUDA_TRY(ctx, cudaFuncSetAttribute(k_dd_scan<TX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem)));
  if (total_items > 0) {
    int per_sm = 0;
    TSK_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dd_scan<TX>, kScanThreads, smem));
    const int64_t grid = std::min<int64_t>(total_items, static_cast<int64_t>(std::max(per_sm, 1)) * ctx->sm_count);
    tsk_prof_scope ps(ctx, TSK_PROF_DIMS);
    k_dd_scan<TX><<<static_cast<unsigned>(grid), kScanThreads, smem, st>>>(Tt, a, total_items);
    TSK_LAUNCH_CHECK(ctx, "k_dd_scan");
  }
  k_dd_exact<TX><<<static_cast<unsigned>((triples * 32 + 255) / 256), 256, 0, st>>>(T, Tt, a, a.sc, a.nn, dim_scores);
  TSK_LAUNCH_CHECK(ctx, "k_dd_exact");
  const int64_t discords = static_cast<int64_t>(a.n_series) * a.K;
  k_dd_select<<<static_cast<unsigned>(discords), 256, 0, st>>>(a, a.sc, a.nn, dim, dim_score, dim_nn);
  TSK_LAUNCH_CHECK(ctx, "k_dd_select");
  if (T_sel && total_samples > 0) {
    const int64_t total = total_samples * a.K;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, static_cast<int64_t>(ctx->sm_count) * 16);
    k_dd_gather<TX><<<static_cast<unsigned>(blocks), 256, 0, st>>>(T, a.cum, a.len, dim, a.n_series, a.d, a.K, total,
                                                                     T_sel);
    TSK_LAUNCH_CHECK(ctx, "k_dd_gather");
  }
  if (T_sel_t && total_samples_t > 0) {
    const int64_t total = total_samples_t * a.K;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, static_cast<int64_t>(ctx->sm_count) * 16);
    k_dd_gather<TX><<<static_cast<unsigned>(blocks), 256, 0, st>>>(Tt, a.cum_t, a.len_t, dim, a.n_series, a.d, a.K,
                                                                     total, T_sel_t);
    TSK_LAUNCH_CHECK(ctx, "k_dd_gather");
  }
  return TSK_OK;
}

}  // namespace

int tsk_dims_window_chunk() { return kTW; }

tsk_status tsk_launch_dims(tsk_ctx* ctx, const void* T, const void* T_train, int t_dtype, int32_t n_series,
                           const int64_t* d_cum, const int32_t* d_len, const int64_t* d_cum_t, const int32_t* d_len_t,
                           const int64_t* d_item_prefix, int64_t total_items, int64_t total_samples,
                           int64_t total_samples_t, int32_t d, const float* R, int32_t k, int32_t m, int32_t excl,
                           int32_t K, const int32_t* idx, const int32_t* grp, int32_t* dim, double* dim_score,
                           int32_t* dim_nn, double* dim_scores, void* T_sel, void* T_sel_train, char* ws) {
  DimArgs a;
  a.cum = d_cum;
  a.len = d_len;
  a.cum_t = d_cum_t;
  a.len_t = d_len_t;
  a.item_prefix = d_item_prefix;
  a.R = R;
  a.idx = idx;
  a.grp = grp;
  const size_t triples = static_cast<size_t>(n_series) * K * d;
  a.m4 = (m + 3) & ~3;
  tsk_carver cv(ws);
  a.best = cv.take<unsigned long long>(triples);
  a.Q = cv.take<float>(triples * a.m4);
  a.qinfo = cv.take<float4>(triples);
  a.sc = cv.take<double>(triples);
  a.nn = cv.take<int32_t>(triples);
  a.n_series = n_series;
  a.d = d;
  a.k = k;
  a.m = m;
  a.excl = excl;
  a.K = K;
  if (t_dtype == TSK_F64)
    return run_dims<double>(ctx, static_cast<const double*>(T), static_cast<const double*>(T_train), a, total_items,
                            dim, dim_score, dim_nn, dim_scores, static_cast<double*>(T_sel),
                            static_cast<double*>(T_sel_train), total_samples, total_samples_t);
  return run_dims<float>(ctx, static_cast<const float*>(T), static_cast<const float*>(T_train), a, total_items, dim,
                         dim_score, dim_nn, dim_scores, static_cast<float*>(T_sel), static_cast<float*>(T_sel_train),
                         total_samples, total_samples_t);
}

size_t tsk_dims_ws_bytes(int32_t n_series, int32_t K, int32_t d, int32_t m) {
  const size_t triples = static_cast<size_t>(n_series) * K * d;
  return tsk_carver::bytes_for(triples, 8) + tsk_carver::bytes_for(triples * ((m + 3) & ~3), 4) +
         tsk_carver::bytes_for(triples, 16) + tsk_carver::bytes_for(triples, 8) + tsk_carver::bytes_for(triples, 4);
}
