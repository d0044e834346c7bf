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
//                       of 32*V diagonals and H rows; lane t walks diagonals
//                       d0 + tV .. d0 + tV + V - 1 down the rows with the float32
//                       recurrence, anchored exactly in float64 at the first row.
//                       Each cell's correlation rho = c * inv_i * inv_j updates the
//                       row maximum (reduced over lanes through shared memory) and
//                       the column maximum (carried from lane to lane as the
//                       band's columns slide).  Keys carry the in-lane diagonal
//                       offset in their 4 low mantissa bits, so a max also knows
//                       its argmax.  Results merge into a packed (key, index)
//                       64-bit word per window with atomicMax.
//   4. k_mp_refine      for every window: its chosen neighbour's distance in
//                       float64, dist = sqrt(2 m (1 - rho)), plus the constant-
//                       window rules.
// The float64 variant (k_mp_diag_f64) is exact: one thread per diagonal, a
// first pass takes the float64 maximum per window, a second pass the lowest
// index attaining it.
#include "tsk_internal.cuh"

#include <algorithm>
#include <cfloat>
#include <cmath>

namespace {

constexpr int kV = 8;                    // diagonals per lane
constexpr int kWarps = 4;                // warps per CTA
constexpr int kD = 32 * kV;              // diagonals per band
constexpr int kTagIn = 15;               // tag of a column maximum inherited from another lane
constexpr int kWinChunk = 1024;          // windows per window-stats CTA
constexpr int kWinThreads = 256;
constexpr int kPad = kD + 4 * kV + 64;   // zeroed slack after each stream's window arrays
constexpr float kEmpty = -3.0f;          // below every correlation
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
__global__ void __launch_bounds__(kWinThreads) k_window_stats(const TX* __restrict__ X, const int64_t* __restrict__ xoff,
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
  const TX* x = X + xoff[q];
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
// ---------------------------------------------------------------------------
struct MpArgs {
  const void* X;
  const int64_t* xoff;
  const int32_t* len;
  const int64_t* woff;
  const int64_t* tile_prefix;
  const int64_t* band_off;
  const int32_t* band_prefix;
  unsigned long long* counter;
  WinArrays wa;
  int64_t total_tiles;
  int n_streams, m, excl, excl4, H;
};

__device__ __forceinline__ float tag_key(float rho, unsigned tag) {
  return __uint_as_float((__float_as_uint(rho) & ~15u) | tag);
}
__device__ __forceinline__ float untag_key(float key) { return __uint_as_float(__float_as_uint(key) & ~15u); }

// Merge the buffered rows/columns of `count` steps into the global profile.
// Slot u of the buffers belongs to row `base + u` (and to column base + u + d0,
// the column that left lane 0 at that step).
template <int V>
__device__ __forceinline__ void flush_rows_cols(float (*rowbuf)[33], const float* cbk, const int* cbr, int count, int base,
                                                int d0, int l, unsigned long long* best, int lane) {
  __syncwarp();
  if (lane < count) {
    const int ir = base + lane;
    float bk = kEmpty;
    int bl = 0;
#pragma unroll 8
    for (int u = 0; u < 32; ++u) {
      const float kk = rowbuf[lane][u];
      if (kk > bk) { bk = kk; bl = u; }
    }
    if (bk > -2.f) {
      const int col = ir + d0 + bl * V + static_cast<int>(__float_as_uint(bk) & 15u);
      atomicMax(&best[ir], tsk_pack(untag_key(bk), col));
    }
    const float ck = cbk[lane];
    const int jc = ir + d0;
    if (ck > -2.f && jc < l) atomicMax(&best[jc], tsk_pack(untag_key(ck), cbr[lane]));
  }
  __syncwarp();
}

template <int V, bool MASKED, typename TX>
__device__ __forceinline__ void mp_tile(const MpArgs& a, const TX* __restrict__ x, int n, int l, int64_t wb, int d0, int r0,
                                        int rEnd, float (*rowbuf)[33], float* cbk, int* cbr, int lane) {
  const double* __restrict__ mu = a.wa.mu + wb;
  const float* __restrict__ inv = a.wa.inv + wb;
  const float* __restrict__ df = a.wa.df + wb;
  const float* __restrict__ dg = a.wa.dg + wb;
  unsigned long long* __restrict__ best = a.wa.best + wb;
  const int dl = d0 + lane * V;
  const int m = a.m;

  // exact anchors c(r0, r0 + dl + v) in float64: sum_t (x[r0+t] - mean_r0) x[c+t]
  float cov[V];
  {
    double acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0.0;
    const double mr = mu[r0];
    for (int t = 0; t < m; ++t) {
      const double av = static_cast<double>(x[r0 + t]) - mr;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int idx = r0 + dl + v + t;
        double xv;
        if (MASKED) xv = idx < n ? static_cast<double>(x[idx]) : 0.0;
        else xv = static_cast<double>(x[idx]);
        acc[v] = fma(av, xv, acc[v]);
      }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) cov[v] = static_cast<float>(acc[v]);
  }

  float cdf[V], cdg[V], cinv[V], ckey[V];
  int cin[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int j = r0 + dl + v;
    cdf[v] = df[j];
    cdg[v] = dg[j];
    cinv[v] = inv[j];
    ckey[v] = kEmpty;
    cin[v] = -1;
  }

  const int nsteps = MASKED ? ((rEnd - r0 + V - 1) / V) * V : (rEnd - r0);
  for (int s0 = 0; s0 < nsteps; s0 += V) {
    const int ib = r0 + s0;
    float rdf[V], rdg[V], rinv[V], ndf[V], ndg[V], ninv[V];
#pragma unroll
    for (int u = 0; u < V; ++u) {
      rdf[u] = df[ib + u];
      rdg[u] = dg[ib + u];
      rinv[u] = inv[ib + u];
      const int j = ib + u + dl + V;
      ndf[u] = df[j];
      ndg[u] = dg[j];
      ninv[u] = inv[j];
    }
#pragma unroll
    for (int s = 0; s < V; ++s) {
      const int i = ib + s;
      float rowk = kEmpty;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int c = (v + s) % V;
        const float rho = (cov[v] * cinv[c]) * rinv[s];
        float key = tag_key(rho, static_cast<unsigned>(v));
        if (MASKED) {
          const int dd = dl + v;
          const bool ok = (dd >= a.excl) && (i + dd < l) && (i < rEnd);
          key = ok ? key : kEmpty;
        }
        rowk = fmaxf(rowk, key);
        ckey[c] = fmaxf(ckey[c], key);
        cov[v] = fmaf(rdf[s], cdg[c], cov[v]);
        cov[v] = fmaf(cdf[c], rdg[s], cov[v]);
      }
      const int slot = (s0 + s) & 31;
      rowbuf[slot][lane] = rowk;
      {
        // the column in slot s % V (diagonal offset 0 of this lane) leaves the lane
        const int c0 = s % V;
        const float kl = ckey[c0];
        const unsigned tag = __float_as_uint(kl) & 15u;
        const int row = (tag == static_cast<unsigned>(kTagIn)) ? cin[c0] : (i - static_cast<int>(tag));
        const float kin = __shfl_down_sync(TSK_FULL_MASK, kl, 1);
        const int rin = __shfl_down_sync(TSK_FULL_MASK, row, 1);
        if (lane == 0) { cbk[slot] = kl; cbr[slot] = row; }
        ckey[c0] = (lane == 31) ? kEmpty : tag_key(kin, kTagIn);
        cin[c0] = rin;
        cdf[c0] = ndf[s];
        cdg[c0] = ndg[s];
        cinv[c0] = ninv[s];
      }
    }
    if (((s0 + V) & 31) == 0) flush_rows_cols<V>(rowbuf, cbk, cbr, 32, r0 + s0 + V - 32, d0, l, best, lane);
  }
  const int rem = nsteps & 31;
  if (rem) flush_rows_cols<V>(rowbuf, cbk, cbr, rem, r0 + nsteps - rem, d0, l, best, lane);
  // columns still inside the band: slot v <-> column r0 + nsteps + dl + v
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int j = r0 + nsteps + dl + v;
    const float kk = ckey[v];
    if (kk > -2.f && j < l) {
      const unsigned tag = __float_as_uint(kk) & 15u;
      const int row = (tag == static_cast<unsigned>(kTagIn)) ? cin[v] : (j - dl - static_cast<int>(tag));
      atomicMax(&best[j], tsk_pack(untag_key(kk), row));
    }
  }
}

template <int V, typename TX>
__global__ void __launch_bounds__(kWarps * 32) k_mp_diag(MpArgs a) {
  __shared__ float rowbuf[kWarps][32][33];
  __shared__ float cbk[kWarps][32];
  __shared__ int cbr[kWarps][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int D = 32 * V;
  for (;;) {
    unsigned long long w = 0;
    if (lane == 0) w = atomicAdd(a.counter, 1ull);
    w = __shfl_sync(TSK_FULL_MASK, w, 0);
    if (static_cast<int64_t>(w) >= a.total_tiles) break;
    const int q = tsk_find_segment<int64_t>(a.tile_prefix, a.n_streams, static_cast<int64_t>(w));
    const int t = static_cast<int>(static_cast<int64_t>(w) - a.tile_prefix[q]);
    const int32_t* bp = a.band_prefix + a.band_off[q];
    const int nb = static_cast<int>(a.band_off[q + 1] - a.band_off[q]) - 1;
    const int b = tsk_find_segment<int32_t>(bp, nb, t);
    const int r0 = (t - bp[b]) * a.H;
    const int n = a.len[q];
    const int l = n - a.m + 1;
    const int d0 = a.excl4 + b * D;
    const int dmin = max(d0, a.excl);
    const int rEnd = min(r0 + a.H, l - dmin);
    const TX* x = static_cast<const TX*>(a.X) + a.xoff[q];
    const int64_t wb = a.woff[q];
    const bool interior = (d0 >= a.excl) && (rEnd == r0 + a.H) && (rEnd - 1 + d0 + D - 1 <= l - 1);
    if (interior)
      mp_tile<V, false, TX>(a, x, n, l, wb, d0, r0, rEnd, rowbuf[wid], cbk[wid], cbr[wid], lane);
    else
      mp_tile<V, true, TX>(a, x, n, l, wb, d0, r0, rEnd, rowbuf[wid], cbk[wid], cbr[wid], lane);
  }
}

// ---------------------------------------------------------------------------
// 3'. exact float64 variant: one thread per (stream, diagonal)
// ---------------------------------------------------------------------------
template <typename TX>
__device__ __forceinline__ double f64_cell_rho(double cov, const double* inv64, int i, int j) {
  return cov * inv64[i] * inv64[j];
}

template <typename TX>
__global__ void __launch_bounds__(128) k_mp_diag_f64(MpArgs a, int pass) {
  const int64_t w = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (w >= a.total_tiles) return;
  const int q = tsk_find_segment<int64_t>(a.tile_prefix, a.n_streams, w);
  const int n = a.len[q];
  const int m = a.m;
  const int l = n - m + 1;
  const int delta = a.excl + static_cast<int>(w - a.tile_prefix[q]);
  const TX* x = static_cast<const TX*>(a.X) + a.xoff[q];
  const int64_t wb = a.woff[q];
  const double* mu = a.wa.mu + wb;
  const double* inv64 = a.wa.inv64 + wb;
  unsigned long long* best = a.wa.best + wb;
  int32_t* bidx = a.wa.bidx + wb;
  double cov = 0.0;
  const double m0 = mu[0];
  for (int t = 0; t < m; ++t) cov = fma(static_cast<double>(x[t]) - m0, static_cast<double>(x[delta + t]), cov);
  for (int i = 0; i + delta < l; ++i) {
    const int j = i + delta;
    const double rho = cov * inv64[i] * inv64[j];
    const unsigned long long key = tsk_ordered_u64(rho);
    if (pass == 0) {
      atomicMax(&best[i], key);
      atomicMax(&best[j], key);
    } else {
      if (key == best[i]) atomicMin(&bidx[i], j);
      if (key == best[j]) atomicMin(&bidx[j], i);
    }
    if (j + 1 < l) {
      const double xa = static_cast<double>(x[i]), xb = static_cast<double>(x[i + m]);
      const double ya = static_cast<double>(x[j]), yb = static_cast<double>(x[j + m]);
      const double dfi = (xb - xa) * 0.5, dfj = (yb - ya) * 0.5;
      const double dgi = (xb - mu[i + 1]) + (xa - mu[i]);
      const double dgj = (yb - mu[j + 1]) + (ya - mu[j]);
      cov = fma(dfi, dgj, cov);
      cov = fma(dfj, dgi, cov);
    }
  }
}

// ---------------------------------------------------------------------------
// 4. refinement: float64 distance to each window's chosen neighbour
// ---------------------------------------------------------------------------
template <typename TX, typename TP>
__global__ void __launch_bounds__(256) k_mp_refine(const TX* __restrict__ X, const int64_t* __restrict__ xoff,
                                                   const int32_t* __restrict__ len, const uint8_t* __restrict__ smask,
                                                   const int64_t* __restrict__ woff, int n_streams, int64_t total, int m,
                                                   int excl, int exact64, WinArrays wa, TP* __restrict__ P,
                                                   int32_t* __restrict__ I) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int q = tsk_find_segment<int64_t>(xoff, n_streams, e);
  if (!smask[q]) return;
  const int n = len[q];
  const int l = n - m + 1;
  const int i = static_cast<int>(e - xoff[q]);
  if (i >= l) {
    P[e] = static_cast<TP>(NAN);
    I[e] = -1;
    return;
  }
  const int64_t wb = woff[q];
  const TX* x = X + xoff[q];
  // lowest admissible constant window
  int jc = -1;
  if (wa.constcnt[q] > 0) {
    const int f = wa.nxt[wb];
    if (f <= i - excl) jc = f;
    else if (i + excl < l) {
      const int g = wa.nxt[wb + i + excl];
      if (g < l) jc = g;
    }
  }
  const double sqm = sqrt(static_cast<double>(m));
  if (wa.inv[wb + i] == 0.f) {
    if (jc >= 0) { P[e] = static_cast<TP>(0); I[e] = jc; return; }
    const int jl = (i >= excl) ? 0 : ((i + excl < l) ? i + excl : -1);
    P[e] = static_cast<TP>(jl >= 0 ? sqm : INFINITY);
    I[e] = jl;
    return;
  }
  int j = -1;
  if (exact64) {
    const int b = wa.bidx[wb + i];  // initialised to 0x7f7f7f7f (no neighbour)
    j = (b >= l) ? -1 : b;
  } else {
    const unsigned long long pk = wa.best[wb + i];
    j = pk ? tsk_unpack_idx(pk) : -1;
  }
  double dist = INFINITY;
  if (j >= 0) {
    if (wa.inv[wb + j] == 0.f) {
      dist = sqm;
    } else {
      const double mi = wa.mu[wb + i];
      double c = 0.0;
      for (int t = 0; t < m; ++t) c = fma(static_cast<double>(x[i + t]) - mi, static_cast<double>(x[j + t]), c);
      const double rho = c / (sqrt(wa.ss[wb + i]) * sqrt(wa.ss[wb + j]));
      dist = sqrt(fmax(0.0, 2.0 * m * (1.0 - rho)));
    }
  }
  if (jc >= 0 && (sqm < dist || (sqm == dist && jc < j))) { dist = sqm; j = jc; }
  P[e] = static_cast<TP>(dist);
  I[e] = j;
}

template <typename TX>
tsk_status run_typed(tsk_ctx* ctx, const TX* X, int32_t n_streams, const tsk_mp_plan& plan, int32_t m, int32_t excl,
                     int32_t precision, void* P, int32_t* I, char* ws) {
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
    TSK_CUDA_TRY(ctx, cudaFuncSetAttribute(k_window_stats<TX>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    k_window_stats<TX><<<static_cast<unsigned>(plan.total_chunks), kWinThreads, smem, st>>>(
        X, plan.xoff, plan.len, plan.woff, plan.chunk_prefix, n_streams, m, f64 ? 1 : 0, wa, ctx->d_err);
    TSK_LAUNCH_CHECK(ctx, "k_window_stats");
    k_next_const<<<n_streams, kWinThreads, 0, st>>>(plan.len, plan.smask, plan.woff, m, wa);
    TSK_LAUNCH_CHECK(ctx, "k_next_const");
  }
  MpArgs a{};
  a.X = X;
  a.xoff = plan.xoff;
  a.len = plan.len;
  a.woff = plan.woff;
  a.tile_prefix = plan.tile_prefix;
  a.band_off = plan.band_off;
  a.band_prefix = plan.band_prefix;
  a.counter = counter;
  a.wa = wa;
  a.total_tiles = plan.total_tiles;
  a.n_streams = n_streams;
  a.m = m;
  a.excl = excl;
  a.excl4 = excl & ~3;
  a.H = plan.H;
  if (plan.total_tiles > 0) {
    if (f64) {
      const int64_t blocks = (plan.total_tiles + 127) / 128;
      for (int pass = 0; pass < 2; ++pass) {
        k_mp_diag_f64<TX><<<static_cast<unsigned>(blocks), 128, 0, st>>>(a, pass);
        TSK_LAUNCH_CHECK(ctx, "k_mp_diag_f64");
      }
    } else {
      int per_sm = 0;
      TSK_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mp_diag<kV, TX>, kWarps * 32, 0));
      per_sm = std::max(per_sm, 1);
      const int64_t want = (plan.total_tiles + kWarps - 1) / kWarps;
      const int64_t grid = std::min<int64_t>(want, static_cast<int64_t>(per_sm) * ctx->sm_count);
      {
        tsk_prof_scope ps(ctx, TSK_PROF_MP_DIAG);
        k_mp_diag<kV, TX><<<static_cast<unsigned>(grid), kWarps * 32, 0, st>>>(a);
      }
      TSK_LAUNCH_CHECK(ctx, "k_mp_diag");
    }
  }
  const int64_t total = plan.total_samples;
  if (total > 0) {
    const int64_t blocks = (total + 255) / 256;
    if (f64)
      k_mp_refine<TX, double><<<static_cast<unsigned>(blocks), 256, 0, st>>>(X, plan.xoff, plan.len, plan.smask, plan.woff, n_streams, total, m, excl, 1, wa, static_cast<double*>(P), I);
    else
      k_mp_refine<TX, float><<<static_cast<unsigned>(blocks), 256, 0, st>>>(X, plan.xoff, plan.len, plan.smask, plan.woff, n_streams, total, m, excl, 0, wa, static_cast<float*>(P), I);
    TSK_LAUNCH_CHECK(ctx, "k_mp_refine");
  }
  return TSK_OK;
}

}  // namespace

int tsk_mp_band_width() { return kD; }
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
    return run_typed<double>(ctx, static_cast<const double*>(X), n_streams, plan, m, excl, precision, P, I, ws);
  return run_typed<float>(ctx, static_cast<const float*>(X), n_streams, plan, m, excl, precision, P, I, ws);
}
