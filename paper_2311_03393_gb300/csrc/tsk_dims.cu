// Discord dimension detection (Alg. 3) for the discords of the time-detection
// phase, and the gather of each chosen raw stream for the optional refinement.
//
// For discord r of series s at window i* in sketch stream g*, every raw stream
// j of the group J_g* = {j : R[j, g*] != 0} is scored by the 1NN distance of
// its own window i* (Def. 6 at a single row, self-join exclusion |t - i*| <
// excl), and j* is the first j (ascending) whose score exceeds every earlier
// one, starting from 0.
//
// Pipeline per call:
//   1. k_dd_scan    one CTA per (series, discord, stream, chunk of 1024 windows):
//                   the distance profile of the query window i* against the
//                   chunk.  The chunk is staged in shared memory shifted by its
//                   first sample, window means and norms come from float64
//                   chunk-local prefix sums, and each thread forms 4 consecutive
//                   sliding dot products with the centred query in float32
//                   (16 FMAs per 2 vector loads).  The largest correlation and
//                   lowest window index merge per (series, discord, stream) in
//                   a packed 64-bit word with atomicMax.
//   2. k_dd_select  one warp per (series, discord): the chosen window of every
//                   stream of the group is re-evaluated exactly (compensated
//                   sums), then the strict running maximum over ascending j.
//   3. k_dd_gather  (optional) copies stream j* of every discord into a
//                   contiguous buffer for a self-join refinement profile.
#include "tsk_internal.cuh"
#include "tsk_rho.cuh"

#include <algorithm>
#include <cmath>

namespace {

constexpr int kTW = 1024;          // windows per scan item
constexpr int kScanThreads = 256;  // 4 windows per thread
constexpr double kConstRelVar = 1e-12;

struct DimArgs {
  const int64_t* cum;          // [n_series + 1] sample offsets of series (per stream)
  const int32_t* len;          // [n_series]
  const int64_t* item_prefix;  // [n_series + 1] scan items before each series
  const float* R;              // d x k
  const int32_t* idx;          // n_series x K
  const int32_t* grp;          // n_series x K
  unsigned long long* best;    // n_series x K x d
  int n_series, d, k, m, excl, K;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(TSK_FULL_MASK, v, o);
  return v;
}

// Sum over the block (256 threads); every thread receives the total.
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int q = 0; q < kScanThreads / 32; ++q) t += red[q];
  return t;
}

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) { return a > b ? a : b; }

template <typename TX>
__global__ void __launch_bounds__(kScanThreads) k_dd_scan(const TX* __restrict__ T, DimArgs a, int64_t total_items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = a.m;
  const int m4 = (m + 3) & ~3;
  const int xs_len = kTW + m4 + 8;                   // staged samples (zero padded)
  float* xs = reinterpret_cast<float*>(smem_raw);     // [xs_len]
  float* qs = xs + xs_len;                            // [m4]
  double* p1 = reinterpret_cast<double*>(qs + m4 + ((m4 & 1) ? 1 : 0));  // [kTW + m] prefix of shifted samples
  double* p2 = p1 + (kTW + m);                        // [kTW + m] prefix of their squares
  __shared__ double red[kScanThreads / 32];
  __shared__ double seg1[kScanThreads], seg2[kScanThreads];
  __shared__ unsigned long long wbest[kScanThreads / 32];

  for (int64_t item = blockIdx.x; item < total_items; item += gridDim.x) {
    const int s = tsk_find_segment<int64_t>(a.item_prefix, a.n_series, item);
    const int n = a.len[s];
    const int l = n - m + 1;
    const int chunks = (l + kTW - 1) / kTW;
    int64_t rem = item - a.item_prefix[s];
    const int c = static_cast<int>(rem % chunks);
    rem /= chunks;
    const int j = static_cast<int>(rem % a.d);
    const int r = static_cast<int>(rem / a.d);
    const int i_star = a.idx[s * a.K + r];
    if (i_star < 0 || i_star >= l) continue;
    const int g_star = a.grp[s * a.K + r];
    if (g_star < 0 || g_star >= a.k || a.R[static_cast<int64_t>(j) * a.k + g_star] == 0.f) continue;
    const int t0 = c * kTW;
    const int nw = min(kTW, l - t0);
    // this chunk holds no admissible window when it lies inside the exclusion zone
    if (t0 > i_star - a.excl && t0 + nw - 1 < i_star + a.excl) continue;
    const TX* x = T + a.cum[s] * static_cast<int64_t>(a.d) + static_cast<int64_t>(j) * n;

    // ---- query: float64 mean and variance, centred float32 copy ----
    double sq = 0.0;
    for (int t = threadIdx.x; t < m; t += kScanThreads) sq += static_cast<double>(x[i_star + t]);
    const double mu_q = block_sum(sq, red) / m;
    double vq = 0.0, sqs = 0.0, nq = 0.0;
    for (int t = threadIdx.x; t < m4; t += kScanThreads) {
      float v = 0.f;
      if (t < m) {
        const double dv = static_cast<double>(x[i_star + t]) - mu_q;
        vq += dv * dv;
        v = static_cast<float>(dv);
      }
      qs[t] = v;
      sqs += static_cast<double>(v);
      nq += static_cast<double>(v) * static_cast<double>(v);
    }
    const double var_q = block_sum(vq, red) / m;
    const double sum_qs = block_sum(sqs, red);
    const double norm_qs = sqrt(block_sum(nq, red));
    const bool q_const = var_q <= kConstRelVar * fmax(1.0, mu_q * mu_q);

    // ---- chunk: samples shifted by the first one, float64 prefix sums ----
    const double x_ref = static_cast<double>(x[t0]);
    const int ns = nw + m - 1;                          // samples the chunk's windows touch
    for (int p = threadIdx.x; p < xs_len; p += kScanThreads)
      xs[p] = (p < ns) ? static_cast<float>(static_cast<double>(x[t0 + p]) - x_ref) : 0.f;
    // segmented inclusive scan of (y, y^2), y = x - x_ref in float64, over ns samples
    const int seg = (ns + kScanThreads - 1) / kScanThreads;
    const int lo = threadIdx.x * seg, hi = min(ns, lo + seg);
    double a1 = 0.0, a2 = 0.0;
    for (int p = lo; p < hi; ++p) {
      const double y = static_cast<double>(x[t0 + p]) - x_ref;
      a1 += y;
      a2 += y * y;
    }
    seg1[threadIdx.x] = a1;
    seg2[threadIdx.x] = a2;
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive scan of the 256 segment totals by one warp
      double c1 = 0.0, c2 = 0.0;
      for (int q = 0; q < kScanThreads / 32; ++q) {
        const int u = q * 32 + threadIdx.x;
        double v1 = seg1[u], v2 = seg2[u];
        double i1 = v1, i2 = v2;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const double t1 = __shfl_up_sync(TSK_FULL_MASK, i1, o), t2 = __shfl_up_sync(TSK_FULL_MASK, i2, o);
          if (threadIdx.x >= o) { i1 += t1; i2 += t2; }
        }
        seg1[u] = c1 + i1 - v1;
        seg2[u] = c2 + i2 - v2;
        c1 += __shfl_sync(TSK_FULL_MASK, i1, 31);
        c2 += __shfl_sync(TSK_FULL_MASK, i2, 31);
      }
    }
    __syncthreads();
    {
      double b1 = seg1[threadIdx.x], b2 = seg2[threadIdx.x];
      if (threadIdx.x == 0) { p1[0] = 0.0; p2[0] = 0.0; }
      for (int p = lo; p < hi; ++p) {
        const double y = static_cast<double>(x[t0 + p]) - x_ref;
        b1 += y;
        b2 += y * y;
        p1[p + 1] = b1;
        p2[p + 1] = b2;
      }
    }
    __syncthreads();

    // ---- 4 sliding dot products per thread ----
    const int w0 = threadIdx.x * 4;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const float4* xs4 = reinterpret_cast<const float4*>(xs);
    const float4* qs4 = reinterpret_cast<const float4*>(qs);
    float4 A = xs4[threadIdx.x];
    for (int kk = 0; kk < m4; kk += 4) {
      const float4 B = xs4[threadIdx.x + (kk >> 2) + 1];
      const float4 q = qs4[kk >> 2];
      const float v[8] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        acc[u] = __fmaf_rn(q.x, v[u + 0], acc[u]);
        acc[u] = __fmaf_rn(q.y, v[u + 1], acc[u]);
        acc[u] = __fmaf_rn(q.z, v[u + 2], acc[u]);
        acc[u] = __fmaf_rn(q.w, v[u + 3], acc[u]);
      }
      A = B;
    }

    // ---- correlations and the chunk's best (largest key, lowest index) ----
    unsigned long long best = 0ull;
    const float inv_q = (norm_qs > 0.0) ? static_cast<float>(1.0 / norm_qs) : 0.f;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int w = w0 + u;
      const int t = t0 + w;
      if (w >= nw || (t > i_star - a.excl && t < i_star + a.excl)) continue;
      const double s1 = p1[w + m] - p1[w], s2 = p2[w + m] - p2[w];
      const double mean_y = s1 / m;
      const double var = fmax(0.0, s2 / m - mean_y * mean_y);
      const double mu_t = x_ref + mean_y;
      const bool t_const = var <= kConstRelVar * fmax(1.0, mu_t * mu_t);
      float key;
      if (q_const) key = t_const ? 1.0f : 0.5f;       // dist 0 to a constant window, sqrt(m) otherwise
      else if (t_const) key = 0.5f;                    // 2m(1 - 1/2) = m
      else {
        const float cov = acc[u] - static_cast<float>(mean_y * sum_qs);
        const float inv_t = static_cast<float>(1.0 / sqrt(m * var));
        key = fminf(1.0f, fmaxf(-1.0f, cov * inv_q * inv_t));
      }
      best = umax64(best, tsk_pack(key, t));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = umax64(best, __shfl_xor_sync(TSK_FULL_MASK, best, o));
    if ((threadIdx.x & 31) == 0) wbest[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long b = 0ull;
#pragma unroll
      for (int q = 0; q < kScanThreads / 32; ++q) b = umax64(b, wbest[q]);
      if (b) atomicMax(&a.best[(static_cast<int64_t>(s) * a.K + r) * a.d + j], b);
    }
    __syncthreads();  // shared buffers are reused by the next item
  }
}

// float64 mean and the constant-window test of x[i .. i+m)
template <typename TX>
__device__ void window_mean_const(const TX* x, int i, int m, double* mean, bool* is_const) {
  double s = 0.0;
  for (int t = 0; t < m; ++t) s += static_cast<double>(x[i + t]);
  const double mu = s / m;
  double v = 0.0;
  for (int t = 0; t < m; ++t) {
    const double dv = static_cast<double>(x[i + t]) - mu;
    v += dv * dv;
  }
  *mean = mu;
  *is_const = (v / m) <= kConstRelVar * fmax(1.0, mu * mu);
}

template <typename TX>
__global__ void __launch_bounds__(256) k_dd_select(const TX* __restrict__ T, DimArgs a, int32_t* __restrict__ dim,
                                                   double* __restrict__ dim_score, int32_t* __restrict__ dim_nn,
                                                   double* __restrict__ dim_scores) {
  const int64_t wid = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= static_cast<int64_t>(a.n_series) * a.K) return;
  const int s = static_cast<int>(wid / a.K);
  const int n = a.len[s];
  const int l = n - a.m + 1;
  const int i_star = a.idx[wid];
  const int g_star = a.grp[wid];
  const bool valid = i_star >= 0 && i_star < l && g_star >= 0 && g_star < a.k;
  double bs = 0.0;     // strict running maximum from 0 over this lane's j (ascending)
  int bj = -1, bnn = -1;
  int first = a.d;     // lowest j of the group
  double first_s = 0.0;
  int first_nn = -1;
  const double m2 = 2.0 * a.m;
  const double sqm = sqrt(static_cast<double>(a.m));
  for (int j = lane; j < a.d; j += 32) {
    double sc = NAN;
    int nn = -1;
    if (valid && a.R[static_cast<int64_t>(j) * a.k + g_star] != 0.f) {
      const TX* x = T + a.cum[s] * static_cast<int64_t>(a.d) + static_cast<int64_t>(j) * n;
      const unsigned long long p = a.best[wid * a.d + j];
      if (p == 0ull) {
        sc = INFINITY;  // no admissible neighbour
      } else {
        nn = tsk_unpack_idx(p);
        double mq, mt;
        bool cq, ct;
        window_mean_const(x, i_star, a.m, &mq, &cq);
        window_mean_const(x, nn, a.m, &mt, &ct);
        if (cq) sc = ct ? 0.0 : sqm;
        else if (ct) sc = sqm;
        else {
          const double rho = tsk::window_rho(x, i_star, nn, a.m, mq, mt);
          sc = sqrt(fmax(0.0, m2 * (1.0 - rho)));
        }
      }
      if (j < first) { first = j; first_s = sc; first_nn = nn; }
      if (sc > bs) { bs = sc; bj = j; bnn = nn; }
    }
    if (dim_scores) dim_scores[wid * a.d + j] = sc;
  }
  // combine lanes: the larger score, then the lower j; and the lowest group member
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double os = __shfl_xor_sync(TSK_FULL_MASK, bs, o);
    const int oj = __shfl_xor_sync(TSK_FULL_MASK, bj, o);
    const int onn = __shfl_xor_sync(TSK_FULL_MASK, bnn, o);
    if (oj >= 0 && (bj < 0 || os > bs || (os == bs && oj < bj))) { bs = os; bj = oj; bnn = onn; }
    const int of = __shfl_xor_sync(TSK_FULL_MASK, first, o);
    const double ofs = __shfl_xor_sync(TSK_FULL_MASK, first_s, o);
    const int ofn = __shfl_xor_sync(TSK_FULL_MASK, first_nn, o);
    if (of < first) { first = of; first_s = ofs; first_nn = ofn; }
  }
  if (lane == 0) {
    if (bj >= 0) { dim[wid] = bj; dim_score[wid] = bs; dim_nn[wid] = bnn; }
    else if (first < a.d) { dim[wid] = first; dim_score[wid] = first_s; dim_nn[wid] = first_nn; }
    else { dim[wid] = -1; dim_score[wid] = NAN; dim_nn[wid] = -1; }
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
  const size_t floats = static_cast<size_t>(kTW + m4 + 8) + m4 + ((m4 & 1) ? 1 : 0);
  return floats * 4 + static_cast<size_t>(2) * (kTW + m) * 8 + 16;
}

template <typename TX>
tsk_status run_dims(tsk_ctx* ctx, const TX* T, const DimArgs& a, int64_t total_items, int32_t* dim, double* dim_score,
                    int32_t* dim_nn, double* dim_scores, TX* T_sel, int64_t total_samples) {
  cudaStream_t st = ctx->stream;
  TSK_CUDA_TRY(ctx, cudaMemsetAsync(a.best, 0, sizeof(unsigned long long) * static_cast<size_t>(a.n_series) * a.K * a.d, st));
  const size_t smem = scan_smem_bytes(a.m);
  TSK_CUDA_TRY(ctx, cudaFuncSetAttribute(k_dd_scan<TX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem)));
  if (total_items > 0) {
    int per_sm = 0;
    TSK_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dd_scan<TX>, kScanThreads, smem));
    const int64_t grid = std::min<int64_t>(total_items, static_cast<int64_t>(std::max(per_sm, 1)) * ctx->sm_count);
    k_dd_scan<TX><<<static_cast<unsigned>(grid), kScanThreads, smem, st>>>(T, a, total_items);
    TSK_LAUNCH_CHECK(ctx, "k_dd_scan");
  }
  const int64_t warps = static_cast<int64_t>(a.n_series) * a.K;
  k_dd_select<TX><<<static_cast<unsigned>((warps * 32 + 255) / 256), 256, 0, st>>>(T, a, dim, dim_score, dim_nn,
                                                                                     dim_scores);
  TSK_LAUNCH_CHECK(ctx, "k_dd_select");
  if (T_sel && total_samples > 0) {
    const int64_t total = total_samples * a.K;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, static_cast<int64_t>(ctx->sm_count) * 16);
    k_dd_gather<TX><<<static_cast<unsigned>(blocks), 256, 0, st>>>(T, a.cum, a.len, dim, a.n_series, a.d, a.K, total,
                                                                     T_sel);
    TSK_LAUNCH_CHECK(ctx, "k_dd_gather");
  }
  return TSK_OK;
}

}  // namespace

int tsk_dims_window_chunk() { return kTW; }

tsk_status tsk_launch_dims(tsk_ctx* ctx, const void* T, int t_dtype, int32_t n_series, const int64_t* d_cum,
                           const int32_t* d_len, const int64_t* d_item_prefix, int64_t total_items,
                           int64_t total_samples, int32_t d, const float* R, int32_t k, int32_t m, int32_t excl,
                           int32_t K, const int32_t* idx, const int32_t* grp, int32_t* dim, double* dim_score,
                           int32_t* dim_nn, double* dim_scores, void* T_sel, char* ws) {
  DimArgs a;
  a.cum = d_cum;
  a.len = d_len;
  a.item_prefix = d_item_prefix;
  a.R = R;
  a.idx = idx;
  a.grp = grp;
  tsk_carver cv(ws);
  a.best = cv.take<unsigned long long>(static_cast<size_t>(n_series) * K * d);
  a.n_series = n_series;
  a.d = d;
  a.k = k;
  a.m = m;
  a.excl = excl;
  a.K = K;
  if (t_dtype == TSK_F64)
    return run_dims<double>(ctx, static_cast<const double*>(T), a, total_items, dim, dim_score, dim_nn, dim_scores,
                            static_cast<double*>(T_sel), total_samples);
  return run_dims<float>(ctx, static_cast<const float*>(T), a, total_items, dim, dim_score, dim_nn, dim_scores,
                         static_cast<float*>(T_sel), total_samples);
}

size_t tsk_dims_ws_bytes(int32_t n_series, int32_t K, int32_t d) {
  return tsk_carver::bytes_for(static_cast<size_t>(n_series) * K * d, 8);
}
