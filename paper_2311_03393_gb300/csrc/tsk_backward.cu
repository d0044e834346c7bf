// Adjoint of the ranked discord scores with respect to the input series T and
// the projection R (the derivative of Def. 3 through the sketch of Alg. 1 and
// the global z-normalisation of Sec. III-A; not itself in the paper).
//
// For a selected score dist(x, y), x = S_g[i:i+m], y = S_g[j:j+m] (j the
// nearest neighbour), rho their correlation and x_hat, y_hat the z-normalised
// windows:  d dist/dx = (rho x_hat - y_hat)/(sigma_x dist),
//           d dist/dy = (rho y_hat - x_hat)/(sigma_y dist).
// dS is non-zero on 2m positions per score, so it is kept compact:
//   k_bw_windows  dS of each score (2 x m values)
//   k_bw_dims     per (series, dim j): a_j = mean(dT_bar_j), b_j = mean(dT_bar_j T_bar_j), dR
//   k_bw_dense    dT_j = (- a_j - T_bar_j b_j) / sigma_j everywhere (one FMA per element)
//   k_bw_scatter  dT_j += (R_jg dS_g) / sigma_j on the 2m positions of each score
#include "tsk_internal.cuh"

#include <algorithm>
#include <cmath>

namespace {

constexpr int kBwThreads = 128;

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(TSK_FULL_MASK, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int u = 0; u < (int)(blockDim.x >> 5); ++u) t += sh[u];
  return t;
}

__global__ void __launch_bounds__(kBwThreads) k_bw_windows(const float* __restrict__ dscore, const int32_t* __restrict__ idx,
                                                           const int32_t* __restrict__ grp, const int32_t* __restrict__ nn,
                                                           int K, const float* __restrict__ S, const int64_t* __restrict__ cum,
                                                           const int32_t* __restrict__ len, int k, int m,
                                                           float* __restrict__ dSc) {
  __shared__ double sh[32];
  const int64_t sr = blockIdx.x;
  const int s = static_cast<int>(sr / K);
  float* out = dSc + sr * 2 * m;
  const int i = idx[sr], g = grp[sr], j = nn[sr];
  const int n = len[s];
  bool ok = i >= 0 && j >= 0 && g >= 0 && g < k && i + m <= n && j + m <= n;
  double mx = 0, my = 0, sx = 0, sy = 0, rho = 0, dist = 0;
  const float* X = S + static_cast<int64_t>(k) * cum[s] + static_cast<int64_t>(ok ? g : 0) * n;
  if (ok) {
    double a = 0, b = 0;
    for (int t = threadIdx.x; t < m; t += kBwThreads) { a += X[i + t]; b += X[j + t]; }
    mx = block_sum(a, sh) / m;
    my = block_sum(b, sh) / m;
    a = 0; b = 0;
    for (int t = threadIdx.x; t < m; t += kBwThreads) {
      const double u = X[i + t] - mx, v = X[j + t] - my;
      a += u * u;
      b += v * v;
    }
    sx = sqrt(block_sum(a, sh) / m);
    sy = sqrt(block_sum(b, sh) / m);
    ok = sx > 0 && sy > 0;
  }
  if (ok) {
    double a = 0, b = 0;
    for (int t = threadIdx.x; t < m; t += kBwThreads) {
      const double u = (X[i + t] - mx) / sx, v = (X[j + t] - my) / sy;
      a += u * v;
      b += (u - v) * (u - v);
    }
    rho = block_sum(a, sh) / m;
    dist = sqrt(block_sum(b, sh));
    ok = dist > 0;
  }
  const double w = ok ? static_cast<double>(dscore[sr]) : 0.0;
  for (int t = threadIdx.x; t < m; t += kBwThreads) {
    float gx = 0.f, gy = 0.f;
    if (ok) {
      const double u = (X[i + t] - mx) / sx, v = (X[j + t] - my) / sy;
      gx = static_cast<float>(w * (rho * u - v) / (sx * dist));
      gy = static_cast<float>(w * (rho * v - u) / (sy * dist));
    }
    out[t] = gx;
    out[m + t] = gy;
  }
}

template <typename TIn>
__global__ void __launch_bounds__(kBwThreads) k_bw_dims(const float* __restrict__ dSc, const int32_t* __restrict__ idx,
                                                        const int32_t* __restrict__ grp, const int32_t* __restrict__ nn,
                                                        int K, const TIn* __restrict__ T, const double* __restrict__ stats,
                                                        const float* __restrict__ R, const int64_t* __restrict__ cum,
                                                        const int32_t* __restrict__ len, int d, int k, int m,
                                                        double* __restrict__ ab, float* __restrict__ dR) {
  __shared__ double sh[32];
  const int s = blockIdx.x / d, j = blockIdx.x % d;
  const int n = len[s];
  const double mu = stats[2 * (static_cast<int64_t>(s) * d + j)];
  const double sg = stats[2 * (static_cast<int64_t>(s) * d + j) + 1];
  if (!(sg > 0)) {
    if (threadIdx.x == 0) { ab[2 * blockIdx.x] = 0; ab[2 * blockIdx.x + 1] = 0; }
    return;
  }
  const double ri = 1.0 / sg;
  const TIn* Tj = T + static_cast<int64_t>(d) * cum[s] + static_cast<int64_t>(j) * n;
  double sa = 0, sb = 0;
  for (int r = 0; r < K; ++r) {
    const int64_t sr = static_cast<int64_t>(s) * K + r;
    const int g = grp[sr];
    if (idx[sr] < 0 || nn[sr] < 0 || g < 0 || g >= k) continue;
    const double Rjg = R[static_cast<int64_t>(j) * k + g];
    const float* v = dSc + sr * 2 * m;
    double dr = 0;
    for (int e = threadIdx.x; e < 2 * m; e += kBwThreads) {
      const int pos = (e < m) ? idx[sr] + e : nn[sr] + (e - m);
      const double tb = (static_cast<double>(Tj[pos]) - mu) * ri;
      sa += Rjg * v[e];
      sb += Rjg * v[e] * tb;
      dr += tb * v[e];
    }
    dr = block_sum(dr, sh);
    if (threadIdx.x == 0 && dr != 0.0) atomicAdd(&dR[static_cast<int64_t>(j) * k + g], static_cast<float>(dr));
  }
  sa = block_sum(sa, sh);
  sb = block_sum(sb, sh);
  if (threadIdx.x == 0) { ab[2 * blockIdx.x] = sa / n; ab[2 * blockIdx.x + 1] = sb / n; }
}

// dT_j[t] = c0 + c1 (T_j[t] - mu_j) with c0 = -a_j / sigma_j, c1 = -b_j / sigma_j^2
// (the same as (-a_j - T_bar_j[t] b_j) / sigma_j), 0 for a constant stream.  A
// CTA takes a chunk of kBwChunk samples of one (series, stream) row at a time,
// the row's constants formed in float64; float32 series take the mean as two
// floats, so the centred sample is exact to float32 rounding, and one FMA per
// element.  Coalesced passes along time.
constexpr int kBwChunk = 4096;  // samples of a row per work item of k_bw_dense

template <typename TIn>
__global__ void __launch_bounds__(256) k_bw_dense(const TIn* __restrict__ T, const double* __restrict__ stats,
                                                  const double* __restrict__ ab, const int64_t* __restrict__ cum,
                                                  const int32_t* __restrict__ len, int n_series, int d,
                                                  int chunks_per_row, float* __restrict__ dT) {
  const int64_t items = static_cast<int64_t>(n_series) * d * chunks_per_row;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int64_t q = it / chunks_per_row;
    const int s = static_cast<int>(q / d), j = static_cast<int>(q % d);
    const int n = len[s];
    const int t0 = static_cast<int>(it % chunks_per_row) * kBwChunk;
    if (t0 >= n) continue;
    const int t1 = min(n, t0 + kBwChunk);
    const int64_t base = static_cast<int64_t>(d) * cum[s] + static_cast<int64_t>(j) * n;
    const double sg = stats[2 * q + 1];
    if (!(sg > 0.0)) {
      for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) dT[base + t] = 0.f;
      continue;
    }
    const double mu = stats[2 * q], r = 1.0 / sg;
    const double c0 = -ab[2 * q] * r, c1 = -ab[2 * q + 1] * r * r;
    if constexpr (sizeof(TIn) == 4) {
      const float muh = static_cast<float>(mu), mul = static_cast<float>(mu - static_cast<double>(muh));
      const float f0 = static_cast<float>(c0), f1 = static_cast<float>(c1);
      for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x)
        dT[base + t] = __fmaf_rn(f1, __fsub_rn(__fsub_rn(T[base + t], muh), mul), f0);
    } else {
      for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x)
        dT[base + t] = static_cast<float>(c0 + c1 * (static_cast<double>(T[base + t]) - mu));
    }
  }
}

__global__ void k_bw_scatter(const float* __restrict__ dSc, const int32_t* __restrict__ idx, const int32_t* __restrict__ grp,
                             const int32_t* __restrict__ nn, int K, const double* __restrict__ stats,
                             const float* __restrict__ R, const int64_t* __restrict__ cum, const int32_t* __restrict__ len,
                             int d, int k, int m, int64_t total, float* __restrict__ dT) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int64_t sr = e / (2 * m);
  const int u = static_cast<int>(e % (2 * m));
  const int s = static_cast<int>(sr / K);
  const int g = grp[sr];
  if (idx[sr] < 0 || nn[sr] < 0 || g < 0 || g >= k) return;
  const float v = dSc[e];
  if (v == 0.f) return;
  const int pos = (u < m) ? idx[sr] + u : nn[sr] + (u - m);
  const int n = len[s];
  const int64_t base = static_cast<int64_t>(d) * cum[s] + pos;
  for (int j = 0; j < d; ++j) {
    const double sg = stats[2 * (static_cast<int64_t>(s) * d + j) + 1];
    if (!(sg > 0)) continue;
    const float add = static_cast<float>(static_cast<double>(R[static_cast<int64_t>(j) * k + g]) * v / sg);
    atomicAdd(&dT[base + static_cast<int64_t>(j) * n], add);
  }
}

}  // namespace

tsk_status tsk_launch_backward(tsk_ctx* ctx, const float* dscore, const int32_t* idx, const int32_t* grp,
                               const int32_t* nn, int32_t K, const void* T, int t_dtype, const double* stats,
                               const float* R, const float* S, int32_t n_series, const int64_t* d_cum,
                               const int32_t* d_len, int32_t max_len, int32_t d, int32_t k,
                               int32_t m, float* dT, float* dR, char* ws) {
  tsk_carver cv(ws);
  const int64_t nsel = static_cast<int64_t>(n_series) * K;
  float* dSc = cv.take<float>(nsel * 2 * m);
  double* ab = cv.take<double>(static_cast<int64_t>(n_series) * d * 2);
  cudaStream_t st = ctx->stream;
  TSK_CUDA_TRY(ctx, cudaMemsetAsync(dR, 0, sizeof(float) * static_cast<size_t>(d) * k, st));
  k_bw_windows<<<static_cast<unsigned>(nsel), kBwThreads, 0, st>>>(dscore, idx, grp, nn, K, S, d_cum, d_len, k, m, dSc);
  TSK_LAUNCH_CHECK(ctx, "k_bw_windows");
  const unsigned nd = static_cast<unsigned>(static_cast<int64_t>(n_series) * d);
  const int chunks_per_row = std::max(1, (max_len + kBwChunk - 1) / kBwChunk);
  const int64_t items = static_cast<int64_t>(nd) * chunks_per_row;
  const unsigned dblocks = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(items, int64_t(ctx->sm_count) * 8)));
  const int64_t sc = nsel * 2 * m;
  const unsigned sblocks = static_cast<unsigned>((sc + 255) / 256);
  if (t_dtype == TSK_F64) {
    k_bw_dims<double><<<nd, kBwThreads, 0, st>>>(dSc, idx, grp, nn, K, static_cast<const double*>(T), stats, R, d_cum, d_len, d, k, m, ab, dR);
    TSK_LAUNCH_CHECK(ctx, "k_bw_dims");
    k_bw_dense<double><<<dblocks, 256, 0, st>>>(static_cast<const double*>(T), stats, ab, d_cum, d_len, n_series, d, chunks_per_row, dT);
  } else {
    k_bw_dims<float><<<nd, kBwThreads, 0, st>>>(dSc, idx, grp, nn, K, static_cast<const float*>(T), stats, R, d_cum, d_len, d, k, m, ab, dR);
    TSK_LAUNCH_CHECK(ctx, "k_bw_dims");
    k_bw_dense<float><<<dblocks, 256, 0, st>>>(static_cast<const float*>(T), stats, ab, d_cum, d_len, n_series, d, chunks_per_row, dT);
  }
  TSK_LAUNCH_CHECK(ctx, "k_bw_dense");
  if (sblocks > 0) {
    k_bw_scatter<<<sblocks, 256, 0, st>>>(dSc, idx, grp, nn, K, stats, R, d_cum, d_len, d, k, m, sc, dT);
    TSK_LAUNCH_CHECK(ctx, "k_bw_scatter");
  }
  return TSK_OK;
}
