// Aggregation over the streams of a series (Def. 5: max over dimensions, the
// lowest stream on ties) and the ranked discords (Alg. 2 extended to a list of
// K by masking |i - i*| < topk_excl after each pick).  The aggregation is one
// grid-stride pass over every window of the batch; the K picks run in one CTA
// per series over the aggregated row (L2-resident by then).
#include "tsk_internal.cuh"

#include <algorithm>
#include <cmath>

namespace {

constexpr int kTopThreads = 1024;

template <typename TP>
__device__ __forceinline__ void better(TP v, int i, TP& bv, int& bi) {
  if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
}

// A[cum[s] + i] = max_g P_g[i], G = its stream (lowest on ties), for every
// window i < l of every series; consecutive threads take consecutive windows.
template <typename TP>
__global__ void __launch_bounds__(256) k_aggregate(const TP* __restrict__ P, const int64_t* __restrict__ cum,
                                                   const int32_t* __restrict__ len, int32_t n_series, int group, int m,
                                                   int64_t total, TP* __restrict__ Abuf, int32_t* __restrict__ Gbuf) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < total; p += stride) {
    const int s = tsk_find_segment<int64_t>(cum, n_series, p);
    const int n = len[s];
    const int i = static_cast<int>(p - cum[s]);
    if (i >= n - m + 1) continue;
    const int64_t pbase = static_cast<int64_t>(group) * cum[s];
    TP a = P[pbase + i];
    int gb = 0;
    for (int g = 1; g < group; ++g) {
      const TP v = P[pbase + static_cast<int64_t>(g) * n + i];
      if (v > a) { a = v; gb = g; }
    }
    Abuf[p] = a;
    Gbuf[p] = gb;
  }
}

template <typename TP>
__global__ void __launch_bounds__(kTopThreads) k_topk(const int32_t* __restrict__ I, const int64_t* __restrict__ cum,
                                                     const int32_t* __restrict__ len, int group, int m, int K, int te,
                                                     int32_t* __restrict__ idx, int32_t* __restrict__ grp,
                                                     TP* __restrict__ score, int32_t* __restrict__ nn,
                                                     TP* __restrict__ Abuf, const int32_t* __restrict__ Gbuf) {
  const int s = blockIdx.x;
  const int n = len[s];
  const int l = n - m + 1;
  const int64_t pbase = static_cast<int64_t>(group) * cum[s];
  TP* A = Abuf + cum[s];
  const int32_t* G = Gbuf + cum[s];
  const TP ninf = static_cast<TP>(-INFINITY);
  __shared__ TP sv[32];
  __shared__ int si[32];
  __shared__ int pick;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int r = 0; r < K; ++r) {
    TP bv = ninf;
    int bi = INT_MAX;
    for (int i = threadIdx.x; i < l; i += kTopThreads) better(A[i], i, bv, bi);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const TP ov = __shfl_xor_sync(TSK_FULL_MASK, bv, o);
      const int oi = __shfl_xor_sync(TSK_FULL_MASK, bi, o);
      better(ov, oi, bv, bi);
    }
    if (lane == 0) { sv[w] = bv; si[w] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      TP v = sv[0];
      int ii = si[0];
      for (int u = 1; u < kTopThreads / 32; ++u) better(sv[u], si[u], v, ii);
      const int64_t o = static_cast<int64_t>(s) * K + r;
      if (v == ninf || ii == INT_MAX) {
        pick = -1;
        idx[o] = -1; grp[o] = -1; nn[o] = -1;
        score[o] = static_cast<TP>(NAN);
      } else {
        pick = ii;
        const int g = G[ii];
        idx[o] = ii;
        grp[o] = g;
        score[o] = v;
        nn[o] = I[pbase + static_cast<int64_t>(g) * n + ii];
      }
    }
    __syncthreads();
    const int p = pick;
    if (p < 0) {
      for (int rr = r + 1 + threadIdx.x; rr < K; rr += kTopThreads) {
        const int64_t o = static_cast<int64_t>(s) * K + rr;
        idx[o] = -1; grp[o] = -1; nn[o] = -1;
        score[o] = static_cast<TP>(NAN);
      }
      break;
    }
    const int lo = max(0, p - te + 1), hi = min(l, p + te);
    for (int i = lo + threadIdx.x; i < hi; i += kTopThreads) A[i] = ninf;
    __syncthreads();
  }
}

}  // namespace

tsk_status tsk_launch_topk(tsk_ctx* ctx, const void* P, int p_dtype, const int32_t* I, int32_t n_series,
                           const int64_t* d_cum, const int32_t* d_len, int32_t group, int32_t m, int32_t K,
                           int32_t topk_excl, int32_t* idx, int32_t* grp, void* score, int32_t* nn, char* ws,
                           int64_t total_samples) {
  tsk_carver cv(ws);
  int32_t* G = cv.take<int32_t>(total_samples);
  const unsigned agg_blocks =
      static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((total_samples + 255) / 256, int64_t(ctx->sm_count) * 8)));
  if (p_dtype == TSK_F64) {
    double* A = cv.take<double>(total_samples);
    k_aggregate<double><<<agg_blocks, 256, 0, ctx->stream>>>(static_cast<const double*>(P), d_cum, d_len, n_series, group, m, total_samples, A, G);
    TSK_LAUNCH_CHECK(ctx, "k_aggregate");
    k_topk<double><<<n_series, kTopThreads, 0, ctx->stream>>>(I, d_cum, d_len, group, m, K, topk_excl, idx, grp, static_cast<double*>(score), nn, A, G);
  } else {
    float* A = cv.take<float>(total_samples);
    k_aggregate<float><<<agg_blocks, 256, 0, ctx->stream>>>(static_cast<const float*>(P), d_cum, d_len, n_series, group, m, total_samples, A, G);
    TSK_LAUNCH_CHECK(ctx, "k_aggregate");
    k_topk<float><<<n_series, kTopThreads, 0, ctx->stream>>>(I, d_cum, d_len, group, m, K, topk_excl, idx, grp, static_cast<float*>(score), nn, A, G);
  }
  TSK_LAUNCH_CHECK(ctx, "k_topk");
  return TSK_OK;
}
