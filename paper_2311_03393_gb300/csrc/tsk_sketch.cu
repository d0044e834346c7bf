// Global z-normalisation and the random-projection sketch S = R^T T_bar
// (Sec. III-A, Alg. 1), plus dimension addition/deletion (Sec. III-C).
//
// The sketch is a dense contraction over d with a tiny output width k; it is
// bound by reading T once.  In bfloat16 mode each element of T is normalised
// in float64, rounded to bfloat16 (nearest even) and fed to the tensor cores;
// products are summed in float32.
#include "tsk_internal.cuh"
#include "tsk_ff.cuh"

#include <algorithm>
#include <cmath>
#include <type_traits>

namespace {

constexpr int kStatThreads = 256;

// ---------------------------------------------------------------------------
// Column statistics: mean and population std of every stream, float64.
// Sums are taken of x - x[0] (a shift that keeps them well conditioned).  For
// float32 series they are accumulated in float-float (the shift is exact as a
// two-sum, squares as product plus fma error), ~2^-44 relative, so the FP64
// pipe is used only for the final combination.
// ---------------------------------------------------------------------------
template <typename TIn>
__global__ void __launch_bounds__(kStatThreads) k_colstats(const TIn* __restrict__ T, const int64_t* __restrict__ off,
                                                           const int32_t* __restrict__ len, double* __restrict__ stats,
                                                           int* __restrict__ err) {
  const int64_t q = blockIdx.x;
  const int64_t base = off[q];
  const int n = len[q];
  const double x0 = tsk_ld(T, base);
  double s1 = 0.0, s2 = 0.0;
  bool bad = false;
  if constexpr (std::is_same<TIn, float>::value) {
    const float xf0 = T[base];
    FF a1{0.f, 0.f}, a2{0.f, 0.f};
    for (int t = threadIdx.x; t < n; t += kStatThreads) {
      const float x = T[base + t];
      bad |= !isfinite(x);
      const FF y = ff_two_sum(x, -xf0);
      a1 = ff_add(a1, y);
      a2 = ff_add(a2, ff_sqr(y));
    }
    s1 = static_cast<double>(a1.h) + static_cast<double>(a1.l);
    s2 = static_cast<double>(a2.h) + static_cast<double>(a2.l);
  } else {
    for (int t = threadIdx.x; t < n; t += kStatThreads) {
      const double x = tsk_ld(T, base + t);
      bad |= !isfinite(x);
      const double y = x - x0;
      s1 += y;
      s2 = fma(y, y, s2);
    }
  }
  if (bad) atomicOr(err, TSK_DEVERR_NONFINITE);
  __shared__ double r1[kStatThreads / 32], r2[kStatThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(TSK_FULL_MASK, s1, o);
    s2 += __shfl_xor_sync(TSK_FULL_MASK, s2, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { r1[w] = s1; r2[w] = s2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int u = 0; u < kStatThreads / 32; ++u) { a += r1[u]; b += r2[u]; }
    const double mean_y = a / n;
    const double var = fmax(0.0, b / n - mean_y * mean_y);
    stats[2 * q + 0] = x0 + mean_y;
    stats[2 * q + 1] = sqrt(var);
  }
}

// Normalised element in float64: (x - mu) / sigma, 0 for a constant stream.
__device__ __forceinline__ double tsk_tbar(double x, double mu, double rinv) { return (x - mu) * rinv; }

// Per-stream constants of the float32 fast path: mu = muh + mul, 1/sigma ~ rh,
// and the two coefficients of its safety threshold.
struct NormC {
  double mu, r;   // float64 mean and 1/sigma (the reference)
  float muh, mul, rh, t1, t2;
};
__device__ __forceinline__ NormC make_normc(double mu, double r) {
  NormC c;
  c.mu = mu;
  c.r = r;
  c.muh = static_cast<float>(mu);
  c.mul = static_cast<float>(mu - static_cast<double>(c.muh));
  c.rh = static_cast<float>(r);
  c.t1 = static_cast<float>(0x1p-21 * r * fabs(mu)) * 1.0001f;  // rounded up
  c.t2 = static_cast<float>(0x1p-21 * r) * 1.0001f;
  return c;
}

// bfloat16 of the float64 value (x - mu) * r, computed without float64 in almost
// all cases.  v = ((x - muh) - mul) * rh in float32 differs from the float64
// value by at most E = 2^-21 |v| + A, A = 2^-45 r (|mu| + |x|) (four float32
// roundings plus the two-term mean's residual).  A float32 ulp of a normal v
// exceeds 2^-24 |v|, so where |v| >= 2^24 A = t1 + t2 |x| the error is below 9
// ulps of v; if v's low 16 bits are then at least 10 ulps from the bfloat16
// rounding midpoint (0x8000), no midpoint lies between v and the float64 value
// and both round (nearest, ties to even) to the same bfloat16.  Otherwise
// (about 1e-3 of elements) the float64 value is formed and rounded.
__device__ __forceinline__ uint16_t tbar_bf16(float x, const NormC& c) {
  const float v = __fmul_rn(__fsub_rn(__fsub_rn(x, c.muh), c.mul), c.rh);
  const float thr = fmaxf(__fmaf_rn(c.t2, fabsf(x), c.t1), 0x1p-100f);
  const uint32_t bits = __float_as_uint(v);
  if (fabsf(v) >= thr && ((bits & 0xffffu) - 0x7ff6u) > 20u) {  // low 16 bits outside 0x8000 +- 10
    const uint32_t rnd = 0x7fffu + ((bits >> 16) & 1u);
    return static_cast<uint16_t>((bits + rnd) >> 16);
  }
  return tsk_f64_to_bf16_bits(tsk_tbar(static_cast<double>(x), c.mu, c.r));
}
__device__ __forceinline__ uint16_t tbar_bf16(double x, const NormC& c) {
  return tsk_f64_to_bf16_bits(tsk_tbar(x, c.mu, c.r));
}

// ---------------------------------------------------------------------------
// bfloat16 tensor-core sketch.
//
// k_sketch_prep turns R into bfloat16 bits, transposed and zero-padded
// (Rt[g][j], kp x dp), and the per-stream statistics into NormC constants, once
// per call.  k_sketch_bf16: one CTA = 64 time points x 64 outputs (blockIdx.y
// picks the group of 64 outputs) x one range of dimensions (blockIdx.z, when
// the grid would otherwise leave SMs idle); 4 warps, one m16 tile of time
// points each, up to 8 n8 tiles; dimensions in stages of 32, the next stage's
// samples loaded into registers while the current stage's MMAs run.  With
// several dimension ranges the partial sums go to a workspace and
// k_sketch_reduce adds them in a fixed order (deterministic).
// ---------------------------------------------------------------------------
constexpr int kSkT = 64;       // time points per CTA
constexpr int kSkThreads = 128;
constexpr int kSkKC = 32;      // dimensions per stage
constexpr int kSkRow = kSkKC + 8;  // padded smem row (80 bytes: conflict-free fragment loads)

__global__ void k_sketch_prep(const float* __restrict__ R, int32_t d, int32_t k, int32_t dp, int32_t kp,
                              const double* __restrict__ stats, int64_t nstreams, uint16_t* __restrict__ Rt,
                              NormC* __restrict__ nc) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nr = static_cast<int64_t>(kp) * dp;
  if (e < nr) {
    const int g = static_cast<int>(e / dp), j = static_cast<int>(e % dp);
    Rt[e] = (g < k && j < d) ? tsk_f64_to_bf16_bits(static_cast<double>(R[static_cast<int64_t>(j) * k + g])) : 0;
  }
  if (e < nstreams) {
    const double mu = stats[2 * e], sg = stats[2 * e + 1];
    nc[e] = make_normc(mu, sg > 0.0 ? 1.0 / sg : 0.0);
  }
}

template <typename TIn, int NTM>
__global__ void __launch_bounds__(kSkThreads, (NTM <= 4 ? 6 : 4)) k_sketch_bf16(const TIn* __restrict__ T, const int64_t* __restrict__ cum,
                                                           const int32_t* __restrict__ len,
                                                           const int64_t* __restrict__ blk_prefix, int32_t n_series,
                                                           int32_t d, int32_t dchunk, const uint16_t* __restrict__ Rt,
                                                           int32_t dp, int32_t k, const NormC* __restrict__ nc,
                                                           float* __restrict__ S, int64_t part_stride) {
  __shared__ __align__(16) uint16_t As[kSkT][kSkRow];
  __shared__ __align__(16) uint16_t Bs[64][kSkRow];
  __shared__ NormC snc[kSkKC];

  const int s = tsk_find_segment<int64_t>(blk_prefix, n_series, static_cast<int64_t>(blockIdx.x));
  const int n = len[s];
  const int t0 = static_cast<int>(blockIdx.x - blk_prefix[s]) * kSkT;
  const int64_t tbase = static_cast<int64_t>(d) * cum[s];
  const int64_t sbase = static_cast<int64_t>(k) * cum[s] + static_cast<int64_t>(blockIdx.z) * part_stride;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const int gbase = static_cast<int>(blockIdx.y) * 64;
  const int NT = min(NTM, (k - gbase + 7) >> 3);  // n8 tiles of this output group (NTM: at most)
  const int jb = static_cast<int>(blockIdx.z) * dchunk;
  const int je = min(d, jb + dchunk);

  float acc[NTM][4];
#pragma unroll
  for (int q = 0; q < NTM; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;

  // this thread's share of a stage: 16 samples (dimension e >> 6, time e & 63 for
  // e = tid + 128 u) and two 8-wide rows of R (output e2 >> 2, dimensions 8 (e2 & 3)..)
  TIn xv[16];
  uint4 rv[2];
  auto load_stage = [&](int j0) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = tid + u * kSkThreads;
      const int j = j0 + (e >> 6), t = t0 + (e & 63);
      xv[u] = (j < je && t < n) ? T[tbase + static_cast<int64_t>(j) * n + t] : TIn(0);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e2 = tid + u * kSkThreads;
      const int g = gbase + (e2 >> 2), jj = j0 + 8 * (e2 & 3);
      rv[u] = *reinterpret_cast<const uint4*>(Rt + static_cast<int64_t>(g) * dp + jj);
    }
  };
  load_stage(jb);
  for (int j0 = jb; j0 < je; j0 += kSkKC) {
    __syncthreads();  // the previous stage's fragments have been read
    if (tid < kSkKC) snc[tid] = (j0 + tid < je) ? nc[static_cast<int64_t>(s) * d + j0 + tid] : make_normc(0.0, 0.0);
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = tid + u * kSkThreads;
      const int jl = e >> 6, tl = e & 63;
      As[tl][jl] = (j0 + jl < je && t0 + tl < n) ? tbar_bf16(xv[u], snc[jl]) : uint16_t(0);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e2 = tid + u * kSkThreads;
      uint4 r = rv[u];
      // dimensions past this range's end contribute nothing
      const int jj = j0 + 8 * (e2 & 3);
      if (jj + 8 > je) {
        uint16_t* h = reinterpret_cast<uint16_t*>(&r);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (jj + q >= je) h[q] = 0;
      }
      *reinterpret_cast<uint4*>(&Bs[e2 >> 2][8 * (e2 & 3)]) = r;
    }
    __syncthreads();
    if (j0 + kSkKC < je) load_stage(j0 + kSkKC);  // overlaps the MMAs below
    const int r0 = warp * 16 + gid;
#pragma unroll
    for (int ks = 0; ks < kSkKC; ks += 16) {
      const uint32_t a0 = *reinterpret_cast<const uint32_t*>(&As[r0][ks + 2 * tig]);
      const uint32_t a1 = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][ks + 2 * tig]);
      const uint32_t a2 = *reinterpret_cast<const uint32_t*>(&As[r0][ks + 2 * tig + 8]);
      const uint32_t a3 = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][ks + 2 * tig + 8]);
#pragma unroll
      for (int nt = 0; nt < NTM; ++nt) {
        if (nt < NT) {
          const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&Bs[nt * 8 + gid][ks + 2 * tig]);
          const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&Bs[nt * 8 + gid][ks + 2 * tig + 8]);
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};\n"
              : "+f"(acc[nt][0]), "+f"(acc[nt][1]), "+f"(acc[nt][2]), "+f"(acc[nt][3])
              : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
      }
    }
  }
#pragma unroll
  for (int nt = 0; nt < NTM; ++nt) {
    if (nt < NT) {
      const int g = gbase + nt * 8 + 2 * tig;
      const int t = t0 + warp * 16 + gid;
      if (t < n) {
        if (g < k) S[sbase + static_cast<int64_t>(g) * n + t] = acc[nt][0];
        if (g + 1 < k) S[sbase + static_cast<int64_t>(g + 1) * n + t] = acc[nt][1];
      }
      if (t + 8 < n) {
        if (g < k) S[sbase + static_cast<int64_t>(g) * n + t + 8] = acc[nt][2];
        if (g + 1 < k) S[sbase + static_cast<int64_t>(g + 1) * n + t + 8] = acc[nt][3];
      }
    }
  }
}

// S = sum over the dimension ranges of the partial sketches, in range order
__global__ void k_sketch_reduce(const float* __restrict__ part, int nparts, int64_t total, float* __restrict__ S) {
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float v = 0.f;
    for (int q = 0; q < nparts; ++q) v += part[static_cast<int64_t>(q) * total + e];
    S[e] = v;
  }
}

// ---------------------------------------------------------------------------
// float32 / float64 sketch on the FMA pipes (one thread per time point).
// ---------------------------------------------------------------------------
template <typename TIn, typename Acc>
__global__ void __launch_bounds__(128) k_sketch_fma(const TIn* __restrict__ T, const int64_t* __restrict__ cum,
                                                    const int32_t* __restrict__ len,
                                                    const int64_t* __restrict__ blk_prefix, int32_t n_series,
                                                    int32_t d, const float* __restrict__ R, int32_t k,
                                                    const double* __restrict__ stats, Acc* __restrict__ S) {
  const int s = tsk_find_segment<int64_t>(blk_prefix, n_series, static_cast<int64_t>(blockIdx.x));
  const int n = len[s];
  const int t = static_cast<int>(blockIdx.x - blk_prefix[s]) * kSkT + static_cast<int>(threadIdx.x);
  if (threadIdx.x >= kSkT || t >= n) return;
  const int64_t tbase = static_cast<int64_t>(d) * cum[s];
  const int64_t sbase = static_cast<int64_t>(k) * cum[s];
  for (int g0 = 0; g0 < k; g0 += 8) {
    Acc acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = Acc(0);
    for (int j = 0; j < d; ++j) {
      const double mu = stats[2 * (static_cast<int64_t>(s) * d + j) + 0];
      const double sg = stats[2 * (static_cast<int64_t>(s) * d + j) + 1];
      const double ri = sg > 0.0 ? 1.0 / sg : 0.0;
      const Acc x = static_cast<Acc>(tsk_tbar(tsk_ld(T, tbase + static_cast<int64_t>(j) * n + t), mu, ri));
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (g0 + u < k) acc[u] = fma(static_cast<Acc>(R[static_cast<int64_t>(j) * k + g0 + u]), x, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (g0 + u < k) S[sbase + static_cast<int64_t>(g0 + u) * n + t] = acc[u];
  }
}

// ---------------------------------------------------------------------------
// Rank-one updates S += op_q r_q T_bar_q (Sec. III-C); one thread per sample.
// ---------------------------------------------------------------------------
template <typename TIn, typename Acc>
__global__ void k_update_dims(Acc* __restrict__ S, const TIn* __restrict__ Td, const int64_t* __restrict__ cum,
                              const int32_t* __restrict__ len, int32_t n_series, int64_t total, int32_t nd,
                              const float* __restrict__ Rrows, const int8_t* __restrict__ op, int32_t k,
                              int32_t precision, const double* __restrict__ stats) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int s = tsk_find_segment<int64_t>(cum, n_series, e);
  const int n = len[s];
  const int t = static_cast<int>(e - cum[s]);
  const int64_t dbase = static_cast<int64_t>(nd) * cum[s];
  const int64_t sbase = static_cast<int64_t>(k) * cum[s];
  for (int q = 0; q < nd; ++q) {
    const double mu = stats[2 * (static_cast<int64_t>(s) * nd + q) + 0];
    const double sg = stats[2 * (static_cast<int64_t>(s) * nd + q) + 1];
    const double ri = sg > 0.0 ? 1.0 / sg : 0.0;
    const double tb = tsk_tbar(tsk_ld(Td, dbase + static_cast<int64_t>(q) * n + t), mu, ri);
    const Acc sign = static_cast<Acc>(op[q]);
    if (precision == TSK_SKETCH_BF16) {
      const float x = tsk_bf16_bits_to_f32(tbar_bf16(Td[dbase + static_cast<int64_t>(q) * n + t], make_normc(mu, ri)));
      for (int g = 0; g < k; ++g) {
        const float r = tsk_bf16_bits_to_f32(tsk_f64_to_bf16_bits(static_cast<double>(Rrows[q * k + g])));
        if (r != 0.f) S[sbase + static_cast<int64_t>(g) * n + t] += sign * static_cast<Acc>(r * x);
      }
    } else {
      const Acc x = static_cast<Acc>(tb);
      for (int g = 0; g < k; ++g) {
        const Acc r = static_cast<Acc>(Rrows[q * k + g]);
        if (r != Acc(0)) S[sbase + static_cast<int64_t>(g) * n + t] = fma(sign * r, x, S[sbase + static_cast<int64_t>(g) * n + t]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Point updates T_j[t] += delta (Sec. III-C), the build's normalisation held
// fixed; one thread per distinct point.  With T given, T is updated in place
// and S moves by R[j,g] times the change of the normalised stored sample (in
// bf16-matched mode: of its bfloat16 rounding), so S stays the sketch of the
// updated series; without T, by R[j,g] * delta / sigma_j.
// ---------------------------------------------------------------------------
template <typename TX, typename Acc>
__global__ void k_point_update(Acc* __restrict__ S, TX* __restrict__ T, const int4* __restrict__ pts,
                               const double* __restrict__ delta, int32_t npts, const int64_t* __restrict__ cum,
                               const int32_t* __restrict__ len, int32_t d, const float* __restrict__ R, int32_t k,
                               int32_t precision, const double* __restrict__ stats) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= npts) return;
  const int4 p = pts[u];
  const int s = p.x, j = p.y, t = p.z;
  const int n = len[s];
  const int64_t st = 2 * (static_cast<int64_t>(s) * d + j);
  const double mu = stats[st], sg = stats[st + 1];
  const double ri = sg > 0.0 ? 1.0 / sg : 0.0;
  Acc* srow = S + static_cast<int64_t>(k) * cum[s] + t;
  if (T) {
    const int64_t pos = cum[s] * d + static_cast<int64_t>(j) * n + t;
    const TX x_old = T[pos];
    const TX x_new = static_cast<TX>(static_cast<double>(x_old) + delta[u]);
    T[pos] = x_new;
    if (precision == TSK_SKETCH_BF16) {
      const NormC c = make_normc(mu, ri);
      const float a = tsk_bf16_bits_to_f32(tbar_bf16(x_old, c));
      const float b = tsk_bf16_bits_to_f32(tbar_bf16(x_new, c));
      for (int g = 0; g < k; ++g) {
        const float r = tsk_bf16_bits_to_f32(tsk_f64_to_bf16_bits(static_cast<double>(R[j * k + g])));
        if (r != 0.f && a != b) atomicAdd(&srow[static_cast<int64_t>(g) * n], static_cast<Acc>(__fmaf_rn(r, b, -(r * a))));
      }
    } else {
      const double dt = tsk_tbar(static_cast<double>(x_new), mu, ri) - tsk_tbar(static_cast<double>(x_old), mu, ri);
      for (int g = 0; g < k; ++g) {
        const double r = static_cast<double>(R[j * k + g]);
        if (r != 0.0) atomicAdd(&srow[static_cast<int64_t>(g) * n], static_cast<Acc>(r * dt));
      }
    }
  } else {
    const double dt = delta[u] * ri;
    for (int g = 0; g < k; ++g) {
      const double r = static_cast<double>(R[j * k + g]);
      if (r != 0.0) atomicAdd(&srow[static_cast<int64_t>(g) * n], static_cast<Acc>(r * dt));
    }
  }
}

}  // namespace

tsk_status tsk_launch_colstats(tsk_ctx* ctx, const void* T, int t_dtype, const int64_t* d_off, const int32_t* d_len,
                               int64_t n_streams, double* stats) {
  if (n_streams <= 0) return TSK_OK;
  if (n_streams > 0x7fffffff) return tsk_fail(ctx, TSK_ERR_UNSUPPORTED, "too many streams");
  const dim3 grid(static_cast<unsigned>(n_streams));
  if (t_dtype == TSK_F64)
    k_colstats<double><<<grid, kStatThreads, 0, ctx->stream>>>(static_cast<const double*>(T), d_off, d_len, stats, ctx->d_err);
  else
    k_colstats<float><<<grid, kStatThreads, 0, ctx->stream>>>(static_cast<const float*>(T), d_off, d_len, stats, ctx->d_err);
  TSK_LAUNCH_CHECK(ctx, "k_colstats");
  return TSK_OK;
}

// Dimension ranges of the bfloat16 sketch: enough CTAs to fill the GPU about 8
// deep, each range at least 256 dimensions.
static void sketch_split(int64_t total_blocks, int32_t d, int32_t k, int sm_count, int* nparts, int* dchunk) {
  const int64_t tiles = total_blocks * ((k + 63) / 64);
  const int64_t want = static_cast<int64_t>(sm_count) * 8;
  int p = static_cast<int>(std::min<int64_t>(std::max<int64_t>(1, (want + tiles - 1) / tiles), std::max(1, d / 256)));
  int c = (d + p - 1) / p;
  c = (c + kSkKC - 1) / kSkKC * kSkKC;
  p = (d + c - 1) / c;
  *nparts = p;
  *dchunk = c;
}

size_t tsk_sketch_ws_bytes(int32_t n_series, int32_t d, int32_t k, int64_t total_blocks, int64_t total_samples,
                           int sm_count) {
  int p = 1, c = d;
  sketch_split(total_blocks, d, k, sm_count, &p, &c);
  const size_t dp = (static_cast<size_t>(d) + kSkKC - 1) / kSkKC * kSkKC + kSkKC;
  const size_t kp = (static_cast<size_t>(k) + 63) / 64 * 64;
  size_t b = tsk_carver::bytes_for(kp * dp, 2) + tsk_carver::bytes_for(static_cast<size_t>(n_series) * d, sizeof(NormC));
  if (p > 1) b += tsk_carver::bytes_for(static_cast<size_t>(p) * k * total_samples, 4);
  return b + 512;
}

tsk_status tsk_launch_sketch(tsk_ctx* ctx, const void* T, int t_dtype, int32_t n_series, const int64_t* d_cum,
                             const int32_t* d_len, const int64_t* d_blk_prefix, int64_t total_blocks, int32_t d,
                             const float* R, int32_t k, int32_t precision, const double* stats, void* S,
                             int64_t total_samples, char* ws) {
  if (total_blocks <= 0) return TSK_OK;
  if (total_blocks > 0x7fffffff) return tsk_fail(ctx, TSK_ERR_UNSUPPORTED, "batch too large");
  const dim3 grid(static_cast<unsigned>(total_blocks));
  const bool f64in = t_dtype == TSK_F64;
  cudaStream_t st = ctx->stream;
  if (precision == TSK_SKETCH_BF16) {
    int parts = 1, dchunk = d;
    sketch_split(total_blocks, d, k, ctx->sm_count, &parts, &dchunk);
    // the stage loop reads R rows 8 dimensions at a time up to one stage past a range
    const int32_t dp = (d + kSkKC - 1) / kSkKC * kSkKC + kSkKC;
    const int32_t kp = (k + 63) / 64 * 64;
    tsk_carver cv(ws);
    uint16_t* Rt = cv.take<uint16_t>(static_cast<size_t>(kp) * dp);
    NormC* nc = cv.take<NormC>(static_cast<size_t>(n_series) * d);
    float* part = parts > 1 ? cv.take<float>(static_cast<size_t>(parts) * k * total_samples) : nullptr;
    const int64_t nstreams = static_cast<int64_t>(n_series) * d;
    const int64_t nprep = std::max<int64_t>(static_cast<int64_t>(kp) * dp, nstreams);
    k_sketch_prep<<<static_cast<unsigned>((nprep + 255) / 256), 256, 0, st>>>(R, d, k, dp, kp, stats, nstreams, Rt, nc);
    TSK_LAUNCH_CHECK(ctx, "k_sketch_prep");
    const dim3 grid_bf16(static_cast<unsigned>(total_blocks), static_cast<unsigned>(kp / 64),
                         static_cast<unsigned>(parts));
    float* out = parts > 1 ? part : static_cast<float*>(S);
    const int64_t pstride = static_cast<int64_t>(k) * total_samples;
    {
      // accumulator tiles per thread: as many n8 tiles as the widest output group needs
      const int nt = std::min(8, (k + 7) / 8);
      const int ntm = nt <= 1 ? 1 : nt <= 2 ? 2 : nt <= 4 ? 4 : 8;
      tsk_prof_scope ps(ctx, TSK_PROF_SKETCH);
      if (f64in) {
        const double* Td = static_cast<const double*>(T);
        switch (ntm) {
          case 1: k_sketch_bf16<double, 1><<<grid_bf16, kSkThreads, 0, st>>>(Td, d_cum, d_len, d_blk_prefix, n_series, d, dchunk, Rt, dp, k, nc, out, pstride); break;
          case 2: k_sketch_bf16<double, 2><<<grid_bf16, kSkThreads, 0, st>>>(Td, d_cum, d_len, d_blk_prefix, n_series, d, dchunk, Rt, dp, k, nc, out, pstride); break;
          case 4: k_sketch_bf16<double, 4><<<grid_bf16, kSkThreads, 0, st>>>(Td, d_cum, d_len, d_blk_prefix, n_series, d, dchunk, Rt, dp, k, nc, out, pstride); break;
          default: k_sketch_bf16<double, 8><<<grid_bf16, kSkThreads, 0, st>>>(Td, d_cum, d_len, d_blk_prefix, n_series, d, dchunk, Rt, dp, k, nc, out, pstride); break;
        }
      } else {
        const float* Tf = static_cast<const float*>(T);
        switch (ntm) {
          case 1: k_sketch_bf16<float, 1><<<grid_bf16, kSkThreads, 0, st>>>(Tf, d_cum, d_len, d_blk_prefix, n_series, d, dchunk, Rt, dp, k, nc, out, pstride); break;
          case 2: k_sketch_bf16<float, 2><<<grid_bf16, kSkThreads, 0, st>>>(Tf, d_cum, d_len, d_blk_prefix, n_series, d, dchunk, Rt, dp, k, nc, out, pstride); break;
          case 4: k_sketch_bf16<float, 4><<<grid_bf16, kSkThreads, 0, st>>>(Tf, d_cum, d_len, d_blk_prefix, n_series, d, dchunk, Rt, dp, k, nc, out, pstride); break;
          default: k_sketch_bf16<float, 8><<<grid_bf16, kSkThreads, 0, st>>>(Tf, d_cum, d_len, d_blk_prefix, n_series, d, dchunk, Rt, dp, k, nc, out, pstride); break;
        }
      }
    }
    TSK_LAUNCH_CHECK(ctx, "k_sketch_bf16");
    if (parts > 1) {
      const int64_t total = pstride;
      const int64_t blocks = std::min<int64_t>((total + 255) / 256, static_cast<int64_t>(ctx->sm_count) * 16);
      k_sketch_reduce<<<static_cast<unsigned>(blocks), 256, 0, st>>>(part, parts, total, static_cast<float*>(S));
      TSK_LAUNCH_CHECK(ctx, "k_sketch_reduce");
    }
  } else if (precision == TSK_SKETCH_FP32) {
    tsk_prof_scope ps(ctx, TSK_PROF_SKETCH);
    if (f64in)
      k_sketch_fma<double, float><<<grid, 128, 0, st>>>(static_cast<const double*>(T), d_cum, d_len, d_blk_prefix, n_series, d, R, k, stats, static_cast<float*>(S));
    else
      k_sketch_fma<float, float><<<grid, 128, 0, st>>>(static_cast<const float*>(T), d_cum, d_len, d_blk_prefix, n_series, d, R, k, stats, static_cast<float*>(S));
    TSK_LAUNCH_CHECK(ctx, "k_sketch_fma<f32>");
  } else {
    tsk_prof_scope ps(ctx, TSK_PROF_SKETCH);
    if (f64in)
      k_sketch_fma<double, double><<<grid, 128, 0, st>>>(static_cast<const double*>(T), d_cum, d_len, d_blk_prefix, n_series, d, R, k, stats, static_cast<double*>(S));
    else
      k_sketch_fma<float, double><<<grid, 128, 0, st>>>(static_cast<const float*>(T), d_cum, d_len, d_blk_prefix, n_series, d, R, k, stats, static_cast<double*>(S));
    TSK_LAUNCH_CHECK(ctx, "k_sketch_fma<f64>");
  }
  return TSK_OK;
}

tsk_status tsk_launch_update_dims(tsk_ctx* ctx, void* S, const void* T_dims, int t_dtype, int32_t n_series,
                                  const int64_t* d_cum, const int32_t* d_len, int64_t total_samples, int32_t nd,
                                  const float* d_Rrows, const int8_t* d_op, int32_t k, int32_t precision,
                                  const double* stats) {
  if (total_samples <= 0) return TSK_OK;
  const int threads = 256;
  const int64_t blocks = (total_samples + threads - 1) / threads;
  if (blocks > 0x7fffffff) return tsk_fail(ctx, TSK_ERR_UNSUPPORTED, "batch too large");
  const bool f64in = t_dtype == TSK_F64;
  if (precision == TSK_SKETCH_FP64) {
    if (f64in)
      k_update_dims<double, double><<<static_cast<unsigned>(blocks), threads, 0, ctx->stream>>>(static_cast<double*>(S), static_cast<const double*>(T_dims), d_cum, d_len, n_series, total_samples, nd, d_Rrows, d_op, k, precision, stats);
    else
      k_update_dims<float, double><<<static_cast<unsigned>(blocks), threads, 0, ctx->stream>>>(static_cast<double*>(S), static_cast<const float*>(T_dims), d_cum, d_len, n_series, total_samples, nd, d_Rrows, d_op, k, precision, stats);
  } else {
    if (f64in)
      k_update_dims<double, float><<<static_cast<unsigned>(blocks), threads, 0, ctx->stream>>>(static_cast<float*>(S), static_cast<const double*>(T_dims), d_cum, d_len, n_series, total_samples, nd, d_Rrows, d_op, k, precision, stats);
    else
      k_update_dims<float, float><<<static_cast<unsigned>(blocks), threads, 0, ctx->stream>>>(static_cast<float*>(S), static_cast<const float*>(T_dims), d_cum, d_len, n_series, total_samples, nd, d_Rrows, d_op, k, precision, stats);
  }
  TSK_LAUNCH_CHECK(ctx, "k_update_dims");
  return TSK_OK;
}

tsk_status tsk_launch_point_update(tsk_ctx* ctx, void* S, void* T, int t_dtype, const int4* d_pts, const double* d_delta,
                                   int32_t npts, const int64_t* d_cum, const int32_t* d_len, int32_t d, const float* R,
                                   int32_t k, int32_t precision, const double* stats) {
  if (npts <= 0) return TSK_OK;
  const unsigned blocks = static_cast<unsigned>((npts + 127) / 128);
  cudaStream_t st = ctx->stream;
  const bool f64s = precision == TSK_SKETCH_FP64;
  if (t_dtype == TSK_F64) {
    if (f64s)
      k_point_update<double, double><<<blocks, 128, 0, st>>>(static_cast<double*>(S), static_cast<double*>(T), d_pts,
                                                             d_delta, npts, d_cum, d_len, d, R, k, precision, stats);
    else
      k_point_update<double, float><<<blocks, 128, 0, st>>>(static_cast<float*>(S), static_cast<double*>(T), d_pts,
                                                            d_delta, npts, d_cum, d_len, d, R, k, precision, stats);
  } else {
    if (f64s)
      k_point_update<float, double><<<blocks, 128, 0, st>>>(static_cast<double*>(S), static_cast<float*>(T), d_pts,
                                                            d_delta, npts, d_cum, d_len, d, R, k, precision, stats);
    else
      k_point_update<float, float><<<blocks, 128, 0, st>>>(static_cast<float*>(S), static_cast<float*>(T), d_pts,
                                                           d_delta, npts, d_cum, d_len, d, R, k, precision, stats);
  }
  TSK_LAUNCH_CHECK(ctx, "k_point_update");
  return TSK_OK;
}
