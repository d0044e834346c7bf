// Global z-normalisation and the random-projection sketch S = R^T T_bar
// (Sec. III-A, Alg. 1), plus dimension addition/deletion (Sec. III-C).
//
// The sketch is a dense contraction over d with a tiny output width k; it is
// bound by reading T once.  In bfloat16 mode each element of T becomes the
// bfloat16 (nearest even) of its float64 normalised value, decided in float32
// with an error interval and in float64 only where that cannot decide, and is
// fed to the tensor cores; products are summed in float32.
#include "tsk_internal.cuh"
#include "tsk_ff.cuh"

#include <cuda.h>  // CUtensorMap and the encoder's signature (the encoder is fetched from the driver at run time)

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
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

// Per-stream constants of the float32 fast path: v = ((x + nmuh) + nmul) * rh
// approximates the float64 value (x - mu) * r, and c0 is the absolute part of
// the bound on their difference.
struct NormC {
  double mu, r;               // float64 mean and 1/sigma (the reference)
  float nmuh, nmul, rh, c0;   // -float(mu), -float(mu - float(mu)), float(r), absolute error term
};
__device__ __forceinline__ NormC make_normc(double mu, double r) {
  NormC c;
  c.mu = mu;
  c.r = r;
  if (fabs(mu) < 1e37 && r < 1e37) {
    const float muh = static_cast<float>(mu);
    c.nmuh = -muh;
    c.nmul = -static_cast<float>(mu - static_cast<double>(muh));
    c.rh = static_cast<float>(r);
    // r = 0 (a constant stream): v = 0 = w exactly
    c.c0 = r > 0.0 ? static_cast<float>((0x1p-46 * r * fabs(mu) + 0x1p-125) * 1.001) : 0.f;
  } else {  // out of the float32 path's range: every element takes the float64 path
    c.nmuh = c.nmul = c.rh = 0.f;
    c.c0 = INFINITY;
  }
  return c;
}

// Packed bfloat16 pair, round to nearest even: element lo in bits 0..15, hi in 16..31.
__device__ __forceinline__ uint32_t cvt_bf16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// bfloat16 (nearest even) of the float64 value w = (x - mu) * r, with float64
// arithmetic only where float32 cannot decide it.  The float32 value v (four
// roundings, mu split in two floats) satisfies |v - w| <= 2^-22 |v| + 2^-47 r |mu|
// (plus 2^-148 near the subnormal range); E = 2^-21 |v| + c0 bounds that with
// a factor 2 to spare.  Rounding is monotone, so if v - E (rounded down) and
// v + E (rounded up) have the same bfloat16, w has it too.  Otherwise (about
// 2e-4 of elements) w is formed in float64 and rounded.
__device__ __forceinline__ uint16_t tbar_bf16(float x, const NormC& c) {
  const float v = __fmul_rn(__fadd_rn(__fadd_rn(x, c.nmuh), c.nmul), c.rh);
  const float e = __fmaf_rn(fabsf(v), 0x1p-21f, c.c0);
  const uint32_t b = cvt_bf16x2(__fsub_rd(v, e), __fadd_ru(v, e));
  if ((b & 0xffffu) == (b >> 16)) return static_cast<uint16_t>(b & 0xffffu);
  return tsk_f64_to_bf16_bits(tsk_tbar(static_cast<double>(x), c.mu, c.r));
}
__device__ __forceinline__ uint16_t tbar_bf16(double x, const NormC& c) {
  return tsk_f64_to_bf16_bits(tsk_tbar(x, c.mu, c.r));
}
// The same for two samples of one stream, packed (x0 in the low half); the
// float32 steps run on pairs.
// The float32 part has no branch: it returns the packed roundings of v - E
// (blo) and v + E (bhi); where they differ float64 must decide.  A caller can
// run several pairs side by side and fix the rare ones afterwards.
__device__ __forceinline__ uint32_t tbar_bf16x2_fast(float x0, float x1, float2 nmuh2, float2 nmul2, float2 rh2, float c0,
                                                     uint32_t& bhi) {
  const float2 v = __fmul2_rn(__fadd2_rn(__fadd2_rn(make_float2(x0, x1), nmuh2), nmul2), rh2);
  const float2 e = make_float2(__fmaf_rn(fabsf(v.x), 0x1p-21f, c0), __fmaf_rn(fabsf(v.y), 0x1p-21f, c0));
  const float2 lo = __ffma2_rd(e, make_float2(-1.f, -1.f), v);
  const float2 hi = __fadd2_ru(v, e);
  bhi = cvt_bf16x2(hi.x, hi.y);
  return cvt_bf16x2(lo.x, lo.y);
}
__device__ __forceinline__ uint32_t tbar_bf16x2_f64(double x0, double x1, const NormC* __restrict__ nc) {
  const double mu = nc->mu, r = nc->r;
  return static_cast<uint32_t>(tsk_f64_to_bf16_bits(tsk_tbar(x0, mu, r))) |
         (static_cast<uint32_t>(tsk_f64_to_bf16_bits(tsk_tbar(x1, mu, r))) << 16);
}

// ---------------------------------------------------------------------------
// bfloat16 tensor-core sketch.
//
// k_sketch_prep turns R into bfloat16 MMA B fragments, in the order the warps
// read them (per stage of 32 dimensions, n8 output tile and lane: one 16-byte
// word holding the lane's fragments of both k16 steps), zero past d and k, and
// the per-stream statistics into NormC constants, once per call.
//
// k_sketch_bf16: a persistent grid (the CTAs resident at once) walks work
// units; a unit is 16 x (4 / wd) time points of one series, one group of up
// to 64 outputs and one range of dimensions (ranges only when the grid would
// otherwise leave SMs idle).  The 4 warps of a CTA split the range into wd
// parts (wd = 4 for d >= 256: a unit is one m16 tile of time points) and run
// independently over their dimensions in stages of 32.  A stage's samples (32
// dimensions x 16 time points) arrive in one of three per-warp shared-memory
// slots kSkSlots stages ahead: one TMA tile (cp.async.bulk.tensor, 64-byte
// swizzle, completion on an mbarrier) for a float32 series whose rows are
// 16-byte aligned, plain loads otherwise.  Lane j converts its 16 samples of
// dimension j in pairs with one set of normalisation constants and writes them
// with two 16-byte stores into the warp's [dimension][time] tile; the A
// fragments come from that tile with ldmatrix.trans.  At the end of a unit the
// wd partial sums of each time tile are added in a fixed order (one CTA
// barrier per unit), and with several dimension ranges k_sketch_reduce adds
// those in a fixed order (deterministic).
// ---------------------------------------------------------------------------
constexpr int kSkBlock = 64;       // time points per block of the batch layout
constexpr int kSkThreads = 128;
constexpr int kSkWarps = kSkThreads / 32;
constexpr int kSkKC = 32;          // dimensions per stage
constexpr int kSkArow = 16 + 8;    // padded tile row: 16 time points (48 bytes: conflict-free stores and ldmatrix rows)

// dimension parts per CTA (warps splitting the dimensions) for d dimensions
__host__ __device__ inline int sketch_wd(int32_t d) { return d >= 256 ? 4 : (d >= 64 ? 2 : 1); }

__device__ __forceinline__ uint32_t pack_bf16_pair(uint16_t lo, uint16_t hi) {
  return static_cast<uint32_t>(lo) | (static_cast<uint32_t>(hi) << 16);
}

__global__ void k_sketch_prep(const float* __restrict__ R, int32_t d, int32_t k, int32_t nstage, int32_t kp,
                              const double* __restrict__ stats, int64_t nstreams, uint4* __restrict__ Rf,
                              NormC* __restrict__ nc) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nr = static_cast<int64_t>(nstage) * (kp / 8) * 32;
  if (e < nr) {
    const int lane = static_cast<int>(e & 31);
    const int64_t w = e >> 5;
    const int g8 = static_cast<int>(w % (kp / 8)), q = static_cast<int>(w / (kp / 8));
    const int g = g8 * 8 + (lane >> 2), j0 = q * kSkKC + 2 * (lane & 3);
    auto rb = [&](int j) -> uint16_t {
      return (g < k && j < d) ? tsk_f64_to_bf16_bits(static_cast<double>(R[static_cast<int64_t>(j) * k + g])) : 0;
    };
    // b0 = (k 2t, 2t+1), b1 = (k 2t+8, 2t+9) of the k16 steps at 0 and 16
    Rf[e] = make_uint4(pack_bf16_pair(rb(j0), rb(j0 + 1)), pack_bf16_pair(rb(j0 + 8), rb(j0 + 9)),
                       pack_bf16_pair(rb(j0 + 16), rb(j0 + 17)), pack_bf16_pair(rb(j0 + 24), rb(j0 + 25)));
  }
  if (e < nstreams) {
    const double mu = stats[2 * e], sg = stats[2 * e + 1];
    nc[e] = make_normc(mu, sg > 0.0 ? 1.0 / sg : 0.0);
  }
}

// 16 consecutive samples (a 16-byte aligned address, or guarded scalar loads)
__device__ __forceinline__ void sk_load16(const float* __restrict__ p, int nv, bool vec, float (&x)[16]) {
  if (vec) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(p) + u);
      x[4 * u] = q.x;
      x[4 * u + 1] = q.y;
      x[4 * u + 2] = q.z;
      x[4 * u + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int u = 0; u < 16; ++u) x[u] = u < nv ? p[u] : 0.f;
  }
}
__device__ __forceinline__ void sk_load16(const double* __restrict__ p, int nv, bool vec, double (&x)[16]) {
  if (vec) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const double2 q = __ldg(reinterpret_cast<const double2*>(p) + u);
      x[2 * u] = q.x;
      x[2 * u + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int u = 0; u < 16; ++u) x[u] = u < nv ? p[u] : 0.0;
  }
}

// A work unit of the persistent sketch kernel, as seen by one warp: its 16
// time points of one series, output group gy and dimensions [jb, je) (empty
// when the time points lie past the series end).
struct SkUnit {
  int s, n, tw, nv, jb, je, gy;
  int64_t tbase, sbase;
};

constexpr int kSkSlots = 3;                      // stages of samples in flight per warp
constexpr int kSkTileBytes = kSkKC * kSkArow * 2;
// one stage: 32 dimensions x 16 samples
__host__ __device__ constexpr int sk_slot_bytes(int elem) { return kSkKC * 16 * elem; }
// dynamic shared memory: [slots: warps x kSkSlots stages][tiles: warps x 1.5 KB][partial sums][mbarriers]
__host__ __device__ constexpr int sk_smem_bytes(int ntm, int elem) {
  return kSkWarps * kSkSlots * sk_slot_bytes(elem) + kSkWarps * kSkTileBytes + 2 * kSkWarps * ntm * 4 * 32 * 4 +
         kSkWarps * kSkSlots * 8 + 16;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the barrier's phase `parity` to complete, at most ~1 s.  Returns
// false after flagging a timeout in the error word (the data are not valid).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, int* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > (1LL << 31)) {
      atomicOr(err, TSK_DEVERR_TIMEOUT);
      return false;
    }
  }
  return true;
}
// 2-D tile (x: time, y: dimension) of the tensor map into shared memory, completing on bar
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// A stage slot holds row r (dimension j0 + r): float32 as 64 bytes at r * 64,
// its 16-byte chunk c at chunk c ^ ((r >> 1) & 3) (the tensor map's 64-byte
// swizzle; slots are 512-byte aligned); float64 as 128 bytes at r * 128, chunk c
// at c ^ (r & 7).  Either way the 32 lanes reading their rows hit distinct banks.
template <typename TIn>
__device__ __forceinline__ int sk_chunk_off(int r, int c) {
  return sizeof(TIn) == 4 ? r * 64 + ((c ^ ((r >> 1) & 3)) << 4) : r * 128 + ((c ^ (r & 7)) << 4);
}

template <typename TIn, int NTM>
__global__ void __launch_bounds__(kSkThreads, sizeof(TIn) == 8 ? 2 : (NTM <= 2 ? 4 : 3)) k_sketch_bf16(
    const __grid_constant__ CUtensorMap tmap, int use_tma, const TIn* __restrict__ T,
    const int64_t* __restrict__ cum, const int32_t* __restrict__ len, const int64_t* __restrict__ blk_prefix,
    int32_t n_series, int64_t n_ctiles, int32_t d, int32_t dchunk, int32_t parts, int32_t wd,
    const uint4* __restrict__ Rf, int32_t kp, int32_t k, const NormC* __restrict__ nc, float* __restrict__ S,
    int64_t part_stride, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sk_smem[];
  constexpr int kSlotBytes = sk_slot_bytes(static_cast<int>(sizeof(TIn)));
  constexpr int kChunks = static_cast<int>(sizeof(TIn));  // 16-byte chunks per row
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned char* slots = sk_smem + warp * (kSkSlots * kSlotBytes);
  uint16_t(*tile)[kSkArow] =
      reinterpret_cast<uint16_t(*)[kSkArow]>(sk_smem + kSkWarps * kSkSlots * kSlotBytes + warp * kSkTileBytes);
  float(*red)[kSkWarps][NTM * 4][32] = reinterpret_cast<float(*)[kSkWarps][NTM * 4][32]>(
      sk_smem + kSkWarps * kSkSlots * kSlotBytes + kSkWarps * kSkTileBytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sk_smem + kSkWarps * kSkSlots * kSlotBytes + kSkWarps * kSkTileBytes +
                                               2 * kSkWarps * NTM * 4 * 32 * 4) +
                   warp * kSkSlots;
  // abort flags, one per unit parity: set by a warp whose copy never landed,
  // read by every warp after that unit's block barrier
  volatile int* abortf = reinterpret_cast<volatile int*>(sk_smem + kSkWarps * kSkSlots * kSlotBytes +
                                                         kSkWarps * kSkTileBytes + 2 * kSkWarps * NTM * 4 * 32 * 4 +
                                                         kSkWarps * kSkSlots * 8);

  const int tsub = warp / wd, dpart = warp % wd;
  const int gid = lane >> 2, tig = lane & 3;
  const int kgroups = kp / 64;
  const int C = static_cast<int>(n_ctiles), G = static_cast<int>(gridDim.x);
  const int wsh = wd == 4 ? 2 : (wd == 2 ? 1 : 0);

  // the TMA path needs the 64-byte swizzle's 512-byte alignment of every slot
  if ((smem_u32(sk_smem) & 1023u) != 0) use_tma = 0;
  if (lane == 0) {
    for (int i = 0; i < kSkSlots; ++i) mbar_init(&bars[i], 1);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  if (tid == 0) abortf[0] = abortf[1] = 0;
  __syncthreads();

  // unit u = c + C (gy + kgroups z): CTA tile c (wd per 64-point block, each
  // 16 x (4 / wd) time points), output group gy, dimension range z.  A CTA
  // walks u = blockIdx.x, + G, ... by updating (c, gy, z) in place.
  auto first_unit = [&](int& c, int& gy, int& z) {
    c = static_cast<int>(blockIdx.x);
    gy = z = 0;
    while (c >= C) {
      c -= C;
      if (++gy == kgroups) { gy = 0; ++z; }
    }
  };
  auto next_unit = [&](int& c, int& gy, int& z) {
    c += G;
    while (c >= C) {
      c -= C;
      if (++gy == kgroups) { gy = 0; ++z; }
    }
  };
  auto decode = [&](int c, int gy, int z, SkUnit& I) {
    I.gy = gy;
    const int blk = c >> wsh;
    I.s = tsk_find_segment<int64_t>(blk_prefix, n_series, static_cast<int64_t>(blk));
    I.n = len[I.s];
    I.tw = (blk - static_cast<int>(blk_prefix[I.s])) * kSkBlock + (c & (wd - 1)) * (16 * (4 / wd)) + 16 * tsub;
    I.nv = min(16, max(0, I.n - I.tw));
    I.tbase = static_cast<int64_t>(d) * cum[I.s];
    I.sbase = static_cast<int64_t>(k) * cum[I.s] + static_cast<int64_t>(z) * part_stride;
    const int rb = z * dchunk, re = min(d, rb + dchunk);
    const int wchunk = ((re - rb + wd - 1) / wd + kSkKC - 1) / kSkKC * kSkKC;
    I.jb = min(re, rb + dpart * wchunk);
    I.je = I.nv > 0 ? min(re, I.jb + wchunk) : I.jb;
  };

  // issue cursor: the next stage of this warp's stream to fetch (unit (pc, pg, pz), dimensions pj..)
  int pc, pg, pz, pj = 0;
  first_unit(pc, pg, pz);
  SkUnit P{};
  auto skip_empty = [&]() {
    while (pz < parts && pj >= P.je) {
      next_unit(pc, pg, pz);
      if (pz < parts) {
        decode(pc, pg, pz, P);
        pj = P.jb;
      }
    }
  };
  if (pz < parts) {
    decode(pc, pg, pz, P);
    pj = P.jb;
    skip_empty();
  }
  // fetch the cursor's stage into slot i: one TMA tile (rows past d and time
  // points past n arrive as zeros), or, without a tensor map, each lane's row
  // by plain loads; then advance the cursor
  unsigned pending = 0;  // bit i: slot i has a stage issued and not yet waited for
  auto issue = [&](int i) {
    if (pz >= parts) return;
    pending |= 1u << i;
    unsigned char* slot = slots + i * kSlotBytes;
    if (use_tma) {
      if (lane == 0) {
        mbar_arrive_expect_tx(&bars[i], kSlotBytes);
        tma_load_2d(slot, &tmap, P.tw, pj, &bars[i]);
      }
    } else {
      const int j = pj + lane;
      TIn x[16];
      if (j < P.je) {
        const TIn* src = T + P.tbase + static_cast<int64_t>(j) * P.n + P.tw;
        sk_load16(src, P.nv, P.nv == 16 && (reinterpret_cast<uintptr_t>(src) & 15u) == 0, x);
      } else {
#pragma unroll
        for (int u = 0; u < 16; ++u) x[u] = TIn(0);
      }
#pragma unroll
      for (int c = 0; c < kChunks; ++c)
        *reinterpret_cast<uint4*>(slot + sk_chunk_off<TIn>(lane, c)) = *reinterpret_cast<const uint4*>(&x[c * (16 / kChunks)]);
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars[i]);
    }
    pj += kSkKC;
    skip_empty();
  };
#pragma unroll
  for (int i = 0; i < kSkSlots; ++i) issue(i);

  float acc[NTM][4];
  const int i8 = lane >> 3, r8 = lane & 7;  // ldmatrix: this lane's row of matrix i8
  int si = 0;          // slot of the next stage to process (stages rotate through the slots)
  unsigned phase = 0;  // bit i: parity of slot i's next completion
  int ord = 0;  // unit ordinal (parity picks the partial-sum buffer)
  bool dead = false;  // warp-uniform: a wait gave up; no more copies are issued
  int uc, ug, uz;
  first_unit(uc, ug, uz);
  for (; uz < parts; next_unit(uc, ug, uz), ++ord) {
    SkUnit I;
    decode(uc, ug, uz, I);
    const int NT = min(NTM, (k - I.gy * 64 + 7) >> 3);  // n8 tiles of this output group (NTM: at most)
#pragma unroll
    for (int q = 0; q < NTM; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
    const NormC* ncs = nc + static_cast<int64_t>(I.s) * d;
    for (int j0 = I.jb; j0 < I.je; j0 += kSkKC) {
      const int j = j0 + lane;
      const bool jv = j < I.je;
      // constants of this lane's dimension and the stage's B fragments (both k16 steps)
      const NormC* cp = ncs + (jv ? j : I.jb);
      const float4 cst = __ldg(reinterpret_cast<const float4*>(&cp->nmuh));
      uint4 bf[NTM];
      {
        const uint4* base = Rf + (static_cast<int64_t>(j0 / kSkKC) * (kp / 8) + I.gy * 8) * 32 + lane;
#pragma unroll
        for (int nt = 0; nt < NTM; ++nt) bf[nt] = __ldg(base + nt * 32);
      }
      if (!__all_sync(TSK_FULL_MASK, mbar_wait_bounded(&bars[si], (phase >> si) & 1u, err))) {
        dead = true;  // leave within one wait limit: the unit's result is not valid
        break;
      }
      pending &= ~(1u << si);
      phase ^= 1u << si;
      TIn x[16];
      {
        const unsigned char* slot = slots + si * kSlotBytes;
        if constexpr (sizeof(TIn) == 4) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float4 q = *reinterpret_cast<const float4*>(slot + sk_chunk_off<TIn>(lane, c));
            x[4 * c] = q.x;
            x[4 * c + 1] = q.y;
            x[4 * c + 2] = q.z;
            x[4 * c + 3] = q.w;
          }
        } else {
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const double2 q = *reinterpret_cast<const double2*>(slot + sk_chunk_off<TIn>(lane, c));
            x[2 * c] = q.x;
            x[2 * c + 1] = q.y;
          }
        }
      }
      // every lane has read the slot (refill it with the stage kSkSlots ahead) and,
      // from the previous stage, the tile's fragments (the tile may be rewritten)
      __syncwarp();
      if (use_tma && lane == 0) asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      issue(si);
      si = si + 1 == kSkSlots ? 0 : si + 1;
      uint32_t pk[8];
      if constexpr (sizeof(TIn) == 4) {
        const float2 nmuh2 = make_float2(cst.x, cst.x), nmul2 = make_float2(cst.y, cst.y), rh2 = make_float2(cst.z, cst.z);
        uint32_t diff = 0;  // nonzero if float32 cannot decide some pair (about 1 in 2500 pairs)
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          uint32_t bhi;
          pk[q] = tbar_bf16x2_fast(x[2 * q], x[2 * q + 1], nmuh2, nmul2, rh2, cst.w, bhi);
          diff |= pk[q] ^ bhi;
        }
        if (diff) {  // find the undecided pairs again and take them in float64
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            uint32_t bhi;
            if (tbar_bf16x2_fast(x[2 * q], x[2 * q + 1], nmuh2, nmul2, rh2, cst.w, bhi) != bhi)
              pk[q] = tbar_bf16x2_f64(x[2 * q], x[2 * q + 1], cp);
          }
        }
      } else {
        const double mu = cp->mu, r = cp->r;
#pragma unroll
        for (int q = 0; q < 8; ++q)
          pk[q] = pack_bf16_pair(tsk_f64_to_bf16_bits(tsk_tbar(x[2 * q], mu, r)), tsk_f64_to_bf16_bits(tsk_tbar(x[2 * q + 1], mu, r)));
      }
      if (!jv || I.nv < 16) {  // zero the samples past the series end or the warp's range end
        const int lim = jv ? I.nv : 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) pk[q] = 2 * q >= lim ? 0u : (2 * q + 1 >= lim ? (pk[q] & 0xffffu) : pk[q]);
      }
      {
        uint4* dst = reinterpret_cast<uint4*>(&tile[lane][0]);
        dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
      }
      __syncwarp();
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        // A fragments (16 time points x 16 dimensions), transposed from the tile
        uint32_t a0, a1, a2, a3;
        const unsigned addr = smem_u32(&tile[16 * ks + (i8 >> 1) * 8 + r8][(i8 & 1) * 8]);
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                     : "=r"(a0), "=r"(a1), "=r"(a2), "=r"(a3)
                     : "r"(addr));
#pragma unroll
        for (int nt = 0; nt < NTM; ++nt) {  // every tile: R is zero past k, those outputs are not stored
          const uint32_t b0 = ks ? bf[nt].z : bf[nt].x, b1 = ks ? bf[nt].w : bf[nt].y;
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};\n"
              : "+f"(acc[nt][0]), "+f"(acc[nt][1]), "+f"(acc[nt][2]), "+f"(acc[nt][3])
              : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
      }
    }
    if (wd > 1) {  // add the dimension parts of each time tile in part order
      float(*rb)[NTM * 4][32] = red[ord & 1];
#pragma unroll
      for (int nt = 0; nt < NTM; ++nt)
#pragma unroll
        for (int c = 0; c < 4; ++c) rb[warp][nt * 4 + c][lane] = acc[nt][c];
      if (dead && lane == 0) abortf[ord & 1] = 1;
      __syncthreads();  // also: every warp has finished reading the buffer of two units ago
      if (abortf[ord & 1]) break;  // every warp of the block leaves at the same unit
      if (dpart != 0) continue;
#pragma unroll
      for (int nt = 0; nt < NTM; ++nt)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float v = rb[warp][nt * 4 + c][lane];
          for (int p = 1; p < wd; ++p) v += rb[warp + p][nt * 4 + c][lane];
          acc[nt][c] = v;
        }
    }
    if (dead) break;  // one warp per time tile (no block barrier): leave alone
    if (I.nv <= 0) continue;
#pragma unroll
    for (int nt = 0; nt < NTM; ++nt) {
      if (nt < NT) {
        const int g = I.gy * 64 + nt * 8 + 2 * tig;
        const int t = I.tw + gid;
        if (t < I.n) {
          if (g < k) S[I.sbase + static_cast<int64_t>(g) * I.n + t] = acc[nt][0];
          if (g + 1 < k) S[I.sbase + static_cast<int64_t>(g + 1) * I.n + t] = acc[nt][1];
        }
        if (t + 8 < I.n) {
          if (g < k) S[I.sbase + static_cast<int64_t>(g) * I.n + t + 8] = acc[nt][2];
          if (g + 1 < k) S[I.sbase + static_cast<int64_t>(g + 1) * I.n + t + 8] = acc[nt][3];
        }
      }
    }
  }
  // after an abort, copies may still be in flight into this block's slots: wait
  // for each (again at most ~1 s) before the block's shared memory is released
  for (int i = 0; i < kSkSlots; ++i)
    if (pending & (1u << i)) mbar_wait_bounded(&bars[i], (phase >> i) & 1u, err);
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
  const int t = static_cast<int>(blockIdx.x - blk_prefix[s]) * kSkBlock + static_cast<int>(threadIdx.x);
  if (threadIdx.x >= kSkBlock || t >= n) return;
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

// Self-test of the failure path: one warp waits, with the sketch kernel's
// bounded wait, on an mbarrier phase that nothing completes (one arrival
// expected, none made).  The wait gives up after ~1 s and flags a timeout in the
// error word; no copy is in flight, so the block simply ends.
__global__ void k_selftest_wait(int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  __syncwarp();
  mbar_wait_bounded(&bar, 0u, err);
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

// Tensor map of one float32 series (d rows of n samples, row stride n * 4 bytes):
// boxes of 16 samples x 32 rows, 64-byte swizzle, zero fill outside the series.
// The encoder comes from the driver through the runtime (no link to libcuda).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static bool sketch_tensor_map(CUtensorMap* map, const void* T, int64_t n, int32_t d) {
  static EncodeTiledFn encode = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<EncodeTiledFn>(fn);
  });
  if (!encode || n <= 0 || d <= 0) return false;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(n), static_cast<cuuint64_t>(d)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(n) * 4};
  const cuuint32_t box[2] = {16, kSkKC};
  const cuuint32_t estr[2] = {1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(T), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Dimension ranges of the bfloat16 sketch: enough CTAs to fill the GPU about 8
// deep, each range at least 256 dimensions.
static void sketch_split(int64_t total_blocks, int32_t d, int32_t k, int sm_count, int* nparts, int* dchunk) {
  const int64_t tiles = total_blocks * sketch_wd(d) * ((k + 63) / 64);
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
  const size_t nstage = (static_cast<size_t>(d) + kSkKC - 1) / kSkKC;
  const size_t kp = (static_cast<size_t>(k) + 63) / 64 * 64;
  size_t b = tsk_carver::bytes_for(nstage * (kp / 8) * 32, sizeof(uint4)) +
             tsk_carver::bytes_for(static_cast<size_t>(n_series) * d, sizeof(NormC));
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
    const int32_t nstage = (d + kSkKC - 1) / kSkKC;
    const int32_t kp = (k + 63) / 64 * 64;
    const int32_t wd = sketch_wd(d);
    tsk_carver cv(ws);
    const int64_t nfrag = static_cast<int64_t>(nstage) * (kp / 8) * 32;
    uint4* Rf = cv.take<uint4>(static_cast<size_t>(nfrag));
    NormC* nc = cv.take<NormC>(static_cast<size_t>(n_series) * d);
    float* part = parts > 1 ? cv.take<float>(static_cast<size_t>(parts) * k * total_samples) : nullptr;
    const int64_t nstreams = static_cast<int64_t>(n_series) * d;
    const int64_t nprep = std::max<int64_t>(nfrag, nstreams);
    k_sketch_prep<<<static_cast<unsigned>((nprep + 255) / 256), 256, 0, st>>>(R, d, k, nstage, kp, stats, nstreams, Rf, nc);
    TSK_LAUNCH_CHECK(ctx, "k_sketch_prep");
    const int64_t n_ctiles = total_blocks * wd;
    const int64_t nunits = n_ctiles * (kp / 64) * parts;
    if (nunits > 0x3fffffff) return tsk_fail(ctx, TSK_ERR_UNSUPPORTED, "batch too large for the sketch");
    float* out = parts > 1 ? part : static_cast<float*>(S);
    const int64_t pstride = static_cast<int64_t>(k) * total_samples;
    {
      // accumulator tiles per thread: as many n8 tiles as the widest output group needs
      const int nt = std::min(8, (k + 7) / 8);
      const int ntm = nt <= 1 ? 1 : nt <= 2 ? 2 : nt <= 4 ? 4 : 8;
      // one float32 series whose rows are 16-byte aligned: stages come by TMA
      CUtensorMap tmap;
      std::memset(&tmap, 0, sizeof(tmap));
      int use_tma = 0;
      if (!f64in && n_series == 1 && total_samples % 4 == 0 && (reinterpret_cast<uintptr_t>(T) & 15u) == 0)
        use_tma = sketch_tensor_map(&tmap, T, total_samples, d) ? 1 : 0;
      tsk_prof_scope ps(ctx, TSK_PROF_SKETCH);
      // persistent grid: as many CTAs as are resident at once (at most one per unit)
      cudaError_t attr_err = cudaSuccess;
      auto launch = [&](auto kern, auto Tp, int smem) {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (attr_err != cudaSuccess) return;
        int per_sm = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSkThreads, smem) != cudaSuccess || per_sm < 1)
          per_sm = 1;
        const int64_t grid = std::min<int64_t>(nunits, static_cast<int64_t>(per_sm) * ctx->sm_count);
        kern<<<static_cast<unsigned>(grid), kSkThreads, smem, st>>>(tmap, use_tma, Tp, d_cum, d_len, d_blk_prefix,
                                                                    n_series, n_ctiles, d, dchunk, parts, wd, Rf, kp, k,
                                                                    nc, out, pstride, ctx->d_err);
      };
      if (f64in) {
        const double* Td = static_cast<const double*>(T);
        switch (ntm) {
          case 1: launch(k_sketch_bf16<double, 1>, Td, sk_smem_bytes(1, 8)); break;
          case 2: launch(k_sketch_bf16<double, 2>, Td, sk_smem_bytes(2, 8)); break;
          case 4: launch(k_sketch_bf16<double, 4>, Td, sk_smem_bytes(4, 8)); break;
          default: launch(k_sketch_bf16<double, 8>, Td, sk_smem_bytes(8, 8)); break;
        }
      } else {
        const float* Tf = static_cast<const float*>(T);
        switch (ntm) {
          case 1: launch(k_sketch_bf16<float, 1>, Tf, sk_smem_bytes(1, 4)); break;
          case 2: launch(k_sketch_bf16<float, 2>, Tf, sk_smem_bytes(2, 4)); break;
          case 4: launch(k_sketch_bf16<float, 4>, Tf, sk_smem_bytes(4, 4)); break;
          default: launch(k_sketch_bf16<float, 8>, Tf, sk_smem_bytes(8, 4)); break;
        }
      }
      if (attr_err != cudaSuccess) return tsk_cuda_fail(ctx, attr_err, "k_sketch_bf16 shared-memory size");
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

tsk_status tsk_launch_selftest_wait(tsk_ctx* ctx) {
  k_selftest_wait<<<1, 32, 0, ctx->stream>>>(ctx->d_err);
  TSK_LAUNCH_CHECK(ctx, "k_selftest_wait");
  return TSK_OK;
}
