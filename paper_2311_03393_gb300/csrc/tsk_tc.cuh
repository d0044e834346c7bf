// Sliding dot products on the tensor cores, shared by the dimension scan
// (Alg. 3) and the incremental profile's row scans.
//
// For a chunk of windows and a batch of up to 16 query windows,
// C[w][r] = sum_t q_r[t] (x[w + t] - x_ref) is the chunk's Hankel matrix of
// windows (windows x taps) times the queries (taps x queries): mma.sync
// m16n8k16 with f16 operands and float32 accumulation.  Element (a, b) of the
// Hankel tile at window w0 and tap t0 is sample w0 + t0 + a + b, so an
// A-fragment register (two consecutive b) is the pair of samples starting at
// w0 + t0 + a + b: every pair is staged once, as one 32-bit word per starting
// sample, and a fragment is three conflict-free 32-bit reads (rows g and g + 8
// share the middle pair).
//
// float32 accuracy from a two-term split of values scaled by a power of two
// into [-1, 1]: v = hi + lo 2^-11 with hi = fp16(v), lo = fp16((v - hi) 2^11),
// so no term is subnormal; C = A_hi B_hi + (A_hi B_lo + A_lo B_hi) 2^-11, the
// dropped lo lo term being 2^-22 of |v||q|.
#pragma once

#include <cuda_fp16.h>
#include <cstdint>

namespace tsk {

constexpr int kTcMaxKT = 32;  // k-tiles of 16 taps a staged query batch holds (m <= 512)

__device__ __forceinline__ uint32_t h2_bits(__half a, __half b) {
  return static_cast<uint32_t>(__half_as_ushort(a)) | (static_cast<uint32_t>(__half_as_ushort(b)) << 16);
}
// v -> (hi, lo) with v ~ hi + lo * 2^-11
__device__ __forceinline__ void split_h(float v, __half& hi, __half& lo) {
  hi = __float2half_rn(v);
  lo = __float2half_rn((v - __half2float(hi)) * 2048.f);
}
__device__ __forceinline__ void mma_f16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                        uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
// power-of-two scale 2^-e with |v| * 2^-e < 1 for |v| <= amax (1 for amax = 0)
__device__ __forceinline__ float pow2_scale(float amax, int* e_out = nullptr) {
  int e = 0;
  if (amax > 0.f) frexpf(amax, &e);
  if (e_out) *e_out = e;
  return ldexpf(1.f, -e);
}

// One 16-window tile times a batch's n-tiles: c1 += A_hi B_hi, c2 += A_hi B_lo + A_lo B_hi.
// Hp, Lp: staged pairs (hi, lo) indexed by starting sample; Bs: [kt][nt][lane] = {hi b0, hi b1, lo b0, lo b1}.
__device__ __forceinline__ void hankel_tile(const uint32_t* __restrict__ Hp, const uint32_t* __restrict__ Lp,
                                            const uint4* __restrict__ Bs, int wb, int KT, int NT, int lane,
                                            float (&c1)[2][4], float (&c2)[2][4]) {
  const int g = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      c1[nt][u] = 0.f;
      c2[nt][u] = 0.f;
    }
  for (int kt = 0; kt < KT; ++kt) {
    const int sp = wb + kt * 16 + g + 2 * tq;
    const uint32_t h0 = Hp[sp], h1 = Hp[sp + 8], h3 = Hp[sp + 16];
    const uint32_t l0 = Lp[sp], l1 = Lp[sp + 8], l3 = Lp[sp + 16];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      if (nt < NT) {
        const uint4 b = Bs[(kt * 2 + nt) * 32 + lane];
        mma_f16(c1[nt], h0, h1, h1, h3, b.x, b.y);
        mma_f16(c2[nt], h0, h1, h1, h3, b.z, b.w);
        mma_f16(c2[nt], l0, l1, l1, l3, b.x, b.y);
      }
    }
  }
}

// B-fragment entry e of a batch (e < KT * NT * 32): lane, n-tile and k-tile of
// the entry, the query slot (column) and first tap it covers.
struct BEntry {
  int lane, nt, kt, slot, tap;
};
__device__ __forceinline__ BEntry b_entry(int e, int NT) {
  BEntry b;
  b.lane = e & 31;
  b.nt = (e >> 5) % NT;
  b.kt = (e >> 5) / NT;
  b.slot = b.nt * 8 + (b.lane >> 2);
  b.tap = b.kt * 16 + 2 * (b.lane & 3);
  return b;
}
// the four taps of an entry: tap, tap + 1 (b0), tap + 8, tap + 9 (b1)
__device__ __forceinline__ uint4 b_pack(const float (&v)[4]) {
  __half h[4], l[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) split_h(v[u], h[u], l[u]);
  return make_uint4(h2_bits(h[0], h[1]), h2_bits(h[2], h[3]), h2_bits(l[0], l[1]), h2_bits(l[2], l[3]));
}
__device__ __forceinline__ int b_tap(const BEntry& b, int u) { return b.tap + (u & 1) + (u >> 1) * 8; }

}  // namespace tsk
