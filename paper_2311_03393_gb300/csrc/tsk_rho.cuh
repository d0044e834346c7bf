// Exact correlation of two windows of one series, shared by the matrix-profile
// refinement and the dimension-detection kernels.
#pragma once

#include <cuda_runtime.h>

namespace tsk {

// Correlation of window i of series xa and window j of series xb (float32),
// accurate to ~1e-12.
// Both windows are centred in float32 with a two-term mean (the centred values
// carry a rounding of at most ~2^-24 of themselves, an input-sized
// perturbation), then sum(ab), sum(aa), sum(bb) are accumulated with
// error-free float32 transforms: each product is p + e with p = fl(ab),
// e = fma(a, b, -p), and each running sum is a (hi, lo) pair updated by a
// two-sum.  All three sums see the same values, so equal windows give rho = 1.
struct DSum {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, pe));
  }
  __device__ __forceinline__ double value() const { return static_cast<double>(hi) + static_cast<double>(lo); }
};

__device__ __forceinline__ double window_rho(const float* __restrict__ xa, int i, const float* __restrict__ xb, int j,
                                             int m, double mi, double mj) {
  const float mih = static_cast<float>(mi), mil = static_cast<float>(mi - static_cast<double>(mih));
  const float mjh = static_cast<float>(mj), mjl = static_cast<float>(mj - static_cast<double>(mjh));
  DSum sab, saa, sbb;
  for (int t = 0; t < m; ++t) {
    const float a = __fsub_rn(__fsub_rn(xa[i + t], mih), mil);
    const float b = __fsub_rn(__fsub_rn(xb[j + t], mjh), mjl);
    sab.add_prod(a, b);
    saa.add_prod(a, a);
    sbb.add_prod(b, b);
  }
  return sab.value() / sqrt(saa.value() * sbb.value());
}
// float64 series: the same correlation with float64 sums
__device__ __forceinline__ double window_rho(const double* __restrict__ xa, int i, const double* __restrict__ xb, int j,
                                             int m, double mi, double mj) {
  double sab = 0.0, saa = 0.0, sbb = 0.0;
  for (int t = 0; t < m; ++t) {
    const double a = xa[i + t] - mi, b = xb[j + t] - mj;
    sab = fma(a, b, sab);
    saa = fma(a, a, saa);
    sbb = fma(b, b, sbb);
  }
  return sab / sqrt(saa * sbb);
}

// windows i and j of one series
template <typename TX>
__device__ __forceinline__ double window_rho(const TX* __restrict__ x, int i, int j, int m, double mi, double mj) {
  return window_rho(x, i, x, j, m, mi, mj);
}

}  // namespace tsk
