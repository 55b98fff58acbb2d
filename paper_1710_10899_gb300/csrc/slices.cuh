// Integer-slice representation of the mixed path's working matrices (internal header).
//
// A matrix is held as NSL FP16 planes of small integers with one power-of-two scale,
//     A = 2^(E-7) sum_{s<NSL} q_s 2^(-8s),  |q_0| <= 128, |q_s| <= 129 (s >= 1),
// so that the tensor cores multiply the planes exactly and accumulate each level
// L = s + t of a product exactly (see fwd_mixed.cu).  Planes are row-major with leading
// dimension ld; plane s starts at q + s * plane.
#pragma once
#include <cuda_fp16.h>
#include "common.cuh"

namespace submat {
namespace slc {

constexpr int NSL = 5;              // integer slices per matrix (levels 0..NSL-1 are kept)

// Knuth's TwoSum (no products, so no contraction hazards).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Slices of v = hi + lo (|v| <= 2^e) as floats q[0..NSL).
__device__ __forceinline__ void make_slices(float hi, float lo, int e, float* q) {
  const float sc = ldexpf(1.f, 7 - e);
  const float yh = hi * sc, yl = lo * sc;           // exact (power-of-two scaling)
  q[0] = rintf(yh);
  float r = __fadd_rn(__fsub_rn(yh, q[0]), yl) * 256.f;
#pragma unroll
  for (int s = 1; s < NSL; ++s) {
    q[s] = rintf(r);
    r = __fsub_rn(r, q[s]) * 256.f;
  }
}

__device__ __forceinline__ void put_slices(__half* q, size_t plane, size_t idx, float hi,
                                           float lo, int e) {
  float v[NSL];
  make_slices(hi, lo, e, v);
#pragma unroll
  for (int s = 0; s < NSL; ++s) q[s * plane + idx] = __float2half_rn(v[s]);
}

// v = 2^(cexp) sum_L 2^(-8L) acc_L as a double-float (hi, lo).
__device__ __forceinline__ void combine_levels(const float* acc, float cscale, float& vh,
                                               float& vl) {
  float s0 = acc[0], e0, t, u;
  two_sum(s0, acc[1] * (1.f / 256.f), t, u);
  s0 = t;
  e0 = u;
  two_sum(s0, acc[2] * (1.f / 65536.f), t, u);
  s0 = t;
  e0 = __fadd_rn(e0, u);
  e0 = __fadd_rn(e0, acc[3] * (1.f / 16777216.f));
  e0 = __fadd_rn(e0, acc[4] * (1.f / 4294967296.f));
  two_sum(s0, e0, t, u);
  vh = t * cscale;
  vl = u * cscale;
}

// ((p+1) d - v) / p for v = vh + vl, in double-float.
__device__ __forceinline__ void t_from_m(float vh, float vl, float d, int p, float& th,
                                         float& tl) {
  float a1, a2;
  two_sum((float)(p + 1) * d, -vh, a1, a2);
  a2 = __fsub_rn(a2, vl);
  two_sum(a1, a2, a1, a2);
  const float pinv = 1.f / (float)p;
  th = a1 * pinv;
  const float rem = __fmaf_rn(-th, (float)p, a1);   // remainder of the division
  tl = __fadd_rn(rem, a2) * pinv;
}

// Exponent e with |v| <= 2^e for the largest magnitude amax (at least -60).
__device__ __forceinline__ int exp_bound(float amax) {
  if (!(amax > 0.f)) return -60;
  int e;
  frexpf(amax, &e);            // amax = f 2^e with f in [0.5, 1)
  return e;
}

struct SliceLoad {     // X(i,k) as double from the slices
  const __half* q;
  size_t plane;
  int ld;
  double scale;        // 2^(e-7)
  __device__ __forceinline__ double operator()(int i, int k) const {
    const size_t e = (size_t)i * ld + k;
    const float a = __half2float(q[e]) + __half2float(q[plane + e]) * (1.f / 256.f);
    const float b = __half2float(q[2 * plane + e]) * (1.f / 65536.f) +
                    __half2float(q[3 * plane + e]) * (1.f / 16777216.f);
    const float c = __half2float(q[4 * plane + e]) * (1.f / 4294967296.f);
    return ((double)a + (double)b + (double)c) * scale;
  }
};

struct SliceLoadF {    // leading 15 bits, FP32 (condition estimate)
  const __half* q;
  size_t plane;
  int ld;
  float scale;
  __device__ __forceinline__ float operator()(int i, int k) const {
    const size_t e = (size_t)i * ld + k;
    return (__half2float(q[e]) + __half2float(q[plane + e]) * (1.f / 256.f)) * scale;
  }
};

}  // namespace slc
}  // namespace submat
