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

// c (alpha d - v) for v = vh + vl, in double-float, with c = ch + cl and alpha = ah + al
// (the step matrix of a scaled step; d is 1 on the diagonal, else 0).
__device__ __forceinline__ void t_affine(float vh, float vl, float d, float ah, float al,
                                         float ch, float cl, float& th, float& tl) {
  float a1, a2;
  two_sum(ah * d, -vh, a1, a2);                     // ah * d is exact
  a2 = __fadd_rn(a2, __fsub_rn(al * d, vl));
  two_sum(a1, a2, a1, a2);
  const float h = __fmul_rn(a1, ch);
  const float err = __fmaf_rn(a1, ch, -h);          // a1 * ch - h exactly
  const float l = __fadd_rn(err, __fadd_rn(__fmul_rn(a1, cl), __fmul_rn(a2, ch)));
  two_sum(h, l, th, tl);
}

// Double-float split of a double by integer operations (FP64 units are scarce): h takes the
// leading 24 significant bits, l the next 29 rounded to 24, so h + l keeps about 48 bits.
// Magnitudes outside [2^-74, 2^100] are not expected here; they keep only h (or 0).
__device__ __forceinline__ void split_dbl(double v, float& h, float& l) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7FF);
  const unsigned sign = (unsigned)(b >> 63) << 31;
  if (ex < 1023 - 74 || ex > 1023 + 100) {
    h = ex < 1023 - 74 ? 0.f : __int_as_float((int)(sign | 0x7F800000u));
    l = 0.f;
    return;
  }
  const unsigned long long frac = b & ((1ull << 52) - 1);
  h = __int_as_float((int)(sign | ((unsigned)(ex - 1023 + 127) << 23) | (unsigned)(frac >> 29)));
  const float r = __uint2float_rn((unsigned)(frac & ((1u << 29) - 1)));       // < 2^29
  const float sc = __int_as_float((int)(((unsigned)(ex - 1075 + 127)) << 23));   // 2^(ex-1075)
  l = __int_as_float(__float_as_int(r * sc) | (int)sign);
}

// (ah + al) (bh + bl) as a double-float.
__device__ __forceinline__ void mul_df(float ah, float al, float bh, float bl, float& h,
                                       float& l) {
  const float p = __fmul_rn(ah, bh);
  const float e = __fmaf_rn(ah, bh, -p);
  two_sum(p, __fadd_rn(e, __fadd_rn(__fmul_rn(ah, bl), __fmul_rn(al, bh))), h, l);
}

// Eight consecutive values of a sliced matrix (scale exponent e) as double-floats.  The
// planes' integers recombine exactly: q0 2^8 + q1 < 2^16 and q2 2^16 + q3 2^8 + q4 < 2^24.
__device__ __forceinline__ void load8_df(const __half* q, size_t plane, size_t idx0, int e,
                                         float* vh, float* vl) {
  uint4 raw[NSL];
#pragma unroll
  for (int k = 0; k < NSL; ++k) raw[k] = *reinterpret_cast<const uint4*>(q + k * plane + idx0);
  const float sc = ldexpf(1.f, e - 7);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    float qq[NSL];
#pragma unroll
    for (int k = 0; k < NSL; ++k) qq[k] = __half2float(reinterpret_cast<const __half*>(&raw[k])[c]);
    const float a = __fmaf_rn(qq[0], 256.f, qq[1]);
    const float b = __fmaf_rn(qq[2], 65536.f, __fmaf_rn(qq[3], 256.f, qq[4]));
    float h, l;
    two_sum(a * (1.f / 256.f), b * (1.f / 4294967296.f), h, l);
    vh[c] = h * sc;
    vl[c] = l * sc;
  }
}

// c (alpha y - v) for y = yh + yl and v = vh + vl, in double-float (c, alpha exact FP32).
__device__ __forceinline__ void aff_df(float vh, float vl, float yh, float yl, float alpha,
                                       float c, float& oh, float& ol) {
  float ah, al, s, e;
  mul_df(yh, yl, alpha, 0.f, ah, al);
  two_sum(ah, -vh, s, e);
  e = __fadd_rn(e, __fsub_rn(al, vl));
  two_sum(s, e, s, e);
  mul_df(s, e, c, 0.f, oh, ol);
}

// One value of a sliced matrix (scale exponent e) as a double-float (see load8_df).
__device__ __forceinline__ void load1_df(const __half* q, size_t plane, size_t idx, int e,
                                         float& vh, float& vl) {
  float qq[NSL];
#pragma unroll
  for (int k = 0; k < NSL; ++k) qq[k] = __half2float(q[k * plane + idx]);
  const float a = __fmaf_rn(qq[0], 256.f, qq[1]);
  const float b = __fmaf_rn(qq[2], 65536.f, __fmaf_rn(qq[3], 256.f, qq[4]));
  const float sc = ldexpf(1.f, e - 7);
  float h, l;
  two_sum(a * (1.f / 256.f), b * (1.f / 4294967296.f), h, l);
  vh = h * sc;
  vl = l * sc;
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
