// Integer-slice representation of the mixed path's working matrices (internal header).
//
// A matrix is held as NSL = 4 FP16 planes of integers with one power-of-two scale,
//     A = 2^(E-9) sum_{s<4} q_s 2^(-10s),  |q_0| <= 513, |q_s| <= 512 (s >= 1),
// 40 bits below the scale 2^E, so that the tensor cores multiply the planes exactly and
// accumulate the low levels L = s + t of a product exactly (see fwd_mixed.cu).  Planes are
// row-major with leading dimension ld; plane s starts at q + s * plane.
#pragma once
#include <cuda_fp16.h>
#include "common.cuh"

namespace submat {
namespace slc {

constexpr int NSL = 4;              // integer slices per matrix
constexpr int Q0B = 9;              // an entry of magnitude 2^E has q_0 = 2^Q0B
constexpr float kRad = 1024.f;      // 2^10: weight ratio of consecutive slices
constexpr float kRadInv = 1.f / 1024.f;

// Knuth's TwoSum (no products, so no contraction hazards).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Slices of v = hi + lo (|v| <= 2^e) as floats q[0..NSL): q_0 = rint(v 2^(9-e)), then the
// remainder times 2^30, rounded to an integer (an error of at most one unit of q_3), is cut
// into balanced base-1024 digits with integer operations, so no bit of the double-float is
// lost to an FP32 rounding of the remainder.
__device__ __forceinline__ void make_slices(float hi, float lo, int e, float* q) {
  const float sc = ldexpf(1.f, Q0B - e);
  const float yh = hi * sc, yl = lo * sc;           // exact (power-of-two scaling)
  const float q0 = rintf(yh);
  const float rh = __fsub_rn(yh, q0);               // exact: |rh| <= 1/2
  int r = __float2int_rn(rh * 1073741824.f) + __float2int_rn(yl * 1073741824.f);
  const int d3 = ((r + 512) & 1023) - 512;          // in [-512, 511]
  r = (r - d3) >> 10;                               // exact: r - d3 is a multiple of 1024
  const int d2 = ((r + 512) & 1023) - 512;
  r = (r - d2) >> 10;
  q[0] = q0;
  q[1] = (float)r;                                  // |r| <= 2^29 / 2^20 + 1
  q[2] = (float)d2;
  q[3] = (float)d3;
}

__device__ __forceinline__ void put_slices(__half* q, size_t plane, size_t idx, float hi,
                                           float lo, int e) {
  float v[NSL];
  make_slices(hi, lo, e, v);
#pragma unroll
  for (int s = 0; s < NSL; ++s) q[s * plane + idx] = __float2half_rn(v[s]);
}

// v = cscale sum_L 2^(-10L) acc_L (levels 0..3) as a double-float (hi, lo); levels 0..2
// join error-free.
__device__ __forceinline__ void combine_levels(const float* acc, float cscale, float& vh,
                                               float& vl) {
  float s0, e0, t, u;
  two_sum(acc[0], acc[1] * kRadInv, s0, e0);
  two_sum(s0, acc[2] * (kRadInv * kRadInv), t, u);
  e0 = __fadd_rn(__fadd_rn(e0, u), acc[3] * (kRadInv * kRadInv * kRadInv));
  two_sum(t, e0, vh, vl);
  vh *= cscale;
  vl *= cscale;
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
// planes' integers recombine exactly: a = q0 2^10 + q1 and b = q2 2^10 + q3 stay below 2^20,
// and v 2^(9-e) = a 2^-10 + b 2^-30.
__device__ __forceinline__ void load8_df(const __half* q, size_t plane, size_t idx0, int e,
                                         float* vh, float* vl) {
  uint4 raw[NSL];
#pragma unroll
  for (int k = 0; k < NSL; ++k) raw[k] = *reinterpret_cast<const uint4*>(q + k * plane + idx0);
  const float sc = ldexpf(1.f, e - Q0B);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    float qq[NSL];
#pragma unroll
    for (int k = 0; k < NSL; ++k) qq[k] = __half2float(reinterpret_cast<const __half*>(&raw[k])[c]);
    const float a = __fmaf_rn(qq[0], kRad, qq[1]);
    const float b = __fmaf_rn(qq[2], kRad, qq[3]);
    float h, l;
    two_sum(a * kRadInv, b * (kRadInv * kRadInv * kRadInv), h, l);
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
  const float a = __fmaf_rn(qq[0], kRad, qq[1]);
  const float b = __fmaf_rn(qq[2], kRad, qq[3]);
  const float sc = ldexpf(1.f, e - Q0B);
  float h, l;
  two_sum(a * kRadInv, b * (kRadInv * kRadInv * kRadInv), h, l);
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
  double scale;        // 2^(e-9)
  __device__ __forceinline__ double operator()(int i, int k) const {
    const size_t e = (size_t)i * ld + k;
    const float a = __half2float(q[e]) + __half2float(q[plane + e]) * kRadInv;   // exact
    const float b = (__half2float(q[2 * plane + e]) +
                     __half2float(q[3 * plane + e]) * kRadInv) * (kRadInv * kRadInv);
    return ((double)a + (double)b) * scale;
  }
};

struct SliceLoadF {    // leading 20 bits, FP32 (condition estimate)
  const __half* q;
  size_t plane;
  int ld;
  float scale;         // 2^(e-9)
  __device__ __forceinline__ float operator()(int i, int k) const {
    const size_t e = (size_t)i * ld + k;
    return (__half2float(q[e]) + __half2float(q[plane + e]) * kRadInv) * scale;
  }
};

}  // namespace slc
}  // namespace submat
