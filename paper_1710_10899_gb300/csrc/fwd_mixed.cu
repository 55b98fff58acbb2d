// Mixed-precision forward: one persistent CTA per SM processes whole submatrices.
//
// Per row j (Alg. 1, Sec. 3.2, Alg. 2):
//   gather S_j (FP64) -> Gershgorin bound lambda_bar = max_k sum_l |S_kl| (FP64)
//   M_0 = S/lambda_bar, X_0 = I; coupled iteration for the inverse p-th root
//       X_{k+1} = X_k T_k,  M_{k+1} = T_k^p M_k
//   (the coupled form of the Newton iteration of Bini, Higham and Meini cited in Sec. 2)
//   with spectrally scaled steps T_k = c_k (alpha_k I - M_k) (scaled_step.cuh); for p >= 2
//   only column pos_j of X is carried (a vector), until ||M - I||_F <= 0.05 (or the tol
//   rule), then X M^(-1/p) with M^(-1/p) as a Taylor polynomial in I - M on that column
//   (taylor_final); for p = 1 X is a product, until ||M - I||_F <= tol sqrt(m), then one
//   Newton update X (2I - M) and FP64 refinement of the column (refine.cuh);
//   F = lambda_bar^(-1/p) X; column residual and condition estimate; write column pos_j.
//
// Arithmetic.  Rounding errors made in any iteration persist in the coupled iteration's
// limit, so every GEMM must be accurate to well below the 1e-6 target, and the tensor
// cores' FP32 accumulation truncates (biased toward zero) when it rounds.  Each working
// matrix is therefore held as four FP16 planes of integers with one power-of-two scale per
// matrix (an error-free splitting in the manner of Ozaki et al.; slices.cuh):
//     A = 2^(E-9) sum_{s<4} q_s 2^(-10s),  |q0| <= 513, |q1..q3| <= 512,
// 40 bits relative to the scale 2^E (E is chosen tight: M's eigenvalues lie in (0,1], those
// of T and of T^i M below bounds that follow from the step constants, so 2^E bounds the
// spectral norm; X's exponent bounds its largest entry, predicted from its last measured
// maximum).  A product is the sum over levels L = s + t <= 3 of 2^(-10L) sum_{s+t=L} Q_s^A Q_t^B
// (ten FP16 products per k-step, FP32 accumulation per level).  The products of these
// integers are exact, and the level-0 and level-1 partial sums are integers bounded through
// the operands' norms: with s0 = 2^(9-b) (b the exponent bias of slice_bias), every row of
// A - alpha I (the affine term below, alpha <= p + 1) has 2-norm at most (p+1) s0 + sqrt(K)/2
// in level-0 units and every column of a spectrally scaled B at most s0 + sqrt(K)/2, while a
// residual slice is at most 512 in magnitude, so by Cauchy-Schwarz level 1 stays below
// 513 sqrt(K) ((p+2) s0 + sqrt(K)) and level 0 far below that; slice_bias takes the smallest
// b that keeps this under 2^24 (b = 0 up to K = 240 for p = 2, b = 1 up to about K = 950).
// Levels 2 and 3 carry weights 2^-20 and 2^-30; the levels dropped (s + t >= 4) weigh 2^-40
// and bound the normwise error of a product near 3 2^-40 K of the scales (2^-40 sqrt(K) for
// slices of either sign).  The epilogue combines the levels in double-float (FP32 pairs)
// and re-splits the result.
//
// GEMM engines (template parameter TC):
//   TC = true  (default): tcgen05.mma kind::f16, M = 128, N = 96, the four level
//              accumulators in one 384-column TMEM buffer, drained in phases (levels
//              combined into shared memory and TMEM released; scaling, slicing and the
//              stores; the mirror images) so the next tile's MMAs overlap the later
//              phases; operands moved by TMA (SWIZZLE_32B, 16-wide k-slices) through a
//              4-stage mbarrier pipeline.  A full-width tile issues the ten plane
//              products of a k-step as six MMAs over B's concatenated planes (N up to
//              192), and the affine term alpha Y (Y = B) enters the accumulators through
//              the level-0 A plane: on the k-steps of the tile's diagonal block the MMA
//              warp subtracts the exact integer alpha' from its diagonal entries in the
//              stage, so A_0 B_t adds -alpha' B_t to level t and the epilogue reads no Y.  Roles: warps 0-7 run the epilogue (two per TMEM
//              lane quarter), warp 8 issues TMA, warp 9 issues MMAs, warps 10-11 apply the
//              iteration's step to the carried column (384 threads).
//              All working matrices are symmetric, so a row-major B read as K-major
//              gives B^T = B to rounding: the engine computes A B^T.
//   TC = false: mma.sync m16n8k16 on 64 x 64 tiles with a cp.async pipeline (the legacy
//              tensor path, kept as the baseline the tcgen05 engine is measured against).
//
// Working matrices live in a per-CTA global scratch: 29 planes of LD x LD halves per CTA
// (LD = the plan's largest order padded to 64, at least 128): two X buffers (p = 1), three
// buffers for M_k and the partial products and one spare, 4 planes each, the gathered S_j
// in FP64 in four planes' space, and one plane for the carried vectors.  A submatrix of order m uses the
// leading mp x mp block (mp = m padded to 16 for tcgen05, 64 for mma.sync); its padding
// rows/columns stay exactly zero.  Rows of a tile beyond mp may hold older data: they only
// reach output entries beyond mp, which are never stored.
#include <cuda_fp16.h>
#include "common.cuh"
#include "refine.cuh"
#include "slices.cuh"
#include "scaled_step.cuh"
#include "tc_prims.cuh"

namespace submat {
namespace {

using namespace slc;

constexpr int E_M = 0;             // |M| <= 1 (eigenvalues of M_k lie in (0, 1])
constexpr int kMatSlots = 6;       // X[2], three M / partial-product buffers, one spare
constexpr int kSPlane = kMatSlots * NSL;          // S_j (FP64) in four planes' space
constexpr int kVecPlane = kSPlane + 4;            // the tracked vectors
constexpr int kPlanesPerCta = kVecPlane + 1;
constexpr double kSliceProducts = NSL * (NSL + 1) / 2;   // FP16 products per GEMM (s + t < NSL)

// Every product of the iteration has the form C = c (alpha Y - A Y), i.e. the step matrix
// T = c (alpha I - A) applied to Y, with A = M_k and Y the B operand (all matrices are
// symmetric polynomials in S, so they commute).  The tcgen05 engine adds -alpha Y to the
// accumulators through its level-0 A plane; the mma.sync engine reads Y's entry at the
// output position.  Flags:
// accumulate ||C - I||_F^2 over the leading m x m block, and/or max |C|.
enum EpiFlag { EPI_NORM = 1, EPI_AMAX = 2 };

struct Mat {
  __half* q;        // NSL planes of LD*LD halves
  int e;            // scale exponent: |entries| <= 2^e
  int plane0;       // index of plane 0 in the tensor map's third dimension
};

struct GemmIO {     // what every GEMM call shares within one submatrix
  int mp, m, p, ld;
  size_t plane;     // ld * ld
  float* norm_part;  // ||.||_F^2 partial sums, one slot per writing warp (summed in order)
  unsigned* amax_s;
  float c, alpha;          // C = c (alpha Y - A B)
};

// Exponent for values bounded by b (with a relative margin for rounding).
__device__ __forceinline__ int exp_of(float b) { return exp_bound(b * (1.f + 1e-6f)); }

// Exponent bias b of the M / partial-product matrices of an order-mp row (entries then
// scale to |q0| <= 2^(9-b)): the smallest b for which alpha' = alpha 2^(9-b) stays an FP16
// integer next to q0 (alpha <= p + 1) and the level-0 / level-1 partial sums of every
// product stay integers below 2^24 (the bounds of the file header).
__device__ __forceinline__ int slice_bias(int mp, int p) {
  const float rk = sqrtf((float)mp);
  for (int b = 0; b < 3; ++b) {
    const float s0 = ldexpf(1.f, Q0B - b);
    if ((float)(p + 1) * s0 <= 2048.f &&
        513.f * rk * ((float)(p + 2) * s0 + rk) < 16777216.f)
      return b;
  }
  return 3;
}
// Exponent bias of the X matrices (p = 1; A = M_k with bias bm): X's exponent bounds its
// entries, not its rows' 2-norms, so a column of X may reach s0 sqrt(K) in level-0 units.
__device__ __forceinline__ int slice_bias_x(int mp, int bm) {
  const float rk = sqrtf((float)mp), k = (float)mp;
  const float sa = 2.f * ldexpf(1.f, Q0B - bm) + 0.5f * rk;   // rows of M - alpha I, alpha <= 2
  for (int b = 0; b < 12; ++b) {
    const float sx = ldexpf(1.f, Q0B - b) + 0.5f;
    if (sa * sx * rk < 16777216.f && 513.f * rk * sa + 513.f * sx * k < 16777216.f) return b;
  }
  return 12;
}

// Slices of 8 consecutive values -> one 16-byte store per plane.
__device__ __forceinline__ void store8_slices(__half* q, size_t plane, size_t idx0,
                                              const float* vh, const float* vl, int e) {
  __align__(16) __half out[NSL][8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    float s[NSL];
    make_slices(vh[c], vl[c], e, s);
#pragma unroll
    for (int k = 0; k < NSL; ++k) out[k][c] = __float2half_rn(s[k]);
  }
#pragma unroll
  for (int k = 0; k < NSL; ++k)
    *reinterpret_cast<uint4*>(q + k * plane + idx0) = *reinterpret_cast<const uint4*>(out[k]);
}

// Warp groups of the tcgen05 CTA, each with a named barrier: BAR = 0 is the whole block
// (__syncthreads); kGemmBar the warps that run a GEMM (epilogue, TMA, MMA: 0..9); kEpiBar
// the epilogue warps 0..7; kVecBar the two vector warps 10..11, which apply an iteration's
// step to the carried vectors while the other warps run that iteration's GEMMs.
constexpr int kGemmBar = 1, kGemmWarps = 10;
constexpr int kVecBar = 2, kVecWarp0 = 10, kVecGroupWarps = 2;
constexpr int kEpiBar = 3, kEpiGroupWarps = 8;
template <int BAR>
__device__ __forceinline__ constexpr int grp_count() {
  return BAR == kGemmBar ? kGemmWarps * 32 : BAR == kVecBar ? kVecGroupWarps * 32 : kEpiGroupWarps * 32;
}
template <int BAR>
__device__ __forceinline__ void grp_sync() {
  if (BAR == 0)
    __syncthreads();
  else
    asm volatile("bar.sync %0, %1;\n" ::"n"(BAR), "n"(grp_count<BAR>()) : "memory");
}
// Barrier of the epilogue warps that also returns whether any of them passed true.
__device__ __forceinline__ bool epi_sync_any(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
      " bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kEpiBar), "n"(kEpiGroupWarps * 32)
      : "memory");
  return r != 0;
}
// Sum of per-warp partial sums in warp order, so the result does not depend on timing (the
// norm steers the step constants and the stopping test).
__device__ __forceinline__ float sum_parts(const float* part, int n) {
  float r = 0.f;
  for (int w = 0; w < n; ++w) r += part[w];
  return r;
}
template <int BAR>
__device__ __forceinline__ int grp_threads() { return BAR == 0 ? (int)blockDim.x : grp_count<BAR>(); }
template <int BAR>
__device__ __forceinline__ int grp_warps() { return grp_threads<BAR>() >> 5; }
// thread and warp index within the group
template <int BAR>
__device__ __forceinline__ int grp_tid() {
  return BAR == kVecBar ? (int)threadIdx.x - kVecWarp0 * 32 : (int)threadIdx.x;
}
template <int BAR>
__device__ __forceinline__ int grp_warp() { return grp_tid<BAR>() >> 5; }

// y[i] = scale * sum_k X(i,k) x[k] for i < m, X from its first NP planes (FP32 result).
// Each warp takes RW rows at a time (their loads are in flight together), eight consecutive
// columns per lane with 16-byte loads; x is zero beyond m up to mp.  x, y in shared memory.
template <int NP, int RW = 4, int BAR = 0>
__device__ void matvec_slices_f32(const __half* q, size_t plane, int ld, float scale,
                                  const float* x, float* y, int m, int mp) {
  const int lane = threadIdx.x & 31, warp = grp_warp<BAR>();
  for (int i0 = warp * RW; i0 < m; i0 += grp_warps<BAR>() * RW) {
    float acc[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) acc[r] = 0.f;
    for (int c0 = lane * 8; c0 < mp; c0 += 256) {
      uint4 raw[RW][NP];
#pragma unroll
      for (int r = 0; r < RW; ++r) {
        const size_t e = (size_t)min(i0 + r, m - 1) * ld + c0;     // rows past m: discarded
#pragma unroll
        for (int k = 0; k < NP; ++k) raw[r][k] = *reinterpret_cast<const uint4*>(q + k * plane + e);
      }
      float xv[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) xv[c] = x[c0 + c];
#pragma unroll
      for (int r = 0; r < RW; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          float v = 0.f, w = 1.f;
#pragma unroll
          for (int k = 0; k < NP; ++k) {
            v = fmaf(__half2float(reinterpret_cast<const __half*>(&raw[r][k])[c]), w, v);
            w *= kRadInv;
          }
          acc[r] = fmaf(v, xv[c], acc[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      const float t = warp_sum_f(acc[r]);
      if (lane == 0 && i0 + r < m) y[i0 + r] = t * scale;
    }
  }
  grp_sync<BAR>();
}

// One pass over the sliced A (scale exponent e) for two products: out[i] = sum_k A(i,k) x[k]
// in FP64 from x given as double-floats (xh, xl), and uo[i] = sum_k A(i,k) u[k] in FP32; all
// vectors zero beyond m up to mp, i < m.  The planes' integers recombine exactly
// (a = q0 2^10 + q1, b = q2 2^10 + q3, A = 2^(e-19) (a + 2^-20 b)) and the products
// a xh are accumulated error-free in double-float, so out keeps about 44 bits.  Each warp
// takes RW rows at a time, eight consecutive columns per lane.
template <int RW = 2, int BAR = 0, bool U = true>
__device__ void matvec2_slices(const __half* q, size_t plane, int ld, int e, const float* xh,
                               const float* xl, double* out, const float* u, float* uo, int m,
                               int mp) {
  const int lane = threadIdx.x & 31, warp = grp_warp<BAR>();
  const double sc = ldexp(1.0, e - Q0B - 10);
  for (int i0 = warp * RW; i0 < m; i0 += grp_warps<BAR>() * RW) {
    float sh[RW], sl[RW], su[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) sh[r] = sl[r] = su[r] = 0.f;
    for (int c0 = lane * 8; c0 < mp; c0 += 256) {
      uint4 raw[RW][NSL];
#pragma unroll
      for (int r = 0; r < RW; ++r) {
        const size_t g = (size_t)min(i0 + r, m - 1) * ld + c0;     // rows past m: discarded
#pragma unroll
        for (int k = 0; k < NSL; ++k) raw[r][k] = *reinterpret_cast<const uint4*>(q + k * plane + g);
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float x = xh[c0 + c], xlo = xl[c0 + c], uv = U ? u[c0 + c] : 0.f;
#pragma unroll
        for (int r = 0; r < RW; ++r) {
          float qq[NSL];
#pragma unroll
          for (int k = 0; k < NSL; ++k)
            qq[k] = __half2float(reinterpret_cast<const __half*>(&raw[r][k])[c]);
          const float a = __fmaf_rn(qq[0], kRad, qq[1]);
          const float b = __fmaf_rn(qq[2], kRad, qq[3]);
          const float pr = __fmul_rn(a, x);
          const float pe = __fmaf_rn(a, x, -pr);          // a x - pr exactly
          float t;
          two_sum(sh[r], pr, sh[r], t);
          sl[r] = __fadd_rn(sl[r], __fadd_rn(t, __fmaf_rn(a, xlo, __fmaf_rn(b * (kRadInv * kRadInv), x, pe))));
          if (U) su[r] = __fmaf_rn(__fmaf_rn(qq[2], kRadInv, a), uv, su[r]);   // FP32, 3 planes
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      float h = sh[r], l = sl[r], uu = su[r];
      for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o);
        const float ol = __shfl_xor_sync(0xffffffffu, l, o);
        if (U) uu += __shfl_xor_sync(0xffffffffu, uu, o);
        float t;
        two_sum(h, oh, h, t);
        l = __fadd_rn(l, __fadd_rn(ol, t));
      }
      if (lane == 0 && i0 + r < m) {
        out[i0 + r] = ((double)h + (double)l) * sc;
        if (U) uo[i0 + r] = uu * (float)sc;
      }
    }
  }
  grp_sync<BAR>();
}

// The step T = c (alpha I - M_k) applied to the vectors carried for p >= 2: y <- T^ny y (FP64
// results of double-float products) and, with track_u, u <- T^p u (FP32).  All vectors live
// in the CTA's global scratch and are zero beyond m up to mp.  Run by a warp group (BAR, see
// grp_sync): inside the tcgen05 engine the vector warps do it during the iteration's GEMMs,
// which read M_k as well but write elsewhere.
struct VecTask {
  const __half* q;          // M_k's planes
  size_t plane;
  int ld, e, m, mp, p;
  int ny;                   // applications of T to y: 1 (A^(-1/p)) or p - 1 (A^(1/p))
  double c, alpha;
  double* y;                // carried column of X (FP64)
  float* u;                 // carried residual vector
  float* yh;                // scratch: y as double-floats
  float* yl;
  double* my;               // scratch: M y
  float* t;                 // scratch: M u
  bool track_u;             // also u <- T^p u (else y only)
};

template <int BAR>
__device__ void vec_task(const VecTask& v) {
  const int gt = grp_tid<BAR>(), gn = grp_threads<BAR>();
  const float cf = (float)v.c, af = (float)v.alpha;
  for (int t = 0; t < (v.track_u ? v.p : v.ny); ++t) {
    if (t < v.ny) {
      // M y (FP64) and M u (FP32) in one pass
      for (int i = gt; i < v.mp; i += gn) {
        float h = 0.f, l = 0.f;
        if (i < v.m) split_dbl(v.y[i], h, l);
        v.yh[i] = h;
        v.yl[i] = l;
      }
      grp_sync<BAR>();
      if (v.track_u)
        matvec2_slices<2, BAR, true>(v.q, v.plane, v.ld, v.e, v.yh, v.yl, v.my, v.u, v.t, v.m, v.mp);
      else
        matvec2_slices<2, BAR, false>(v.q, v.plane, v.ld, v.e, v.yh, v.yl, v.my, v.u, v.t, v.m, v.mp);
      for (int i = gt; i < v.m; i += gn) v.y[i] = v.c * (v.alpha * v.y[i] - v.my[i]);
      if (!v.track_u) {
        grp_sync<BAR>();
        continue;
      }
    } else {
      matvec_slices_f32<3, 8, BAR>(v.q, v.plane, v.ld, ldexpf(1.f, v.e - Q0B), v.u, v.t, v.m, v.mp);
    }
    for (int i = gt; i < v.m; i += gn) v.u[i] = cf * (af * v.u[i] - v.t[i]);
    grp_sync<BAR>();
  }
}

// Final step of the p >= 2 path: the Taylor polynomial P(E) = sum_{j<=J} c_j E^j of
// (I - E)^(-1/p), c_0 = 1, c_j = c_{j-1} (1/p + j - 1) / j, E = I - M, applied ny times to
// y (FP64 results of double-float products) and p times to u (FP32), by Horner:
// a <- c_j v + a - M a, j = J-1 .. 0, from a = c_J v.  While both still need applications
// one pass over M serves both (matvec2_slices); the applications to u alone use degree Ju
// (the residual check needs far less accuracy than the column).  ay, au: scratch vectors
// (mp).  All threads.
constexpr float kTaylorStop = 0.05f;    // iterate until ||M - I||_F <= this (p >= 2)
constexpr int kTaylorMaxDeg = 12;
template <int RWY>       // rows per warp of the passes that serve y (loads in flight)
__device__ void taylor_final(const VecTask& v, int Jy, int Ju, double* ay, float* au) {
  const int gt = threadIdx.x, gn = blockDim.x;
  double cj[kTaylorMaxDeg + 1];
  cj[0] = 1.0;
  for (int j = 1; j <= kTaylorMaxDeg; ++j)
    cj[j] = cj[j - 1] * (1.0 / (double)v.p + (double)(j - 1)) / (double)j;
  for (int app = 0; app < v.p; ++app) {         // u needs p applications, y ny <= p - 1
    const bool ydo = app < v.ny;
    const int J = ydo ? Jy : Ju;
    for (int i = gt; i < v.mp; i += gn) {
      if (ydo) ay[i] = i < v.m ? cj[J] * v.y[i] : 0.0;
      au[i] = i < v.m ? (float)cj[J] * v.u[i] : 0.f;
    }
    __syncthreads();
    for (int j = J - 1; j >= 0; --j) {
      if (ydo) {
        for (int i = gt; i < v.mp; i += gn) {
          float h = 0.f, l = 0.f;
          if (i < v.m) split_dbl(ay[i], h, l);
          v.yh[i] = h;
          v.yl[i] = l;
        }
        __syncthreads();
        matvec2_slices<RWY, 0, true>(v.q, v.plane, v.ld, v.e, v.yh, v.yl, v.my, au, v.t, v.m, v.mp);
        for (int i = gt; i < v.m; i += gn) ay[i] = cj[j] * v.y[i] + (ay[i] - v.my[i]);
      } else {
        matvec_slices_f32<3, 8, 0>(v.q, v.plane, v.ld, ldexpf(1.f, v.e - Q0B), au, v.t, v.m, v.mp);
      }
      for (int i = gt; i < v.m; i += gn) au[i] = (float)cj[j] * v.u[i] + (au[i] - v.t[i]);
      __syncthreads();
    }
    for (int i = gt; i < v.m; i += gn) {
      if (ydo) v.y[i] = ay[i];
      v.u[i] = au[i];
    }
    __syncthreads();
  }
}

// Largest eigenvalue of the SPD X (power method, FP32, two leading planes).
__device__ float power_max_slices(const __half* q, size_t plane, int ld, float scale, int m,
                                  int mp, float* a_s, float* b_s, float* red_s, int iters) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < mp; i += blockDim.x)
    a_s[i] = i < m ? 1.f + (float)(((unsigned)i * 2654435761u) >> 22) * (1.f / 1024.f) : 0.f;
  for (int i = tid; i < mp; i += blockDim.x) b_s[i] = 0.f;
  __syncthreads();
  float lam = 0.f;
  for (int it = 0; it < iters; ++it) {
    matvec_slices_f32<2>(q, plane, ld, scale, a_s, b_s, m, mp);
    float na = 0.f, nb = 0.f;
    for (int i = tid; i < m; i += blockDim.x) { na += a_s[i] * a_s[i]; nb += b_s[i] * b_s[i]; }
    na = warp_sum_f(na);
    nb = warp_sum_f(nb);
    if (lane == 0) { red_s[warp] = na; red_s[kMaxWarps + warp] = nb; }
    __syncthreads();
    float ta = 0.f, tb = 0.f;
    for (int w = 0; w < nwarps(); ++w) { ta += red_s[w]; tb += red_s[kMaxWarps + w]; }
    lam = sqrtf(tb / ta);
    const float inv = tb > 0.f ? rsqrtf(tb) : 0.f;
    for (int i = tid; i < m; i += blockDim.x) a_s[i] = b_s[i] * inv;
    __syncthreads();
  }
  return lam;
}

// Starting lower end of M_0's spectrum (scaled_step.cuh): power steps on I - M_0 in FP32
// with M_0 from its two leading planes, from a fixed +-1 vector.  ||(I - M_0) v|| for a unit
// v never exceeds 1 - lambda_min(M_0), so the estimate errs towards a larger lower end (the
// raw estimate; the steps are steered with half of it).  a_s, b_s: mp floats; zero beyond m.
__device__ float start_lo_slices(const __half* q, size_t plane, int ld, int e, int m, int mp,
                                 float* a_s, float* b_s, float* red_s) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float inv_n = rsqrtf((float)m);
  for (int i = tid; i < mp; i += blockDim.x) {
    a_s[i] = i < m ? ((i % 3 == 0) ? inv_n : -inv_n) : 0.f;
    b_s[i] = 0.f;
  }
  __syncthreads();
  float nb = 1.f;
  for (int t = 0; t < kStartLoSteps; ++t) {
    matvec_slices_f32<2, 8>(q, plane, ld, ldexpf(1.f, e - Q0B), a_s, b_s, m, mp);   // b = M_0 a
    float part = 0.f;
    for (int i = tid; i < m; i += blockDim.x) {
      const float d = a_s[i] - b_s[i];
      b_s[i] = d;
      part += d * d;
    }
    part = warp_sum_f(part);
    if (lane == 0) red_s[warp] = part;
    __syncthreads();
    float tot = 0.f;
    for (int w = 0; w < nwarps(); ++w) tot += red_s[w];
    nb = sqrtf(tot);
    if (nb == 0.f) return 1.f;      // a lies in M_0's eigenvalue 1 (m = 1): Newton steps
    if (!(nb > 0.f)) return kLoMin;
    const float inv = 1.f / nb;
    for (int i = tid; i < m; i += blockDim.x) a_s[i] = b_s[i] * inv;
    __syncthreads();
  }
  return 1.f - nb;
}

// start_lo_slices with M_0 held in shared memory as FP32 (row stride mp; rows and columns
// beyond m zero): the same power steps, each warp taking four rows at a time.
__device__ float start_lo_smem(const float* __restrict__ Mf, int m, int mp, float* a_s,
                               float* b_s, float* red_s) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = nwarps();
  const float inv_n = rsqrtf((float)m);
  for (int i = tid; i < mp; i += blockDim.x) {
    a_s[i] = i < m ? ((i % 3 == 0) ? inv_n : -inv_n) : 0.f;
    b_s[i] = 0.f;
  }
  __syncthreads();
  float nb = 1.f;
  for (int t = 0; t < kStartLoSteps; ++t) {
    for (int i0 = warp * 4; i0 < m; i0 += nw * 4) {          // b = M_0 a
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      for (int jj = lane; jj < mp; jj += 32) {
        const float av = a_s[jj];
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r] = fmaf(Mf[min(i0 + r, m - 1) * mp + jj], av, acc[r]);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float v = warp_sum_f(acc[r]);
        if (lane == 0 && i0 + r < m) b_s[i0 + r] = v;
      }
    }
    __syncthreads();
    float part = 0.f;
    for (int i = tid; i < m; i += blockDim.x) {
      const float d = a_s[i] - b_s[i];
      b_s[i] = d;
      part += d * d;
    }
    part = warp_sum_f(part);
    if (lane == 0) red_s[warp] = part;
    __syncthreads();
    float tot = 0.f;
    for (int w = 0; w < nw; ++w) tot += red_s[w];
    nb = sqrtf(tot);
    if (nb == 0.f) return 1.f;      // a lies in M_0's eigenvalue 1 (m = 1): Newton steps
    if (!(nb > 0.f)) return kLoMin;
    const float inv = 1.f / nb;
    for (int i = tid; i < m; i += blockDim.x) a_s[i] = b_s[i] * inv;
    __syncthreads();
  }
  return 1.f - nb;
}

// ======================================================================================
// tcgen05 engine
// ======================================================================================
// Output tiles of 128 rows x 96 columns (the last column tile of a row block is 16 to 96
// wide: padded orders are multiples of 16).  A tcgen05.mma costs a fixed ~45 cycles below
// N ~ 96 (measured), so 96-wide tiles keep the tensor pipe on the work instead of the
// overhead.  The four 96-column level accumulators fill one 384-column TMEM buffer; the
// epilogue drains it in phases: phase 1 (a thread per TMEM lane, i.e. per tile row)
// combines the levels into double-floats staged in shared memory and releases TMEM, so the
// next tile's MMAs run during the rest; phase 2 (the affine step, slicing and stores) maps
// consecutive threads to consecutive 8-column chunks of a row, so a warp's global loads and
// stores cover whole row segments instead of 32 rows; phase 3 writes the mirror images of
// the entries that fall in skipped tiles (see tc_skip) from the slices left in shared
// memory, a thread per tile row, so that those stores are
// contiguous too.  Operands move by TMA in 16-wide k-slices (32-byte rows, SWIZZLE_32B)
// through a 4-stage mbarrier pipeline.
constexpr int TC_M = 128, TC_N = 96, TC_K = 16;        // tile and k-slice
constexpr int TC_STAGES = 4;
constexpr int TC_A_PLANE = TC_M * TC_K * 2;            // 4096 B
constexpr int TC_B_PLANE = TC_N * TC_K * 2;            // 3072 B
constexpr int TC_STAGE_BYTES = NSL * (TC_A_PLANE + TC_B_PLANE);   // 28672 B
constexpr int TC_STAGE_AREA = TC_STAGES * TC_STAGE_BYTES;         // 114688 B
// Staging area: per tile row, 4 x TC_CH 16-byte units (unit (k, ch) of row r holds the
// double-floats of entries (r, 8 ch + 2k), (r, 8 ch + 2k + 1) after phase 1, and plane k
// of entries (r, 8 ch .. 8 ch + 7) after phase 2), plus one unit of padding: the odd row
// stride makes a thread-per-row access (phases 1 and 3) and a thread-per-chunk access
// (phase 2) both free of bank conflicts.
constexpr int TC_CH = TC_N / 8;                        // 8-column chunks per tile row (12)
constexpr int TC_SROW = 4 * TC_CH + 1;                 // units per staged row (49)
constexpr int TC_STAGING_BYTES = TC_M * TC_SROW * 16;  // 100352 B
constexpr float kAlphaQuantum = 1.f / 64.f;            // alpha' = alpha 2^(9 - e) is an integer
constexpr int TC_BUF_COLS = NSL * TC_N;                // 384 TMEM columns
static_assert(TC_SROW >= NSL * TC_CH + 1, "staging units hold every plane of a chunk");
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;           // polls before a wait gives up
constexpr uint32_t TC_TMEM_COLS = 512;
static_assert(TC_BUF_COLS <= (int)TC_TMEM_COLS, "TMEM budget");
static_assert(TC_STAGE_BYTES % 1024 == 0 || TC_STAGE_BYTES % 256 == 0, "swizzle atoms");
// tcgen05 CTA: warps 0-7 run the epilogue (warp w: TMEM lane quarter w % 4, column half
// w / 4 of the tile), warp 8 issues TMA, warp 9 issues MMAs, warps 10-11 run the vector
// steps (12 warps keep the 168-register budget of 10).
constexpr int TC_EPI_WARPS = kEpiGroupWarps;
constexpr int TC_THREADS = (kVecWarp0 + kVecGroupWarps) * 32;
static_assert(kGemmWarps == TC_EPI_WARPS + 2 && kVecWarp0 == kGemmWarps, "warp roles");
constexpr int TC_TMA_WARP = TC_EPI_WARPS, TC_MMA_WARP = TC_EPI_WARPS + 1;
constexpr int TC_EPI_COLS = TC_N * 4 / TC_EPI_WARPS;  // tile columns per epilogue warp (48)

struct TcState {            // pipeline counters; each role keeps its own copy
  uint32_t pit = 0;         // stages issued (TMA)
  uint32_t cit = 0;         // stages consumed (MMA)
  uint32_t tmt = 0;         // tiles accumulated (MMA)
  uint32_t ept = 0;         // tiles drained (epilogue)
};

struct TcCtx {
  unsigned char* stages;    // 1024-aligned shared memory
  uint4* staging;           // [TC_M][TC_SROW] units of the tile being drained
  uint64_t* full;           // [TC_STAGES]
  uint64_t* empty;          // [TC_STAGES]
  uint64_t* tmem_full;      // accumulators ready
  uint64_t* tmem_empty;     // accumulators read (phase 1 done)
  int* abort_s;
  uint32_t tmem;
  const CUtensorMap* tm_a;
  const CUtensorMap* tm_b;
};

// Output tiles of a symmetric product: row block tm (128 rows) needs only the column tiles
// that reach its diagonal block, tn >= skip(tm) = floor(128 tm / 96); the tiles left of them
// lie wholly below the diagonal and are written as mirror images by the tiles above
// (mirror_needed).  All three roles enumerate the tiles in the same order.
__device__ __forceinline__ int tc_skip(int tm) { return (TC_M * tm) / TC_N; }
__device__ __forceinline__ int tc_ntiles(int ntm, int ntn) {
  int n = 0;
  for (int tm = 0; tm < ntm; ++tm) n += max(0, ntn - tc_skip(tm));
  return n;
}
__device__ __forceinline__ void tc_tile(int t, int ntn, int& tm, int& tn) {
  tm = 0;
  for (;;) {
    const int cnt = max(0, ntn - tc_skip(tm));
    if (t < cnt) break;
    t -= cnt;
    ++tm;
  }
  tn = tc_skip(tm) + t;
}
// Entry (i, j) computed in row block tm is also stored at (j, i) when (j, i) lies in a
// skipped tile: j's row block is below tm and i's column tile there is skipped.
__device__ __forceinline__ bool mirror_needed(int i, int j, int tm) {
  const int tmj = j / TC_M;
  return tmj > tm && (i / TC_N) < tc_skip(tmj);
}

// Planes of the eight entries (row, j0..j0+7): one 16-byte store per plane to C, and the
// planes to the staging units su[0], su[TC_CH], ... when keep (for the mirror pass).
__device__ __forceinline__ void store8_planes(__half* q, size_t plane, int ld, int row, int j0,
                                              const float* vh, const float* vl, int e,
                                              uint4* su, bool keep) {
  __align__(16) __half out[NSL][8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    float s[NSL];
    make_slices(vh[c], vl[c], e, s);
#pragma unroll
    for (int k = 0; k < NSL; ++k) out[k][c] = __float2half_rn(s[k]);
  }
  const size_t idx0 = (size_t)row * ld + j0;
#pragma unroll
  for (int k = 0; k < NSL; ++k) {
    const uint4 v = *reinterpret_cast<const uint4*>(out[k]);
    *reinterpret_cast<uint4*>(q + k * plane + idx0) = v;
    if (keep) su[k * TC_CH] = v;
  }
}

// Half index of element (row q, column k) of a K-major 16-wide tile in the 32-byte swizzle
// that TMA writes and the MMA reads: 32-byte rows, the two 16-byte halves of row q swapped
// when bit 2 of q is set (address bit 4 ^= address bit 7; the tile is 256-byte aligned).
__device__ __forceinline__ int sw32_index(int q, int k) {
  return q * TC_K + (((k >> 3) ^ ((q >> 2) & 1)) << 3) + (k & 7);
}

// The MMAs of one k-step.  A full-width tile (N = 96) concatenates B's planes: the four B
// planes of a stage lie back to back (96 rows each), and level L = s + t of A_s B_t sits at
// TMEM columns 96 L, so A_s times B planes t0..t1 is one MMA with N = 96 (t1 - t0 + 1) whose
// output columns start at 96 (s + t0).  The ten plane products (s + t <= 3) become six MMAs
// (N = 192, 192, 144, 144, 192, 96), each reading its A plane once.  A last tile narrower
// than 64 columns issues the ten products separately with N = nw.
__device__ __forceinline__ void mma_kstep_full(uint32_t d0, uint64_t da0, uint64_t db0,
                                               uint32_t acc0) {
  constexpr uint32_t i192 = tc::idesc_f16(TC_M, 192), i144 = tc::idesc_f16(TC_M, 144),
                     i96 = tc::idesc_f16(TC_M, 96);
  constexpr uint64_t PA = TC_A_PLANE >> 4, RB = (TC_K * 2) >> 4;   // 16-byte units
  static_assert(NSL == 4, "the MMA list below is written for four planes");
  // s = 0: B rows 0..383 -> columns 0..383 (overwrite at the first k-step)
  tc::mma_f16(d0 + 0, da0, db0 + 0 * RB, i192, acc0);
  tc::mma_f16(d0 + 192, da0, db0 + 192 * RB, i192, acc0);
  // s = 1: B rows 0..287 -> columns 96..383
  tc::mma_f16(d0 + 96, da0 + PA, db0 + 0 * RB, i144, 1u);
  tc::mma_f16(d0 + 240, da0 + PA, db0 + 144 * RB, i144, 1u);
  // s = 2: B rows 0..191 -> columns 192..383; s = 3: B rows 0..95 -> columns 288..383
  tc::mma_f16(d0 + 192, da0 + 2 * PA, db0, i192, 1u);
  tc::mma_f16(d0 + 288, da0 + 3 * PA, db0, i96, 1u);
}
__device__ __forceinline__ void mma_kstep_narrow(uint32_t d0, uint64_t da0, uint64_t db0,
                                                 uint32_t idesc, uint32_t acc0) {
#pragma unroll
  for (int L = 0; L < NSL; ++L) {
#pragma unroll
    for (int sa_i = 0; sa_i <= L; ++sa_i) {
      const uint64_t da = da0 + (uint64_t)((sa_i * TC_A_PLANE) >> 4);
      const uint64_t db = db0 + (uint64_t)(((L - sa_i) * TC_B_PLANE) >> 4);
      tc::mma_f16(d0 + L * TC_N, da, db, idesc, sa_i != 0 ? 1u : acc0);
    }
  }
}
// C = A B^T on the tcgen05 engine (see the header comment).  All TC_THREADS threads call it.
// The GEMMs of one iteration run back to back with the GEMM warps' barrier between them;
// full_in / full_out make the first one start and the last one end with a whole-block
// barrier, between which the vector warps run the iteration's vector step vt (given with the
// first GEMM; it reads only M_k, the A operand of all of them, and the carried vectors).
// Returns false if a pipeline wait timed out (the CTA then stops); a time-out in a GEMM that
// does not end with full_out is reported by the iteration's last GEMM.
__device__ bool gemm_tc(const TcCtx& c, TcState& st, Mat A, Mat B, Mat C, Mat Y, int flags,
                        const GemmIO& io, const VecTask* vt, bool full_in, bool full_out) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mp = io.mp;
  const int ntm = (mp + TC_M - 1) / TC_M, ntn = (mp + TC_N - 1) / TC_N, KT = mp / TC_K;
  const int ntiles = tc_ntiles(ntm, ntn);
  // generic-proxy writes (planes, shared vectors) before async-proxy reads/writes
  tc::fence_proxy_async_global();
  tc::fence_proxy_async_shared();
  if (warp >= kVecWarp0) {                             // ---- vector warps
    if (full_in) {
      __syncthreads();
      if (vt) vec_task<kVecBar>(*vt);
    }
    if (!full_out) return true;
    __syncthreads();
    return *c.abort_s == 0;
  }
  if (full_in) __syncthreads(); else grp_sync<kGemmBar>();

  if (warp == TC_TMA_WARP) {
    if (lane == 0) {                                   // ---- TMA producer
      for (int t = 0; t < ntiles && !*c.abort_s; ++t) {
        int tm, tn;
        tc_tile(t, ntn, tm, tn);
        for (int kt = 0; kt < KT; ++kt) {
          const uint32_t s = st.pit % TC_STAGES, round = st.pit / TC_STAGES;
          if (round > 0 && !tc::mbar_wait(&c.empty[s], (round - 1) & 1, TC_WAIT_LIMIT)) {
            *c.abort_s = 1;
            break;
          }
          unsigned char* sa = c.stages + s * TC_STAGE_BYTES;
          unsigned char* sb = sa + NSL * TC_A_PLANE;
          tc::mbar_arrive_expect_tx(&c.full[s], TC_STAGE_BYTES);
#pragma unroll
          for (int q = 0; q < NSL; ++q)
            tc::tma_load_3d(sa + q * TC_A_PLANE, c.tm_a, kt * TC_K, tm * TC_M, A.plane0 + q,
                            &c.full[s]);
#pragma unroll
          for (int q = 0; q < NSL; ++q)
            tc::tma_load_3d(sb + q * TC_B_PLANE, c.tm_b, kt * TC_K, tn * TC_N, B.plane0 + q,
                            &c.full[s]);
          ++st.pit;
        }
      }
    }
  } else if (warp == TC_MMA_WARP) {                    // ---- MMA issuer
    // The whole warp runs the loops (waits, votes and the diagonal patch); lane 0 issues the
    // MMAs and commits.  Every wait is taken by all lanes and combined by a vote, so the
    // warp's control flow stays uniform even if a wait gives up.
    // -alpha' = -alpha 2^(9 - e_A), an integer of at most 2^11 (alpha is a multiple of
    // 1/64, e_A <= 3; slice_bias keeps (p + 1) 2^(9 - e_A) <= 2^11), next to the diagonal's
    // q0 in [0, 513] (M_k is positive definite)
    const __half nz = __float2half_rn(-ldexpf(io.alpha, Q0B - A.e));
    for (int t = 0; t < ntiles; ++t) {
      if (__any_sync(0xffffffffu, *c.abort_s != 0)) break;
      int tm, tn;
      tc_tile(t, ntn, tm, tn);
      const int nw = min(TC_N, mp - tn * TC_N);        // 96, or 16..80 for the last tile
      // tiles of 64 columns or more take the concatenated MMAs at the full width (their
      // extra columns, beyond nw, are never read)
      const bool full = nw >= 64;
      const uint32_t idesc = tc::idesc_f16(TC_M, nw);
      // k-steps inside the tile's diagonal block carry the affine term
      const int kd0 = tm * (TC_M / TC_K), kd1 = min(KT, kd0 + TC_M / TC_K);
      // the single accumulator buffer is free once the epilogue has read the previous tile
      const bool freed = st.tmt < 1 || tc::mbar_wait(c.tmem_empty, (st.tmt - 1) & 1, TC_WAIT_LIMIT);
      if (!__all_sync(0xffffffffu, freed)) {
        *c.abort_s = 1;
        break;
      }
      tc::tc_fence_after();
      const uint32_t d0 = c.tmem;
      bool ok = true;
      for (int kt = 0; kt < KT; ++kt) {
        const uint32_t s = st.cit % TC_STAGES;
        const bool got = tc::mbar_wait(&c.full[s], (st.cit / TC_STAGES) & 1, TC_WAIT_LIMIT);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        if (kt >= kd0 && kt < kd1) {
          // the affine term: A_0 - alpha' I on this k-step's 16 diagonal entries of the
          // stage's level-0 A plane (integers of at most 2^11 stay exact in FP16), so the
          // products A_0 B_t add -alpha' B_t to level t; lane k patches entry k and hands
          // its write to the tensor core's proxy before lane 0 issues
          if (lane < TC_K) {
            __half* a0 = reinterpret_cast<__half*>(c.stages + s * TC_STAGE_BYTES);
            const int idx = sw32_index((kt - kd0) * TC_K + lane, lane);
            a0[idx] = __hadd(a0[idx], nz);
            tc::fence_proxy_async_shared();
          }
          __syncwarp();
        }
        if (lane == 0) {
          // operand descriptors of the stage; every offset added below is a compile-time
          // constant added to the 14-bit start-address field (no carry: shared addresses
          // stay below 2^18 bytes)
          const uint32_t sa = tc::saddr(c.stages + s * TC_STAGE_BYTES);
          const uint64_t da0 = tc::desc_sw32(sa);
          const uint64_t db0 = tc::desc_sw32(sa + NSL * TC_A_PLANE);
          const uint32_t acc0 = kt != 0;             // the first k-step overwrites
          if (full)
            mma_kstep_full(d0, da0, db0, acc0);
          else
            mma_kstep_narrow(d0, da0, db0, idesc, acc0);
          tc::mma_commit(&c.empty[s]);               // frees the stage when these MMAs finish
        }
        __syncwarp();
        ++st.cit;
      }
      if (!ok) {
        *c.abort_s = 1;
        break;
      }
      if (lane == 0) tc::mma_commit(c.tmem_full);     // accumulators of tile t ready
      __syncwarp();
      ++st.tmt;
    }
  } else {                                             // ---- epilogue (TMEM lanes 0..127)
    const int q4 = warp & 3, half = warp >> 2;
    const int etid = tid;                              // 0 .. 255 (warps 0..7)
    // the level sums count in units of cscale = 2^(A.e + B.e - 18) and already hold
    // A B - alpha Y (alpha' sits on the level-0 A plane's diagonal), so C = -c cscale w
    const float c_s = -ldexpf(io.c, A.e + B.e - 2 * Q0B);
    float nrm = 0.f, amax = 0.f;
    const int rt = q4 * 32 + lane;                    // phase 1: this thread's tile row
    for (int t = 0; t < ntiles; ++t) {
      // the epilogue warps meet at barriers below, so they leave together (at once if an
      // earlier GEMM of the iteration already gave up)
      const bool timed_out = *c.abort_s || !tc::mbar_wait(c.tmem_full, st.ept & 1, TC_WAIT_LIMIT);
      if (epi_sync_any(timed_out)) {
        *c.abort_s = 1;
        break;
      }
      tc::tc_fence_after();
      int tm, tn;
      tc_tile(t, ntn, tm, tn);
      const int nw = min(TC_N, mp - tn * TC_N);
      const int nch = nw / 8;
      // tile-uniform: do any of its columns reach a later row block (mirror images)?
      const bool tile_mirror = (tn * TC_N + nw - 1) / TC_M > tm;
      // phase 1: w = acc0 + 2^-10 acc1 + 2^-20 acc2 (error-free sums) + 2^-30 acc3 as a
      // double-float into the staging units of row rt.  Level 2 must not be rounded to
      // FP32: when a matrix's entries lie far below its power-of-two scale (or the affine
      // term cancels level 0), levels 0 and 1 are nearly empty and level 2 carries the value
      {
        const int cb = half * TC_EPI_COLS;              // this warp's columns [cb, cb + 48)
        const int ce = min(cb + TC_EPI_COLS, nw);
        const uint32_t tbase = c.tmem + ((uint32_t)(q4 * 32) << 16);
        uint4* srow = c.staging + rt * TC_SROW;
        for (int c0 = cb; c0 < ce; c0 += 8) {          // warp-uniform bounds
          float acc[NSL][8];
#pragma unroll
          for (int L = 0; L < NSL; ++L) tc::tmem_ld8(tbase + L * TC_N + c0, acc[L]);
          tc::tmem_ld_wait();
#pragma unroll
          for (int k2 = 0; k2 < 4; ++k2) {
            float w4[4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int k = 2 * k2 + h;
              float s0, e0, t, u;
              two_sum(acc[0][k], acc[1][k] * kRadInv, s0, e0);
              two_sum(s0, acc[2][k] * (kRadInv * kRadInv), t, u);
              e0 = __fadd_rn(__fadd_rn(e0, u), acc[3][k] * (kRadInv * kRadInv * kRadInv));
              float wh, wl;
              two_sum(t, e0, wh, wl);
              w4[2 * h] = wh;
              w4[2 * h + 1] = wl;
            }
            srow[k2 * TC_CH + c0 / 8] = make_uint4(__float_as_uint(w4[0]), __float_as_uint(w4[1]),
                                                   __float_as_uint(w4[2]), __float_as_uint(w4[3]));
          }
        }
      }
      // the accumulators are read: the next tile's MMAs may start
      tc::tc_fence_before();
      tc::mbar_arrive(c.tmem_empty);
      ++st.ept;
      grp_sync<kEpiBar>();                             // staging complete
      // phase 2: C = c (alpha Y - A B) for (row, 8-column chunk) tasks, consecutive threads
      // on consecutive chunks of a row
      for (int task = etid; task < TC_M * TC_CH; task += TC_EPI_WARPS * 32) {
        const int r = task / TC_CH, ch = task - r * TC_CH;
        const int row = tm * TC_M + r;
        if (row >= mp || ch >= nch) continue;
        const int j0 = tn * TC_N + ch * 8;
        uint4* su = c.staging + r * TC_SROW + ch;
        float wv[16];
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
          const uint4 u = su[k2 * TC_CH];
          wv[4 * k2] = __uint_as_float(u.x);
          wv[4 * k2 + 1] = __uint_as_float(u.y);
          wv[4 * k2 + 2] = __uint_as_float(u.z);
          wv[4 * k2 + 3] = __uint_as_float(u.w);
        }
        float oh[8], ol[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          // out = -c cscale (wh + wl), as a double-float
          const float wh = wv[2 * k], wl = wv[2 * k + 1];
          oh[k] = __fmul_rn(c_s, wh);
          ol[k] = __fmaf_rn(c_s, wl, __fmaf_rn(c_s, wh, -oh[k]));
        }
        store8_planes(C.q, io.plane, io.ld, row, j0, oh, ol, C.e, su, tile_mirror);
        if (flags & EPI_AMAX) {
#pragma unroll
          for (int k = 0; k < 8; ++k) amax = fmaxf(amax, fabsf(oh[k]));
        }
        if (flags & EPI_NORM) {
          // the whole chunk is mirrored or none of it (chunks never straddle a row block)
          const bool mchunk = tile_mirror && mirror_needed(row, j0, tm);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int jj = j0 + k;
            const bool in = (row < io.m) && (jj < io.m);
            const float d = (row == jj) ? 1.f : 0.f;
            const float ev = in ? __fadd_rn(__fsub_rn(oh[k], d), ol[k]) : 0.f;
            nrm += mchunk ? 2.f * ev * ev : ev * ev;   // a mirrored entry counts twice
          }
        }
      }
      if (tile_mirror) {
        grp_sync<kEpiBar>();                           // slices of the tile in the staging area
        // phase 3: entry (i, j) also at (j, i) where that lies in a skipped tile.  A task is
        // a chunk of 8 columns reaching a later row block times 32 tile rows (one warp, a
        // lane per row, so each store covers 32 consecutive columns); whether a chunk is
        // mirrored depends only on its row block (chunks never straddle one) and on the rows'
        // 96-column tile (32 aligned rows never straddle one), so tasks are warp-uniform.
        const int ch_lo = max(0, ((tm + 1) * TC_M - tn * TC_N) / 8);
        const int ntask = (nch - ch_lo) * (TC_M / 32);
        for (int task = warp; task < ntask; task += TC_EPI_WARPS) {
          const int ch = ch_lo + task / (TC_M / 32), r = (task % (TC_M / 32)) * 32 + lane;
          const int row = tm * TC_M + r, j0 = tn * TC_N + ch * 8;
          if (row >= mp || !mirror_needed(row, j0, tm)) continue;
          const uint4* su = c.staging + r * TC_SROW + ch;
#pragma unroll
          for (int k = 0; k < NSL; ++k) {
            const uint4 v = su[k * TC_CH];            // the planes left by phase 2
            const __half* hv = reinterpret_cast<const __half*>(&v);
            __half* dst = C.q + k * io.plane + (size_t)j0 * io.ld + row;
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) dst[(size_t)cc * io.ld] = hv[cc];
          }
        }
      }
      grp_sync<kEpiBar>();                             // staging free for the next tile
    }
    if (flags & EPI_NORM) {
      nrm = warp_sum_f(nrm);
      if (lane == 0) io.norm_part[warp] = nrm;      // warps 0..7
    }
    if (flags & EPI_AMAX) {
      for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      if (lane == 0) atomicMax(io.amax_s, __float_as_uint(amax));
    }
  }
  // the planes written here are read next by TMA (async proxy) through L2
  __threadfence();
  tc::fence_proxy_async_global();
  if (!full_out) {
    grp_sync<kGemmBar>();
    return true;
  }
  __syncthreads();
  return *c.abort_s == 0;
}

// ======================================================================================
// mma.sync engine (baseline)
// ======================================================================================
constexpr int BM = 64;             // CTA output tile (64 x 64)
constexpr int BK = 32;             // k-slice per pipeline stage
constexpr int SY_STAGES = 4;
constexpr int A_LD = BK + 8;       // padded smem row (halves) of an A tile plane
constexpr int B_LD = BM + 8;       // padded smem row (halves) of a B tile plane
constexpr int A_PLANE = BM * A_LD;
constexpr int B_PLANE = BK * B_LD;
constexpr int SY_STAGE = NSL * (A_PLANE + B_PLANE);      // halves per pipeline stage
constexpr int SY_STAGE_AREA = SY_STAGES * SY_STAGE * 2;  // bytes

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}
__device__ __forceinline__ void ldsm_x4(uint32_t* r, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t* r, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C = A B (mp x mp, sliced, row-major ld).  All eight warps work on one 64 x 64 output tile
// at a time (warps 2 x 4, 32 x 16 each), 4-stage cp.async pipeline over k.
__device__ void gemm_sync(Mat A, Mat B, Mat C, Mat Y, int flags, const GemmIO& io,
                          __half* smem) {
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 2, wn = warp & 3;      // 2 x 4 warps
  const int mp = io.mp, ld = io.ld;
  const int nt = mp / BM;
  const int KT = mp / BK;
  const size_t plane = io.plane;
  const float cscale = ldexpf(1.f, A.e + B.e - 2 * Q0B);
  float nrm = 0.f;
  float amax = 0.f;

  for (int t = 0; t < nt * nt; ++t) {
    const int i0 = (t / nt) * BM, j0 = (t % nt) * BM;
    float acc[NSL][2][2][4];
#pragma unroll
    for (int l = 0; l < NSL; ++l)
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[l][a][b][c] = 0.f;

    auto load_stage = [&](int st, int kt) {
      __half* s = smem + st * SY_STAGE;
      const int k0 = kt * BK;
#pragma unroll
      for (int c = tid; c < BM * 4; c += kThreads) {
        const int r = c >> 2, q = (c & 3) * 8;
        const size_t g = (size_t)(i0 + r) * ld + k0 + q;
#pragma unroll
        for (int l = 0; l < NSL; ++l) cp_async16(s + l * A_PLANE + r * A_LD + q, A.q + l * plane + g);
      }
#pragma unroll
      for (int c = tid; c < BK * 8; c += kThreads) {
        const int r = c >> 3, q = (c & 7) * 8;
        const size_t g = (size_t)(k0 + r) * ld + j0 + q;
#pragma unroll
        for (int l = 0; l < NSL; ++l)
          cp_async16(s + NSL * A_PLANE + l * B_PLANE + r * B_LD + q, B.q + l * plane + g);
      }
    };

#pragma unroll
    for (int s = 0; s < SY_STAGES - 1; ++s) {
      if (s < KT) load_stage(s, s);
      cp_async_commit();
    }
    for (int kt = 0; kt < KT; ++kt) {
      cp_async_wait<SY_STAGES - 2>();
      __syncthreads();
      const int nk = kt + SY_STAGES - 1;
      if (nk < KT) load_stage(nk % SY_STAGES, nk);
      cp_async_commit();
      const __half* s = smem + (kt % SY_STAGES) * SY_STAGE;
#pragma unroll
      for (int kk = 0; kk < BK; kk += 16) {
        uint32_t af[NSL][2][4], bf[NSL][2][2];
#pragma unroll
        for (int l = 0; l < NSL; ++l) {
#pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            const int row = wm * 32 + mt * 16 + (lane & 15);
            const int col = kk + (lane >> 4) * 8;
            ldsm_x4(af[l][mt], s + l * A_PLANE + row * A_LD + col);
          }
          const int krow = kk + (lane & 15);
          const int col = wn * 16 + (lane >> 4) * 8;
          uint32_t r[4];
          ldsm_x4_t(r, s + NSL * A_PLANE + l * B_PLANE + krow * B_LD + col);
          bf[l][0][0] = r[0]; bf[l][0][1] = r[1];
          bf[l][1][0] = r[2]; bf[l][1][1] = r[3];
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int n = 0; n < 2; ++n) {
#pragma unroll
            for (int L = 0; L < NSL; ++L)
#pragma unroll
              for (int sa = 0; sa <= L; ++sa) mma16816(acc[L][mt][n], af[sa][mt], bf[L - sa][n]);
          }
      }
    }
    cp_async_wait<0>();
    __syncthreads();

    const int g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int n = 0; n < 2; ++n)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int c2 = 0; c2 < 2; ++c2) {
            const int ci = 2 * h + c2;
            const int i = i0 + wm * 32 + mt * 16 + g + h * 8;
            const int jj = j0 + wn * 16 + n * 8 + 2 * q + c2;
            const float lv[NSL] = {acc[0][mt][n][ci], acc[1][mt][n][ci], acc[2][mt][n][ci],
                                   acc[3][mt][n][ci]};
            float vh, vl, yh, yl, oh, ol;
            combine_levels(lv, cscale, vh, vl);
            const size_t idx = (size_t)i * ld + jj;
            load1_df(Y.q, plane, idx, Y.e, yh, yl);
            aff_df(vh, vl, yh, yl, io.alpha, io.c, oh, ol);
            put_slices(C.q, plane, idx, oh, ol, C.e);
            if (flags & EPI_AMAX) amax = fmaxf(amax, fabsf(oh));
            if (flags & EPI_NORM) {
              const bool in = (i < io.m) && (jj < io.m);
              const float d = (i == jj) ? 1.f : 0.f;
              const float ev = in ? __fadd_rn(__fsub_rn(oh, d), ol) : 0.f;
              nrm += ev * ev;
            }
          }
  }
  if (flags & EPI_NORM) {
    nrm = warp_sum_f(nrm);
    if (lane == 0) io.norm_part[warp] = nrm;        // warps 0..7
  }
  if (flags & EPI_AMAX) {
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) atomicMax(io.amax_s, __float_as_uint(amax));
  }
  // The next GEMM reads these planes with cp.async.cg, which reads L2 and bypasses L1.
  __threadfence();
  __syncthreads();
}

// ======================================================================================
// small-submatrix engine: the whole working set in shared memory, warp-level mma.sync
// ======================================================================================
// Orders up to kSmallMaxM: every sliced matrix lives in shared memory (leading dimension
// kSmallLD; 80-byte rows make the eight row addresses of an ldmatrix fall in distinct banks),
// the gathered S_j in the CTA's global scratch.  A product of padded order mp (16 or 32) is
// (mp/16) x (mp/8) warp tiles of 16 x 8, one per warp, each running the ten plane products
// of every 16-wide k-step with mma.sync m16n8k16 into four per-level FP32 accumulators (the
// same exact level arithmetic as the other engines), then C = c (alpha Y - A B) from Y's
// shared-memory planes.  Two CTAs of 256 threads share an SM.
constexpr int kSmallMaxM = 32;
constexpr int kSmallLD = 40;
constexpr int kSmallPlanes = 5 * NSL + 1;  // X[2], three M / partial-product buffers, vectors
constexpr int kSmallVecPlane = 5 * NSL;
constexpr int kSmallVmax = 64;             // length of the shared vectors y_s, v_s, w_s, R_s
constexpr int kSmallCtasPerSm = 2;
static_assert(kSmallMaxM == SUBMAT_SMALL_MAX_M, "the header's limit of the small engine");
static_assert(kSmallMaxM + 8 <= kSmallLD && kSmallLD % 8 == 0, "padded rows, 16-byte aligned");
static_assert(44 * kSmallLD <= (int)(kSmallLD * kSmallLD * 2), "vectors fit their plane");

__device__ __forceinline__ void ldsm_x2_t(uint32_t* r, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(smem_u32(p)));
}

__device__ void gemm_small(Mat A, Mat B, Mat C, Mat Y, int flags, const GemmIO& io) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mp = io.mp;
  const int ntn = mp / 8, ntiles = (mp / 16) * ntn;
  const size_t plane = io.plane;
  const float cscale = ldexpf(1.f, A.e + B.e - 2 * Q0B);
  float nrm = 0.f, amax = 0.f;
  for (int t = warp; t < ntiles; t += kWarps) {
    const int i0 = (t / ntn) * 16, j0 = (t % ntn) * 8;
    float acc[NSL][4];
#pragma unroll
    for (int l = 0; l < NSL; ++l)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[l][c] = 0.f;
    for (int k0 = 0; k0 < mp; k0 += 16) {
      uint32_t af[NSL][4], bf[NSL][2];
#pragma unroll
      for (int l = 0; l < NSL; ++l) {
        ldsm_x4(af[l], A.q + l * plane + (size_t)(i0 + (lane & 15)) * kSmallLD + k0 + (lane >> 4) * 8);
        ldsm_x2_t(bf[l], B.q + l * plane + (size_t)(k0 + (lane & 15)) * kSmallLD + j0);
      }
#pragma unroll
      for (int L = 0; L < NSL; ++L)
#pragma unroll
        for (int sa = 0; sa <= L; ++sa) mma16816(acc[L], af[sa], bf[L - sa]);
    }
    const int g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int ci = 0; ci < 4; ++ci) {
      const int i = i0 + g + (ci >> 1) * 8, jj = j0 + 2 * q + (ci & 1);
      const float lv[NSL] = {acc[0][ci], acc[1][ci], acc[2][ci], acc[3][ci]};
      float vh, vl, yh, yl, oh, ol;
      combine_levels(lv, cscale, vh, vl);
      const size_t idx = (size_t)i * kSmallLD + jj;
      load1_df(Y.q, plane, idx, Y.e, yh, yl);
      aff_df(vh, vl, yh, yl, io.alpha, io.c, oh, ol);
      put_slices(C.q, plane, idx, oh, ol, C.e);
      if (flags & EPI_AMAX) amax = fmaxf(amax, fabsf(oh));
      if (flags & EPI_NORM) {
        const bool in = (i < io.m) && (jj < io.m);
        const float d = (i == jj) ? 1.f : 0.f;
        const float ev = in ? __fadd_rn(__fsub_rn(oh, d), ol) : 0.f;
        nrm += ev * ev;
      }
    }
  }
  if (flags & EPI_NORM) {
    nrm = warp_sum_f(nrm);
    if (lane == 0) io.norm_part[warp] = nrm;        // warps 0..7 (0 where no tile)
  }
  if (flags & EPI_AMAX) {
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) atomicMax(io.amax_s, __float_as_uint(amax));
  }
  __syncthreads();
}

// ======================================================================================
// the per-submatrix kernel
// ======================================================================================
constexpr size_t kSmemTail = 256;                       // barriers and flags
// Engines of the kernel template (template parameter ENG).
constexpr int ENG_TC = 0, ENG_SYNC = 1, ENG_SMALL = 2;
// small engine: shared vectors (y_s, v_s, w_s, red_s, R_s), then the planes
constexpr size_t kSmallVecBytes =
    ((3 * kSmallVmax + kRedDoubles) * sizeof(double) + kSmallVmax * sizeof(int32_t) + 1023) /
    1024 * 1024;
constexpr size_t kSmallPlaneBytes = (size_t)kSmallLD * kSmallLD * sizeof(__half);
// shared memory before the barrier tail: tcgen05: TMA stages + the epilogue's staging area;
// mma.sync: its cp.async stages; small: vectors + resident planes
template <int ENG>
__host__ __device__ constexpr size_t stage_area() {
  return ENG == ENG_TC ? (size_t)TC_STAGE_AREA + TC_STAGING_BYTES
         : ENG == ENG_SYNC ? (size_t)SY_STAGE_AREA
                           : kSmallVecBytes + kSmallPlanes * kSmallPlaneBytes;
}
// vectors used between GEMMs alias the stage area
constexpr size_t kVecBytes = 4 * SUBMAT_MAX_M * sizeof(double) + kRedDoubles * sizeof(double) +
                             SUBMAT_MAX_M * sizeof(int32_t);
static_assert(kVecBytes <= (size_t)SY_STAGE_AREA, "vector area must fit in the stage area");
// the Taylor finish's vectors follow it (3 doubles and 5 floats per entry)
static_assert(kVecBytes + SUBMAT_MAX_M * sizeof(int2) <= (size_t)TC_STAGE_AREA,
              "the gather's row extents must fit in the idle stage area");
static_assert(kVecBytes % 16 == 0, "16-byte aligned areas after the vectors");
// tcgen05 engine: room for M_0 in FP32 after the vectors, in the idle stage and staging areas
constexpr size_t kMfBytes = (size_t)TC_STAGE_AREA + TC_STAGING_BYTES - kVecBytes;
static_assert(kVecBytes + 44 * (size_t)SUBMAT_MAX_M <= (size_t)SY_STAGE_AREA &&
                  kVecBytes + 44 * (size_t)SUBMAT_MAX_M <= (size_t)TC_STAGE_AREA + TC_STAGING_BYTES,
              "finish vectors must fit in the idle stage area");

template <int ENG>
__global__ void __launch_bounds__(ENG == ENG_TC ? TC_THREADS : kThreads,
                                  ENG == ENG_SMALL ? kSmallCtasPerSm : 1)
    fwd_mixed_kernel(const __grid_constant__ FwdArgs a) {
  constexpr bool TC = ENG == ENG_TC, SMALL = ENG == ENG_SMALL;
  constexpr int VMAX = SMALL ? kSmallVmax : SUBMAT_MAX_M;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  double* y_s = reinterpret_cast<double*>(sm);
  double* v_s = y_s + VMAX;
  double* w_s = v_s + VMAX;
  double* red_s = w_s + VMAX;                         // kRedDoubles doubles
  int32_t* R_s = reinterpret_cast<int32_t*>(red_s + kRedDoubles);
  unsigned char* tail = sm + stage_area<ENG>();
  uint64_t* bars = reinterpret_cast<uint64_t*>(tail);  // full, empty [TC_STAGES], tmem_full, tmem_empty
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(tail + 96);
  int* abort_s = reinterpret_cast<int*>(tail + 100);
  float* norm_part = reinterpret_cast<float*>(tail + 112);   // [kMaxWarps]
  unsigned* amax_s = reinterpret_cast<unsigned*>(tail + 108);
  __shared__ int job_s;

  const int tid = threadIdx.x;
  // the sliced matrices: the CTA's global scratch (tcgen05, mma.sync) or shared memory
  // (small engine, whose S_j takes the CTA's global scratch instead)
  const int LD = SMALL ? kSmallLD : a.ld;
  const size_t plane = (size_t)LD * LD;
  char* scr = a.scratch + (size_t)blockIdx.x * a.scratch_stride;
  __half* hb = SMALL ? reinterpret_cast<__half*>(sm + kSmallVecBytes) : reinterpret_cast<__half*>(scr);
  double* S = SMALL ? reinterpret_cast<double*>(scr) : reinterpret_cast<double*>(hb + kSPlane * plane);
  const int plane_base = blockIdx.x * kPlanesPerCta;
  const int vec_plane = SMALL ? kSmallVecPlane : kVecPlane;

  TcCtx tcx{};
  TcState tst;
  if (TC) {
    if (tid == 0) {
      for (int i = 0; i < 2 * TC_STAGES + 1; ++i) tc::mbar_init(&bars[i], 1);
      tc::mbar_init(&bars[2 * TC_STAGES + 1], TC_EPI_WARPS * 32);
      *abort_s = 0;
      tc::fence_mbar_init();
    }
    if ((tid >> 5) == 0) tc::tmem_alloc(tmem_holder, TC_TMEM_COLS);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    tcx.stages = sm;
    tcx.full = bars;
    tcx.empty = bars + TC_STAGES;
    tcx.tmem_full = bars + 2 * TC_STAGES;
    tcx.tmem_empty = bars + 2 * TC_STAGES + 1;
    tcx.staging = reinterpret_cast<uint4*>(sm + TC_STAGE_AREA);
    tcx.abort_s = abort_s;
    tcx.tmem = *tmem_holder;
    tcx.tm_a = &a.tm_a;
    tcx.tm_b = &a.tm_b;
  } else {
    if (tid == 0) *abort_s = 0;
    __syncthreads();
  }
  if (TC && a.stall != nullptr && *a.stall != 0) {
    // test aid (submat_test_stall): wait on a barrier that nothing signals, before any copy
    // or tensor-core operation is issued, so the bounded wait gives up and the CTA unwinds
    uint64_t* never = bars + 2 * TC_STAGES + 2;
    if (tid == 0) {
      tc::mbar_init(never, 1);
      tc::fence_mbar_init();
      if (!tc::mbar_wait(never, 0, TC_WAIT_LIMIT)) *abort_s = 1;
    }
    __syncthreads();
  }

  int pending = -1;          // a row taken from the queue and left unfinished by a time-out
  for (;;) {
    if (tid == 0) job_s = atomicAdd(a.queue, 1);
    __syncthreads();
    const int idx = job_s;
    __syncthreads();
    if (idx >= a.n) break;
    if (*abort_s) {
      pending = a.order[idx];
      break;
    }
    const int j = a.order[idx];
    const int m = a.m[j];
    const int pos = a.pos[j];
    const int p = a.p;
    // padded order: the tcgen05 engine needs multiples of its 16-wide k-step (and of 16 for
    // an MMA's N), the mma.sync engine multiples of its 64 x 64 tiles
    const int mp = (TC || SMALL) ? (m + 15) / 16 * 16 : pad_mixed(m);

    // Two X buffers (p = 1 only) and three buffers for M_k and the partial products T^s M_k
    // (M_k is the A operand of all p products of an iteration and stays in place).
    Mat X[2] = {{hb + 0 * NSL * plane, 0, plane_base + 0 * NSL},
                {hb + 1 * NSL * plane, 0, plane_base + 1 * NSL}};
    const int eb = slice_bias(mp, p);          // M_k and the partial products
    const int ebx = slice_bias_x(mp, eb);      // X (p = 1)
    const int e_m = E_M + eb;
    Mat B3[3] = {{hb + 2 * NSL * plane, e_m, plane_base + 2 * NSL},
                 {hb + 3 * NSL * plane, e_m, plane_base + 3 * NSL},
                 {hb + 4 * NSL * plane, e_m, plane_base + 4 * NSL}};
    // vectors carried for p >= 2 and their scratch, in the last plane (32 LD bytes)
    double* yg = reinterpret_cast<double*>(hb + vec_plane * plane);   // column pos of X_k
    float* ug = reinterpret_cast<float*>(yg + LD);               // residual vector
    float* yhg = ug + LD;
    float* ylg = yhg + LD;
    double* myg = reinterpret_cast<double*>(ylg + LD);
    float* tg = reinterpret_cast<float*>(myg + LD);
    double* ayg = reinterpret_cast<double*>(tg + LD);            // Horner accumulators of
    float* aug = reinterpret_cast<float*>(ayg + LD);             // the final step

    // the tcgen05 engine keeps the rows' extents in its idle stage area (no static shared
    // array, which would leave no room for the fourth TMA stage)
    double lam;
    if constexpr (TC)
      lam = gather_rows(a.rowptr, a.colind, a.vals_in, j, m, R_s, S, red_s,
                        reinterpret_cast<int2*>(sm + kVecBytes));
    else
      lam = gather_submatrix(a.rowptr, a.colind, a.vals_in, j, m, R_s, S, red_s);
    const double inv_lam = 1.0 / lam;

    // M_0 = S / lambda_bar (leading mp x mp, eight consecutive columns per thread), in
    // double-float FP32 from the integer split of the FP64 values; also ||M_0 - I||_F^2.
    // The tcgen05 engine also keeps M_0's leading FP32 words in its idle stage area, when
    // they fit, for the power steps below.
    float* Mf = nullptr;
    if constexpr (TC) {
      if ((size_t)mp * mp * sizeof(float) <= kMfBytes) Mf = reinterpret_cast<float*>(sm + kVecBytes);
    }
    const int mp8 = mp / 8;
    float ih, il;
    split_dbl(inv_lam, ih, il);
    {
      // two chunks per thread and step, their loads in flight together
      float nrm = 0.f;
      const int total = mp * mp8, nt = blockDim.x;
      for (int e0 = tid; e0 < total; e0 += 2 * nt) {
        double sv[2][8];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int e = e0 + h * nt;
          const int i = e / mp8, j0 = (e % mp8) * 8;
#pragma unroll
          for (int c = 0; c < 8; ++c)
            sv[h][c] = (e < total && i < m && j0 + c < m) ? S[i * m + j0 + c] : 0.0;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int e = e0 + h * nt;
          if (e >= total) break;
          const int i = e / mp8, j0 = (e % mp8) * 8;
          float mh[8], ml[8];
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const int jj = j0 + c;
            mh[c] = ml[c] = 0.f;
            if (i < m && jj < m) {
              float sh, sl;
              split_dbl(sv[h][c], sh, sl);
              mul_df(sh, sl, ih, il, mh[c], ml[c]);
              const float ev = __fadd_rn(__fsub_rn(mh[c], i == jj ? 1.f : 0.f), ml[c]);
              nrm += ev * ev;
            }
          }
          store8_slices(B3[0].q, plane, (size_t)i * LD + j0, mh, ml, e_m);
          if (Mf) {
            float4* mf = reinterpret_cast<float4*>(Mf + (size_t)i * mp + j0);
            mf[0] = make_float4(mh[0], mh[1], mh[2], mh[3]);
            mf[1] = make_float4(mh[4], mh[5], mh[6], mh[7]);
          }
        }
      }
      nrm = warp_sum_f(nrm);
      if ((tid & 31) == 0) norm_part[tid >> 5] = nrm;
    }
    __syncthreads();
    float nrm2 = sum_parts(norm_part, nwarps());

    // lower end of M_0's spectrum: the raw estimate gives the condition estimate
    // lambda_bar / lambda_min(S) = 1 / lambda_min(M_0), half of it steers the steps
    const float lo_raw =
        Mf ? start_lo_smem(Mf, m, mp, reinterpret_cast<float*>(v_s),
                           reinterpret_cast<float*>(w_s), reinterpret_cast<float*>(red_s))
           : start_lo_slices(B3[0].q, plane, LD, e_m, m, mp, reinterpret_cast<float*>(v_s),
                             reinterpret_cast<float*>(w_s), reinterpret_cast<float*>(red_s));
    float lo = 0.5f * lo_raw;

    // tracked vector (p >= 2): the column y of X (the residual vector u is formed after the
    // last iteration, see below)
    const bool track = (p >= 2);
    // A^(-1/p): y_0 = e_pos and y <- T y per step; A^(1/p): y_0 = M_0 e_pos and
    // y <- T^(p-1) y, since S^(1/p) e_pos = lambda_bar^(1/p) X^(p-1) M_0 e_pos at the limit
    const int ny = a.sign < 0 ? 1 : p - 1;
    if (track) {
      for (int i = tid; i < mp; i += blockDim.x) {
        const double s0 = i < m ? S[pos * m + i] * inv_lam : 0.0;
        yg[i] = a.sign < 0 ? ((i == pos) ? 1.0 : 0.0) : s0;
      }
    }
    __threadfence();             // planes are read next through L2 (cp.async.cg / TMA)
    __syncthreads();

    GemmIO io{mp, m, p, LD, plane, norm_part, amax_s, 0.f, 0.f};
    // vt: vector work to run with this GEMM (tcgen05: on the vector warps during this and
    // the iteration's later GEMMs; mma.sync: before the GEMM on all warps).  first / last:
    // the GEMM starts / ends an iteration's sequence (see gemm_tc).
    auto gemm = [&](Mat A, Mat B, Mat C, Mat Y, int flags, const VecTask* vt, bool first = true,
                    bool last = true) -> bool {
      if (TC) return gemm_tc(tcx, tst, A, B, C, Y, flags, io, vt, first, last);
      if (vt) vec_task<0>(*vt);
      if (SMALL)
        gemm_small(A, B, C, Y, flags, io);
      else
        gemm_sync(A, B, C, Y, flags, io, reinterpret_cast<__half*>(sm));
      return true;
    };
    auto vec_of = [&](const Mat& Mk, double c, double alpha, bool track_u) {
      return VecTask{Mk.q, plane, LD, Mk.e, m, mp, p, ny, c, alpha, yg, ug, yhg, ylg, myg, tg,
                     track_u};
    };

    int xc = 0, mi = 0;
    int n_gemm = 0;
    const float tol2 = (float)(a.tol * a.tol * (double)m);
    const float stag2 = 1e-4f * (float)m;       // (1e-2)^2 m
    int iters = 0;
    float prev2 = 3.0e38f, xmax = 1.f;
    bool bad = !(nrm2 == nrm2), stop = false;

    // Iteration k: T_k = c_k (alpha_k I - M_k) with constants for the interval
    // [max(lo_k, 1 - ||M_k - I||_F), 1] (the Frobenius norm bounds the distance of every
    // eigenvalue from 1); X_{k+1} = X_k T_k (tracked as vectors for p >= 2, a product for
    // p = 1), M_{k+1} = T_k^p M_k as p products with M_k as the A operand.
    while (!bad) {
      // p >= 2: close enough to I for the final Taylor step (see below)
      if (track && nrm2 <= kTaylorStop * kTaylorStop) break;
      const ScaledStep st = scaled_step(fmaxf(lo, 1.f - sqrtf(nrm2)), p, kAlphaQuantum);
      io.c = st.c;
      io.alpha = st.alpha;
      const Mat Mk = B3[mi];
      const VecTask vt = vec_of(Mk, (double)st.c, (double)st.alpha, false);
      if (track) {
        // the vector step runs with the first product below
      } else if (iters == 0) {
        // X_1 = T_0 (elementwise from M_0)
        X[0].e = exp_of(st.tmax) + ebx;
        xmax = st.tmax;
        for (int e = tid; e < mp * mp8; e += blockDim.x) {
          const int i = e / mp8, j0 = (e % mp8) * 8;
          const size_t g = (size_t)i * LD + j0;
          float vh[8], vl[8], th[8], tl[8];
          load8_df(Mk.q, plane, g, Mk.e, vh, vl);
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            th[c] = tl[c] = 0.f;
            if (i < m && j0 + c < m)
              t_affine(vh[c], vl[c], i == j0 + c ? 1.f : 0.f, st.alpha, 0.f, st.c, 0.f, th[c],
                       tl[c]);
          }
          store8_slices(X[0].q, plane, g, th, tl, X[0].e);
        }
        __threadfence();
        __syncthreads();
      } else {
        // X_{k+1} = c (alpha X_k - X_k M_k); X_k, T_k SPD and commuting with T_k <= tmax I,
        // so the largest entry (a diagonal one) grows at most by tmax
        X[xc ^ 1].e = exp_of(xmax * st.tmax) + ebx;
        if (tid == 0) *amax_s = 0u;
        __syncthreads();
        if (!gemm(Mk, X[xc], X[xc ^ 1], X[xc], EPI_AMAX, nullptr)) { stop = true; break; }
        ++n_gemm;
        xmax = __uint_as_float(*amax_s);
        xc ^= 1;
      }
      // M_{k+1} = T_k^p M_k: P_s = c (alpha P_{s-1} - M_k P_{s-1}), P_0 = M_k
      int src = mi, dst = (mi + 1) % 3;
      for (int s = 1; s <= p; ++s) {
        const bool last = (s == p);
        B3[dst].e = last ? e_m : exp_of(partial_bound(st, s)) + eb;
        if (!gemm(Mk, B3[src], B3[dst], B3[src], last ? EPI_NORM : 0,
                  (track && s == 1) ? &vt : nullptr, s == 1, last)) {
          stop = true;
          break;
        }
        ++n_gemm;
        src = dst;
        dst = 3 - mi - dst;                     // the buffer that is neither M_k nor P_s
      }
      if (stop) break;
      mi = src;
      lo = st.lo_next;
      ++iters;
      nrm2 = sum_parts(norm_part, kEpiGroupWarps);  // the GEMM ended with a block barrier
      if (!(nrm2 == nrm2) || nrm2 > 1e30f) { bad = true; break; }
      if (nrm2 <= tol2 || iters >= a.k_max) break;
      // at the rounding-error floor (only after a Newton step: a scaled step maps the
      // interval's upper end below 1 and may shrink the norm less while converging fast)
      if (st.newton && nrm2 <= stag2 && nrm2 > 0.25f * prev2) break;
      prev2 = nrm2;
    }
    if (stop) {
      pending = j;
      break;
    }

    // last step.  p >= 2: X_K M_K^(-1/p) is the limit (M_K = X_K^p M_0, all commuting), so
    // the carried column takes M_K^(-1/p) = (I - E)^(-1/p), E = I - M_K, as its Taylor
    // polynomial of degree J in E (Horner, one pass over M_K per degree), J chosen from
    // ||E||_2 <= ||E||_F so that the tail is below 1e-9; this lets the iteration stop at
    // ||E||_F <= kTaylorStop instead of converging to the rounding floor (one GEMM iteration
    // fewer on average).  p = 1: Newton's X (2I - M) as a product, then FP64 refinement.
    double resid = 1e300;
    float kest = 0.f;
    const double c = pow(lam, -1.0 / (double)p);               // F = c X
    if (!bad && track) {
      const double c_out = a.sign < 0 ? c : pow(lam, 1.0 / (double)p);
      // the finish's vectors: in shared memory (the GEMMs' stage and staging areas are idle
      // now), y, its Horner accumulator and M y as doubles, then u, y's double-float split,
      // M u and u's accumulator as floats; the small engine keeps its shared vector plane
      double *yf = yg, *ayf = ayg, *myf = myg;
      float *uf = ug, *yhf = yhg, *ylf = ylg, *tf = tg, *auf = aug;
      if (!SMALL) {
        yf = reinterpret_cast<double*>(sm + kVecBytes);
        ayf = yf + mp;
        myf = ayf + mp;
        uf = reinterpret_cast<float*>(myf + mp);
        yhf = uf + mp;
        ylf = yhf + mp;
        tf = ylf + mp;
        auf = tf + mp;
        for (int i = tid; i < mp; i += blockDim.x) yf[i] = yg[i];
      }
      // residual vector u = M_K e_pos (row pos of the symmetric M_K = X_K^p M_0, up to the
      // products' rounding), carried through the last step with y
      for (int i = tid; i < mp; i += blockDim.x) {
        float h = 0.f, l = 0.f;
        if (i < m) load1_df(B3[mi].q, plane, (size_t)pos * LD + i, B3[mi].e, h, l);
        uf[i] = h + l;
      }
      __syncthreads();
      const float eps = sqrtf(nrm2);
      auto degree = [&](float target) {      // tail eps^(J+1) / (1 - eps) <= target
        int J = 1;
        while (J < kTaylorMaxDeg && !(powf(eps, (float)(J + 1)) <= target * (1.f - eps))) ++J;
        return J;
      };
      // y's tail far below the 1e-6 target; u only feeds the 1e-3 residual test
      const VecTask vf{B3[mi].q, plane, LD, B3[mi].e, m, mp, p, ny, 0.0, 0.0,
                       yf, uf, yhf, ylf, myf, tf, true};
      taylor_final<SMALL ? 2 : 4>(vf, degree(1e-9f), degree(1e-5f), ayf, auf);
      // column pos of the result (lambda_bar^(-1/p) X e_pos, or lambda_bar^(1/p) X^(p-1)
      // M_0 e_pos for A^(1/p)) and the residual F^p s_pos - e_pos = u - e_pos of
      // F = lambda_bar^(-1/p) X
      float r = 0.f;
      for (int i = tid; i < m; i += blockDim.x) {
        y_s[i] = c_out * yf[i];
        const float d = uf[i] - (i == pos ? 1.f : 0.f);
        r += d * d;
      }
      r = warp_sum_f(r);
      if ((tid & 31) == 0) reinterpret_cast<float*>(red_s)[tid >> 5] = r;
      __syncthreads();
      float tot = 0.f;
      for (int w = 0; w < nwarps(); ++w) tot += reinterpret_cast<float*>(red_s)[w];
      __syncthreads();
      resid = sqrt((double)tot);
      kest = lo_raw > 0.f ? 1.f / lo_raw : 3.0e38f;
    } else if (!bad) {
      io.c = 1.f;                                // p = 1: X (2 I - M)
      io.alpha = 2.f;
      X[xc ^ 1].e = exp_of(xmax * 2.f) + ebx;
      if (tid == 0) *amax_s = 0u;
      __syncthreads();
      if (!gemm(B3[mi], X[xc], X[xc ^ 1], X[xc], EPI_AMAX, nullptr)) {
        pending = j;
        break;
      }
      ++n_gemm;
      xc ^= 1;
      SliceLoad xl{X[xc].q, plane, LD, ldexp(1.0, X[xc].e - Q0B)};
      const float xs = ldexpf(1.f, X[xc].e - Q0B);
      resid = refine_column(xl, c, S, m, pos, p, a.refine_steps, y_s, v_s, w_s, red_s);
      if (a.sign > 0) {          // A^(1/1): column pos of S itself (the iteration still checks S)
        for (int i = tid; i < m; i += blockDim.x) y_s[i] = S[pos * m + i];
        __syncthreads();
      }
      // condition estimate lambda_bar / lambda_min = lambda_max(X) (X ~ (S/lambda_bar)^(-1))
      kest = power_max_slices(X[xc].q, plane, LD, xs, m, mp, reinterpret_cast<float*>(v_s),
                              reinterpret_cast<float*>(w_s), reinterpret_cast<float*>(red_s), 6);
    }
    const bool illcond = !bad && !(kest <= (float)a.kappa_max);
    const bool ok = !bad && (resid <= a.resid_tol) && !illcond;
    if (ok) {
      double* out = a.vals_out + a.rowptr[j];
      for (int k = tid; k < m; k += blockDim.x) out[k] = y_s[k];
    }
    if (tid == 0) {
      if (!ok) {
        const int slot = atomicAdd(&a.ctr->n_fallback, 1);
        a.fallback_list[slot] = j;
      }
      if (illcond) atomicAdd(&a.ctr->n_illcond, 1ull);
      atomicMax(&a.ctr->iters_max, iters);
      atomicAdd(&a.ctr->iters_sum, (unsigned long long)iters);
      atomic_max_nonneg(&a.ctr->resid_max_bits, resid);
      atomicAdd(&a.ctr->flops_fp64, refine_flops(m, p, a.refine_steps));
      // ten FP16 slice products per GEMM, counted with the true order m
      atomicAdd(&a.ctr->flops_tensor, (double)n_gemm * kSliceProducts * 2.0 * (double)m * m * m);
      // the method's own count: (p+1) dense products of order m per iteration (+ p = 1's
      // final X product), whatever this engine executes for them
      atomicAdd(&a.ctr->flops_alg,
                ((double)iters * (p + 1) + (p == 1 ? 1.0 : 0.0)) * 2.0 * (double)m * m * m);
    }
    __syncthreads();
  }

  __syncthreads();
  if (*abort_s) {
    // a pipeline wait gave up: the row this CTA left unfinished and every row it takes from
    // the queue from now on are written as NaN (plain stores; nothing else is issued)
    if (tid == 0) atomicExch(&a.ctr->error, 1);
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int j = pending;;) {
      if (j >= 0) {
        double* out = a.vals_out + a.rowptr[j];
        for (int k = tid; k < a.m[j]; k += blockDim.x) out[k] = nan;
      }
      __syncthreads();
      if (tid == 0) job_s = atomicAdd(a.queue, 1);
      __syncthreads();
      const int idx = job_s;
      __syncthreads();
      if (idx >= a.n) break;
      j = a.order[idx];
    }
  }
  if (TC) {
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if ((tid >> 5) == 0) tc::tmem_dealloc(tcx.tmem, TC_TMEM_COLS);
  }
}

}  // namespace

template <int ENG>
static size_t smem_bytes() {
  return stage_area<ENG>() + kSmemTail + 1024;       // + alignment slack
}
size_t smem_fwd_mixed() { return smem_bytes<ENG_TC>(); }

size_t scratch_mixed(int ld) { return (size_t)kPlanesPerCta * ld * ld * sizeof(__half); }

size_t scratch_small() { return (size_t)kSmallMaxM * kSmallMaxM * sizeof(double); }

int small_engine_max_m() { return kSmallMaxM; }

cudaError_t launch_fwd_mixed(const FwdArgs& a, int grid, cudaStream_t s) {
  if (a.engine == ENG_SYNC)
    fwd_mixed_kernel<ENG_SYNC><<<grid, kThreads, smem_bytes<ENG_SYNC>(), s>>>(a);
  else if (a.engine == ENG_SMALL)
    fwd_mixed_kernel<ENG_SMALL><<<grid, kThreads, smem_bytes<ENG_SMALL>(), s>>>(a);
  else
    fwd_mixed_kernel<ENG_TC><<<grid, TC_THREADS, smem_bytes<ENG_TC>(), s>>>(a);
  return cudaGetLastError();
}

int mixed_ctas_per_sm(int engine) { return engine == ENG_SMALL ? kSmallCtasPerSm : 1; }

cudaError_t set_attr_mixed() {
  cudaError_t e = cudaFuncSetAttribute(fwd_mixed_kernel<ENG_TC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes<ENG_TC>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fwd_mixed_kernel<ENG_SMALL>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem_bytes<ENG_SMALL>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fwd_mixed_kernel<ENG_SYNC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_bytes<ENG_SYNC>());
}

}  // namespace submat
