// Mixed-precision forward: one persistent CTA per SM processes whole submatrices.
//
// Per row j (Alg. 1, Sec. 3.2, Alg. 2):
//   gather S_j (FP64) -> Gershgorin bound lambda_bar = max_k sum_l |S_kl| (FP64)
//   M_0 = S/lambda_bar, X_0 = I; coupled Newton iteration for the inverse p-th root
//       T_k = ((p+1) I - M_k) / p,  X_{k+1} = X_k T_k,  M_{k+1} = T_k^p M_k
//   (the coupled form of the Newton iteration of Bini, Higham and Meini cited in Sec. 2)
//   until ||M - I||_F <= tol sqrt(m), then one more X update; F = lambda_bar^(-1/p) X;
//   FP64 column residual (refine.cuh) and condition estimate; write column pos_j.
//
// Arithmetic.  Rounding errors made in any iteration persist in the coupled iteration's
// limit, so every GEMM must be accurate to well below the 1e-6 target, and the tensor
// cores' FP32 accumulation truncates (biased toward zero) when it rounds.  Each working
// matrix A is therefore held as five FP16 planes of small integers with one power-of-two
// scale per matrix (an error-free splitting in the manner of Ozaki et al.):
//     A = 2^(E-7) sum_{s<5} q_s 2^(-8s),  |q0| <= 128, |q1..q4| <= 129,
// about 39 significant bits relative to the largest entry (E is chosen tight: M's
// eigenvalues lie in (0,1], those of T and of T^i M in [1,2) and (0,2); X's exponent is
// measured after every product).  A product is the sum over levels L = s + t <= 4 of
// 2^(-8L) sum_{s+t=L} Q_s^A Q_t^B (15 FP16 MMAs, m16n8k16, FP32 accumulation per level).
// The products of these integers are exact, and every level-0 partial sum is an integer
// below 2^14 K, so for K <= 1024 the tensor cores accumulate level 0 exactly (level 1
// below 2^15 K: exact for K <= 512, and its weight is 2^-8 anyway); levels 2..4 carry
// weights 2^-16..2^-32.  The levels dropped (s + t >= 5) bound the normwise error of a
// product near 2^-39 sqrt(K) of max|A| max|B|.  The epilogue combines the levels in
// double-float (FP32 pairs) and re-splits the result.  (With four planes, the ~2^-31
// per-product error, kept by every iteration, left ~6e-7 in the result; measured.)
//
// Working matrices live in a per-CTA global scratch (mostly L2-resident): X (2 buffers),
// T (2), M (2), each 5 planes of mp x mp halves (mp = m padded to 64), plus the gathered
// S_j in FP64.  Padding rows/columns stay exactly zero.
#include <cuda_fp16.h>
#include "common.cuh"
#include "refine.cuh"

namespace submat {
namespace {

constexpr int NSL = 5;             // integer slices per matrix
constexpr int BM = 64;             // CTA output tile (64 x 64)
constexpr int BK = 32;             // k-slice per pipeline stage
constexpr int STAGES = 3;
constexpr int A_LD = BK + 8;       // padded smem row (halves) of an A tile plane
constexpr int B_LD = BM + 8;       // padded smem row (halves) of a B tile plane
constexpr int A_PLANE = BM * A_LD;
constexpr int B_PLANE = BK * B_LD;
constexpr int STAGE = NSL * (A_PLANE + B_PLANE);       // halves per pipeline stage
constexpr int E_M = 0;             // |M| <= 1 (eigenvalues of M_k lie in (0, 1])
constexpr int E_T = 1;             // |T| <= 2 (eigenvalues of T_k lie in [1, (p+1)/p))
constexpr int E_P = 1;             // |T^i M| <= 2 for i < p (eigenvalues below ((p+1)/p)^i < e)

enum Epi { EPI_FIXED = 0, EPI_M = 1, EPI_STAGE = 2 };

struct Mat {
  __half* q;        // NSL planes of mp*mp halves
  int e;            // scale exponent: |entries| <= 2^e
};

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

// Double-float helpers (Knuth's TwoSum; no products, so no contraction hazards).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Writes the slices of v = hi + lo (|v| <= 2^e) at element idx of the planes.
__device__ __forceinline__ void put_slices(__half* q, size_t plane, size_t idx, float hi,
                                           float lo, int e) {
  const float sc = ldexpf(1.f, 7 - e);
  const float yh = hi * sc, yl = lo * sc;           // exact (power-of-two scaling)
  const float q0 = rintf(yh);
  float r = __fadd_rn(__fsub_rn(yh, q0), yl) * 256.f;
  const float q1 = rintf(r);
  r = __fsub_rn(r, q1) * 256.f;
  const float q2 = rintf(r);
  r = __fsub_rn(r, q2) * 256.f;
  const float q3 = rintf(r);
  r = __fsub_rn(r, q3) * 256.f;
  const float q4 = rintf(r);
  q[idx] = __float2half_rn(q0);
  q[plane + idx] = __float2half_rn(q1);
  q[2 * plane + idx] = __float2half_rn(q2);
  q[3 * plane + idx] = __float2half_rn(q3);
  q[4 * plane + idx] = __float2half_rn(q4);
}

// Exponent e with |v| <= 2^e for the largest magnitude amax (at least -60).
__device__ __forceinline__ int exp_bound(float amax) {
  if (!(amax > 0.f)) return -60;
  int e;
  frexpf(amax, &e);            // amax = f 2^e with f in [0.5, 1)
  return e;
}

// C = A B (mp x mp, sliced, row-major ld mp).  All eight warps work on one 64 x 64 output
// tile at a time (warps 2 x 4, 32 x 16 each), 3-stage cp.async pipeline over k.
//   EPI_FIXED: write C's slices with exponent C.e
//   EPI_M:     also T_next = ((p+1) I - C)/p (masked to the leading m x m block) and
//              sum (C - I)^2 over that block into *norm2_s
//   EPI_STAGE: write C as FP32 pairs (hi plane at stage_hi, lo at stage_lo) and the
//              largest |C| into *amax_s (float bits, atomicMax)
__device__ void gemm_sliced(Mat A, Mat B, Mat C, int mp, int m, int epi, Mat Tn, int p,
                            float* stage_hi, float* stage_lo, __half* smem, float* norm2_s,
                            unsigned* amax_s) {
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 2, wn = warp & 3;      // 2 x 4 warps
  const int nt = mp / BM;
  const int KT = mp / BK;
  const size_t plane = (size_t)mp * mp;
  const float cscale = ldexpf(1.f, A.e + B.e - 14);
  const float pinv = 1.f / (float)p;
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
      __half* s = smem + st * STAGE;
      const int k0 = kt * BK;
      // A planes: 64 rows x 4 chunks of 8 halves; B planes: 32 rows x 8 chunks
#pragma unroll
      for (int c = tid; c < BM * 4; c += kThreads) {
        const int r = c >> 2, q = (c & 3) * 8;
        const size_t g = (size_t)(i0 + r) * mp + k0 + q;
#pragma unroll
        for (int l = 0; l < NSL; ++l) cp_async16(s + l * A_PLANE + r * A_LD + q, A.q + l * plane + g);
      }
#pragma unroll
      for (int c = tid; c < BK * 8; c += kThreads) {
        const int r = c >> 3, q = (c & 7) * 8;
        const size_t g = (size_t)(k0 + r) * mp + j0 + q;
#pragma unroll
        for (int l = 0; l < NSL; ++l)
          cp_async16(s + NSL * A_PLANE + l * B_PLANE + r * B_LD + q, B.q + l * plane + g);
      }
    };

    // prologue: STAGES-1 stages in flight
#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
      if (s < KT) load_stage(s, s);
      cp_async_commit();
    }
    for (int kt = 0; kt < KT; ++kt) {
      cp_async_wait<STAGES - 2>();
      __syncthreads();
      // refill the stage consumed in the previous iteration
      const int nk = kt + STAGES - 1;
      if (nk < KT) load_stage(nk % STAGES, nk);
      cp_async_commit();
      const __half* s = smem + (kt % STAGES) * STAGE;
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

    // epilogue
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
            // v = 2^(eA+eB-14) sum_L 2^(-8L) acc_L, in double-float
            float s0 = acc[0][mt][n][ci], e0 = 0.f, t, u;
            two_sum(s0, acc[1][mt][n][ci] * (1.f / 256.f), t, u);
            s0 = t; e0 = u;
            two_sum(s0, acc[2][mt][n][ci] * (1.f / 65536.f), t, u);
            s0 = t; e0 = __fadd_rn(e0, u);
            e0 = __fadd_rn(e0, acc[3][mt][n][ci] * (1.f / 16777216.f));
            e0 = __fadd_rn(e0, acc[4][mt][n][ci] * (1.f / 4294967296.f));
            two_sum(s0, e0, t, u);
            const float vh = t * cscale, vl = u * cscale;
            const size_t idx = (size_t)i * mp + jj;
            if (epi == EPI_STAGE) {
              stage_hi[idx] = vh;
              stage_lo[idx] = vl;
              amax = fmaxf(amax, fabsf(vh));
            } else {
              put_slices(C.q, plane, idx, vh, vl, C.e);
              if (epi == EPI_M) {
                const bool in = (i < m) && (jj < m);
                const float d = (i == jj) ? 1.f : 0.f;
                float th = 0.f, tl = 0.f;
                if (in) {
                  // ((p+1) d - v) / p in double-float
                  float a1, a2;
                  two_sum((float)(p + 1) * d, -vh, a1, a2);
                  a2 = __fsub_rn(a2, vl);
                  two_sum(a1, a2, a1, a2);
                  th = a1 * pinv;
                  // remainder of the division, exact up to one rounding of the FMA
                  const float rem = __fmaf_rn(-th, (float)p, a1);
                  tl = __fadd_rn(rem, a2) * pinv;
                }
                put_slices(Tn.q, plane, idx, th, tl, Tn.e);
                const float ev = in ? __fadd_rn(__fsub_rn(vh, d), vl) : 0.f;
                nrm += ev * ev;
              }
            }
          }
  }
  if (epi == EPI_M) {
    nrm = warp_sum_f(nrm);
    if (lane == 0) atomicAdd(norm2_s, nrm);
  }
  if (epi == EPI_STAGE) {
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) atomicMax(amax_s, __float_as_uint(amax));
  }
  // The next GEMM reads these planes with cp.async.cg, which reads L2 and bypasses L1:
  // the stores must have reached L2 (GPU scope) before the barrier releases the readers.
  __threadfence();
  __syncthreads();
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

__global__ void __launch_bounds__(kThreads, 1) fwd_mixed_kernel(FwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __half* gemm_smem = reinterpret_cast<__half*>(smem_raw);
  double* y_s = reinterpret_cast<double*>(smem_raw + STAGES * STAGE * sizeof(__half));
  double* v_s = y_s + SUBMAT_MAX_M;
  double* w_s = v_s + SUBMAT_MAX_M;
  double* red_s = w_s + SUBMAT_MAX_M;          // 2*kWarps doubles
  float* norm2_s = reinterpret_cast<float*>(red_s + 2 * kWarps);
  unsigned* amax_s = reinterpret_cast<unsigned*>(norm2_s + 1);
  int32_t* R_s = reinterpret_cast<int32_t*>(norm2_s + 4);
  __shared__ int job_s;

  char* scr = a.scratch + (size_t)blockIdx.x * a.scratch_stride;
  const int tid = threadIdx.x;

  for (;;) {
    if (tid == 0) job_s = atomicAdd(&a.ctr->queue, 1);
    __syncthreads();
    const int idx = job_s;
    __syncthreads();
    if (idx >= a.n) break;
    const int j = a.order[idx];
    const int m = a.m[j];
    const int pos = a.pos[j];
    const int p = a.p;
    const int mp = pad_mixed(m);
    const size_t plane = (size_t)mp * mp;
    const size_t mat = NSL * plane;             // halves per sliced matrix

    double* S = reinterpret_cast<double*>(scr);
    __half* hb = reinterpret_cast<__half*>(scr + (((size_t)m * m * sizeof(double) + 255) / 256) * 256);
    Mat X[2] = {{hb + 0 * mat, E_T}, {hb + 1 * mat, E_T}};
    Mat T[2] = {{hb + 2 * mat, E_T}, {hb + 3 * mat, E_T}};
    Mat M[2] = {{hb + 4 * mat, E_M}, {hb + 5 * mat, E_M}};

    const double lam = gather_submatrix(a.rowptr, a.colind, a.vals_in, j, m, R_s, S, red_s);
    const double inv_lam = 1.0 / lam;

    // M_0 = S / lambda_bar, T_0 = ((p+1) I - M_0)/p, X_1 = X_0 T_0 = T_0.
    for (size_t e = tid; e < plane; e += blockDim.x) {
      const int i = (int)(e / mp), jj = (int)(e % mp);
      double mv = 0.0, tv = 0.0;
      if (i < m && jj < m) {
        mv = S[i * m + jj] * inv_lam;
        tv = ((i == jj ? (double)(p + 1) : 0.0) - mv) / (double)p;
      }
      const float mh = (float)mv, ml = (float)(mv - (double)mh);
      const float th = (float)tv, tl = (float)(tv - (double)th);
      put_slices(M[0].q, plane, e, mh, ml, E_M);
      put_slices(T[0].q, plane, e, th, tl, E_T);
      put_slices(X[0].q, plane, e, th, tl, E_T);
    }
    if (tid == 0) *norm2_s = 0.f;
    __threadfence();             // planes are read next through L2 (cp.async.cg)
    __syncthreads();

    int xc = 0, tc = 0, mc = 0;
    int n_gemm = 0;
    const float tol2 = (float)(a.tol * a.tol * (double)m);
    const float stag2 = 1e-4f * (float)m;       // (1e-2)^2 m
    int iters = 1;
    float nrm2 = 0.f, prev2 = 3.0e38f;
    bool bad = false;

    // X_{k+1} = X_k T_k through the staging planes (the free M buffer), then re-split
    // with the exponent of the largest entry.
    auto x_update = [&]() {
      float* st_hi = reinterpret_cast<float*>(M[mc ^ 1].q);
      float* st_lo = st_hi + plane;
      if (tid == 0) *amax_s = 0u;
      __syncthreads();
      gemm_sliced(X[xc], T[tc], X[xc ^ 1], mp, m, EPI_STAGE, T[tc], p, st_hi, st_lo, gemm_smem,
                  norm2_s, amax_s);
      const int ex = exp_bound(__uint_as_float(*amax_s));
      X[xc ^ 1].e = ex;
      for (size_t e = tid; e < plane; e += blockDim.x)
        put_slices(X[xc ^ 1].q, plane, e, st_hi[e], st_lo[e], ex);
      __threadfence();           // read next through L2 (cp.async.cg)
      __syncthreads();
      xc ^= 1;
      ++n_gemm;
    };

    for (;;) {
      // M <- T^p M, the last product also writes T_next and ||M - I||_F^2
      Mat cur = M[mc];
      int free_slot = mc ^ 1;
      for (int s = 1; s <= p; ++s) {
        const bool last = (s == p);
        Mat dst = M[free_slot];
        dst.e = last ? E_M : E_P;
        M[free_slot].e = dst.e;
        if (last) {
          if (tid == 0) *norm2_s = 0.f;
          __syncthreads();
        }
        gemm_sliced(T[tc], cur, dst, mp, m, last ? EPI_M : EPI_FIXED, T[tc ^ 1], p, nullptr,
                    nullptr, gemm_smem, norm2_s, amax_s);
        ++n_gemm;
        cur = dst;
        mc = free_slot;
        free_slot ^= 1;
      }
      tc ^= 1;
      nrm2 = *norm2_s;
      __syncthreads();
      if (!(nrm2 == nrm2) || nrm2 > 1e30f) { bad = true; break; }
      if (nrm2 <= tol2 || iters >= a.k_max) break;
      if (nrm2 <= stag2 && nrm2 > 0.25f * prev2) break;     // at the rounding-error floor
      prev2 = nrm2;
      x_update();
      ++iters;
    }
    if (!bad) x_update();

    double resid = 1e300;
    float kest = 0.f;
    if (!bad) {
      const double c = pow(lam, -1.0 / (double)p);
      SliceLoad xl{X[xc].q, plane, mp, ldexp(1.0, X[xc].e - 7)};
      resid = refine_column(xl, c, S, m, pos, p, a.refine_steps, y_s, v_s, w_s, red_s);
      // condition estimate lambda_bar / lambda_min = lambda_max(X)^p (X ~ (S/lambda_bar)^(-1/p))
      SliceLoadF xf{X[xc].q, plane, mp, ldexpf(1.f, X[xc].e - 7)};
      const float lx = power_max_eig(xf, m, reinterpret_cast<float*>(v_s),
                                     reinterpret_cast<float*>(w_s),
                                     reinterpret_cast<float*>(red_s), 8);
      kest = powf(lx, (float)p);
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
      // fifteen FP16 slice products per GEMM, counted with the true order m
      atomicAdd(&a.ctr->flops_tensor, (double)n_gemm * 15.0 * 2.0 * (double)m * m * m);
    }
    __syncthreads();
  }
}

}  // namespace

size_t smem_fwd_mixed() {
  return STAGES * STAGE * sizeof(__half) + 3 * SUBMAT_MAX_M * sizeof(double) +
         2 * kWarps * sizeof(double) + 4 * sizeof(float) + SUBMAT_MAX_M * sizeof(int32_t);
}

size_t scratch_mixed(int mp) {
  const size_t s = (((size_t)mp * mp * sizeof(double) + 255) / 256) * 256;
  return s + 6 * NSL * (size_t)mp * mp * sizeof(__half);
}

cudaError_t launch_fwd_mixed(const FwdArgs& a, int grid, cudaStream_t s) {
  fwd_mixed_kernel<<<grid, kThreads, smem_fwd_mixed(), s>>>(a);
  return cudaGetLastError();
}

cudaError_t set_attr_mixed() {
  return cudaFuncSetAttribute(fwd_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_fwd_mixed());
}

}  // namespace submat
