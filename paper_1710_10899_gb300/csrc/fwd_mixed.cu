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
// matrix is therefore held as five FP16 planes of small integers with one power-of-two
// scale per matrix (an error-free splitting in the manner of Ozaki et al.; slices.cuh):
//     A = 2^(E-7) sum_{s<5} q_s 2^(-8s),  |q0| <= 128, |q1..q4| <= 129,
// about 39 significant bits relative to the largest entry (E is chosen tight: M's
// eigenvalues lie in (0,1], those of T and of T^i M in [1,2) and (0,2); X's exponent is
// measured after every product).  A product is the sum over levels L = s + t <= 4 of
// 2^(-8L) sum_{s+t=L} Q_s^A Q_t^B (15 FP16 MMAs per k-step, FP32 accumulation per level).
// The products of these integers are exact, and every level-0 partial sum is an integer
// below 2^14 K, so for K <= 1024 the tensor cores accumulate level 0 exactly (level 1
// below 2^15 K: exact for K <= 512, and its weight is 2^-8 anyway); levels 2..4 carry
// weights 2^-16..2^-32.  The levels dropped (s + t >= 5) bound the normwise error of a
// product near 2^-39 sqrt(K) of max|A| max|B|.  The epilogue combines the levels in
// double-float (FP32 pairs) and re-splits the result.  (With four planes, the ~2^-31
// per-product error, kept by every iteration, left ~6e-7 in the result; measured.)
//
// GEMM engines (template parameter TC):
//   TC = true  (default): tcgen05.mma kind::f16, M = 128, N = 64, the five level
//              accumulators in TMEM (5 x 64 of 512 columns), operands moved by TMA
//              (SWIZZLE_64B, 32-wide k-slices) through a 3-stage mbarrier pipeline.
//              Roles: warp 0 issues TMA, warp 1 issues MMAs, warps 4-7 run the epilogue.
//              All working matrices are symmetric, so a row-major B read as K-major
//              gives B^T = B to rounding: the engine computes A B^T.
//   TC = false: mma.sync m16n8k16 on 64 x 64 tiles with a cp.async pipeline (the legacy
//              tensor path, kept as the baseline the tcgen05 engine is measured against).
//
// Working matrices live in a per-CTA global scratch: 34 planes of LD x LD halves per CTA
// (LD = the plan's largest order padded to 64): X, T, M (two buffers each) x 5 planes, then
// the gathered S_j in FP64 in the last four planes' space.  A submatrix of order m uses the
// leading mp x mp block (mp = m padded to 64); its padding rows/columns stay exactly zero.
#include <cuda_fp16.h>
#include "common.cuh"
#include "refine.cuh"
#include "slices.cuh"
#include "tc_prims.cuh"

namespace submat {
namespace {

using namespace slc;

constexpr int E_M = 0;             // |M| <= 1 (eigenvalues of M_k lie in (0, 1])
constexpr int E_T = 1;             // |T| <= 2 (eigenvalues of T_k lie in [1, (p+1)/p))
constexpr int E_P = 1;             // |T^i M| <= 2 for i < p (eigenvalues below ((p+1)/p)^i < e)
constexpr int kPlanesPerCta = 34;  // 6 matrices x 5 planes + 4 planes of room for S_j (FP64)

enum Epi { EPI_FIXED = 0, EPI_M = 1, EPI_X = 2 };

struct Mat {
  __half* q;        // NSL planes of LD*LD halves
  int e;            // scale exponent: |entries| <= 2^e
  int plane0;       // index of plane 0 in the tensor map's third dimension
};

struct GemmIO {     // what every GEMM call shares within one submatrix
  int mp, m, p, ld;
  size_t plane;     // ld * ld
  float* norm2_s;
  unsigned* amax_s;
};

// Slices of 16 consecutive values -> two 16-byte stores per plane.
__device__ __forceinline__ void store16_slices(__half* q, size_t plane, size_t idx0,
                                               const float* vh, const float* vl, int e) {
  __align__(16) __half out[NSL][16];
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    float s[NSL];
    make_slices(vh[c], vl[c], e, s);
#pragma unroll
    for (int k = 0; k < NSL; ++k) out[k][c] = __float2half_rn(s[k]);
  }
#pragma unroll
  for (int k = 0; k < NSL; ++k) {
    uint4* dst = reinterpret_cast<uint4*>(q + k * plane + idx0);
    const uint4* src = reinterpret_cast<const uint4*>(out[k]);
    dst[0] = src[0];
    dst[1] = src[1];
  }
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

// y[i] = scale * sum_k X(i,k) x[k] for i < m, X from its first NP planes (FP32 result).
// One warp per row, eight consecutive columns per lane with 16-byte loads; x is zero
// beyond m up to mp.  x, y in shared memory.
template <int NP>
__device__ void matvec_slices_f32(const __half* q, size_t plane, int ld, float scale,
                                  const float* x, float* y, int m, int mp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < m; i += kWarps) {
    float acc = 0.f;
    for (int c0 = lane * 8; c0 < mp; c0 += 256) {
      const size_t e = (size_t)i * ld + c0;
      uint4 raw[NP];
#pragma unroll
      for (int k = 0; k < NP; ++k) raw[k] = *reinterpret_cast<const uint4*>(q + k * plane + e);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        float v = 0.f, w = 1.f;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          v = fmaf(__half2float(reinterpret_cast<const __half*>(&raw[k])[c]), w, v);
          w *= (1.f / 256.f);
        }
        acc = fmaf(v, x[c0 + c], acc);
      }
    }
    acc = warp_sum_f(acc);
    if (lane == 0) y[i] = acc * scale;
  }
  __syncthreads();
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
    if (lane == 0) { red_s[warp] = na; red_s[kWarps + warp] = nb; }
    __syncthreads();
    float ta = 0.f, tb = 0.f;
    for (int w = 0; w < kWarps; ++w) { ta += red_s[w]; tb += red_s[kWarps + w]; }
    lam = sqrtf(tb / ta);
    const float inv = tb > 0.f ? rsqrtf(tb) : 0.f;
    for (int i = tid; i < m; i += blockDim.x) a_s[i] = b_s[i] * inv;
    __syncthreads();
  }
  return lam;
}

// Residual ||e_pos - F^p s_pos||_2 of the converged iterate F = c X (p >= 2, no column step):
// a failure test against a threshold of order 1e-3, so FP32 with three planes suffices.
__device__ float column_residual_f32(const __half* q, size_t plane, int ld, float xscale,
                                     double c, const double* S, int m, int mp, int pos, int p,
                                     float* a_s, float* b_s, float* red_s) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < mp; i += blockDim.x) {
    a_s[i] = i < m ? (float)S[pos * m + i] : 0.f;       // s_pos (S = S^T)
    b_s[i] = 0.f;
  }
  __syncthreads();
  float* u = a_s;
  float* v = b_s;
  const float sc = (float)c * xscale;
  for (int t = 0; t < p; ++t) {
    matvec_slices_f32<3>(q, plane, ld, sc, u, v, m, mp);
    float* tmp = u; u = v; v = tmp;
  }
  float r = 0.f;
  for (int i = tid; i < m; i += blockDim.x) {
    const float d = (i == pos ? 1.f : 0.f) - u[i];
    r += d * d;
  }
  r = warp_sum_f(r);
  if (lane == 0) red_s[warp] = r;
  __syncthreads();
  float tot = 0.f;
  for (int w = 0; w < kWarps; ++w) tot += red_s[w];
  __syncthreads();
  return sqrtf(tot);
}

// ======================================================================================
// tcgen05 engine
// ======================================================================================
constexpr int TC_M = 128, TC_N = 64, TC_K = 32;        // tile and k-slice
constexpr int TC_STAGES = 3;
constexpr int TC_A_PLANE = TC_M * TC_K * 2;            // 8192 B
constexpr int TC_B_PLANE = TC_N * TC_K * 2;            // 4096 B
constexpr int TC_STAGE_BYTES = NSL * (TC_A_PLANE + TC_B_PLANE);   // 61440 B
constexpr int TC_STAGE_AREA = TC_STAGES * TC_STAGE_BYTES;         // 184320 B
constexpr uint32_t TC_IDESC = tc::idesc_f16(TC_M, TC_N);
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;           // polls before a wait gives up
constexpr uint32_t TC_TMEM_COLS = 512;

struct TcState {            // pipeline counters; each role keeps its own copy
  uint32_t pit = 0;         // stages issued (TMA)
  uint32_t cit = 0;         // stages consumed (MMA)
  uint32_t tmt = 0;         // tiles accumulated (MMA)
  uint32_t ept = 0;         // tiles drained (epilogue)
};

struct TcCtx {
  unsigned char* stages;    // 1024-aligned shared memory
  uint64_t* full;           // [TC_STAGES]
  uint64_t* empty;          // [TC_STAGES]
  uint64_t* tmem_full;
  uint64_t* tmem_empty;
  int* abort_s;
  uint32_t tmem;
  const CUtensorMap* tm_a;
  const CUtensorMap* tm_b;
};

// C = A B^T on the tcgen05 engine (see the header comment).  All 256 threads call it.
// Returns false if a pipeline wait timed out (the CTA then stops).
__device__ bool gemm_tc(const TcCtx& c, TcState& st, Mat A, Mat B, Mat C, int epi, Mat Tn,
                        const GemmIO& io) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mp = io.mp;
  const int ntm = (mp + TC_M - 1) / TC_M, ntn = mp / TC_N, KT = mp / TC_K;
  const int ntiles = ntm * ntn;
  // generic-proxy writes (planes, staging, shared vectors) before async-proxy reads/writes
  tc::fence_proxy_async_global();
  tc::fence_proxy_async_shared();
  __syncthreads();

  if (warp == 0) {
    if (lane == 0) {                                   // ---- TMA producer
      for (int t = 0; t < ntiles && !*c.abort_s; ++t) {
        const int tm = t / ntn, tn = t % ntn;
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
  } else if (warp == 1) {
    if (lane == 0) {                                   // ---- MMA issuer
      for (int t = 0; t < ntiles && !*c.abort_s; ++t) {
        if (st.tmt > 0 && !tc::mbar_wait(c.tmem_empty, (st.tmt - 1) & 1, TC_WAIT_LIMIT)) {
          *c.abort_s = 1;
          break;
        }
        tc::tc_fence_after();
        bool ok = true;
        for (int kt = 0; kt < KT; ++kt) {
          const uint32_t s = st.cit % TC_STAGES;
          if (!tc::mbar_wait(&c.full[s], (st.cit / TC_STAGES) & 1, TC_WAIT_LIMIT)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t sa = tc::saddr(c.stages + s * TC_STAGE_BYTES);
          const uint32_t sb = sa + NSL * TC_A_PLANE;
#pragma unroll
          for (int kk = 0; kk < TC_K / 16; ++kk) {
#pragma unroll
            for (int L = 0; L < NSL; ++L) {
#pragma unroll
              for (int sa_i = 0; sa_i <= L; ++sa_i) {
                const uint64_t da = tc::desc_sw64(sa + sa_i * TC_A_PLANE + kk * 32);
                const uint64_t db = tc::desc_sw64(sb + (L - sa_i) * TC_B_PLANE + kk * 32);
                tc::mma_f16(c.tmem + L * TC_N, da, db, TC_IDESC,
                            (kt | kk | sa_i) != 0 ? 1u : 0u);
              }
            }
          }
          tc::mma_commit(&c.empty[s]);                 // frees the stage when these finish
          ++st.cit;
        }
        if (!ok) {
          *c.abort_s = 1;
          break;
        }
        tc::mma_commit(c.tmem_full);                   // the tile's accumulators are ready
        ++st.tmt;
      }
    }
  } else if (warp >= 4) {                              // ---- epilogue (TMEM lanes 0..127)
    const int q4 = warp - 4;
    const float cscale = ldexpf(1.f, A.e + B.e - 14);
    float nrm = 0.f, amax = 0.f;
    for (int t = 0; t < ntiles; ++t) {
      if (!tc::mbar_wait(c.tmem_full, st.ept & 1, TC_WAIT_LIMIT)) {
        *c.abort_s = 1;
        break;
      }
      tc::tc_fence_after();
      const int tm = t / ntn, tn = t % ntn;
      const int row = tm * TC_M + q4 * 32 + lane;
      for (int c0 = 0; c0 < TC_N; c0 += 16) {
        float acc[NSL][16];
#pragma unroll
        for (int L = 0; L < NSL; ++L)
          tc::tmem_ld16(c.tmem + ((uint32_t)(q4 * 32) << 16) + L * TC_N + c0, acc[L]);
        tc::tmem_ld_wait();
        if (row < mp) {
          float vh[16], vl[16];
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const float lv[NSL] = {acc[0][k], acc[1][k], acc[2][k], acc[3][k], acc[4][k]};
            combine_levels(lv, cscale, vh[k], vl[k]);
          }
          const int j0 = tn * TC_N + c0;
          const size_t idx0 = (size_t)row * io.ld + j0;
          store16_slices(C.q, io.plane, idx0, vh, vl, C.e);
          if (epi == EPI_X) {
#pragma unroll
            for (int k = 0; k < 16; ++k) amax = fmaxf(amax, fabsf(vh[k]));
          } else {
            if (epi == EPI_M) {
              float th[16], tl[16];
#pragma unroll
              for (int k = 0; k < 16; ++k) {
                const int jj = j0 + k;
                const bool in = (row < io.m) && (jj < io.m);
                const float d = (row == jj) ? 1.f : 0.f;
                th[k] = 0.f;
                tl[k] = 0.f;
                if (in) t_from_m(vh[k], vl[k], d, io.p, th[k], tl[k]);
                const float ev = in ? __fadd_rn(__fsub_rn(vh[k], d), vl[k]) : 0.f;
                nrm += ev * ev;
              }
              store16_slices(Tn.q, io.plane, idx0, th, tl, Tn.e);
            }
          }
        }
      }
      tc::tc_fence_before();
      tc::mbar_arrive(c.tmem_empty);
      ++st.ept;
    }
    if (epi == EPI_M) {
      nrm = warp_sum_f(nrm);
      if (lane == 0) atomicAdd(io.norm2_s, nrm);
    }
    if (epi == EPI_X) {
      for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      if (lane == 0) atomicMax(io.amax_s, __float_as_uint(amax));
    }
  }
  // the planes written here are read next by TMA (async proxy) through L2
  __threadfence();
  tc::fence_proxy_async_global();
  __syncthreads();
  return *c.abort_s == 0;
}

// ======================================================================================
// mma.sync engine (baseline)
// ======================================================================================
constexpr int BM = 64;             // CTA output tile (64 x 64)
constexpr int BK = 32;             // k-slice per pipeline stage
constexpr int SY_STAGES = 3;
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
// at a time (warps 2 x 4, 32 x 16 each), 3-stage cp.async pipeline over k.
__device__ void gemm_sync(Mat A, Mat B, Mat C, int epi, Mat Tn, const GemmIO& io,
                          __half* smem) {
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 2, wn = warp & 3;      // 2 x 4 warps
  const int mp = io.mp, ld = io.ld;
  const int nt = mp / BM;
  const int KT = mp / BK;
  const size_t plane = io.plane;
  const float cscale = ldexpf(1.f, A.e + B.e - 14);
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
                                   acc[3][mt][n][ci], acc[4][mt][n][ci]};
            float vh, vl;
            combine_levels(lv, cscale, vh, vl);
            const size_t idx = (size_t)i * ld + jj;
            put_slices(C.q, plane, idx, vh, vl, C.e);
            if (epi == EPI_X) {
              amax = fmaxf(amax, fabsf(vh));
            } else {
              if (epi == EPI_M) {
                const bool in = (i < io.m) && (jj < io.m);
                const float d = (i == jj) ? 1.f : 0.f;
                float th = 0.f, tl = 0.f;
                if (in) t_from_m(vh, vl, d, io.p, th, tl);
                put_slices(Tn.q, plane, idx, th, tl, Tn.e);
                const float ev = in ? __fadd_rn(__fsub_rn(vh, d), vl) : 0.f;
                nrm += ev * ev;
              }
            }
          }
  }
  if (epi == EPI_M) {
    nrm = warp_sum_f(nrm);
    if (lane == 0) atomicAdd(io.norm2_s, nrm);
  }
  if (epi == EPI_X) {
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) atomicMax(io.amax_s, __float_as_uint(amax));
  }
  // The next GEMM reads these planes with cp.async.cg, which reads L2 and bypasses L1.
  __threadfence();
  __syncthreads();
}

// ======================================================================================
// the per-submatrix kernel
// ======================================================================================
constexpr size_t kSmemTail = 256;                       // barriers and flags
template <bool TC>
__host__ __device__ constexpr size_t stage_area() { return TC ? (size_t)TC_STAGE_AREA : (size_t)SY_STAGE_AREA; }
// vectors used between GEMMs alias the stage area
constexpr size_t kVecBytes = 3 * SUBMAT_MAX_M * sizeof(double) + 2 * kWarps * sizeof(double) +
                             SUBMAT_MAX_M * sizeof(int32_t);
static_assert(kVecBytes <= (size_t)SY_STAGE_AREA, "vector area must fit in the stage area");

template <bool TC>
__global__ void __launch_bounds__(kThreads, 1) fwd_mixed_kernel(const __grid_constant__ FwdArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  double* y_s = reinterpret_cast<double*>(sm);
  double* v_s = y_s + SUBMAT_MAX_M;
  double* w_s = v_s + SUBMAT_MAX_M;
  double* red_s = w_s + SUBMAT_MAX_M;                 // 2*kWarps doubles
  int32_t* R_s = reinterpret_cast<int32_t*>(red_s + 2 * kWarps);
  unsigned char* tail = sm + stage_area<TC>();
  uint64_t* bars = reinterpret_cast<uint64_t*>(tail);  // full[3], empty[3], tmem_full, tmem_empty
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(tail + 64);
  int* abort_s = reinterpret_cast<int*>(tail + 68);
  float* norm2_s = reinterpret_cast<float*>(tail + 72);
  unsigned* amax_s = reinterpret_cast<unsigned*>(tail + 76);
  __shared__ int job_s;

  const int tid = threadIdx.x;
  const int LD = a.ld;
  const size_t plane = (size_t)LD * LD;
  char* scr = a.scratch + (size_t)blockIdx.x * a.scratch_stride;
  __half* hb = reinterpret_cast<__half*>(scr);
  double* S = reinterpret_cast<double*>(hb + 30 * plane);
  const int plane_base = blockIdx.x * kPlanesPerCta;

  TcCtx tcx{};
  TcState tst;
  if (TC) {
    if (tid == 0) {
      for (int i = 0; i < 2 * TC_STAGES + 1; ++i) tc::mbar_init(&bars[i], 1);
      tc::mbar_init(&bars[2 * TC_STAGES + 1], 128);
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
    tcx.abort_s = abort_s;
    tcx.tmem = *tmem_holder;
    tcx.tm_a = &a.tm_a;
    tcx.tm_b = &a.tm_b;
  } else {
    if (tid == 0) *abort_s = 0;
    __syncthreads();
  }

  for (;;) {
    if (tid == 0) job_s = atomicAdd(&a.ctr->queue, 1);
    __syncthreads();
    const int idx = job_s;
    __syncthreads();
    if (idx >= a.n || *abort_s) break;
    const int j = a.order[idx];
    const int m = a.m[j];
    const int pos = a.pos[j];
    const int p = a.p;
    const int mp = pad_mixed(m);

    Mat X[2] = {{hb + 0 * NSL * plane, E_T, plane_base + 0}, {hb + 1 * NSL * plane, E_T, plane_base + 5}};
    Mat T[2] = {{hb + 2 * NSL * plane, E_T, plane_base + 10}, {hb + 3 * NSL * plane, E_T, plane_base + 15}};
    Mat M[2] = {{hb + 4 * NSL * plane, E_M, plane_base + 20}, {hb + 5 * NSL * plane, E_M, plane_base + 25}};

    const double lam = gather_submatrix(a.rowptr, a.colind, a.vals_in, j, m, R_s, S, red_s);
    const double inv_lam = 1.0 / lam;

    // M_0 = S / lambda_bar, T_0 = ((p+1) I - M_0)/p, X_1 = X_0 T_0 = T_0 (leading mp x mp),
    // eight consecutive columns per thread; one FP64 product and one FP64 difference per
    // entry, the rest in double-float FP32.
    const int mp8 = mp / 8;
    for (int e = tid; e < mp * mp8; e += blockDim.x) {
      const int i = e / mp8, j0 = (e % mp8) * 8;
      float mh[8], ml[8], th[8], tl[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int jj = j0 + c;
        mh[c] = ml[c] = th[c] = tl[c] = 0.f;
        if (i < m && jj < m) {
          const double mv = S[i * m + jj] * inv_lam;
          mh[c] = (float)mv;
          ml[c] = (float)(mv - (double)mh[c]);
          t_from_m(mh[c], ml[c], i == jj ? 1.f : 0.f, p, th[c], tl[c]);
        }
      }
      const size_t g = (size_t)i * LD + j0;
      store8_slices(M[0].q, plane, g, mh, ml, E_M);
      store8_slices(T[0].q, plane, g, th, tl, E_T);
      store8_slices(X[0].q, plane, g, th, tl, E_T);
    }
    if (tid == 0) *norm2_s = 0.f;
    __threadfence();             // planes are read next through L2 (cp.async.cg / TMA)
    __syncthreads();

    GemmIO io{mp, m, p, LD, plane, norm2_s, amax_s};
    auto gemm = [&](Mat A, Mat B, Mat C, int epi, Mat Tn) -> bool {
      if (TC) return gemm_tc(tcx, tst, A, B, C, epi, Tn, io);
      gemm_sync(A, B, C, epi, Tn, io, reinterpret_cast<__half*>(sm));
      return true;
    };

    int xc = 0, tc_i = 0, mc = 0;
    int n_gemm = 0;
    const float tol2 = (float)(a.tol * a.tol * (double)m);
    const float stag2 = 1e-4f * (float)m;       // (1e-2)^2 m
    int iters = 1;
    float nrm2 = 0.f, prev2 = 3.0e38f;
    bool bad = false, stop = false;

    // X_{k+1} = X_k T_k, sliced directly with a predicted exponent: X_k and T_k are SPD and
    // commute, and T_k <= (p+1)/p I, so X_{k+1} <= (p+1)/p X_k in the Loewner order and the
    // largest entry (a diagonal one) grows at most by (p+1)/p.  The epilogue measures the
    // new largest entry for the next prediction.
    float xmax = (float)(p + 1) / (float)p;      // |X_1| = |T_0| <= (p+1)/p
    auto x_update = [&]() -> bool {
      X[xc ^ 1].e = exp_bound(xmax * ((float)(p + 1) / (float)p) * (1.f + 1e-6f));
      if (tid == 0) *amax_s = 0u;
      __syncthreads();
      if (!gemm(X[xc], T[tc_i], X[xc ^ 1], EPI_X, T[tc_i])) return false;
      xmax = __uint_as_float(*amax_s);
      xc ^= 1;
      ++n_gemm;
      return true;
    };

    for (;;) {
      // M <- T^p M, the last product also writes T_next and ||M - I||_F^2
      Mat cur = M[mc];
      int free_slot = mc ^ 1;
      for (int s = 1; s <= p && !stop; ++s) {
        const bool last = (s == p);
        M[free_slot].e = last ? E_M : E_P;
        Mat dst = M[free_slot];
        if (last) {
          if (tid == 0) *norm2_s = 0.f;
          __syncthreads();
        }
        if (!gemm(T[tc_i], cur, dst, last ? EPI_M : EPI_FIXED, T[tc_i ^ 1])) stop = true;
        ++n_gemm;
        cur = dst;
        mc = free_slot;
        free_slot ^= 1;
      }
      if (stop) break;
      tc_i ^= 1;
      nrm2 = *norm2_s;
      __syncthreads();
      if (!(nrm2 == nrm2) || nrm2 > 1e30f) { bad = true; break; }
      if (nrm2 <= tol2 || iters >= a.k_max) break;
      if (nrm2 <= stag2 && nrm2 > 0.25f * prev2) break;     // at the rounding-error floor
      prev2 = nrm2;
      if (!x_update()) { stop = true; break; }
      ++iters;
    }
    if (stop) break;
    if (!bad && !x_update()) break;

    double resid = 1e300;
    float kest = 0.f;
    if (!bad) {
      const double c = pow(lam, -1.0 / (double)p);
      SliceLoad xl{X[xc].q, plane, LD, ldexp(1.0, X[xc].e - 7)};
      const float xs = ldexpf(1.f, X[xc].e - 7);
      if (p >= 2 && a.refine_steps < 1) {
        for (int i = tid; i < m; i += blockDim.x) y_s[i] = c * xl(i, pos);
        resid = column_residual_f32(X[xc].q, plane, LD, xs, c, S, m, mp, pos, p,
                                    reinterpret_cast<float*>(v_s), reinterpret_cast<float*>(w_s),
                                    reinterpret_cast<float*>(red_s));
      } else {
        resid = refine_column(xl, c, S, m, pos, p, a.refine_steps, y_s, v_s, w_s, red_s);
      }
      // condition estimate lambda_bar / lambda_min = lambda_max(X)^p (X ~ (S/lambda_bar)^(-1/p))
      const float lx = power_max_slices(X[xc].q, plane, LD, xs, m, mp,
                                        reinterpret_cast<float*>(v_s),
                                        reinterpret_cast<float*>(w_s),
                                        reinterpret_cast<float*>(red_s), 6);
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

  __syncthreads();
  if (*abort_s && tid == 0) atomicExch(&a.ctr->error, 1);
  if (TC) {
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if ((tid >> 5) == 0) tc::tmem_dealloc(tcx.tmem, TC_TMEM_COLS);
  }
}

}  // namespace

template <bool TC>
static size_t smem_bytes() {
  return stage_area<TC>() + kSmemTail + 1024;       // + alignment slack
}
size_t smem_fwd_mixed() { return smem_bytes<true>(); }

size_t scratch_mixed(int ld) { return (size_t)kPlanesPerCta * ld * ld * sizeof(__half); }

cudaError_t launch_fwd_mixed(const FwdArgs& a, int grid, cudaStream_t s) {
  if (a.engine == 1)
    fwd_mixed_kernel<false><<<grid, kThreads, smem_bytes<false>(), s>>>(a);
  else
    fwd_mixed_kernel<true><<<grid, kThreads, smem_bytes<true>(), s>>>(a);
  return cudaGetLastError();
}

cudaError_t set_attr_mixed() {
  cudaError_t e = cudaFuncSetAttribute(fwd_mixed_kernel<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes<true>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fwd_mixed_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_bytes<false>());
}

}  // namespace submat
