// FP64 register-tiled GEMM of the FP64 forward path (internal header).
#pragma once
#include "common.cuh"

namespace submat {
namespace fp64 {

constexpr int TB = 64;     // output tile
constexpr int TK = 16;     // k-slice

enum Epi { EPI_STORE = 0, EPI_M = 1 };

// C = A B for FP64 mp x mp matrices (row-major, ld mp), or C = yc (ya Y - A B) if Y is
// given (the step matrix yc (ya I - A) applied to the symmetric Y).  EPI_M adds
// sum (C - I)^2 over the leading m x m block to *norm2_s and, if Tn is given, writes the
// next step matrix Tn = tc (ta I - C) / td there (zero elsewhere; Newton's step is
// ta = p+1, tc = 1, td = p).
static __device__ void gemm64(const double* __restrict__ A, const double* __restrict__ B,
                       double* __restrict__ C, int mp, int m, int epi, double* __restrict__ Tn,
                       double tc, double ta, double td, double* smem, double* norm2_s,
                       const double* __restrict__ Y = nullptr, double yc = 0.0,
                       double ya = 0.0) {
  double* As = smem;                 // [TK][TB]
  double* Bs = smem + TK * TB;       // [TK][TB]
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int nt = mp / TB;
  double nrm = 0.0;
  for (int t = 0; t < nt * nt; ++t) {
    const int i0 = (t / nt) * TB, j0 = (t % nt) * TB;
    double acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
    for (int k0 = 0; k0 < mp; k0 += TK) {
#pragma unroll
      for (int q = 0; q < (TB * TK) / kThreads; ++q) {
        const int e = tid + q * kThreads;
        const int ii = e / TK, kk = e % TK;
        As[kk * TB + ii] = A[(size_t)(i0 + ii) * mp + k0 + kk];
        const int kb = e / TB, jj = e % TB;
        Bs[kb * TB + jj] = B[(size_t)(k0 + kb) * mp + j0 + jj];
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < TK; ++kk) {
        double av[4], bv[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) av[r] = As[kk * TB + ty + 16 * r];
#pragma unroll
        for (int c = 0; c < 4; ++c) bv[c] = Bs[kk * TB + tx + 16 * c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = i0 + ty + 16 * r, jj = j0 + tx + 16 * c;
        const size_t idx = (size_t)i * mp + jj;
        const double v = Y ? yc * (ya * Y[idx] - acc[r][c]) : acc[r][c];
        C[idx] = v;
        if (epi == EPI_M) {
          const bool in = (i < m) && (jj < m);
          const double d = (i == jj) ? 1.0 : 0.0;
          if (Tn) Tn[idx] = in ? tc * (ta * d - v) / td : 0.0;
          const double e = in ? v - d : 0.0;
          nrm += e * e;
        }
      }
  }
  if (epi == EPI_M) {          // added in warp order: the result does not depend on timing
    nrm = warp_sum(nrm);
    __syncthreads();           // the tile buffers are no longer read
    if ((tid & 31) == 0) smem[tid >> 5] = nrm;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < nwarps(); ++w) t += smem[w];
      *norm2_s += t;
    }
  }
  __syncthreads();
}

}  // namespace fp64
}  // namespace submat
