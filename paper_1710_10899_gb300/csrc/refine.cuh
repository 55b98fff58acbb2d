// FP64 column refinement and residual check of one submatrix result (internal header).
//
// After the coupled iteration, F = c * X (c = lambda_bar^(-1/p)) approximates S^(-1/p) to
// working precision.  Only column pos of F is kept (Alg. 2), so the FP64 work is done on
// that column alone, with O(p m^2) matrix-vector products:
//
//   p = 1:  iterative refinement of S y = e_pos with F as approximate inverse,
//           y <- y + F (e_pos - S y)  (each sweep contracts the error by ||I - F S||);
//   p >= 2: one Newton step on the column, y = F ((p+1) e_pos - F^p s_pos) / p, with
//           s_pos = column pos of S; it removes the part of the error that commutes with S.
//
// The residual ||e_pos - F^p s_pos||_2 (column pos of F^p S - I, i.e. the paper's residual
// X^p A - I of Sec. 4.1 restricted to the submatrix) is returned for the fallback test.
#pragma once
#include "common.cuh"

namespace submat {

// out[i] = c * sum_k F(i,k) in[k], i < m.  One warp per row.  in/out in shared memory.
template <class FLoad>
__device__ __forceinline__ void matvec_rows(const FLoad& F, double c, const double* in,
                                            double* out, int m) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < m; i += nwarps()) {
    double s = 0.0;
    for (int k = lane; k < m; k += 32) s = fma(F(i, k), in[k], s);
    s = warp_sum(s);
    if (lane == 0) out[i] = c * s;
  }
  __syncthreads();
}

__device__ __forceinline__ double block_norm2(const double* v, int m, double* red_s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s += v[i] * v[i];
  s = warp_sum(s);
  if (lane == 0) red_s[warp] = s;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < nwarps(); ++w) t += red_s[w];
  __syncthreads();
  return sqrt(t);
}

struct DenseLoad {     // row-major FP64 m x m
  const double* a;
  int ld;
  __device__ __forceinline__ double operator()(int i, int k) const { return a[i * ld + k]; }
};

// Refines column pos of F = c*X (X given by xload) and writes it to y_s.  S: FP64 m x m
// (ld m).  v_s, w_s: scratch vectors (shared, m doubles).  Returns the residual.
template <class XLoad>
__device__ double refine_column(const XLoad& X, double c, const double* S, int m, int pos,
                                int p, int steps, double* y_s, double* v_s, double* w_s,
                                double* red_s) {
  const int tid = threadIdx.x;
  DenseLoad Sl{S, m};
  double resid;
  if (p == 1) {
    for (int i = tid; i < m; i += blockDim.x) y_s[i] = c * X(i, pos);
    __syncthreads();
    const int sweeps = steps < 1 ? 1 : steps;
    resid = 0.0;
    for (int t = 0; t < sweeps; ++t) {
      matvec_rows(Sl, 1.0, y_s, v_s, m);                       // v = S y
      for (int i = tid; i < m; i += blockDim.x) v_s[i] = (i == pos ? 1.0 : 0.0) - v_s[i];
      __syncthreads();
      const double r = block_norm2(v_s, m, red_s);             // ||e - S y||
      if (t == 0) resid = r;
      if (t < steps) {
        matvec_rows(X, c, v_s, w_s, m);                        // w = F (e - S y)
        for (int i = tid; i < m; i += blockDim.x) y_s[i] += w_s[i];
        __syncthreads();
      }
    }
  } else {
    for (int i = tid; i < m; i += blockDim.x) v_s[i] = S[pos * m + i];   // s_pos (S = S^T)
    __syncthreads();
    double* a = v_s;
    double* b = w_s;
    for (int t = 0; t < p; ++t) {                               // a = F^p s_pos
      matvec_rows(X, c, a, b, m);
      double* tmp = a; a = b; b = tmp;
    }
    for (int i = tid; i < m; i += blockDim.x) b[i] = (i == pos ? 1.0 : 0.0) - a[i];
    __syncthreads();
    resid = block_norm2(b, m, red_s);                          // ||e - F^p s||
    if (steps >= 1) {
      // u = ((p+1) e - F^p s) / p = e + (e - F^p s) / p
      for (int i = tid; i < m; i += blockDim.x)
        a[i] = (i == pos ? 1.0 : 0.0) + b[i] / (double)p;
      __syncthreads();
      matvec_rows(X, c, a, y_s, m);                           // y = F u
    } else {
      for (int i = tid; i < m; i += blockDim.x) y_s[i] = c * X(i, pos);
      __syncthreads();
    }
  }
  return resid;
}

// Largest eigenvalue of the (symmetric positive definite) X, estimated by `iters` steps of
// the power method in FP32 from a fixed positive start vector.  a_s, b_s: m floats each.
template <class XLoad>
__device__ float power_max_eig(const XLoad& X, int m, float* a_s, float* b_s, float* red_s,
                               int iters) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < m; i += blockDim.x)
    a_s[i] = 1.f + (float)(((unsigned)i * 2654435761u) >> 22) * (1.f / 1024.f);
  __syncthreads();
  float lam = 0.f;
  for (int it = 0; it < iters; ++it) {
    for (int i = warp; i < m; i += nwarps()) {
      float s = 0.f;
      for (int k = lane; k < m; k += 32) s = fmaf((float)X(i, k), a_s[k], s);
      s = warp_sum_f(s);
      if (lane == 0) b_s[i] = s;
    }
    __syncthreads();
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

// FP64 flops of refine_column (for the report).
__host__ __device__ __forceinline__ double refine_flops(int m, int p, int steps) {
  const double mv = 2.0 * m * (double)m;
  if (p == 1) {
    const int sweeps = steps < 1 ? 1 : steps;
    return sweeps * mv + steps * mv;
  }
  return p * mv + (steps >= 1 ? mv : 0.0);
}

}  // namespace submat
