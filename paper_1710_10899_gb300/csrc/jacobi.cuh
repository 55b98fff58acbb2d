// FP64 cyclic Jacobi eigendecomposition of one symmetric submatrix per CTA (internal header).
// Round-robin ordering: ceil(m/2) disjoint rotations per step run in parallel; rotation
// from the symmetric 2x2 Schur decomposition of Golub & Van Loan (Alg. 8.4.1).
#pragma once
#include "common.cuh"

namespace submat {
namespace jac {

constexpr int kMaxSweeps = 30;

// Eigendecomposition of the symmetric m x m matrix A (ld m, global) in place: on return
// A's diagonal holds the eigenvalues and V (ld m) the eigenvectors (columns).
// pair_s: 2*ceil(m/2) ints, cs_s: 2*ceil(m/2) doubles (shared).  Returns the sweeps used,
// or -1 if A holds a non-finite value (nothing is decomposed then).
static __device__ int jacobi_eig(double* __restrict__ A, double* __restrict__ V, int m, int* pair_s,
                          double* cs_s, double* red_s) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < m * m; e += blockDim.x) V[e] = (e / m == e % m) ? 1.0 : 0.0;
  __syncthreads();
  const int mm = m + (m & 1);
  const int np = mm / 2;
  int sweep = 0;
  for (; sweep < kMaxSweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = tid; e < m * m; e += blockDim.x) {
      const double v = A[e];
      tot += v * v;
      if (e / m != e % m) off += v * v;
    }
    off = warp_sum(off);
    tot = warp_sum(tot);
    if (lane == 0) { red_s[warp] = off; red_s[kMaxWarps + warp] = tot; }
    __syncthreads();
    double so = 0.0, st = 0.0;
    for (int w = 0; w < nwarps(); ++w) { so += red_s[w]; st += red_s[kMaxWarps + w]; }
    __syncthreads();
    if (!(st <= 1.7e308)) return -1;     // NaN or infinity somewhere in A
    if (m == 1 || !(so > 1e-28 * st)) break;       // off(A) <= 1e-14 ||A||_F
    for (int s = 0; s < mm - 1; ++s) {
      for (int k = tid; k < np; k += blockDim.x) {
        int p, q;
        if (k == 0) { p = s; q = mm - 1; }
        else { p = (s + k) % (mm - 1); q = (s - k + mm - 1) % (mm - 1); }
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, sn = 0.0;
        if (q < m) {
          const double apq = A[p * m + q];
          if (apq != 0.0) {
            const double tau = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            sn = t * c;
          }
        }
        pair_s[2 * k] = p; pair_s[2 * k + 1] = q;
        cs_s[2 * k] = c; cs_s[2 * k + 1] = sn;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int e = tid; e < np * m; e += blockDim.x) {
        const int k = e / m, i = e % m;
        const int p = pair_s[2 * k], q = pair_s[2 * k + 1];
        if (q >= m) continue;
        const double c = cs_s[2 * k], sn = cs_s[2 * k + 1];
        if (sn == 0.0) continue;
        const double ap = A[i * m + p], aq = A[i * m + q];
        A[i * m + p] = c * ap - sn * aq;
        A[i * m + q] = sn * ap + c * aq;
        const double vp = V[i * m + p], vq = V[i * m + q];
        V[i * m + p] = c * vp - sn * vq;
        V[i * m + q] = sn * vp + c * vq;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int e = tid; e < np * m; e += blockDim.x) {
        const int k = e / m, i = e % m;
        const int p = pair_s[2 * k], q = pair_s[2 * k + 1];
        if (q >= m) continue;
        const double c = cs_s[2 * k], sn = cs_s[2 * k + 1];
        if (sn == 0.0) continue;
        const double ap = A[p * m + i], aq = A[q * m + i];
        A[p * m + i] = c * ap - sn * aq;
        A[q * m + i] = sn * ap + c * aq;
      }
      __syncthreads();
    }
  }
  return sweep;
}

}  // namespace jac
}  // namespace submat
