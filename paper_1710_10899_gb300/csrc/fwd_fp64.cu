// All-FP64 forward: the same per-submatrix pipeline as the mixed path (gather, Gershgorin
// scaling, coupled Newton iteration, FP64 column refinement, scatter), with every GEMM in
// FP64 on the CUDA cores.  It is the accuracy reference on the GPU and the baseline the
// mixed-precision path is measured against.
#include "common.cuh"
#include "refine.cuh"
#include "fp64_gemm.cuh"

namespace submat {
namespace {

using namespace fp64;

__global__ void __launch_bounds__(kThreads, 1) fwd_fp64_kernel(FwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* gsm = reinterpret_cast<double*>(smem_raw);              // 2*TK*TB
  double* y_s = gsm + 2 * TK * TB;
  double* v_s = y_s + SUBMAT_MAX_M;
  double* w_s = v_s + SUBMAT_MAX_M;
  double* red_s = w_s + SUBMAT_MAX_M;
  double* norm2_s = red_s + kWarps;
  int32_t* R_s = reinterpret_cast<int32_t*>(norm2_s + 2);
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
    const int mp = pad_fp64(m);
    const size_t mat = (size_t)mp * mp;
    double* S = reinterpret_cast<double*>(scr);
    double* w = S + (((size_t)m * m + 31) / 32) * 32;
    double* X[2] = {w, w + mat};
    double* T[2] = {w + 2 * mat, w + 3 * mat};
    double* M[2] = {w + 4 * mat, w + 5 * mat};

    const double lam = gather_submatrix(a.rowptr, a.colind, a.vals_in, j, m, R_s, S, red_s);
    const double inv_lam = 1.0 / lam;
    for (size_t e = tid; e < mat; e += blockDim.x) {
      const int i = (int)(e / mp), jj = (int)(e % mp);
      double mv = 0.0, tv = 0.0;
      if (i < m && jj < m) {
        mv = S[i * m + jj] * inv_lam;
        tv = ((i == jj ? (double)(p + 1) : 0.0) - mv) / (double)p;
      }
      M[0][e] = mv;
      T[0][e] = tv;
      X[0][e] = tv;
    }
    if (tid == 0) *norm2_s = 0.0;
    __syncthreads();

    int xc = 0, tc = 0, mc = 0, iters = 1;
    bool bad = false;
    const double tol2 = a.tol * a.tol * (double)m;
    const double stag2 = 1e-8 * (double)m;      // (1e-4)^2 m
    double prev2 = 1e300;
    for (;;) {
      const double* cur = M[mc];
      int free_slot = mc ^ 1;
      for (int s = 1; s <= p; ++s) {
        const bool last = (s == p);
        double* dst = M[free_slot];
        if (last) {
          if (tid == 0) *norm2_s = 0.0;
          __syncthreads();
        }
        gemm64(T[tc], cur, dst, mp, m, last ? EPI_M : EPI_STORE, T[tc ^ 1], p, gsm, norm2_s);
        cur = dst;
        mc = free_slot;
        free_slot ^= 1;
      }
      tc ^= 1;
      const double nrm2 = *norm2_s;
      __syncthreads();
      if (!(nrm2 == nrm2) || nrm2 > 1e300) { bad = true; break; }
      if (nrm2 <= tol2 || iters >= a.k_max) break;
      if (nrm2 <= stag2 && nrm2 > 0.25 * prev2) break;      // at the rounding-error floor
      prev2 = nrm2;
      gemm64(X[xc], T[tc], X[xc ^ 1], mp, m, EPI_STORE, nullptr, p, gsm, norm2_s);
      xc ^= 1;
      ++iters;
    }
    if (!bad) {
      gemm64(X[xc], T[tc], X[xc ^ 1], mp, m, EPI_STORE, nullptr, p, gsm, norm2_s);
      xc ^= 1;
    }
    double resid = 1e300;
    if (!bad) {
      const double c = pow(lam, -1.0 / (double)p);
      DenseLoad xl{X[xc], mp};
      resid = refine_column(xl, c, S, m, pos, p, a.refine_steps, y_s, v_s, w_s, red_s);
    }
    const bool ok = !bad && (resid <= a.resid_tol);
    if (ok) {
      double* out = a.vals_out + a.rowptr[j];
      for (int k = tid; k < m; k += blockDim.x) out[k] = y_s[k];
    }
    if (tid == 0) {
      if (!ok) {
        const int slot = atomicAdd(&a.ctr->n_fallback, 1);
        a.fallback_list[slot] = j;
      }
      atomicMax(&a.ctr->iters_max, iters);
      atomicAdd(&a.ctr->iters_sum, (unsigned long long)iters);
      atomic_max_nonneg(&a.ctr->resid_max_bits, resid);
      const double m3 = (double)m * m * m;
      atomicAdd(&a.ctr->flops_fp64,
                (double)iters * (p + 1) * 2.0 * m3 + refine_flops(m, p, a.refine_steps));
    }
    __syncthreads();
  }
}

}  // namespace

size_t smem_fwd_fp64() {
  return (2 * TK * TB + 3 * SUBMAT_MAX_M + kWarps + 2) * sizeof(double) +
         SUBMAT_MAX_M * sizeof(int32_t);
}

size_t scratch_fp64(int mp) {
  return ((((size_t)mp * mp + 31) / 32) * 32 + 6 * (size_t)mp * mp) * sizeof(double);
}

cudaError_t launch_fwd_fp64(const FwdArgs& a, int grid, cudaStream_t s) {
  fwd_fp64_kernel<<<grid, kThreads, smem_fwd_fp64(), s>>>(a);
  return cudaGetLastError();
}

cudaError_t set_attr_fp64() {
  return cudaFuncSetAttribute(fwd_fp64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_fwd_fp64());
}

}  // namespace submat
