// All-FP64 forward: the same per-submatrix pipeline as the mixed path (gather, Gershgorin
// scaling, coupled iteration with spectrally scaled steps and a final Newton step, the
// column of X carried as a vector for p >= 2, FP64 column refinement for p = 1, scatter),
// with every GEMM in FP64 on the CUDA cores.  It is the
// accuracy reference on the GPU and the baseline the mixed-precision path is measured
// against.
#include "common.cuh"
#include "refine.cuh"
#include "fp64_gemm.cuh"
#include "scaled_step.cuh"

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
  double* norm2_s = red_s + kRedDoubles;
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
    double* X[2] = {w, w + mat};                                 // p = 1 only
    double* B3[3] = {w + 2 * mat, w + 3 * mat, w + 4 * mat};     // M_k and T^s M_k

    const double lam = gather_submatrix(a.rowptr, a.colind, a.vals_in, j, m, R_s, S, red_s);
    const double inv_lam = 1.0 / lam;
    double nrm = 0.0;
    for (size_t e = tid; e < mat; e += blockDim.x) {
      const int i = (int)(e / mp), jj = (int)(e % mp);
      double mv = 0.0;
      if (i < m && jj < m) {
        mv = S[i * m + jj] * inv_lam;
        const double ev = mv - (i == jj ? 1.0 : 0.0);
        nrm += ev * ev;
      }
      B3[0][e] = mv;
    }
    nrm = warp_sum(nrm);
    if ((tid & 31) == 0) red_s[tid >> 5] = nrm;
    __syncthreads();
    double nrm2 = 0.0;
    for (int w = 0; w < nwarps(); ++w) nrm2 += red_s[w];     // in warp order
    float lo = 0.5f * start_lo(S, m, inv_lam, v_s, w_s, red_s, kStartLoSteps);

    // tracked vectors (p >= 2): y = X_k e_pos (A^(-1/p)) or X_k^(p-1) M_0 e_pos (A^(1/p)) in
    // y_s, u = X_k^p M_0 e_pos in v_s
    const bool track = (p >= 2);
    const int ny = a.sign < 0 ? 1 : p - 1;
    if (track) {
      for (int i = tid; i < m; i += blockDim.x) {
        v_s[i] = S[pos * m + i] * inv_lam;
        y_s[i] = a.sign < 0 ? ((i == pos) ? 1.0 : 0.0) : v_s[i];
      }
    }
    __syncthreads();
    auto vec_step = [&](const double* Mk, double c, double alpha) {
      DenseLoad Ml{Mk, mp};
      for (int t = 0; t < ny; ++t) {
        matvec_rows(Ml, 1.0, y_s, w_s, m);
        for (int i = tid; i < m; i += blockDim.x) y_s[i] = c * (alpha * y_s[i] - w_s[i]);
        __syncthreads();
      }
      for (int t = 0; t < p; ++t) {
        matvec_rows(Ml, 1.0, v_s, w_s, m);
        for (int i = tid; i < m; i += blockDim.x) v_s[i] = c * (alpha * v_s[i] - w_s[i]);
        __syncthreads();
      }
    };

    int xc = 0, mi = 0, iters = 0;
    bool bad = !(nrm2 == nrm2);
    const double tol2 = a.tol * a.tol * (double)m;
    const double stag2 = 1e-8 * (double)m;      // (1e-4)^2 m
    double prev2 = 1e300;
    // iteration k as in the mixed path: T_k = c_k (alpha_k I - M_k) for the interval
    // [max(lo_k, 1 - ||M_k - I||_F), 1]; M_{k+1} = T_k^p M_k with M_k as the A operand
    while (!bad) {
      const ScaledStep st = scaled_step(fmaxf(lo, (float)(1.0 - sqrt(nrm2))), p);
      const double c = st.newton ? 1.0 / (double)p : (double)st.c;
      const double alpha = st.newton ? (double)(p + 1) : (double)st.alpha;
      const double* Mk = B3[mi];
      if (track) {
        vec_step(Mk, c, alpha);
      } else if (iters == 0) {
        for (size_t e = tid; e < mat; e += blockDim.x) {
          const int i = (int)(e / mp), jj = (int)(e % mp);
          X[0][e] = (i < m && jj < m) ? c * ((i == jj ? alpha : 0.0) - Mk[e]) : 0.0;
        }
        __syncthreads();
      } else {
        gemm64(X[xc], Mk, X[xc ^ 1], mp, m, EPI_STORE, nullptr, 0.0, 0.0, 1.0, gsm, norm2_s,
               X[xc], c, alpha);
        xc ^= 1;
      }
      int src = mi, dst = (mi + 1) % 3;
      for (int s = 1; s <= p; ++s) {
        const bool last = (s == p);
        if (last) {
          if (tid == 0) *norm2_s = 0.0;
          __syncthreads();
        }
        gemm64(Mk, B3[src], B3[dst], mp, m, last ? EPI_M : EPI_STORE, nullptr, 0.0, 0.0, 1.0,
               gsm, norm2_s, B3[src], c, alpha);
        src = dst;
        dst = 3 - mi - dst;
      }
      mi = src;
      lo = st.lo_next;
      ++iters;
      nrm2 = *norm2_s;
      __syncthreads();
      if (!(nrm2 == nrm2) || nrm2 > 1e300) { bad = true; break; }
      if (nrm2 <= tol2 || iters >= a.k_max) break;
      // at the rounding-error floor (only after a Newton step, as in the mixed path)
      if (st.newton && nrm2 <= stag2 && nrm2 > 0.25 * prev2) break;
      prev2 = nrm2;
    }
    // last step: Newton's T = ((p+1) I - M)/p, whose first-order part is M^(-1/p)
    double resid = 1e300;
    const double cl = pow(lam, -1.0 / (double)p);
    if (!bad && track) {
      vec_step(B3[mi], 1.0 / (double)p, (double)(p + 1));
      const double c_out = a.sign < 0 ? cl : pow(lam, 1.0 / (double)p);
      for (int i = tid; i < m; i += blockDim.x) {
        w_s[i] = v_s[i] - (i == pos ? 1.0 : 0.0);
        y_s[i] *= c_out;
      }
      __syncthreads();
      resid = block_norm2(w_s, m, red_s);                    // ||F^p s_pos - e_pos||
    } else if (!bad) {
      gemm64(X[xc], B3[mi], X[xc ^ 1], mp, m, EPI_STORE, nullptr, 0.0, 0.0, 1.0, gsm, norm2_s,
             X[xc], 1.0, 2.0);                                // p = 1: X (2 I - M)
      xc ^= 1;
      DenseLoad xl{X[xc], mp};
      resid = refine_column(xl, cl, S, m, pos, p, a.refine_steps, y_s, v_s, w_s, red_s);
      if (a.sign > 0) {          // A^(1/1): column pos of S itself (the iteration still checks S)
        for (int i = tid; i < m; i += blockDim.x) y_s[i] = S[pos * m + i];
        __syncthreads();
      }
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
      const double n_gemm = track ? (double)iters * p : (double)iters * 2.0;   // + final X (p = 1)
      atomicAdd(&a.ctr->flops_fp64,
                n_gemm * 2.0 * m3 + refine_flops(m, p, a.refine_steps));
      // the method's own count: (p+1) dense products per iteration (+ p = 1's final one)
      atomicAdd(&a.ctr->flops_alg, ((double)iters * (p + 1) + (p == 1 ? 1.0 : 0.0)) * 2.0 * m3);
    }
    __syncthreads();
  }
}

}  // namespace

size_t smem_fwd_fp64() {
  return (2 * TK * TB + 3 * SUBMAT_MAX_M + kRedDoubles + 2) * sizeof(double) +
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
