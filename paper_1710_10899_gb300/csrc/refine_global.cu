// Global refinement of the submatrix result on a fixed sparsity pattern (Sec. 4.5: the
// submatrix method's result as the starting guess of a Newton iteration for A^(-1/p), with
// every product restricted to the pattern, as a sparse iteration has to be).
//
// On a symmetric pattern P (CSR, sorted rows) with values L, R given on P, the restricted
// product is C[i][j] = sum over k in P_i and P_j of L[i][k] R[k][j] for (i, j) in P; R[k][j]
// is read as R^T[j][k], the values of R^T on P gathered through the plan's transposed map.
// One CTA per row i stages P_i and L's row in shared memory; a warp takes an entry (i, j),
// its lanes walk row j of R^T (32 entries at a time, in order), locate each column in P_i by
// bisection, and combine by a fixed butterfly, so a call gives the same bits every time.
// The step: R = A X (then R <- R X, p - 1 more times), X <- ((p + 1) X - X R) / p,
// X <- (X + X^T) / 2, all in FP64, from the symmetric part of the given start.
#include <algorithm>
#include "common.cuh"

namespace submat {
namespace {

constexpr int kRefThreads = 256;

__global__ void __launch_bounds__(kRefThreads) masked_product_kernel(
    const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind, int32_t n,
    const double* __restrict__ L, const double* __restrict__ Rt, double* __restrict__ C) {
  __shared__ int32_t P_s[SUBMAT_MAX_M];
  __shared__ double L_s[SUBMAT_MAX_M];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const int ib = rowptr[i], mi = rowptr[i + 1] - ib;
    for (int k = tid; k < mi; k += blockDim.x) {
      P_s[k] = colind[ib + k];
      L_s[k] = L[ib + k];
    }
    __syncthreads();
    for (int q = warp; q < mi; q += nw) {
      const int j = P_s[q], jb = rowptr[j], je = rowptr[j + 1];
      double sum = 0.0;
      for (int e0 = jb; e0 < je; e0 += 32) {
        const int e = e0 + lane;
        double v = 0.0;
        if (e < je) {
          const int pk = find_sorted(P_s, mi, colind[e]);    // k = colind[e] in P_i?
          if (pk >= 0) v = L_s[pk] * Rt[e];
        }
        sum += warp_sum(v);
      }
      if (lane == 0) C[ib + q] = sum;
    }
    __syncthreads();
  }
}

// out[e] = c1 * x[e] + c2 * y[e]
__global__ void axpby_kernel(double c1, const double* __restrict__ x, double c2,
                             const double* __restrict__ y, double* __restrict__ out, int64_t nnz) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = c1 * x[e] + c2 * y[e];
}

int blocks_for(int64_t work, int threads) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, 152 * 16));
}

}  // namespace

cudaError_t refine_masked_product(const int32_t* rowptr, const int32_t* colind, int32_t n,
                                  const double* L, const double* Rt, double* C, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  masked_product_kernel<<<std::min(n, 152 * 8), kRefThreads, 0, s>>>(rowptr, colind, n, L, Rt, C);
  return cudaGetLastError();
}

cudaError_t refine_axpby(double c1, const double* x, double c2, const double* y, double* out,
                         int64_t nnz, cudaStream_t s) {
  if (nnz <= 0) return cudaSuccess;
  axpby_kernel<<<blocks_for(nnz, 256), 256, 0, s>>>(c1, x, c2, y, out, nnz);
  return cudaGetLastError();
}

}  // namespace submat
