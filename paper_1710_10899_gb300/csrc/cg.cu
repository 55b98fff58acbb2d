// Conjugate gradients on A x = b, plain or with the submatrix method's K ~ A^(-1/2) as the
// preconditioner in the form of Sec. 4.4: CG on K^T A K y = K^T b, then x = K y.
//
// Kernels: CSR products (a warp per row, lanes over the row, a fixed butterfly), the values
// of K^T gathered through the plan's transposed map, and dot products reduced in a fixed
// order (per-block partial sums over a fixed grid, then one block), so a solve gives the
// same bits on every call.  The host drives the iteration and reads two scalars per step.
#include <algorithm>
#include <cmath>
#include "common.cuh"

namespace submat {
namespace {

constexpr int kDotBlocks = 256, kDotThreads = 256;

__global__ void spmv_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                            const double* __restrict__ vals, const double* __restrict__ x,
                            double* __restrict__ y, int32_t n) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    double s = 0.0;
    for (int e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) s = fma(vals[e], x[colind[e]], s);
    s = warp_sum(s);
    if (lane == 0) y[i] = s;
  }
}

// kt[e] for e = (r, c): K's value at (c, r), the entry tpos[e] of row c.
__global__ void transpose_vals_kernel(const int32_t* __restrict__ rowptr,
                                      const int32_t* __restrict__ colind,
                                      const int32_t* __restrict__ tpos,
                                      const double* __restrict__ vals, double* __restrict__ kt,
                                      int64_t nnz) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    kt[e] = vals[rowptr[colind[e]] + tpos[e]];
}

// Block sum of one value per thread, in a fixed order.
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// part[block] = the block's share of x . y (elements strided by the grid, in order).
__global__ void dot_partial_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                   int32_t n, double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    s = fma(x[i], y[i], s);
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// out = sum of the kDotBlocks partial sums, in order.
__global__ void dot_final_kernel(const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < kDotBlocks; i += blockDim.x) s += part[i];
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) *out = t;
}

// x += alpha p, r -= alpha q, and the partial sums of r . r (as dot_partial_kernel).
__global__ void cg_update_kernel(double alpha, double* __restrict__ x, double* __restrict__ r,
                                 const double* __restrict__ p, const double* __restrict__ q,
                                 int32_t n, double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    s = fma(ri, ri, s);
  }
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// p = r + beta p
__global__ void cg_dir_kernel(double beta, const double* __restrict__ r, double* __restrict__ p,
                              int32_t n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], r[i]);
}

int spmv_blocks(int32_t n) { return (int)std::min<int64_t>(((int64_t)n * 32 + 255) / 256, 65535); }

}  // namespace

cudaError_t cg_spmv(const int32_t* rowptr, const int32_t* colind, const double* vals,
                    const double* x, double* y, int32_t n, cudaStream_t s) {
  spmv_kernel<<<spmv_blocks(n), 256, 0, s>>>(rowptr, colind, vals, x, y, n);
  return cudaGetLastError();
}

cudaError_t cg_transpose_vals(const int32_t* rowptr, const int32_t* colind, const int32_t* tpos,
                              const double* vals, double* kt, int64_t nnz, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((nnz + 255) / 256, 65535);
  if (blocks > 0) transpose_vals_kernel<<<blocks, 256, 0, s>>>(rowptr, colind, tpos, vals, kt, nnz);
  return cudaGetLastError();
}

// *out = x . y (device scalar); part: kDotBlocks doubles of scratch.
cudaError_t cg_dot(const double* x, const double* y, int32_t n, double* part, double* out,
                   cudaStream_t s) {
  dot_partial_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(x, y, n, part);
  dot_final_kernel<<<1, kDotThreads, 0, s>>>(part, out);
  return cudaGetLastError();
}

// x += alpha p, r -= alpha q, *rr = r . r
cudaError_t cg_update(double alpha, double* x, double* r, const double* p, const double* q,
                      int32_t n, double* part, double* rr, cudaStream_t s) {
  cg_update_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(alpha, x, r, p, q, n, part);
  dot_final_kernel<<<1, kDotThreads, 0, s>>>(part, rr);
  return cudaGetLastError();
}

cudaError_t cg_dir(double beta, const double* r, double* p, int32_t n, cudaStream_t s) {
  cg_dir_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(beta, r, p, n);
  return cudaGetLastError();
}

size_t cg_dot_scratch() { return kDotBlocks; }

}  // namespace submat
