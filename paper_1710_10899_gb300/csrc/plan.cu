// Plan kernels: pattern checks and the integer part of Alg. 1 (m_j, pos_j).
#include "common.cuh"

namespace submat {
namespace {

// flags[0] bits: 1 = column index out of range, 2 = not strictly ascending in a row,
//                4 = pattern not symmetric, 8 = diagonal entry missing.
__global__ void check_pattern_kernel(const int32_t* __restrict__ rowptr,
                                     const int32_t* __restrict__ colind, int32_t n,
                                     int32_t* flags) {
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
    const int b = rowptr[r], e = rowptr[r + 1];
    int bits = 0;
    for (int k = b + lane; k < e; k += 32) {
      const int c = colind[k];
      if (c < 0 || c >= n) { bits |= 1; continue; }
      if (k + 1 < e && colind[k + 1] <= c) bits |= 2;
      // (c, r) must be stored: binary search r in row c
      int lo = rowptr[c], hi = rowptr[c + 1] - 1, hit = 0;
      while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int v = colind[mid];
        if (v == r) { hit = 1; break; }
        if (v < r) lo = mid + 1; else hi = mid - 1;
      }
      if (!hit) bits |= 4;
    }
    for (int o = 16; o > 0; o >>= 1) bits |= __shfl_xor_sync(0xffffffffu, bits, o);
    if (lane == 0 && bits) atomicOr(flags, bits);
  }
}

// m[j] = |R_j|, pos[j] = R_j.indexof(j) (or -1 and flag 8 when the diagonal is missing).
__global__ void plan_rows_kernel(const int32_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ colind, int32_t n, int32_t* m,
                                 int32_t* pos, int32_t* flags) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int b = rowptr[j], e = rowptr[j + 1];
  m[j] = e - b;
  int lo = b, hi = e - 1, hit = -1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int v = colind[mid];
    if (v == j) { hit = mid; break; }
    if (v < j) lo = mid + 1; else hi = mid - 1;
  }
  pos[j] = hit >= 0 ? hit - b : -1;
  if (hit < 0) atomicOr(flags, 8);
}

}  // namespace

cudaError_t launch_check_pattern(const int32_t* rowptr, const int32_t* colind, int32_t n,
                                 int32_t* flags, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int blocks = (int)((n * 32LL + 255) / 256 < 65536 ? (n * 32LL + 255) / 256 : 65536);
  check_pattern_kernel<<<blocks, 256, 0, s>>>(rowptr, colind, n, flags);
  return cudaGetLastError();
}

cudaError_t launch_plan_rows(const int32_t* rowptr, const int32_t* colind, int32_t n,
                             int32_t* m, int32_t* pos, int32_t* flags, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  plan_rows_kernel<<<(n + 255) / 256, 256, 0, s>>>(rowptr, colind, n, m, pos, flags);
  return cudaGetLastError();
}

}  // namespace submat
