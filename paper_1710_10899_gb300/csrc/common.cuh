// Internal declarations shared by the translation units of libsubmat.so.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/submat.h"

namespace submat {

constexpr int kThreads = 256;          // threads per CTA of the per-submatrix kernels
constexpr int kWarps = kThreads / 32;
constexpr int kMaxWarps = 16;          // largest CTA any helper below runs in (512 threads)
constexpr int kRedDoubles = 2 * kMaxWarps;   // shared reduction scratch of the helpers

// Device-side counters of one forward / backward call (zeroed before each call).
struct DevCounters {
  int32_t queue;              // persistent work queue head (rows handed out)
  int32_t n_fallback;         // rows appended to the fallback list
  int32_t fb_queue;           // fallback work queue head
  int32_t iters_max;
  unsigned long long iters_sum;
  unsigned long long n_notspd;
  unsigned long long resid_max_bits;   // max of non-negative doubles, compared as bits
  double flops_fp64;
  double flops_tensor;
  unsigned long long n_illcond;        // rows sent to the fallback by the condition estimate
  int32_t error;                       // a device pipeline wait timed out
};

// Arguments of the forward kernels.
struct FwdArgs {
  CUtensorMap tm_a;          // mixed tcgen05 engine: A tiles (32 x 128) of the scratch planes
  CUtensorMap tm_b;          //                       B tiles (32 x 48)
  int32_t ld;                // mixed path: leading dimension of the scratch planes
  int32_t engine;            // mixed path: 0 = tcgen05, 1 = mma.sync
  const int32_t* rowptr;
  const int32_t* colind;
  const int32_t* m;          // [n] row sizes
  const int32_t* pos;        // [n] position of the diagonal inside the row
  const int32_t* order;      // [n] rows by decreasing size
  int32_t n;
  int32_t p;
  const double* vals_in;
  double* vals_out;
  DevCounters* ctr;
  int32_t* fallback_list;    // [n]
  char* scratch;             // per-CTA working storage
  size_t scratch_stride;     // bytes per CTA
  int32_t k_max;
  double tol;
  double resid_tol;
  int32_t refine_steps;
  double kappa_max;
};

struct BwdArgs {
  const int32_t* rowptr;
  const int32_t* colind;
  const int32_t* m;
  const int32_t* pos;
  const int32_t* order;
  int32_t n;
  int32_t p;
  const double* vals;        // saved forward input
  const double* grad_out;
  double* grad_in;
  DevCounters* ctr;
  char* scratch;
  size_t scratch_stride;
};

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_plan_rows(const int32_t* rowptr, const int32_t* colind, int32_t n,
                             int32_t* m, int32_t* pos, int32_t* flags, cudaStream_t s);
cudaError_t launch_check_pattern(const int32_t* rowptr, const int32_t* colind, int32_t n,
                                 int32_t* flags, cudaStream_t s);
cudaError_t launch_fwd_mixed(const FwdArgs& a, int grid, cudaStream_t s);
cudaError_t launch_fwd_fp64(const FwdArgs& a, int grid, cudaStream_t s);
cudaError_t launch_fallback(const FwdArgs& a, int grid, cudaStream_t s);
cudaError_t launch_backward(const BwdArgs& a, int grid, cudaStream_t s);

// Dynamic shared memory of each kernel (bytes), for cudaFuncSetAttribute at plan time.
size_t smem_fwd_mixed();
size_t smem_fwd_fp64();
size_t smem_fallback();
size_t smem_backward();
// Message returned by submat_last_error() on this thread.
void set_last_error(const std::string& msg);

// Per-CTA scratch bytes: mixed path for plane leading dimension ld, others for order mp.
size_t scratch_mixed(int ld);
size_t scratch_fp64(int mp);
size_t scratch_eig(int mp);

// Padding of a submatrix order to the tile granularity of the mixed GEMM.
__host__ __device__ inline int pad_mixed(int m) { return (m + 63) / 64 * 64; }
__host__ __device__ inline int pad_fp64(int m) { return (m + 63) / 64 * 64; }

}  // namespace submat

// ------------------------------------------------------------------------------------
// Device helpers used by several kernels (header-only, internal linkage).
// ------------------------------------------------------------------------------------
#ifdef __CUDACC__
namespace submat {

__device__ __forceinline__ int nwarps() { return (int)(blockDim.x >> 5); }

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Index of key in the ascending array a[0..len), or -1.
__device__ __forceinline__ int find_sorted(const int32_t* a, int len, int32_t key) {
  int lo = 0, hi = len - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int32_t v = a[mid];
    if (v == key) return mid;
    if (v < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// Algorithm 1 for row j (value part): S[k*m + l] = A[R[k]][R[l]] in FP64 (zero where not
// stored), R staged in shared memory (R_s, m ints), and the Gershgorin bound
// max_k sum_l |S_kl| returned to every thread.  red_s: kRedDoubles doubles of shared memory.
static __device__ double gather_submatrix(const int32_t* __restrict__ rowptr,
                                   const int32_t* __restrict__ colind,
                                   const double* __restrict__ vals, int j, int m,
                                   int32_t* R_s, double* __restrict__ S, double* red_s) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int base = rowptr[j];
  for (int k = tid; k < m; k += blockDim.x) R_s[k] = colind[base + k];
  for (int e = tid; e < m * m; e += blockDim.x) S[e] = 0.0;
  __syncthreads();
  double wmax = 0.0;
  const int nw = nwarps();
  for (int k = warp; k < m; k += nw) {
    const int r = R_s[k];
    const int b = rowptr[r], e_end = rowptr[r + 1];
    double sum = 0.0;
    for (int e = b + lane; e < e_end; e += 32) {
      const int l = find_sorted(R_s, m, colind[e]);
      if (l >= 0) {
        const double v = vals[e];
        S[k * m + l] = v;
        sum += fabs(v);
      }
    }
    sum = warp_sum(sum);
    wmax = fmax(wmax, sum);
    // a NaN row sum must survive the max
    if (sum != sum) wmax = sum;
  }
  if (lane == 0) red_s[warp] = wmax;
  __syncthreads();
  double lam = red_s[0];
  for (int w = 1; w < nw; ++w) {
    const double v = red_s[w];
    lam = (v != v || lam != lam) ? (v + lam) : fmax(lam, v);
  }
  __syncthreads();
  return lam;
}

// Atomic max of a non-negative double (NaN counts as +inf).
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
  if (v != v) v = __longlong_as_double(0x7ff0000000000000ll);
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

}  // namespace submat
#endif
