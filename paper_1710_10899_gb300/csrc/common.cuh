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
  int32_t run_queue[4];                // work-queue heads of the mixed path's engine launches
  double flops_alg;                    // sum over rows of k_j (p+1) 2 m_j^3 (+ 2 m_j^3 for
                                       // p = 1's final X product): executed iterations k_j,
                                       // true orders m_j, every product counted as a dense GEMM
};

// Arguments of the forward kernels.
struct FwdArgs {
  CUtensorMap tm_a;          // mixed tcgen05 engine: A tiles (16 x 128) of the scratch planes
  CUtensorMap tm_b;          //                       B tiles (16 x 96)
  int32_t ld;                // mixed path: leading dimension of the scratch planes
  int32_t engine;            // mixed path: 0 = tcgen05, 1 = mma.sync, 2 = small (shared memory)
  int32_t* queue;            // mixed path: work-queue head of this launch (its rows: order[0, n))
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
  int32_t sign;              // -1: A^(-1/p), +1: A^(1/p)
  const int32_t* stall;      // tcgen05 engine: nonzero makes every CTA first wait on a barrier
                             // that nothing signals (exercises the bounded wait; see
                             // submat_test_stall)
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
  int32_t sign;              // -1: A^(-1/p), +1: A^(1/p)
  // deterministic scatter: when gbuf is set, rows j in [j0, j1) write G_j (m_j x m_j,
  // row-major) to gbuf + gofs[j] - gofs[j0] instead of adding it into grad_in, and the
  // other rows are skipped
  double* gbuf;
  const int64_t* gofs;       // [n+1] exclusive prefix sums of m_j^2
  int32_t j0, j1;
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
// Transposed positions of the plan: for the entry e = (r, j) of row r, tpos[e] = the index
// of r in row j's column list (the position of row r in R_j).
cudaError_t launch_transposed_positions(const int32_t* rowptr, const int32_t* colind,
                                        int32_t n, int32_t* tpos, cudaStream_t s);
// grad_in[e] += sum over j in R_r and R_c, j0 <= j < j1, of G_j(r, c) (e = (r, c)), the
// G_j stored by a deterministic backward wave; each entry's sum in a fixed order.
cudaError_t launch_grad_gather(const int32_t* rowptr, const int32_t* colind, const int32_t* tpos,
                               const int32_t* m, const int64_t* gofs, const double* gbuf,
                               int32_t n, int32_t j0, int32_t j1, double* grad_in,
                               cudaStream_t s);

// Conjugate-gradient pieces (cg.cu).  cg_dot / cg_update reduce in a fixed order through
// cg_dot_scratch() doubles of part.
cudaError_t cg_spmv(const int32_t* rowptr, const int32_t* colind, const double* vals,
                    const double* x, double* y, int32_t n, cudaStream_t s);
cudaError_t cg_transpose_vals(const int32_t* rowptr, const int32_t* colind, const int32_t* tpos,
                              const double* vals, double* kt, int64_t nnz, cudaStream_t s);
cudaError_t cg_dot(const double* x, const double* y, int32_t n, double* part, double* out,
                   cudaStream_t s);
cudaError_t cg_update(double alpha, double* x, double* r, const double* p, const double* q,
                      int32_t n, double* part, double* rr, cudaStream_t s);
cudaError_t cg_dir(double beta, const double* r, double* p, int32_t n, cudaStream_t s);
size_t cg_dot_scratch();

// Global refinement pieces (refine_global.cu): C = (L R) restricted to the pattern, R given
// through R^T's values on the (symmetric) pattern; out = c1 x + c2 y.
cudaError_t refine_masked_product(const int32_t* rowptr, const int32_t* colind, int32_t n,
                                  const double* L, const double* Rt, double* C, cudaStream_t s);
cudaError_t refine_axpby(double c1, const double* x, double c2, const double* y, double* out,
                         int64_t nnz, cudaStream_t s);

// Mixed-path engines (FwdArgs::engine) and their limits.
constexpr int kEngineTc = 0, kEngineSync = 1, kEngineSmall = 2;
int mixed_ctas_per_sm(int engine);    // CTAs per SM of a mixed-path engine
int small_engine_max_m();             // largest order the small engine takes
size_t scratch_small();               // small engine: global scratch bytes per CTA

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

// |v| of a double as a float from its leading bits (integer operations only: FP64 units are
// scarce); relative error below 2^-20, NaN stays NaN, magnitudes beyond the float range give
// 0 or inf.
__device__ __forceinline__ float abs_f32_approx(double v) {
  const unsigned hi = (unsigned)__double2hiint(v) & 0x7FFFFFFFu;
  const int ex = (int)(hi >> 20);
  if (ex == 0x7FF) return __int_as_float(0x7FC00000);
  if (ex <= 1023 - 127) return 0.f;
  if (ex >= 1023 + 128) return __int_as_float(0x7F800000);
  return __int_as_float((int)(((unsigned)(ex - 1023 + 127) << 23) | ((hi & 0xFFFFFu) << 3)));
}

// Positions of U keys in the sorted a[0..len) (or -1), by a branchless bisection whose U
// chains run interleaved (each step is U independent shared-memory reads).  Keys < 0 give -1.
template <int U>
__device__ __forceinline__ void find_sorted_u(const int32_t* a, int len, const int* key,
                                              int* pos) {
  int base[U];
#pragma unroll
  for (int u = 0; u < U; ++u) base[u] = 0;
  for (int n = len; n > 1;) {
    const int half = n >> 1;
#pragma unroll
    for (int u = 0; u < U; ++u) base[u] = (a[base[u] + half] <= key[u]) ? base[u] + half : base[u];
    n -= half;
  }
#pragma unroll
  for (int u = 0; u < U; ++u) pos[u] = (key[u] >= 0 && len > 0 && a[base[u]] == key[u]) ? base[u] : -1;
}

// Algorithm 1 for row j (value part): S[k*m + l] = A[R[k]][R[l]] in FP64 (zero where not
// stored), R staged in shared memory (R_s, m ints), and the Gershgorin bound
// max_k sum_l |S_kl| returned to every thread (summed in FP32 and enlarged by 1e-4, which
// covers the rounding; any bound above the largest eigenvalue serves).  The extents of all
// m pattern rows are loaded first, in parallel; then each warp takes one row at a time, with
// the first 32 U entries of its next row already requested, and locates a row's entries in
// R by interleaved bisections.  red_s: kRedDoubles doubles of shared memory; ext_s: m int2
// of shared memory for the rows' extents [rowptr[R_k], rowptr[R_k + 1]).
static __device__ double gather_rows(const int32_t* __restrict__ rowptr,
                                     const int32_t* __restrict__ colind,
                                     const double* __restrict__ vals, int j, int m,
                                     int32_t* R_s, double* __restrict__ S, double* red_s,
                                     int2* ext_s) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int base = rowptr[j];
  for (int k = tid; k < m; k += blockDim.x) {
    const int r = colind[base + k];
    R_s[k] = r;
    ext_s[k] = make_int2(rowptr[r], rowptr[r + 1]);
  }
  for (int e = tid; e < m * m; e += blockDim.x) S[e] = 0.0;
  __syncthreads();
  float wmax = 0.f;
  const int nw = nwarps();
  constexpr int U = 8;
  int ncol[U];
  double nv[U];
  auto load_chunk = [&](int e0, int e_end, int* col, double* v) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * 32 + lane;
      col[u] = e < e_end ? colind[e] : -1;
      v[u] = e < e_end ? vals[e] : 0.0;
    }
  };
  if (warp < m) load_chunk(ext_s[warp].x, ext_s[warp].y, ncol, nv);
  for (int k = warp; k < m; k += nw) {
    const int b = ext_s[k].x, e_end = ext_s[k].y;
    int col[U];
    double v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      col[u] = ncol[u];
      v[u] = nv[u];
    }
    if (k + nw < m) load_chunk(ext_s[k + nw].x, ext_s[k + nw].y, ncol, nv);   // next row
    float sum = 0.f;
    for (int e0 = b;;) {
      int l[U];
      find_sorted_u<U>(R_s, m, col, l);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (l[u] >= 0) {
          S[k * m + l[u]] = v[u];
          sum += abs_f32_approx(v[u]);
        }
      }
      e0 += 32 * U;
      if (e0 >= e_end) break;
      load_chunk(e0, e_end, col, v);                 // rows longer than 32 U entries
    }
    sum = warp_sum_f(sum);
    // a NaN row sum must survive the max
    wmax = (sum != sum || wmax != wmax) ? sum + wmax : fmaxf(wmax, sum);
  }
  if (lane == 0) red_s[warp] = (double)wmax;
  __syncthreads();
  double lam = red_s[0];
  for (int w = 1; w < nw; ++w) {
    const double v = red_s[w];
    lam = (v != v || lam != lam) ? (v + lam) : fmax(lam, v);
  }
  __syncthreads();
  return lam * (1.0 + 1e-4);
}

// gather_rows with the extents in a static shared array of SUBMAT_MAX_M entries.
static __device__ double gather_submatrix(const int32_t* __restrict__ rowptr,
                                          const int32_t* __restrict__ colind,
                                          const double* __restrict__ vals, int j, int m,
                                          int32_t* R_s, double* __restrict__ S, double* red_s) {
  __shared__ int2 ext_s[SUBMAT_MAX_M];
  return gather_rows(rowptr, colind, vals, j, m, R_s, S, red_s, ext_s);
}

// Atomic max of a non-negative double (NaN counts as +inf).
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
  if (v != v) v = __longlong_as_double(0x7ff0000000000000ll);
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

}  // namespace submat
#endif
