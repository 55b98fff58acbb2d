// FP64 symmetric eigendecomposition of one submatrix per CTA (cyclic Jacobi, round-robin
// ordering so that m/2 disjoint rotations run in parallel), and the two kernels built on it:
//
//   fallback: rows whose mixed/FP64 Newton result failed its residual test are recomputed
//             from S = V diag(lambda) V^T as column pos of V diag(lambda^(-1/p)) V^T;
//             a non-positive (or non-finite) eigenvalue marks the row NaN (not SPD).
//   backward: the Daleckii-Krein adjoint (Higham, Functions of Matrices, Thm. 3.11):
//             for L = <g, column pos of f(S)>, f(x) = x^(-1/p), and the symmetrised
//             cotangent Gbar = (g e_pos^T + e_pos g^T)/2,
//             dL/dS = V (Gamma o (V^T Gbar V)) V^T,  Gamma_ab = divided difference of f,
//             with V^T Gbar V = (u w^T + w u^T)/2, u = V^T g, w = V^T e_pos; the result is
//             added into the gradient of every stored entry (R[k], R[l]).
//
// Rotation: the symmetric 2x2 Schur decomposition of Golub & Van Loan (Alg. 8.4.1).
#include <algorithm>
#include "common.cuh"
#include "jacobi.cuh"
#include "jacobi_df.cuh"

namespace submat {
namespace {

using namespace jac;

__device__ void gather_dense(const int32_t* rowptr, const int32_t* colind, const double* vals,
                             int j, int m, int32_t* R_s, double* S, double* red_s) {
  (void)gather_submatrix(rowptr, colind, vals, j, m, R_s, S, red_s);
}

__global__ void __launch_bounds__(kThreads) fallback_kernel(FwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* cs_s = reinterpret_cast<double*>(smem_raw);               // SUBMAT_MAX_M
  double* lam_s = cs_s + SUBMAT_MAX_M;                                // SUBMAT_MAX_M
  double* red_s = lam_s + SUBMAT_MAX_M;                               // kRedDoubles
  int32_t* pair_s = reinterpret_cast<int32_t*>(red_s + kRedDoubles);  // SUBMAT_MAX_M
  int32_t* R_s = pair_s + SUBMAT_MAX_M;                               // SUBMAT_MAX_M
  __shared__ int job_s;
  __shared__ int bad_s;
  char* scr = a.scratch + (size_t)blockIdx.x * a.scratch_stride;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) job_s = atomicAdd(&a.ctr->fb_queue, 1);
    __syncthreads();
    const int idx = job_s;
    __syncthreads();
    if (idx >= a.ctr->n_fallback) break;
    const int j = a.fallback_list[idx];
    const int m = a.m[j], pos = a.pos[j], p = a.p;
    double* A = reinterpret_cast<double*>(scr);
    double* V = A + (size_t)m * m;
    gather_dense(a.rowptr, a.colind, a.vals_in, j, m, R_s, A, red_s);
    const int sweeps = jacobi_eig(A, V, m, pair_s, cs_s, red_s);
    if (tid == 0) bad_s = sweeps < 0 ? 1 : 0;
    __syncthreads();
    for (int i = tid; i < m; i += blockDim.x) {
      const double l = A[i * m + i];
      if (!(l > 0.0) || !(l < 1e308)) bad_s = 1;
      lam_s[i] = pow(l, (double)a.sign / (double)p) * V[pos * m + i];   // f(l) = l^(sign/p)
    }
    __syncthreads();
    double* out = a.vals_out + a.rowptr[j];
    const bool bad = bad_s != 0;
    for (int k = tid; k < m; k += blockDim.x) {
      double s = 0.0;
      for (int i = 0; i < m; ++i) s = fma(V[k * m + i], lam_s[i], s);
      out[k] = bad ? __longlong_as_double(0x7ff8000000000000ll) : s;
    }
    if (tid == 0 && bad) atomicAdd(&a.ctr->n_notspd, 1ull);
    if (tid == 0) atomicAdd(&a.ctr->flops_fp64, 12.0 * (double)m * m * m + 2.0 * m * m);
    __syncthreads();
  }
}

// Shared memory of the backward kernel, laid out per row.  Rows of order up to kBwdSmallM:
// the per-row vectors sized kBwdSmallM, then the upper triangle of the submatrix packed as
// double-floats (the Jacobi's working matrix) and, when they fit after it (orders up to
// about 135), the transposed eigenvectors; the gather's row extents use the triangle's
// space before it is filled.  Larger rows: the vectors sized SUBMAT_MAX_M and the extents;
// their Jacobi runs in global memory.
constexpr size_t kBwdSmem = 230400;
constexpr int kBwdSmallM = 240;
constexpr size_t kBwdSmallVecBytes =
    (4 * kBwdSmallM + kRedDoubles) * sizeof(double) + 2 * kBwdSmallM * sizeof(int32_t);
constexpr int kPackedCap = (int)((kBwdSmem - kBwdSmallVecBytes) / sizeof(float2));
static_assert((4 * SUBMAT_MAX_M + kRedDoubles) * sizeof(double) +
                  2 * SUBMAT_MAX_M * sizeof(int32_t) + SUBMAT_MAX_M * sizeof(int2) <=
              kBwdSmem, "the large-row layout");
static_assert(kBwdSmallM * (kBwdSmallM + 1) / 2 > kPackedCap, "packed orders end below kBwdSmallM");

// The backward's per-step Jacobi work is latency-bound at 8 warps; 16 warps (128 registers
// each, the whole register file) hide twice as much.
constexpr int kBwdThreads = 512;
static_assert(kBwdThreads / 32 <= kMaxWarps, "reduction scratch");

__global__ void __launch_bounds__(kBwdThreads, 1) backward_kernel(BwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int job_s;
  __shared__ int bad_s;
  char* scr = a.scratch + (size_t)blockIdx.x * a.scratch_stride;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (;;) {
    if (tid == 0) job_s = atomicAdd(&a.ctr->queue, 1);
    __syncthreads();
    const int idx = job_s;
    __syncthreads();
    if (idx >= a.n) break;
    const int j = a.order[idx];
    if (a.gbuf && (j < a.j0 || j >= a.j1)) continue;     // another wave's row
    const int m = a.m[j], pos = a.pos[j], p = a.p;
    // this row's shared-memory layout (see kBwdSmem)
    const bool packed = m * (m + 1) / 2 <= kPackedCap;
    const int vl = packed ? kBwdSmallM : SUBMAT_MAX_M;
    double* cs_s = reinterpret_cast<double*>(smem_raw);             // vl
    double* al_s = cs_s + vl;                                         // alpha = lambda^(1/p)
    double* u_s = al_s + vl;                                          // V^T g
    double* w_s = u_s + vl;                                           // V^T e_pos
    double* red_s = w_s + vl;                                         // kRedDoubles
    int32_t* pair_s = reinterpret_cast<int32_t*>(red_s + kRedDoubles);   // vl
    int32_t* R_s = pair_s + vl;                                       // vl
    float2* P_s = reinterpret_cast<float2*>(R_s + vl);               // kPackedCap (packed)
    double* A = reinterpret_cast<double*>(scr);
    double* V = A + (size_t)m * m;
    double* W = V + (size_t)m * m;
    (void)gather_rows(a.rowptr, a.colind, a.vals, j, m, R_s, A, red_s,
                      reinterpret_cast<int2*>(P_s));                  // extents: m int2
    // the eigendecomposition in double-float (jacobi_df.cuh): with A's upper triangle packed
    // in shared memory when it fits (eigenvectors transposed after it when they fit too,
    // else in W), else in place in A, V
    int sweeps;
    if (packed) {
      for (int e = tid; e < m * m; e += blockDim.x) {
        const int r = e / m, c = e - r * m;
        if (r <= c) P_s[jdf::pidx(r, c, m)] = jdf::split(A[e]);
      }
      __syncthreads();
      const int tri = m * (m + 1) / 2;
      float2* Vt = tri + m * m <= kPackedCap ? P_s + tri : reinterpret_cast<float2*>(W);
      sweeps = jdf::jacobi_eig_df_packed(P_s, Vt, m, pair_s, reinterpret_cast<float*>(cs_s), red_s);
      for (int e = tid; e < m * m; e += blockDim.x) {
        const int i = e / m, k = e - i * m;
        V[e] = jdf::join(Vt[k * m + i]);
        if (i == k) A[e] = jdf::join(P_s[jdf::pidx(i, i, m)]);
      }
    } else {
      float2* A2 = reinterpret_cast<float2*>(A);
      float2* V2 = reinterpret_cast<float2*>(V);
      for (int e = tid; e < m * m; e += blockDim.x) A2[e] = jdf::split(A[e]);
      __syncthreads();
      sweeps = jdf::jacobi_eig_df(A2, V2, m, pair_s, reinterpret_cast<float*>(cs_s), red_s);
      for (int e = tid; e < m * m; e += blockDim.x) {
        A[e] = jdf::join(A2[e]);
        V[e] = jdf::join(V2[e]);
      }
    }
    if (tid == 0) bad_s = sweeps < 0 ? 1 : 0;
    __syncthreads();
    const double* g = a.grad_out + a.rowptr[j];
    for (int i = tid; i < m; i += blockDim.x) {
      const double l = A[i * m + i];
      if (!(l > 0.0) || !(l < 1e308)) bad_s = 1;
      al_s[i] = pow(l, 1.0 / (double)p);
      w_s[i] = V[pos * m + i];
    }
    // u = V^T g: one warp per component
    for (int i = warp; i < m; i += nwarps()) {
      double s = 0.0;
      for (int k = lane; k < m; k += 32) s = fma(V[k * m + i], g[k], s);
      s = warp_sum(s);
      if (lane == 0) u_s[i] = s;
    }
    __syncthreads();
    if (bad_s) {
      if (tid == 0) atomicAdd(&a.ctr->n_notspd, 1ull);
      if (a.gbuf) {              // no contribution, as in the atomic scatter
        double* gj = a.gbuf + (a.gofs[j] - a.gofs[a.j0]);
        for (int e = tid; e < m * m; e += blockDim.x) gj[e] = 0.0;
      }
      __syncthreads();
      continue;
    }
    // Q_ab = Gamma_ab (u_a w_b + w_a u_b) / 2, stored in A (the eigenvalues are in al_s)
    for (int e = tid; e < m * m; e += blockDim.x) {
      const int x = e / m, y = e % m;
      const double ax = al_s[x], ay = al_s[y];
      double ssum = 0.0, px = 1.0;
      for (int i = 0; i < p; ++i) {
        double py = 1.0;
        for (int t = 0; t < p - 1 - i; ++t) py *= ay;
        ssum += px * py;
        px *= ax;
      }
      // divided difference of f(l) = l^(sign/p) in the eigenvalues' p-th roots ax, ay
      const double gam = a.sign > 0 ? 1.0 / ssum : -1.0 / (ax * ay * ssum);
      A[e] = gam * 0.5 * (u_s[x] * w_s[y] + w_s[x] * u_s[y]);
    }
    __syncthreads();
    // W = V Q, then G = W V^T over A: double-float GEMMs on the FP32 units (jdf::gemm_df),
    // staged in the shared memory after the row's vectors (the packed triangle is done)
    jdf::gemm_df<false>(V, A, W, m, P_s);
    jdf::gemm_df<true>(W, V, A, m, P_s);
    if (a.gbuf) {                // deterministic: keep G_j for the gather pass
      double* gj = a.gbuf + (a.gofs[j] - a.gofs[a.j0]);
      for (int e = tid; e < m * m; e += blockDim.x) gj[e] = A[e];
      if (tid == 0) atomicAdd(&a.ctr->flops_fp64, 16.0 * (double)m * m * m);
      __syncthreads();
      continue;
    }
    // scatter-add G[k][l] into the stored entry (R[k], R[l])
    for (int k = warp; k < m; k += nwarps()) {
      const int r = R_s[k];
      for (int e = a.rowptr[r] + lane; e < a.rowptr[r + 1]; e += 32) {
        const int l = find_sorted(R_s, m, a.colind[e]);
        if (l >= 0) atomicAdd(a.grad_in + e, A[k * m + l]);
      }
    }
    if (tid == 0) atomicAdd(&a.ctr->flops_fp64, 16.0 * (double)m * m * m);
    __syncthreads();
  }
}

// tpos[e] for e = (r, j): the index of r in row j's sorted column list.
__global__ void transposed_positions_kernel(const int32_t* __restrict__ rowptr,
                                            const int32_t* __restrict__ colind, int32_t n,
                                            int32_t* __restrict__ tpos) {
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += warps)
    for (int e = rowptr[r] + lane; e < rowptr[r + 1]; e += 32) {
      const int j = colind[e];
      tpos[e] = find_sorted(colind + rowptr[j], rowptr[j + 1] - rowptr[j], r);
    }
}

// One CTA per row r (grid-stride), one warp per stored entry (r, c) of it: the rows j of
// R_c (32 at a time, lanes in ascending order) that also lie in R_r (a bisection in R_r,
// staged in shared memory) and in [j0, j1) contribute G_j(k, l), k = position of r in R_j,
// l = position of c in R_j.  Lanes combine by a fixed butterfly and the 32-row chunks in
// order, so the sum does not depend on timing.
__global__ void __launch_bounds__(256) grad_gather_kernel(
    const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
    const int32_t* __restrict__ tpos, const int32_t* __restrict__ mrow,
    const int64_t* __restrict__ gofs, const double* __restrict__ gbuf, int32_t n, int32_t j0,
    int32_t j1, double* __restrict__ grad_in) {
  __shared__ int32_t R_s[SUBMAT_MAX_M];      // R_r
  __shared__ int32_t K_s[SUBMAT_MAX_M];      // position of r in R_j for each j in R_r
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int64_t base = gofs[j0];
  for (int r = blockIdx.x; r < n; r += gridDim.x) {
    const int rb = rowptr[r], mr = rowptr[r + 1] - rb;
    for (int i = tid; i < mr; i += blockDim.x) {
      R_s[i] = colind[rb + i];
      K_s[i] = tpos[rb + i];
    }
    __syncthreads();
    for (int ci = warp; ci < mr; ci += nw) {
      const int c = R_s[ci], cb = rowptr[c], ce = rowptr[c + 1];
      double sum = 0.0;
      for (int q0 = cb; q0 < ce; q0 += 32) {
        const int q = q0 + lane;
        double v = 0.0;
        if (q < ce) {
          const int j = colind[q];
          if (j >= j0 && j < j1) {
            const int idx = find_sorted(R_s, mr, j);
            if (idx >= 0) {
              const int mj = mrow[j];
              v = gbuf[(gofs[j] - base) + (int64_t)K_s[idx] * mj + tpos[q]];
            }
          }
        }
        sum += warp_sum(v);
      }
      if (lane == 0) grad_in[rb + ci] += sum;
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_transposed_positions(const int32_t* rowptr, const int32_t* colind,
                                        int32_t n, int32_t* tpos, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>(((int64_t)n * 32 + 255) / 256, 65535);
  transposed_positions_kernel<<<blocks, 256, 0, s>>>(rowptr, colind, n, tpos);
  return cudaGetLastError();
}

cudaError_t launch_grad_gather(const int32_t* rowptr, const int32_t* colind, const int32_t* tpos,
                               const int32_t* m, const int64_t* gofs, const double* gbuf,
                               int32_t n, int32_t j0, int32_t j1, double* grad_in,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int blocks = std::min(n, 152 * 8);
  grad_gather_kernel<<<blocks, 256, 0, s>>>(rowptr, colind, tpos, m, gofs, gbuf, n, j0, j1,
                                            grad_in);
  return cudaGetLastError();
}

size_t smem_fallback() {
  return (2 * SUBMAT_MAX_M + kRedDoubles) * sizeof(double) + 2 * SUBMAT_MAX_M * sizeof(int32_t);
}
size_t smem_backward() { return kBwdSmem; }
size_t scratch_eig(int mp) { return 3 * (size_t)mp * mp * sizeof(double); }

cudaError_t launch_fallback(const FwdArgs& a, int grid, cudaStream_t s) {
  fallback_kernel<<<grid, kThreads, smem_fallback(), s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_backward(const BwdArgs& a, int grid, cudaStream_t s) {
  backward_kernel<<<grid, kBwdThreads, smem_backward(), s>>>(a);
  return cudaGetLastError();
}
cudaError_t set_attr_eig() {
  cudaError_t e = cudaFuncSetAttribute(fallback_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_fallback());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_backward());
}

}  // namespace submat
