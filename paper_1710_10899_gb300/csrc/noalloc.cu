// submat_invroot_noalloc: the FP64 forward for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a memory pool or arena owned by
// another framework, allocation-free sections of an application, or hosts that forbid device
// allocations after start-up.  This entry point needs no plan (submat_plan allocates) and
// allocates nothing: its working storage is the file-scope device array below, which every
// GPU that loads the library keeps until the process exits.  The caller passes the CSR
// pattern, the values and the output buffer, all in device memory.
//
// Per row j it runs the FP64 path's steps (Alg. 1 gather, Gershgorin scaling, coupled
// Newton iteration in FP64, FP64 column refinement) and, if the residual test fails, the
// FP64 Jacobi eigendecomposition of the same submatrix in the same CTA, then writes column
// pos_j into row j (Alg. 2).  m_j and pos_j are found on the fly from rowptr/colind.
//
// Sharing: every call uses the same array and the array keeps the last call's contents;
// the control block at its start (work counter, status) is cleared by each call.  Calls that
// overlap on the GPU (two streams, or two host threads) race on the array and must be
// serialised by the caller.
#include <mutex>
#include <string>

#include "common.cuh"
#include "refine.cuh"
#include "fp64_gemm.cuh"
#include "jacobi.cuh"

namespace submat {
namespace {

constexpr size_t kCtrlBytes = 256;
constexpr size_t kNoallocBytes = (size_t)SUBMAT_NOALLOC_SCRATCH_MIB << 20;

// Working storage: [control block | per-CTA slots].
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

struct NoallocCtrl {
  int32_t queue;       // rows handed out
  int32_t status;      // bit 1: row longer than m_max or empty, 2: no diagonal, 4: not SPD,
                       // 8: an extent or column index out of range
};

struct NoallocArgs {
  const int32_t* rowptr;
  const int32_t* colind;
  int64_t nnz;
  int32_t n;
  int32_t p;
  int32_t m_max;
  const double* vals_in;
  double* vals_out;
  NoallocCtrl* ctrl;
  char* slots;
  size_t slot_stride;
};

size_t slot_bytes(int mp) {
  return ((((size_t)mp * mp + 31) / 32) * 32 + 6 * (size_t)mp * mp) * sizeof(double);
}

// The caller's pattern is not validated by a plan here, so before anything of row j is read
// beyond rowptr[j..j+1]: its extent [base, base + m) and the extents of the rows named by its
// column indices must lie in [0, nnz], and those indices in [0, n).  The gather reads nothing
// else (other rows' column indices are only compared with R_j, never used as addresses).
// All threads call it; returns the block-wide verdict.
__device__ bool row_in_bounds(const NoallocArgs& a, int base, int m, int* flag_s) {
  if (threadIdx.x == 0) *flag_s = 0;
  __syncthreads();
  const bool ext_ok = base >= 0 && (int64_t)base + m <= a.nnz;
  if (ext_ok) {
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
      const int32_t r = a.colind[base + k];
      bool ok = r >= 0 && r < a.n;
      if (ok) {
        const int32_t b = a.rowptr[r], e = a.rowptr[r + 1];
        ok = b >= 0 && b <= e && (int64_t)e <= a.nnz;
      }
      if (!ok) *flag_s = 1;
    }
  }
  __syncthreads();
  const bool ok = ext_ok && *flag_s == 0;
  __syncthreads();
  return ok;
}

__global__ void __launch_bounds__(kThreads, 1) noalloc_fp64_kernel(NoallocArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* gsm = reinterpret_cast<double*>(smem_raw);              // 2*TK*TB
  double* y_s = gsm + 2 * fp64::TK * fp64::TB;
  double* v_s = y_s + SUBMAT_MAX_M;
  double* w_s = v_s + SUBMAT_MAX_M;
  double* red_s = w_s + SUBMAT_MAX_M;                                // kRedDoubles
  double* norm2_s = red_s + kRedDoubles;
  int32_t* R_s = reinterpret_cast<int32_t*>(norm2_s + 2);          // SUBMAT_MAX_M
  int32_t* pair_s = R_s + SUBMAT_MAX_M;                              // SUBMAT_MAX_M
  __shared__ int job_s, bad_s, oob_s;
  char* scr = a.slots + (size_t)blockIdx.x * a.slot_stride;
  const int tid = threadIdx.x;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);

  for (;;) {
    if (tid == 0) job_s = atomicAdd(&a.ctrl->queue, 1);
    __syncthreads();
    const int j = job_s;
    __syncthreads();
    if (j >= a.n) break;
    const int base = a.rowptr[j];
    const int m = a.rowptr[j + 1] - base;
    double* out = a.vals_out + base;
    if (m < 1 || m > a.m_max) {
      for (int k = tid; k < (m > 0 ? m : 0); k += blockDim.x)
        if (base + k >= 0 && (int64_t)base + k < a.nnz) out[k] = nan;
      if (tid == 0) atomicOr(&a.ctrl->status, 1);
      __syncthreads();
      continue;
    }
    if (!row_in_bounds(a, base, m, &oob_s)) {
      // the row's own extent may be the bad one: write only inside [0, nnz)
      for (int k = tid; k < m; k += blockDim.x)
        if (base + k >= 0 && (int64_t)base + k < a.nnz) out[k] = nan;
      if (tid == 0) atomicOr(&a.ctrl->status, 8);
      __syncthreads();
      continue;
    }
    const int pos = find_sorted(a.colind + base, m, j);
    if (pos < 0) {
      for (int k = tid; k < m; k += blockDim.x) out[k] = nan;
      if (tid == 0) atomicOr(&a.ctrl->status, 2);
      __syncthreads();
      continue;
    }
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
    __syncthreads();

    int xc = 0, tc = 0, mc = 0, iters = 1;
    bool bad = false;
    const double tol2 = 1e-14 * (double)m;              // ||M - I||_F <= 1e-7 sqrt(m)
    const double stag2 = 1e-8 * (double)m;
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
        fp64::gemm64(T[tc], cur, dst, mp, m, last ? fp64::EPI_M : fp64::EPI_STORE, T[tc ^ 1], 1.0,
                     (double)(p + 1), (double)p, gsm, norm2_s);   // Newton's step
        cur = dst;
        mc = free_slot;
        free_slot ^= 1;
      }
      tc ^= 1;
      const double nrm2 = *norm2_s;
      __syncthreads();
      if (!(nrm2 == nrm2) || nrm2 > 1e300) { bad = true; break; }
      if (nrm2 <= tol2 || iters >= 40) break;
      if (nrm2 <= stag2 && nrm2 > 0.25 * prev2) break;
      prev2 = nrm2;
      fp64::gemm64(X[xc], T[tc], X[xc ^ 1], mp, m, fp64::EPI_STORE, nullptr, 0.0, 0.0, 1.0, gsm,
                   norm2_s);
      xc ^= 1;
      ++iters;
    }
    double resid = 1e300;
    if (!bad) {
      fp64::gemm64(X[xc], T[tc], X[xc ^ 1], mp, m, fp64::EPI_STORE, nullptr, 0.0, 0.0, 1.0, gsm,
                   norm2_s);
      xc ^= 1;
      DenseLoad xl{X[xc], mp};
      resid = refine_column(xl, pow(lam, -1.0 / (double)p), S, m, pos, p, p == 1 ? 2 : 0,
                            y_s, v_s, w_s, red_s);
    }
    if (!bad && resid <= 1e-3) {
      for (int k = tid; k < m; k += blockDim.x) out[k] = y_s[k];
    } else {
      // FP64 eigendecomposition of the same submatrix, in this CTA's slot
      double* A = w;
      double* V = w + (size_t)m * m;
      gather_submatrix(a.rowptr, a.colind, a.vals_in, j, m, R_s, A, red_s);
      const int sweeps = jac::jacobi_eig(A, V, m, pair_s, v_s, red_s);
      if (tid == 0) bad_s = sweeps < 0 ? 1 : 0;
      __syncthreads();
      for (int i = tid; i < m; i += blockDim.x) {
        const double l = A[i * m + i];
        if (!(l > 0.0) || !(l < 1e308)) bad_s = 1;
        w_s[i] = pow(l, -1.0 / (double)p) * V[pos * m + i];
      }
      __syncthreads();
      const bool fail = bad_s != 0;
      for (int k = tid; k < m; k += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s = fma(V[k * m + i], w_s[i], s);
        out[k] = fail ? nan : s;
      }
      if (tid == 0 && fail) atomicOr(&a.ctrl->status, 4);
    }
    __syncthreads();
  }
}

size_t smem_noalloc() {
  return (2 * fp64::TK * fp64::TB + 3 * SUBMAT_MAX_M + kRedDoubles + 2) * sizeof(double) +
         2 * SUBMAT_MAX_M * sizeof(int32_t);
}

// Per-device set-up: the device address of the array and the kernel's shared-memory limit.
struct DeviceSetup {
  bool done = false;
  char* base = nullptr;
  int n_sm = 0;
};
constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

}  // namespace
}  // namespace submat

using namespace submat;

extern "C" submat_status submat_invroot_noalloc(int32_t n, int64_t nnz, const int32_t* rowptr,
                                                const int32_t* colind, int32_t p, int32_t m_max,
                                                const double* vals_in, double* vals_out,
                                                void* stream) {
  auto fail = [&](submat_status s, const std::string& msg) {
    set_last_error(msg);
    return s;
  };
  set_last_error("");
  if (n < 0 || nnz < 0 || nnz > INT32_MAX) return fail(SUBMAT_EINVAL, "bad n or nnz");
  if (p < 1) return fail(SUBMAT_EINVAL, "p must be >= 1");
  if (n == 0) return SUBMAT_OK;
  if (!rowptr || !colind || !vals_in || !vals_out) return fail(SUBMAT_EINVAL, "NULL pointer");
  if (m_max < 1 || m_max > SUBMAT_NOALLOC_MAX_M)
    return fail(SUBMAT_ETOOBIG, "m_max must be in [1, " + std::to_string(SUBMAT_NOALLOC_MAX_M) +
                                    "] for the no-allocation entry point");
  const char* a0 = reinterpret_cast<const char*>(vals_in);
  const char* b0 = reinterpret_cast<const char*>(vals_out);
  const size_t bytes = (size_t)nnz * sizeof(double);
  if (a0 < b0 + bytes && b0 < a0 + bytes) return fail(SUBMAT_EINVAL, "vals_out overlaps vals_in");
  const size_t slot = (slot_bytes(pad_fp64(m_max)) + 255) / 256 * 256;
  const size_t n_slots = (kNoallocBytes - kCtrlBytes) / slot;
  if (n_slots < 1)
    return fail(SUBMAT_ETOOBIG, "m_max too large for the " +
                                    std::to_string(SUBMAT_NOALLOC_SCRATCH_MIB) + " MiB scratch");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(SUBMAT_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(SUBMAT_ECUDA, "device index out of range");
  DeviceSetup& ds = g_setup[dev];
  {
    // once per device, with that device current: the device address of the array (its name
    // is only a host-side stand-in in host code) and the kernel's shared-memory limit
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!ds.done) {
      void* ptr = nullptr;
      cudaError_t se = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (se == cudaSuccess)
        se = cudaFuncSetAttribute(noalloc_fp64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_noalloc());
      if (se == cudaSuccess) se = cudaDeviceGetAttribute(&ds.n_sm, cudaDevAttrMultiProcessorCount, dev);
      if (se != cudaSuccess) return fail(SUBMAT_ECUDA, std::string("set-up: ") + cudaGetErrorString(se));
      ds.base = static_cast<char*>(ptr);
      ds.done = true;
    }
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  NoallocArgs a{};
  a.rowptr = rowptr;
  a.colind = colind;
  a.nnz = nnz;
  a.n = n;
  a.p = p;
  a.m_max = m_max;
  a.vals_in = vals_in;
  a.vals_out = vals_out;
  a.ctrl = reinterpret_cast<NoallocCtrl*>(ds.base);
  a.slots = ds.base + kCtrlBytes;
  a.slot_stride = slot;
  int grid = ds.n_sm;
  if ((size_t)grid > n_slots) grid = (int)n_slots;
  if (grid > n) grid = n;
  e = cudaMemsetAsync(ds.base, 0, kCtrlBytes, s);
  if (e == cudaSuccess) {
    noalloc_fp64_kernel<<<grid, kThreads, smem_noalloc(), s>>>(a);
    e = cudaGetLastError();
  }
  NoallocCtrl ctrl{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ctrl, ds.base, sizeof(ctrl), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(SUBMAT_ECUDA, cudaGetErrorString(e));
  if (ctrl.status & 8)
    return fail(SUBMAT_EINVAL, "a row extent or column index lies outside [0, nnz] / [0, n)");
  if (ctrl.status & 1) return fail(SUBMAT_ETOOBIG, "a row is empty or longer than m_max");
  if (ctrl.status & 2) return fail(SUBMAT_ENODIAG, "a row does not store its diagonal entry");
  if (ctrl.status & 4) return fail(SUBMAT_ENOTSPD, "a submatrix is not positive definite");
  return SUBMAT_OK;
}
