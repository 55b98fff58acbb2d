// C ABI of libsubmat.so (declared in include/submat.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "common.cuh"
#include "engine_table.h"

namespace submat {
cudaError_t set_attr_mixed();
cudaError_t set_attr_fp64();
cudaError_t set_attr_eig();
}  // namespace submat

using namespace submat;

namespace {

thread_local std::string g_last_error;

submat_status fail(submat_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

#define CUDA_TRY(expr)                                                                  \
  do {                                                                                  \
    cudaError_t err_ = (expr);                                                          \
    if (err_ != cudaSuccess) {                                                          \
      return fail(err_ == cudaErrorMemoryAllocation ? SUBMAT_ENOMEM : SUBMAT_ECUDA,     \
                  std::string(#expr) + ": " + cudaGetErrorString(err_));                \
    }                                                                                   \
  } while (0)

// One persistent launch of the mixed forward: an engine over order[begin, begin + count).
struct EngineRun {
  int engine = 0;
  int32_t begin = 0, count = 0;
  int grid = 0;
};

struct GraphEntry {
  const double* in = nullptr;
  double* out = nullptr;
  cudaGraphExec_t exec = nullptr;
};

// Makes the plan's device current for one call and restores the caller's on every return.
struct DeviceScope {
  int prev = 0;
  bool switched = false;
  cudaError_t enter(int dev) {
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess || prev == dev) return e;
    e = cudaSetDevice(dev);
    switched = e == cudaSuccess;
    return e;
  }
  ~DeviceScope() {
    if (switched) cudaSetDevice(prev);
  }
};

// No C++ exception leaves the C ABI: a failed host allocation becomes SUBMAT_ENOMEM.
#define SUBMAT_NOTHROW(call)                                       \
  try {                                                            \
    return call;                                                   \
  } catch (const std::bad_alloc&) {                                \
    return fail(SUBMAT_ENOMEM, "host allocation failed");          \
  } catch (const std::exception& e_) {                             \
    return fail(SUBMAT_EINVAL, std::string("host: ") + e_.what()); \
  } catch (...) {                                                  \
    return fail(SUBMAT_EINVAL, "host: unknown exception");         \
  }

}  // namespace

namespace submat {
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace submat

struct submat_plan_s {
  int device = 0;
  int n_sm = 0;
  int32_t n = 0;
  int32_t row_begin = 0, row_end = 0;   // rows this plan computes (its shard; all by default)
  int32_t n_jobs = 0;                   // row_end - row_begin
  int64_t nnz = 0;
  int32_t p = 1;
  submat_opts opts{};
  int32_t* d_rowptr = nullptr;
  int32_t* d_colind = nullptr;
  int32_t* d_m = nullptr;
  int32_t* d_pos = nullptr;
  int32_t* d_order = nullptr;
  int32_t* d_fallback = nullptr;
  int32_t* d_flags = nullptr;
  int32_t* d_stall = nullptr;         // submat_test_stall's flag, read by the tcgen05 forward
  DevCounters* d_ctr = nullptr;       // forward counters
  DevCounters* d_ctr_bwd = nullptr;   // backward counters
  char* d_scratch = nullptr;
  size_t stride = 0;
  int grid = 0;
  double* d_saved = nullptr;
  bool have_fwd = false;
  int32_t m_max = 0;
  int32_t ld = 0;                     // mixed path: leading dimension of the scratch planes
  double sum_m3 = 0.0;
  CUtensorMap tm_a{}, tm_b{};         // mixed path, tcgen05 engine
  cudaStream_t last_stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  double* d_host_in = nullptr;     // device staging of submat_invroot_host
  double* d_host_out = nullptr;
  // deterministic backward (allocated by the first one): row sizes, transposed positions,
  // offsets of the per-row gradients G_j, the waves' buffer and the waves' row ranges
  std::vector<int32_t> h_m;
  int32_t* d_tpos = nullptr;
  int64_t* d_gofs = nullptr;
  double* d_gbuf = nullptr;
  std::vector<std::pair<int32_t, int32_t>> waves;
  double* d_cg = nullptr;          // submat_pcg work vectors (allocated by the first call)
  double* d_ref = nullptr;         // submat_refine work arrays (allocated by the first call)
  std::vector<GraphEntry> graphs;
  std::vector<EngineRun> runs;        // mixed path: engine launches by size bucket
};

namespace {

void release(submat_plan_t P) {
  if (!P) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(P->device);
  for (auto& g : P->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
  for (auto& e : P->ev)
    if (e) cudaEventDestroy(e);
  cudaFree(P->d_host_in);
  cudaFree(P->d_host_out);
  cudaFree(P->d_tpos);
  cudaFree(P->d_gofs);
  cudaFree(P->d_gbuf);
  cudaFree(P->d_cg);
  cudaFree(P->d_ref);
  cudaFree(P->d_rowptr);
  cudaFree(P->d_colind);
  cudaFree(P->d_m);
  cudaFree(P->d_pos);
  cudaFree(P->d_order);
  cudaFree(P->d_fallback);
  cudaFree(P->d_flags);
  cudaFree(P->d_stall);
  cudaFree(P->d_ctr);
  cudaFree(P->d_ctr_bwd);
  cudaFree(P->d_scratch);
  cudaFree(P->d_saved);
  cudaSetDevice(prev);
  delete P;
}

// The plan's transposed map (computed once): tpos[e] for e = (r, j) is the position of r in
// row j's column list.
cudaError_t ensure_tpos(submat_plan_t P, cudaStream_t s) {
  if (P->d_tpos || P->nnz == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(&P->d_tpos, (size_t)P->nnz * sizeof(int32_t));
  if (e != cudaSuccess) return e;
  return launch_transposed_positions(P->d_rowptr, P->d_colind, P->n, P->d_tpos, s);
}

// Queue the forward of plan P on stream s.
submat_status enqueue_forward(submat_plan_t P, const double* in, double* out, cudaStream_t s,
                              bool capturing) {
  const unsigned evf = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  FwdArgs a{};
  a.rowptr = P->d_rowptr;
  a.colind = P->d_colind;
  a.m = P->d_m;
  a.pos = P->d_pos;
  a.order = P->d_order;
  a.n = P->n_jobs;                      // rows of this plan (d_order holds them)
  a.p = P->p;
  a.vals_in = in;
  a.vals_out = out;
  a.ctr = P->d_ctr;
  a.fallback_list = P->d_fallback;
  a.scratch = P->d_scratch;
  a.scratch_stride = P->stride;
  a.k_max = P->opts.k_max;
  a.tol = P->opts.tol;
  a.resid_tol = P->opts.resid_tol;
  a.refine_steps = P->opts.refine_steps;
  a.kappa_max = P->opts.kappa_max;
  a.sign = P->opts.root_sign;
  a.ld = P->ld;
  a.engine = kEngineTc;
  a.queue = &P->d_ctr->queue;
  a.tm_a = P->tm_a;
  a.tm_b = P->tm_b;
  a.stall = P->d_stall;
  CUDA_TRY(cudaMemcpyAsync(P->d_saved, in, (size_t)P->nnz * sizeof(double),
                           cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemsetAsync(P->d_ctr, 0, sizeof(DevCounters), s));
  CUDA_TRY(cudaEventRecordWithFlags(P->ev[0], s, evf));
  if (P->opts.precision == SUBMAT_PREC_FP64) {
    CUDA_TRY(launch_fwd_fp64(a, P->grid, s));
  } else {
    for (size_t r = 0; r < P->runs.size(); ++r) {    // longest rows first, one engine per run
      const EngineRun& run = P->runs[r];
      FwdArgs b = a;
      b.engine = run.engine;
      b.order = P->d_order + run.begin;
      b.n = run.count;
      b.queue = &P->d_ctr->run_queue[r];
      b.scratch_stride = run.engine == kEngineSmall ? scratch_small() : P->stride;
      CUDA_TRY(launch_fwd_mixed(b, run.grid, s));
    }
  }
  CUDA_TRY(cudaEventRecordWithFlags(P->ev[1], s, evf));
  CUDA_TRY(launch_fallback(a, P->grid, s));
  CUDA_TRY(cudaEventRecordWithFlags(P->ev[2], s, evf));
  return SUBMAT_OK;
}

}  // namespace

extern "C" {

submat_status submat_shard_rows(int32_t n, const int32_t* rowptr, int32_t count, int32_t rank,
                               int32_t* row_begin, int32_t* row_end) {
  g_last_error.clear();
  if (!rowptr || !row_begin || !row_end || n < 0) return fail(SUBMAT_EINVAL, "bad argument");
  if (count < 1 || rank < 0 || rank >= count)
    return fail(SUBMAT_EINVAL, "shard rank must lie in [0, count)");
  // cumulative cost of the rows (m_j^3) and the first row reaching each quantile
  double total = 0.0;
  for (int32_t j = 0; j < n; ++j) {
    const double m = (double)(rowptr[j + 1] - rowptr[j]);
    total += m * m * m;
  }
  auto start = [&](int32_t k) -> int32_t {
    if (k <= 0) return 0;
    if (k >= count) return n;
    const double target = total * (double)k / (double)count;
    double acc = 0.0;
    for (int32_t j = 0; j < n; ++j) {
      if (acc >= target) return j;
      const double m = (double)(rowptr[j + 1] - rowptr[j]);
      acc += m * m * m;
    }
    return n;
  };
  *row_begin = start(rank);
  *row_end = start(rank + 1);
  return SUBMAT_OK;
}

void submat_default_opts(submat_opts* o) {
  if (!o) return;
  o->precision = SUBMAT_PREC_MIXED_F16;
  o->k_max = 40;
  o->tol = 0.0;
  o->resid_tol = 1e-3;
  o->refine_steps = -1;
  o->use_graph = 1;
  o->kappa_max = 100.0;
  o->root_sign = -1;
  o->grad_deterministic = 0;
  o->grad_wave_mib = 0;
  o->shard_count = 0;
  o->shard_rank = 0;
  o->small_max_m = kTunedSmallMaxM;
  o->sync_max_m = kTunedSyncMaxM;
}

const char* submat_status_string(submat_status s) {
  switch (s) {
    case SUBMAT_OK: return "ok";
    case SUBMAT_EINVAL: return "invalid argument";
    case SUBMAT_ENODIAG: return "diagonal entry not stored";
    case SUBMAT_ENOTSYM: return "pattern not symmetric";
    case SUBMAT_ETOOBIG: return "row longer than SUBMAT_MAX_M";
    case SUBMAT_ENOMEM: return "out of memory";
    case SUBMAT_ECUDA: return "CUDA error";
    case SUBMAT_ENOTSPD: return "submatrix not positive definite";
    case SUBMAT_ENOFWD: return "no forward on this plan";
    case SUBMAT_ETIMEOUT: return "device pipeline wait timed out";
  }
  return "unknown status";
}

const char* submat_last_error(void) { return g_last_error.c_str(); }

static submat_status plan_impl(const submat_csr* csr, int32_t p, const submat_opts* opts,
                               submat_plan_t* out) {
  g_last_error.clear();
  if (!out) return fail(SUBMAT_EINVAL, "out is NULL");
  *out = nullptr;
  if (!csr) return fail(SUBMAT_EINVAL, "csr is NULL");
  if (p < 1) return fail(SUBMAT_EINVAL, "p must be >= 1");
  if (csr->n < 0 || csr->nnz < 0) return fail(SUBMAT_EINVAL, "negative size");
  if (csr->nnz > INT32_MAX) return fail(SUBMAT_EINVAL, "nnz exceeds int32 indexing");
  if (csr->n > csr->nnz)       // every row stores at least its diagonal entry
    return fail(SUBMAT_ENODIAG, "fewer stored entries than rows: a row lacks its diagonal");
  if (!csr->rowptr || (csr->nnz > 0 && !csr->colind))
    return fail(SUBMAT_EINVAL, "NULL rowptr/colind");

  submat_opts o;
  submat_default_opts(&o);
  if (opts) o = *opts;
  if (o.precision != SUBMAT_PREC_FP64 && o.precision != SUBMAT_PREC_MIXED_F16 &&
      o.precision != SUBMAT_PREC_MIXED_F16_SYNC)
    return fail(SUBMAT_EINVAL, "unknown precision");
  if (o.k_max < 1) o.k_max = 40;
  if (!(o.tol > 0.0)) o.tol = (o.precision == SUBMAT_PREC_FP64) ? 1e-7 : 1e-4;
  if (!(o.resid_tol > 0.0)) o.resid_tol = 1e-3;
  if (o.refine_steps < 0) o.refine_steps = (p == 1) ? 2 : 0;
  if (!(o.kappa_max > 0.0)) o.kappa_max = 100.0;
  if (o.root_sign != -1 && o.root_sign != 1) return fail(SUBMAT_EINVAL, "root_sign must be -1 or +1");
  if (o.grad_deterministic != 0 && o.grad_deterministic != 1)
    return fail(SUBMAT_EINVAL, "grad_deterministic must be 0 or 1");
  if (o.grad_wave_mib <= 0) o.grad_wave_mib = SUBMAT_GRAD_WAVE_MIB;
  if (o.shard_count <= 1) {
    o.shard_count = 1;
    if (o.shard_rank != 0) return fail(SUBMAT_EINVAL, "shard_rank must be 0 without shards");
  } else if (o.shard_rank < 0 || o.shard_rank >= o.shard_count) {
    return fail(SUBMAT_EINVAL, "shard_rank must lie in [0, shard_count)");
  }
  if (o.precision != SUBMAT_PREC_FP64 && p > SUBMAT_MIXED_MAX_P)
    return fail(SUBMAT_EINVAL, "the mixed-precision modes take p <= SUBMAT_MIXED_MAX_P (" +
                                   std::to_string(SUBMAT_MIXED_MAX_P) + "); use SUBMAT_PREC_FP64");
  if (o.small_max_m < 0) o.small_max_m = kTunedSmallMaxM;
  if (o.sync_max_m < 0) o.sync_max_m = kTunedSyncMaxM;
  if (o.small_max_m > small_engine_max_m())
    return fail(SUBMAT_EINVAL, "small_max_m exceeds SUBMAT_SMALL_MAX_M");

  const int32_t n = csr->n;
  const int64_t nnz = csr->nnz;
  const size_t rp_bytes = ((size_t)n + 1) * sizeof(int32_t);
  std::vector<int32_t> h_rowptr((size_t)n + 1);
  if (csr->on_device) {
    CUDA_TRY(cudaMemcpy(h_rowptr.data(), csr->rowptr, rp_bytes, cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(h_rowptr.data(), csr->rowptr, rp_bytes);
  }
  if (h_rowptr[0] != 0 || h_rowptr[n] != nnz)
    return fail(SUBMAT_EINVAL, "rowptr[0] must be 0 and rowptr[n] must be nnz");
  int32_t m_max = 0;
  double sum_m3 = 0.0;
  for (int32_t j = 0; j < n; ++j) {
    const int32_t len = h_rowptr[j + 1] - h_rowptr[j];
    if (len < 0) return fail(SUBMAT_EINVAL, "rowptr not nondecreasing");
    if (len == 0) return fail(SUBMAT_ENODIAG, "empty row " + std::to_string(j));
    if (len > SUBMAT_MAX_M)
      return fail(SUBMAT_ETOOBIG, "row " + std::to_string(j) + " has " + std::to_string(len) +
                                      " entries (max " + std::to_string(SUBMAT_MAX_M) + ")");
    m_max = std::max(m_max, len);
    sum_m3 += (double)len * len * len;
  }

  submat_plan_t P = new (std::nothrow) submat_plan_s();
  if (!P) return fail(SUBMAT_ENOMEM, "host allocation");
  // released on every early return (and on a host exception); handed out at the end
  std::unique_ptr<submat_plan_s, void (*)(submat_plan_t)> owner(P, release);
  P->n = n;
  P->nnz = nnz;
  P->p = p;
  P->opts = o;
  P->m_max = m_max;
  {
    submat_status sst = submat_shard_rows(n, h_rowptr.data(), o.shard_count, o.shard_rank,
                                          &P->row_begin, &P->row_end);
    if (sst != SUBMAT_OK) return sst;
  }
  P->n_jobs = P->row_end - P->row_begin;
  sum_m3 = 0.0;
  for (int32_t j = P->row_begin; j < P->row_end; ++j) {
    const double len = (double)(h_rowptr[j + 1] - h_rowptr[j]);
    sum_m3 += len * len * len;
  }
  P->sum_m3 = sum_m3;
  auto bail = [](submat_status st) { return st; };   // the owner releases P
#define PLAN_TRY(expr)                                                              \
  do {                                                                              \
    cudaError_t err_ = (expr);                                                      \
    if (err_ != cudaSuccess) {                                                      \
      fail(err_ == cudaErrorMemoryAllocation ? SUBMAT_ENOMEM : SUBMAT_ECUDA,        \
           std::string(#expr) + ": " + cudaGetErrorString(err_));                   \
      return bail(err_ == cudaErrorMemoryAllocation ? SUBMAT_ENOMEM : SUBMAT_ECUDA); \
    }                                                                               \
  } while (0)

  PLAN_TRY(cudaGetDevice(&P->device));
  PLAN_TRY(cudaDeviceGetAttribute(&P->n_sm, cudaDevAttrMultiProcessorCount, P->device));
  PLAN_TRY(set_attr_mixed());
  PLAN_TRY(set_attr_fp64());
  PLAN_TRY(set_attr_eig());
  const size_t nb = (size_t)(n > 0 ? n : 1);
  PLAN_TRY(cudaMalloc(&P->d_rowptr, rp_bytes));
  PLAN_TRY(cudaMalloc(&P->d_colind, (nnz > 0 ? nnz : 1) * sizeof(int32_t)));
  PLAN_TRY(cudaMalloc(&P->d_m, nb * sizeof(int32_t)));
  PLAN_TRY(cudaMalloc(&P->d_pos, nb * sizeof(int32_t)));
  PLAN_TRY(cudaMalloc(&P->d_order, nb * sizeof(int32_t)));
  PLAN_TRY(cudaMalloc(&P->d_fallback, nb * sizeof(int32_t)));
  PLAN_TRY(cudaMalloc(&P->d_flags, sizeof(int32_t)));
  PLAN_TRY(cudaMalloc(&P->d_stall, sizeof(int32_t)));
  PLAN_TRY(cudaMemset(P->d_stall, 0, sizeof(int32_t)));
  PLAN_TRY(cudaMalloc(&P->d_ctr, sizeof(DevCounters)));
  PLAN_TRY(cudaMalloc(&P->d_ctr_bwd, sizeof(DevCounters)));
  PLAN_TRY(cudaMemset(P->d_ctr, 0, sizeof(DevCounters)));
  PLAN_TRY(cudaMemset(P->d_ctr_bwd, 0, sizeof(DevCounters)));
  PLAN_TRY(cudaMemcpy(P->d_rowptr, h_rowptr.data(), rp_bytes, cudaMemcpyHostToDevice));
  if (nnz > 0)
    PLAN_TRY(cudaMemcpy(P->d_colind, csr->colind, nnz * sizeof(int32_t),
                        csr->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
  PLAN_TRY(cudaMemset(P->d_flags, 0, sizeof(int32_t)));
  PLAN_TRY(launch_check_pattern(P->d_rowptr, P->d_colind, n, P->d_flags, 0));
  int32_t flags = 0;
  PLAN_TRY(cudaMemcpy(&flags, P->d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (flags & 1) { fail(SUBMAT_EINVAL, "column index out of range"); return bail(SUBMAT_EINVAL); }
  if (flags & 2) {
    fail(SUBMAT_EINVAL, "column indices not strictly ascending within a row");
    return bail(SUBMAT_EINVAL);
  }
  if (flags & 4) { fail(SUBMAT_ENOTSYM, "pattern not symmetric"); return bail(SUBMAT_ENOTSYM); }
  PLAN_TRY(launch_plan_rows(P->d_rowptr, P->d_colind, n, P->d_m, P->d_pos, P->d_flags, 0));
  PLAN_TRY(cudaMemcpy(&flags, P->d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (flags & 8) {
    fail(SUBMAT_ENODIAG, "a row does not store its diagonal entry");
    return bail(SUBMAT_ENODIAG);
  }
  // The plan's rows (its shard) by decreasing size (longest first), ties by index: counting
  // sort on m.
  std::vector<int32_t> h_m(nb), order(nb);
  if (n > 0) PLAN_TRY(cudaMemcpy(h_m.data(), P->d_m, n * sizeof(int32_t), cudaMemcpyDeviceToHost));
  {
    std::vector<int64_t> start(SUBMAT_MAX_M + 2, 0);
    for (int32_t j = P->row_begin; j < P->row_end; ++j) start[SUBMAT_MAX_M - h_m[j]]++;
    int64_t acc = 0;
    for (auto& v : start) { const int64_t c = v; v = acc; acc += c; }
    for (int32_t j = P->row_begin; j < P->row_end; ++j) order[start[SUBMAT_MAX_M - h_m[j]]++] = j;
  }
  if (P->n_jobs > 0)
    PLAN_TRY(cudaMemcpy(P->d_order, order.data(), P->n_jobs * sizeof(int32_t),
                        cudaMemcpyHostToDevice));
  P->h_m.assign(h_m.begin(), h_m.begin() + n);

  const int mp = std::max(pad_mixed(m_max), pad_fp64(m_max));
  const bool mixed = o.precision != SUBMAT_PREC_FP64;
  // mixed path: planes of LD x LD halves (LD >= one 128-row tile); 34 planes per CTA hold
  // the six sliced matrices, S_j and, for the fallback, 3 m^2 doubles
  P->ld = std::max(128, mp);
  size_t stride = mixed ? scratch_mixed(P->ld) : std::max(scratch_eig(mp), scratch_fp64(mp));
  stride = (stride + 1023) / 1024 * 1024;
  P->stride = stride;
  P->grid = std::max(1, std::min(P->n_sm, P->n_jobs));
  // the mixed path's engine runs: the plan's rows are ordered by decreasing m, so each size
  // bucket is one contiguous run of the order (tcgen05, then mma.sync, then small)
  size_t scratch_bytes = stride * (size_t)P->grid;
  if (mixed) {
    int32_t cnt[3] = {0, 0, 0};
    for (int32_t j = P->row_begin; j < P->row_end; ++j) {
      const int32_t mj = h_m[j];
      int e = kEngineTc;
      if (o.precision == SUBMAT_PREC_MIXED_F16_SYNC) e = kEngineSync;
      else if (mj <= o.small_max_m) e = kEngineSmall;
      else if (mj <= o.sync_max_m) e = kEngineSync;
      cnt[e]++;
    }
    int32_t begin = 0;
    for (int e : {kEngineTc, kEngineSync, kEngineSmall}) {
      if (cnt[e] == 0) continue;
      EngineRun run;
      run.engine = e;
      run.begin = begin;
      run.count = cnt[e];
      run.grid = std::max(1, std::min(P->n_sm * mixed_ctas_per_sm(e), cnt[e]));
      if (e == kEngineSmall)
        scratch_bytes = std::max(scratch_bytes, scratch_small() * (size_t)run.grid);
      P->runs.push_back(run);
      begin += cnt[e];
    }
  }
  PLAN_TRY(cudaMalloc(&P->d_scratch, scratch_bytes));
  if (mixed && o.precision == SUBMAT_PREC_MIXED_F16) {
    // TMA descriptors over all CTAs' planes: dims (LD cols, LD rows, planes), 32-byte swizzle
    PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t ge = cudaGetDriverEntryPoint("cuTensorMapEncodeTiled",
                                             reinterpret_cast<void**>(&encode),
                                             cudaEnableDefault, &q);
    if (ge != cudaSuccess || q != cudaDriverEntryPointSuccess || !encode) {
      fail(SUBMAT_ECUDA, "cuTensorMapEncodeTiled not available");
      return bail(SUBMAT_ECUDA);
    }
    const uint64_t planes = (uint64_t)(stride / ((size_t)P->ld * P->ld * 2)) * P->grid;
    cuuint64_t dims[3] = {(cuuint64_t)P->ld, (cuuint64_t)P->ld, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)P->ld * 2, (cuuint64_t)P->ld * P->ld * 2};
    cuuint32_t elem[3] = {1, 1, 1};
    cuuint32_t box_a[3] = {16, 128, 1}, box_b[3] = {16, 96, 1};   // 16-wide k-slices
    CUresult r1 = encode(&P->tm_a, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, P->d_scratch, dims, strides,
                         box_a, elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    CUresult r2 = encode(&P->tm_b, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, P->d_scratch, dims, strides,
                         box_b, elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS) {
      fail(SUBMAT_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r1) + ", " +
                             std::to_string((int)r2) + ")");
      return bail(SUBMAT_ECUDA);
    }
  }
  PLAN_TRY(cudaMalloc(&P->d_saved, (nnz > 0 ? nnz : 1) * sizeof(double)));
  PLAN_TRY(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking));
  for (auto& e : P->ev) PLAN_TRY(cudaEventCreate(&e));
  PLAN_TRY(cudaDeviceSynchronize());
#undef PLAN_TRY
  *out = owner.release();
  return SUBMAT_OK;
}

static submat_status invroot_impl(submat_plan_t P, const double* in, double* out, void* stream,
                                  int32_t sync) {
  g_last_error.clear();
  if (!P) return fail(SUBMAT_EINVAL, "plan is NULL");
  if (P->n == 0) return SUBMAT_OK;
  if (!in || !out) return fail(SUBMAT_EINVAL, "NULL value array");
  const char* a0 = reinterpret_cast<const char*>(in);
  const char* b0 = reinterpret_cast<const char*>(out);
  const size_t bytes = (size_t)P->nnz * sizeof(double);
  if (a0 < b0 + bytes && b0 < a0 + bytes) return fail(SUBMAT_EINVAL, "vals_out overlaps vals_in");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  DeviceScope dev;
  CUDA_TRY(dev.enter(P->device));
  submat_status st = SUBMAT_OK;
  if (P->opts.use_graph) {
    GraphEntry* ge = nullptr;
    for (auto& g : P->graphs)
      if (g.in == in && g.out == out) ge = &g;
    if (!ge) {
      if (P->graphs.size() >= 8) {
        cudaGraphExecDestroy(P->graphs.front().exec);
        P->graphs.erase(P->graphs.begin());
      }
      cudaGraph_t graph = nullptr;
      CUDA_TRY(cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal));
      st = enqueue_forward(P, in, out, P->cap_stream, true);
      cudaError_t ce = cudaStreamEndCapture(P->cap_stream, &graph);
      if (st != SUBMAT_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      CUDA_TRY(ce);
      GraphEntry g;
      g.in = in;
      g.out = out;
      cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
      cudaGraphDestroy(graph);
      CUDA_TRY(ie);
      P->graphs.push_back(g);
      ge = &P->graphs.back();
    }
    CUDA_TRY(cudaGraphLaunch(ge->exec, s));
  } else {
    st = enqueue_forward(P, in, out, s, false);
    if (st != SUBMAT_OK) return st;
  }
  P->last_stream = s;
  P->have_fwd = true;
  if (sync) {
    CUDA_TRY(cudaStreamSynchronize(s));
    DevCounters c;
    CUDA_TRY(cudaMemcpy(&c, P->d_ctr, sizeof(c), cudaMemcpyDeviceToHost));
    if (c.error) return fail(SUBMAT_ETIMEOUT, "a device pipeline wait timed out");
    if (c.n_notspd > 0)
      return fail(SUBMAT_ENOTSPD, std::to_string(c.n_notspd) + " submatrices not SPD");
  }
  return SUBMAT_OK;
}

static submat_status invroot_host_impl(submat_plan_t P, const double* in, double* out,
                                       void* stream) {
  g_last_error.clear();
  if (!P) return fail(SUBMAT_EINVAL, "plan is NULL");
  if (P->n == 0) return SUBMAT_OK;
  if (!in || !out) return fail(SUBMAT_EINVAL, "NULL value array");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)P->nnz * sizeof(double);
  DeviceScope dev;
  CUDA_TRY(dev.enter(P->device));
  if (!P->d_host_in) {
    CUDA_TRY(cudaMalloc(&P->d_host_in, bytes));
    CUDA_TRY(cudaMalloc(&P->d_host_out, bytes));
  }
  CUDA_TRY(cudaMemcpyAsync(P->d_host_in, in, bytes, cudaMemcpyHostToDevice, s));
  submat_status st = invroot_impl(P, P->d_host_in, P->d_host_out, stream, 0);
  if (st != SUBMAT_OK) return st;
  CUDA_TRY(cudaMemcpyAsync(out, P->d_host_out, bytes, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  DevCounters c;
  CUDA_TRY(cudaMemcpy(&c, P->d_ctr, sizeof(c), cudaMemcpyDeviceToHost));
  if (c.error) return fail(SUBMAT_ETIMEOUT, "a device pipeline wait timed out");
  if (c.n_notspd > 0)
    return fail(SUBMAT_ENOTSPD, std::to_string(c.n_notspd) + " submatrices not SPD");
  return SUBMAT_OK;
}

static submat_status backward_impl(submat_plan_t P, const double* grad_out, double* grad_in,
                                   void* stream) {
  g_last_error.clear();
  if (!P) return fail(SUBMAT_EINVAL, "plan is NULL");
  if (!P->have_fwd) return fail(SUBMAT_ENOFWD, "backward before forward");
  if (P->n == 0) return SUBMAT_OK;
  if (!grad_out || !grad_in) return fail(SUBMAT_EINVAL, "NULL gradient array");
  {
    const char* a0 = reinterpret_cast<const char*>(grad_out);
    const char* b0 = reinterpret_cast<const char*>(grad_in);
    const size_t bytes = (size_t)P->nnz * sizeof(double);
    if (a0 < b0 + bytes && b0 < a0 + bytes)
      return fail(SUBMAT_EINVAL, "grad_in overlaps grad_out");
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  DeviceScope dev;
  CUDA_TRY(dev.enter(P->device));
  BwdArgs a{};
  a.rowptr = P->d_rowptr;
  a.colind = P->d_colind;
  a.m = P->d_m;
  a.pos = P->d_pos;
  a.order = P->d_order;
  a.n = P->n_jobs;                      // rows of this plan (d_order holds them)
  a.p = P->p;
  a.vals = P->d_saved;
  a.grad_out = grad_out;
  a.grad_in = grad_in;
  a.ctr = P->d_ctr_bwd;
  a.scratch = P->d_scratch;
  a.scratch_stride = P->stride;
  a.sign = P->opts.root_sign;
  CUDA_TRY(cudaMemsetAsync(grad_in, 0, (size_t)P->nnz * sizeof(double), s));
  CUDA_TRY(cudaMemsetAsync(P->d_ctr_bwd, 0, sizeof(DevCounters), s));
  if (!P->opts.grad_deterministic) {
    CUDA_TRY(launch_backward(a, P->grid, s));
  } else {
    if (!P->d_gbuf) {
      // G_j offsets and waves of at most grad_wave_mib MiB
      cudaFree(P->d_gofs);                     // left by an earlier call that ran out of memory
      P->d_gofs = nullptr;
      std::vector<int64_t> gofs((size_t)P->n + 1, 0);
      for (int32_t j = 0; j < P->n; ++j) gofs[j + 1] = gofs[j] + (int64_t)P->h_m[j] * P->h_m[j];
      const int64_t cap = (int64_t)P->opts.grad_wave_mib * 1024 * 1024 / (int64_t)sizeof(double);
      P->waves.clear();
      int64_t wave_max = 0;
      for (int32_t j0 = P->row_begin; j0 < P->row_end;) {       // the plan's rows only
        int32_t j1 = j0 + 1;
        while (j1 < P->row_end && gofs[j1 + 1] - gofs[j0] <= cap) ++j1;
        P->waves.emplace_back(j0, j1);
        wave_max = std::max(wave_max, gofs[j1] - gofs[j0]);
        j0 = j1;
      }
      CUDA_TRY(cudaMalloc(&P->d_gofs, gofs.size() * sizeof(int64_t)));
      CUDA_TRY(cudaMemcpy(P->d_gofs, gofs.data(), gofs.size() * sizeof(int64_t),
                          cudaMemcpyHostToDevice));
      CUDA_TRY(cudaMalloc(&P->d_gbuf, (size_t)wave_max * sizeof(double)));
    }
    CUDA_TRY(ensure_tpos(P, s));
    a.gbuf = P->d_gbuf;
    a.gofs = P->d_gofs;
    for (const auto& w : P->waves) {
      a.j0 = w.first;
      a.j1 = w.second;
      CUDA_TRY(cudaMemsetAsync(&P->d_ctr_bwd->queue, 0, sizeof(int32_t), s));   // job queue
      CUDA_TRY(launch_backward(a, P->grid, s));
      CUDA_TRY(launch_grad_gather(P->d_rowptr, P->d_colind, P->d_tpos, P->d_m, P->d_gofs,
                                  P->d_gbuf, P->n, w.first, w.second, grad_in, s));
    }
  }
  P->last_stream = s;
  return SUBMAT_OK;
}

static submat_status pcg_impl(submat_plan_t P, const double* vals_a, const double* vals_k,
                              const double* b, double* x, double tol, int32_t max_iter,
                              int32_t* iters, double* rel_resid, void* stream) {
  g_last_error.clear();
  if (!P) return fail(SUBMAT_EINVAL, "plan is NULL");
  if (!vals_a || !b || !x) return fail(SUBMAT_EINVAL, "NULL array");
  if (iters) *iters = 0;
  if (rel_resid) *rel_resid = 0.0;
  if (P->n == 0) return SUBMAT_OK;
  if (!(tol > 0.0)) tol = 1e-6;
  if (max_iter <= 0) max_iter = 2 * P->n;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  DeviceScope dev;
  CUDA_TRY(dev.enter(P->device));
  const int32_t n = P->n;
  const size_t nd = (size_t)n;
  if (!P->d_cg) {
    const size_t words = 6 * nd + (size_t)P->nnz + cg_dot_scratch() + 2;
    CUDA_TRY(cudaMalloc(&P->d_cg, words * sizeof(double)));
  }
  double* r = P->d_cg;
  double* p = r + nd;
  double* q = p + nd;
  double* t1 = q + nd;
  double* t2 = t1 + nd;
  double* y = t2 + nd;                      // the iterate (x itself without K)
  double* kt = y + nd;                      // K^T's values
  double* part = kt + P->nnz;
  double* scal = part + cg_dot_scratch();
  const bool pre = vals_k != nullptr;
  double* it_x = pre ? y : x;
  if (pre) {
    CUDA_TRY(ensure_tpos(P, s));
    CUDA_TRY(cg_transpose_vals(P->d_rowptr, P->d_colind, P->d_tpos, vals_k, kt, P->nnz, s));
    CUDA_TRY(cg_spmv(P->d_rowptr, P->d_colind, kt, b, r, n, s));          // r = K^T b
  } else {
    CUDA_TRY(cudaMemcpyAsync(r, b, nd * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  CUDA_TRY(cudaMemsetAsync(it_x, 0, nd * sizeof(double), s));
  CUDA_TRY(cudaMemcpyAsync(p, r, nd * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cg_dot(r, r, n, part, scal, s));
  double rr = 0.0;
  CUDA_TRY(cudaMemcpyAsync(&rr, scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  const double bnorm = std::sqrt(rr);
  int32_t it = 0;
  submat_status st = SUBMAT_OK;
  while (bnorm > 0.0 && std::sqrt(rr) > tol * bnorm && it < max_iter) {
    if (pre) {                                                            // q = K^T A K p
      CUDA_TRY(cg_spmv(P->d_rowptr, P->d_colind, vals_k, p, t1, n, s));
      CUDA_TRY(cg_spmv(P->d_rowptr, P->d_colind, vals_a, t1, t2, n, s));
      CUDA_TRY(cg_spmv(P->d_rowptr, P->d_colind, kt, t2, q, n, s));
    } else {                                                              // q = A p
      CUDA_TRY(cg_spmv(P->d_rowptr, P->d_colind, vals_a, p, q, n, s));
    }
    CUDA_TRY(cg_dot(p, q, n, part, scal, s));
    double pq = 0.0;
    CUDA_TRY(cudaMemcpyAsync(&pq, scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (!(pq > 0.0) || !std::isfinite(pq)) {      // the operator is not positive definite
      st = fail(SUBMAT_ENOTSPD, "CG: p^T A p <= 0");
      break;
    }
    const double alpha = rr / pq;
    CUDA_TRY(cg_update(alpha, it_x, r, p, q, n, part, scal + 1, s));
    double rr_new = 0.0;
    CUDA_TRY(cudaMemcpyAsync(&rr_new, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cg_dir(rr_new / rr, r, p, n, s));
    rr = rr_new;
    ++it;
  }
  if (pre) CUDA_TRY(cg_spmv(P->d_rowptr, P->d_colind, vals_k, y, x, n, s));   // x = K y
  CUDA_TRY(cudaStreamSynchronize(s));
  if (iters) *iters = it;
  if (rel_resid) *rel_resid = bnorm > 0.0 ? std::sqrt(rr) / bnorm : 0.0;
  P->last_stream = s;
  return st;
}

static submat_status refine_impl(submat_plan_t P, const double* a_vals, const double* x_in,
                                 int32_t p, int32_t iters, double* x_out, void* stream) {
  g_last_error.clear();
  if (!P) return fail(SUBMAT_EINVAL, "plan is NULL");
  if (!a_vals || !x_in || !x_out) return fail(SUBMAT_EINVAL, "NULL array");
  if (p < 1 || iters < 0) return fail(SUBMAT_EINVAL, "p must be >= 1 and iters >= 0");
  if (P->n == 0) return SUBMAT_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  DeviceScope dev;
  CUDA_TRY(dev.enter(P->device));
  const int64_t nnz = P->nnz;
  if (!P->d_ref) CUDA_TRY(cudaMalloc(&P->d_ref, 4 * (size_t)nnz * sizeof(double)));
  CUDA_TRY(ensure_tpos(P, s));
  double* x = P->d_ref;              // the iterate
  double* r = x + nnz;               // R = A X^i
  double* t = r + nnz;               // transposed values
  double* c = t + nnz;               // a restricted product
  const int32_t* rp = P->d_rowptr;
  const int32_t* ci = P->d_colind;
  // X = (X0 + X0^T) / 2
  CUDA_TRY(cg_transpose_vals(rp, ci, P->d_tpos, x_in, t, nnz, s));
  CUDA_TRY(refine_axpby(0.5, x_in, 0.5, t, x, nnz, s));
  for (int32_t it = 0; it < iters; ++it) {
    // R = A X (X symmetric: X^T's values are X's), then R <- R X, p - 1 times
    CUDA_TRY(refine_masked_product(rp, ci, P->n, a_vals, x, r, s));
    for (int32_t k = 1; k < p; ++k) {
      CUDA_TRY(refine_masked_product(rp, ci, P->n, r, x, c, s));
      CUDA_TRY(cudaMemcpyAsync(r, c, (size_t)nnz * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    // X <- ((p + 1) X - X R) / p, then X <- (X + X^T) / 2
    CUDA_TRY(cg_transpose_vals(rp, ci, P->d_tpos, r, t, nnz, s));
    CUDA_TRY(refine_masked_product(rp, ci, P->n, x, t, c, s));
    CUDA_TRY(refine_axpby((double)(p + 1) / p, x, -1.0 / p, c, c, nnz, s));
    CUDA_TRY(cg_transpose_vals(rp, ci, P->d_tpos, c, t, nnz, s));
    CUDA_TRY(refine_axpby(0.5, c, 0.5, t, x, nnz, s));
  }
  CUDA_TRY(cudaMemcpyAsync(x_out, x, (size_t)nnz * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  P->last_stream = s;
  return SUBMAT_OK;
}

submat_status submat_get_report(submat_plan_t P, submat_report* r) {
  g_last_error.clear();
  if (!P || !r) return fail(SUBMAT_EINVAL, "NULL argument");
  std::memset(r, 0, sizeof(*r));
  r->n_rows = P->n_jobs;
  r->m_max = P->m_max;
  r->sum_m3 = P->sum_m3;
  if (P->n == 0) return SUBMAT_OK;
  CUDA_TRY(cudaStreamSynchronize(P->last_stream));
  DevCounters c;
  CUDA_TRY(cudaMemcpy(&c, P->d_ctr, sizeof(c), cudaMemcpyDeviceToHost));
  r->iters_max = c.iters_max;
  r->iters_sum = (int64_t)c.iters_sum;
  r->n_fallback = c.n_fallback;
  r->n_notspd = (int64_t)c.n_notspd;
  double mr;
  unsigned long long bits = c.resid_max_bits;
  std::memcpy(&mr, &bits, sizeof(mr));
  r->max_resid = mr;
  r->flops_tensor = c.flops_tensor;
  r->flops_fp64 = c.flops_fp64;
  r->n_illcond = (int64_t)c.n_illcond;
  r->flops_alg = c.flops_alg;
  if (P->have_fwd) {
    CUDA_TRY(cudaEventElapsedTime(&r->ms_kernel, P->ev[0], P->ev[1]));
    CUDA_TRY(cudaEventElapsedTime(&r->ms_fallback, P->ev[1], P->ev[2]));
  }
  return SUBMAT_OK;
}

submat_status submat_plan_rows(submat_plan_t P, int32_t* m, int32_t* pos) {
  g_last_error.clear();
  if (!P || (P->n > 0 && (!m || !pos))) return fail(SUBMAT_EINVAL, "NULL argument");
  if (P->n == 0) return SUBMAT_OK;
  CUDA_TRY(cudaMemcpy(m, P->d_m, P->n * sizeof(int32_t), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(pos, P->d_pos, P->n * sizeof(int32_t), cudaMemcpyDeviceToHost));
  return SUBMAT_OK;
}

submat_status submat_test_stall(submat_plan_t P, int32_t on) {
  g_last_error.clear();
  if (!P) return fail(SUBMAT_EINVAL, "plan is NULL");
  DeviceScope dev;
  CUDA_TRY(dev.enter(P->device));
  const int32_t v = on != 0 ? 1 : 0;
  CUDA_TRY(cudaDeviceSynchronize());          // no forward of this plan reads the flag now
  CUDA_TRY(cudaMemcpy(P->d_stall, &v, sizeof(v), cudaMemcpyHostToDevice));
  return SUBMAT_OK;
}

submat_status submat_plan_shape(submat_plan_t P, int32_t* n, int64_t* nnz) {
  if (!P) return fail(SUBMAT_EINVAL, "plan is NULL");
  if (n) *n = P->n;
  if (nnz) *nnz = P->nnz;
  return SUBMAT_OK;
}

void submat_plan_destroy(submat_plan_t P) { release(P); }

submat_status submat_plan(const submat_csr* csr, int32_t p, const submat_opts* opts,
                          submat_plan_t* out) {
  SUBMAT_NOTHROW(plan_impl(csr, p, opts, out))
}

submat_status submat_invroot(submat_plan_t P, const double* in, double* out, void* stream,
                             int32_t sync) {
  SUBMAT_NOTHROW(invroot_impl(P, in, out, stream, sync))
}

submat_status submat_invroot_host(submat_plan_t P, const double* in, double* out, void* stream) {
  SUBMAT_NOTHROW(invroot_host_impl(P, in, out, stream))
}

submat_status submat_invroot_backward(submat_plan_t P, const double* grad_out, double* grad_in,
                                      void* stream) {
  SUBMAT_NOTHROW(backward_impl(P, grad_out, grad_in, stream))
}

submat_status submat_refine(submat_plan_t P, const double* a_vals, const double* x_in, int32_t p,
                            int32_t iters, double* x_out, void* stream) {
  SUBMAT_NOTHROW(refine_impl(P, a_vals, x_in, p, iters, x_out, stream))
}

submat_status submat_pcg(submat_plan_t P, const double* vals_a, const double* vals_k,
                         const double* b, double* x, double tol, int32_t max_iter,
                         int32_t* iters, double* rel_resid, void* stream) {
  SUBMAT_NOTHROW(pcg_impl(P, vals_a, vals_k, b, x, tol, max_iter, iters, rel_resid, stream))
}

}  // extern "C"
