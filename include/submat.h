/*
 * submat.h -- C ABI of the GB300 submatrix-method library (libsubmat.so).
 *
 * The submatrix method (Lass et al., PASC'18, Sec. 3) approximates A^(-1/p) for a large
 * sparse symmetric positive definite matrix A while keeping A's sparsity pattern:
 *
 *   Algorithm 1 (Sec. 3.1): for every row j, R_j = the stored column indices of row j
 *       (ascending), S_j[k][l] = A[R_j[k]][R_j[l]] (zero where not stored).
 *   Sec. 3.2: F_j = S_j^(-1/p), the principal inverse p-th root of S_j.
 *   Algorithm 2 (Sec. 3.3) with the row-based CSR storage of Sec. 3.4: the result has A's
 *       rowptr/colind, and row j holds column pos_j = R_j.indexof(j) of F_j.
 *
 * All calls return a submat_status and never throw or abort.  Value arrays are FP64 and
 * in A's CSR order.  Device pointers are CUDA device (or managed) memory of the device
 * that was current when the plan was made; the caller owns them.  Calls are ordered on
 * the stream passed in (a cudaStream_t, NULL = legacy default stream); a plan must not be
 * used from two streams at the same time.
 */
#ifndef SUBMAT_H
#define SUBMAT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SUBMAT_API __attribute__((visibility("default")))
#else
#define SUBMAT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SUBMAT_OK = 0,
  SUBMAT_EINVAL = 1,    /* bad argument: NULL pointer, p < 1, unsorted/duplicate/out-of-range
                           column index, negative sizes, vals_out aliasing vals_in or
                           grad_in aliasing grad_out                                      */
  SUBMAT_ENODIAG = 2,   /* a row does not store its diagonal entry (Alg. 2 needs
                           R.indexof(j))                                                  */
  SUBMAT_ENOTSYM = 3,   /* the pattern is not symmetric                                    */
  SUBMAT_ETOOBIG = 4,   /* a row has more entries than SUBMAT_MAX_M                        */
  SUBMAT_ENOMEM = 5,    /* a device or host allocation failed                              */
  SUBMAT_ECUDA = 6,     /* a CUDA runtime call failed (the message is in submat_last_error) */
  SUBMAT_ENOTSPD = 7,   /* some submatrix is not positive definite or holds a non-finite
                           value; its output row is NaN, the others are valid            */
  SUBMAT_ENOFWD = 8,    /* backward called before any forward on this plan                 */
  SUBMAT_ETIMEOUT = 9   /* a device-side pipeline wait gave up (the rows not done are NaN)  */
} submat_status;

/* Largest submatrix order (row length) the library accepts. */
#define SUBMAT_MAX_M 1536

/*
 * Precision of the submatrix operation.  The iteration's products run on FP16 tensor cores
 * rather than as single TF32 or BF16 products: rounding errors made in any step of the
 * coupled iteration stay in its limit (X_inf = X_k M_k^(-1/p) from any iterate on), so a
 * low-precision phase followed by FP64 refinement leaves ~1e-3 (TF32) or ~1e-2 (BF16) for
 * p >= 2, and the tensor cores' FP32 accumulation truncates.  Each matrix is therefore split
 * into four FP16 planes of 10-bit integers whose low level sums the FP32 accumulators hold
 * exactly (an error-free splitting in the manner of Ozaki et al.), 40 bits below its scale;
 * FP64 stays for the gather, the scaling, the column output and its residual, the p = 1
 * refinement and the eigendecomposition fallback.
 */
enum {
  SUBMAT_PREC_FP64 = 0,       /* coupled Newton iteration entirely in FP64 (CUDA cores)     */
  SUBMAT_PREC_MIXED_F16 = 1,  /* coupled Newton iteration on the tensor cores (tcgen05) with
                                 every matrix split into four FP16 planes of 10-bit integers,
                                 accumulated per level (10 FP16 products per product),
                                 then the FP64 column residual check                       */
  SUBMAT_PREC_MIXED_F16_SYNC = 2  /* the same arithmetic on the legacy mma.sync tensor path
                                 (kept as the baseline of the tcgen05 engine)               */
};

typedef struct {
  int32_t n;               /* order of A                                                 */
  int64_t nnz;             /* stored entries                                             */
  const int32_t* rowptr;   /* [n+1], rowptr[0] = 0, nondecreasing, rowptr[n] = nnz        */
  const int32_t* colind;   /* [nnz], strictly ascending within each row, in [0, n)        */
  int32_t on_device;       /* 0: host pointers, 1: device pointers                       */
} submat_csr;

typedef struct {
  int32_t precision;       /* SUBMAT_PREC_*; default SUBMAT_PREC_MIXED_F16               */
  int32_t k_max;           /* iteration cap of the coupled iteration; default 40         */
  double tol;              /* stop when ||M - I||_F <= tol * sqrt(m) (or when it stops
                              decreasing below 1e-2 sqrt(m)), then do one more X update;
                              the mixed path for p >= 2 also stops once ||M - I||_F <= 0.05
                              and finishes with a Taylor polynomial of M^(-1/p) on the
                              carried column instead; default 1e-4 (mixed) / 1e-7 (FP64);
                              <= 0 selects the default                                    */
  double resid_tol;        /* a row whose FP64 column residual ||e_pos - F^p s_pos||_2
                              exceeds this goes to the FP64 eigendecomposition fallback;
                              default 1e-3                                                */
  int32_t refine_steps;    /* FP64 column refinement: p = 1: iterative-refinement sweeps
                              (default 2); p >= 2: 1 = one Newton step on the column,
                              0 = none (default 0: once the iteration has converged the
                              step amplifies the part of the error that does not commute
                              with S_j); < 0 selects the default                          */
  int32_t use_graph;       /* capture the forward launches into a CUDA graph; default 1  */
  double kappa_max;        /* mixed path: a row whose condition estimate
                              lambda_bar / lambda_min (power iteration on the converged
                              iterate) exceeds this goes to the FP64 fallback; default 100 */
  int32_t root_sign;       /* -1 (default): the inverse p-th root A^(-1/p); +1: the positive
                              p-th root A^(1/p), the same method with f(S) = S^(1/p)
                              (Sec. 4.2), computed from the same iteration as
                              S^(1/p) e_pos = S (S^(-1/p))^(p-1) e_pos; any other value is
                              SUBMAT_EINVAL.  submat_invroot_noalloc is inverse only.     */
  int32_t grad_deterministic; /* 0 (default): submat_invroot_backward adds each submatrix's
                              contributions to grad_in with atomic adds (their order, and so
                              the last bits, vary from call to call); 1: each stored entry
                              sums its contributions in a fixed order (the contributing rows
                              j ascending, in waves of at most grad_wave_mib MiB of
                              per-submatrix gradients), so repeated calls give identical
                              bits.  Costs device memory for the waves' gradients, nnz int32
                              and n+1 int64, allocated by the first such backward; any other
                              value is SUBMAT_EINVAL.                                     */
  int32_t grad_wave_mib;   /* deterministic backward: largest device buffer of per-
                              submatrix gradients per wave, in MiB (a wave holds at least
                              one row); <= 0 selects SUBMAT_GRAD_WAVE_MIB                  */
  int32_t shard_count;     /* 0 or 1 (default): the plan computes every row; k > 1: only
                              the rows of shard shard_rank of k (submat_shard_rows), for one
                              GPU of k each given the whole matrix (Sec. 6.1.1): the forward
                              writes only those rows' segments of vals_out, the backward
                              gives those rows' contribution to grad_in (the shards'
                              grad_in add up to the full gradient)                         */
  int32_t shard_rank;      /* 0 .. shard_count-1                                          */
  int32_t small_max_m;     /* SUBMAT_PREC_MIXED_F16: rows of order m <= small_max_m take the
                              small-submatrix engine (every working matrix in shared memory,
                              warp-level mma.sync tiles); 0 disables it; at most
                              SUBMAT_SMALL_MAX_M; < 0 selects the tuned default            */
  int32_t sync_max_m;      /* SUBMAT_PREC_MIXED_F16: rows with small_max_m < m <= sync_max_m
                              take the mma.sync engine (64 x 64 tiles), larger rows the
                              tcgen05 engine (128 x 96 tiles in tensor memory); < 0 selects
                              the tuned default.  The rows are ordered by decreasing m, so
                              each engine gets one contiguous run of the work queue and one
                              persistent launch                                           */
} submat_opts;

/* Largest order the small-submatrix engine takes. */
#define SUBMAT_SMALL_MAX_M 32

typedef struct {
  int64_t n_rows;          /* submatrices processed by the last forward                  */
  int32_t m_max;           /* largest submatrix order                                    */
  int32_t iters_max;       /* largest iteration count of the last forward                */
  int64_t iters_sum;       /* sum of iteration counts                                    */
  int64_t n_fallback;      /* rows recomputed by the FP64 eigendecomposition fallback    */
  int64_t n_notspd;        /* rows with a non-positive eigenvalue or non-finite input    */
  double max_resid;        /* largest FP64 column residual seen before the fallback      */
  double sum_m3;           /* sum over rows of m^3 (true sizes)                           */
  double flops_tensor;     /* tensor-core flops executed by the last forward: sum over
                              rows of (GEMMs executed) * 10 FP16 slice products *
                              2 m_j^3 (true m_j; p GEMMs per iteration for p >= 2;
                              two for p = 1, plus its final X product)                   */
  double flops_fp64;       /* FP64 flops of the last forward (FP64 path: iterations;
                              mixed path: column refinement; both: fallback)             */
  float ms_kernel;         /* device time of the last forward's main (Newton) kernel,
                              from CUDA events recorded around it on the launch stream   */
  float ms_fallback;       /* device time of the last forward's fallback kernel          */
  int64_t n_illcond;       /* rows sent to the fallback by the condition estimate        */
  double flops_alg;        /* the method's flops of the last forward, independent of the
                              engine: sum over rows of k_j (p+1) 2 m_j^3 with the executed
                              iteration count k_j and the true order m_j, every product
                              counted as a dense GEMM (p = 1 adds 2 m_j^3 for its final X
                              product); divide by ms_kernel for the roofline rate        */
} submat_report;

typedef struct submat_plan_s* submat_plan_t;

/*
 * Row range [*row_begin, *row_end) of shard rank of count (host call; no GPU needed).
 * Every worker holds the whole matrix and takes a contiguous range of rows, as in
 * Sec. 6.1.1, with the boundaries at the quantiles of the rows' cost m_j^3 instead of equal
 * row counts (the load imbalance Sec. 6.1.3 describes): shard k starts at the first row
 * whose cumulative cost reaches k/count of the total.  rowptr: host array of n+1 entries.
 * SUBMAT_EINVAL for count < 1, rank outside [0, count) or NULL pointers.
 */
SUBMAT_API submat_status submat_shard_rows(int32_t n, const int32_t* rowptr, int32_t count,
                                           int32_t rank, int32_t* row_begin, int32_t* row_end);

/* Fill *opts with the defaults. */
SUBMAT_API void submat_default_opts(submat_opts* opts);

/* Largest root order of the mixed-precision paths: beyond it the affine term and the
 * level sums of the integer slices could no longer be kept exact (SUBMAT_PREC_FP64 takes
 * any p >= 1). */
#define SUBMAT_MIXED_MAX_P 10

/*
 * Build a plan for A's pattern and the root order p >= 1 (Alg. 1, index part; p at most
 * SUBMAT_MIXED_MAX_P for the mixed-precision modes, else SUBMAT_EINVAL).
 * Checks the pattern (SUBMAT_EINVAL / ENODIAG / ENOTSYM / ETOOBIG; n > nnz means some row
 * lacks its diagonal: ENODIAG), computes m_j and
 * pos_j on the device, orders the rows by decreasing m_j for the persistent scheduler,
 * and allocates the per-CTA working storage.  The plan keeps device copies of rowptr and
 * colind; the caller's arrays may be freed afterwards.  opts may be NULL (defaults).
 */
SUBMAT_API submat_status submat_plan(const submat_csr* csr, int32_t p, const submat_opts* opts,
                          submat_plan_t* out);

/*
 * Forward: vals_out = the submatrix method's approximation of A^(-1/p) (A^(1/p) with
 * root_sign = +1) on A's pattern (Alg. 1, Sec. 3.2, Alg. 2).  vals_in and vals_out are device arrays of nnz doubles in
 * CSR order; they must not overlap.  A's values must be symmetric (A[r][c] = A[c][r]).
 * The plan keeps a device copy of vals_in for the backward.  Returns SUBMAT_ENOTSPD (after
 * writing every other row) when some submatrix is not positive definite.  Stream-ordered;
 * the status of the numerics (ENOTSPD) needs a stream synchronisation and is only
 * returned when sync != 0; with sync == 0 the call returns SUBMAT_OK after queueing the
 * work and submat_get_report gives the counts later.
 */
SUBMAT_API submat_status submat_invroot(submat_plan_t plan, const double* vals_in, double* vals_out,
                             void* stream, int32_t sync);

/*
 * Forward on host buffers: copies vals_in (nnz doubles, host memory; pinned memory makes
 * the copies asynchronous) to plan-owned device memory on the stream, runs
 * submat_invroot, copies the result back into vals_out (host, nnz doubles) and
 * synchronises the stream.  The device buffers are allocated on the first call and kept
 * by the plan.  Returns SUBMAT_ENOTSPD and SUBMAT_ETIMEOUT like submat_invroot with
 * sync != 0.
 */
SUBMAT_API submat_status submat_invroot_host(submat_plan_t plan, const double* vals_in,
                                             double* vals_out, void* stream);

/* Default largest buffer of per-submatrix gradients of a deterministic backward wave. */
#define SUBMAT_GRAD_WAVE_MIB 4096

/*
 * Backward (Daleckii-Krein adjoint; Higham, Functions of Matrices, Thm. 3.11, with
 * f(x) = x^(root_sign/p)):
 * grad_in = dL/dvals for L = sum(grad_out * vals_out) of the last forward, with respect to
 * A's stored values, the (r,c)/(c,r) pair sharing one symmetric perturbation.  For each row
 * j the submatrix is regathered from the saved vals_in and decomposed again (recomputation,
 * no stored iterates) by a cyclic Jacobi with the matrix and eigenvectors held as
 * double-floats (FP32 pairs, ~44 significant bits; the rotation angles, the divided
 * differences and the products with the eigenvectors in FP64).  grad_out and grad_in are
 * device arrays of nnz doubles that must not overlap; grad_in is overwritten.  Returns
 * SUBMAT_ENOFWD if no forward ran on this plan.
 * With opts.grad_deterministic = 1 the per-submatrix gradients G_j of a wave of rows are
 * stored, and each entry (r, c) then adds G_j(r, c) over the wave's rows j whose patterns
 * hold both r and c (the transposed map of the plan: j in R_r and R_c), without atomics.
 */
SUBMAT_API submat_status submat_invroot_backward(submat_plan_t plan, const double* grad_out,
                                      double* grad_in, void* stream);

/*
 * Conjugate gradients on A x = b for A on the plan's pattern (Sec. 4.4, the submatrix
 * method as a preconditioner).  vals_a: A's values (device, nnz doubles, SPD); b, x:
 * device arrays of n doubles (x is overwritten; it starts from zero).  With vals_k == NULL
 * plain CG; otherwise K (values vals_k on the same pattern, CSR, e.g. the result of
 * submat_invroot with p = 2, K ~ A^(-1/2)) is applied as in Sec. 4.4: CG on
 * K^T A K y = K^T b, then x = K y.  Stops when the 2-norm of the iterated system's residual
 * is at most tol (<= 0: 1e-6) times that of its right-hand side, or after max_iter
 * (<= 0: 2n) steps; *iters and *rel_resid (either may be NULL) receive the step count and
 * that final ratio.  Dot products are reduced in a fixed order, so repeated calls give the
 * same bits.  Synchronous on the stream.  Work vectors (6n + nnz doubles) are allocated by
 * the plan's first call.  Returns SUBMAT_ENOTSPD if p^T A p <= 0 occurs (x then holds the
 * last iterate, mapped by K when given).
 */
SUBMAT_API submat_status submat_pcg(submat_plan_t plan, const double* vals_a, const double* vals_k,
                                    const double* b, double* x, double tol, int32_t max_iter,
                                    int32_t* iters, double* rel_resid, void* stream);

/*
 * Global refinement of an approximate inverse p-th root on the plan's pattern (Sec. 4.5:
 * the submatrix method's result as the starting guess of a Newton iteration for A^(-1/p),
 * every product restricted to the pattern as a sparse iteration has to be).  From the
 * symmetric part X of x_in, `iters` steps of
 *     R = A X, then R <- R X (p - 1 more times);  X <- ((p + 1) X - X R) / p;
 *     X <- (X + X^T) / 2,
 * each product C = L R restricted to the pattern: C[i][j] = sum over k with (i, k) and
 * (k, j) stored of L[i][k] R[k][j], for every stored (i, j).  FP64, a fixed summation order
 * (identical bits on every call).  a_vals, x_in, x_out: device arrays of nnz doubles on the
 * plan's pattern (A's values and the start, e.g. the result of submat_invroot; on a pattern
 * wider than A's, such as that of A^2, A's values are zero where A stores nothing); x_out may
 * alias x_in.  The plan's p and precision are not used.  Synchronous on the stream; work
 * arrays of 4 nnz doubles (and the plan's transposed map) are allocated by the first call.
 * The step converges only from a start that commutes with A closely enough: for p = 1
 * (Newton-Schulz for the inverse) the error E maps to -E A E, for p >= 2 error components
 * that couple eigenvalues far apart grow.
 */
SUBMAT_API submat_status submat_refine(submat_plan_t plan, const double* a_vals,
                                       const double* x_in, int32_t p, int32_t iters,
                                       double* x_out, void* stream);

/* Counters of the last forward (synchronises the plan's stream). */
SUBMAT_API submat_status submat_get_report(submat_plan_t plan, submat_report* out);

/*
 * The integer plan as computed on the device (Alg. 1 index part): m[j] = |R_j| and
 * pos[j] = R_j.indexof(j), copied into the caller's host arrays of n int32 each.
 */
SUBMAT_API submat_status submat_plan_rows(submat_plan_t plan, int32_t* m, int32_t* pos);

/*
 * Test aid for the bounded device waits (the paper has no counterpart).  While on != 0,
 * every CTA of the plan's tcgen05 engine launch (SUBMAT_PREC_MIXED_F16, rows above the
 * small and mma.sync buckets) first waits on a pipeline barrier that nothing signals, before
 * it issues any copy or tensor-core operation; the wait gives up after its poll limit (on
 * the order of a second), the CTA writes NaN to every row it takes from its work queue, and
 * submat_invroot returns SUBMAT_ETIMEOUT (with sync != 0; submat_get_report still works).
 * Rows of the other engines are computed as usual.  on = 0 restores normal operation.
 * Other precisions ignore the flag.  Synchronises the device.
 */
SUBMAT_API submat_status submat_test_stall(submat_plan_t plan, int32_t on);

/* Order n and entry count nnz of the plan's pattern. */
SUBMAT_API submat_status submat_plan_shape(submat_plan_t plan, int32_t* n, int64_t* nnz);

/*
 * No-allocation forward (the paper has no counterpart; it is a deployment aid).
 *
 * Some callers cannot call cudaMalloc: code running inside another framework's memory pool
 * or arena, allocation-free sections of an application, or hosts that forbid device
 * allocations after start-up.  submat_plan allocates, so such callers use this call
 * instead: it needs no plan and allocates nothing.  It runs the FP64 path (gather,
 * Gershgorin scaling, coupled Newton iteration in FP64, FP64 column refinement, and the
 * FP64 Jacobi eigendecomposition for rows whose residual test fails) with its working
 * storage in one file-scope device array of SUBMAT_NOALLOC_SCRATCH_MIB MiB, which every GPU
 * that loads the library holds until the process exits.
 *
 *   n, nnz, rowptr, colind  A's pattern in device memory (sorted, unique, symmetric, every
 *                           diagonal stored).  Before touching a row's data the kernel checks
 *                           that the row's extent and the extents of the rows its column
 *                           indices name lie in [0, nnz] and that those indices lie in
 *                           [0, n); a row that fails gets NaN and the call SUBMAT_EINVAL.
 *                           Sortedness and symmetry are not re-checked (see submat_plan)
 *   p                       root order, >= 1
 *   m_max                   the caller's bound on the row lengths, 1..SUBMAT_NOALLOC_MAX_M;
 *                           larger values return SUBMAT_ETOOBIG before any GPU work, and a
 *                           row longer than m_max (or empty) gets NaN and SUBMAT_ETOOBIG
 *   vals_in, vals_out       device arrays of nnz doubles, not overlapping
 *   stream                  cudaStream_t; the call is synchronous: it waits for the stream
 *                           and reads a status word back before it returns
 *
 * Returns SUBMAT_ENODIAG / SUBMAT_ENOTSPD as the plan-based calls do (affected rows NaN).
 * The first call on a device looks up the array's device address and sets the kernel's
 * shared-memory limit on that device; make that first call before any stream capture.
 * Every call shares the array, and the array keeps the last call's contents (the call
 * clears its own control block): calls that overlap on the GPU race, so serialise them.
 * It uses at most as many CTAs as the array has slots for pad(m_max) (about 18 for
 * m_max = 256), so it is slower than submat_invroot.
 */
#define SUBMAT_NOALLOC_SCRATCH_MIB 64
#define SUBMAT_NOALLOC_MAX_M 1024
SUBMAT_API submat_status submat_invroot_noalloc(int32_t n, int64_t nnz, const int32_t* rowptr,
                                                const int32_t* colind, int32_t p, int32_t m_max,
                                                const double* vals_in, double* vals_out,
                                                void* stream);

/* Release every resource of the plan.  NULL is ignored. */
SUBMAT_API void submat_plan_destroy(submat_plan_t plan);

/* Static description of a status code. */
SUBMAT_API const char* submat_status_string(submat_status s);

/* Message of the last failing call on this thread ("" if none). */
SUBMAT_API const char* submat_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SUBMAT_H */
