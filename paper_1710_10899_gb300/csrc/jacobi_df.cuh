// Cyclic Jacobi eigendecomposition of one symmetric submatrix per CTA with the matrix and
// the eigenvectors held as double-floats (FP32 pairs, ~44 significant bits) (internal
// header).  The O(m^3) rotation updates run on the FP32 units: an FP64 operation costs
// 64 FP32 operations' time on this GPU, and a double-float rotation update takes about 20
// FP32 operations for the 2 of FP64.  The O(m) rotation angles per step are computed in
// double-float too (angle_df).  Same ordering and rotation as jacobi.cuh (round-robin pairs; the symmetric 2x2 Schur
// decomposition of Golub & Van Loan, Alg. 8.4.1); it stops at off(A) <= 1e-12 ||A||_F or,
// below 1e-9 ||A||_F, once a sweep shrinks off(A) by less than half (the rounding floor of
// double-floats; FP64's 1e-14 bound they cannot reach).
#pragma once
#include "common.cuh"
#include "slices.cuh"

namespace submat {
namespace jdf {

constexpr int kMaxSweeps = 30;
constexpr int kVtU = 8;        // eigenvector elements in flight per thread (packed variant)

__device__ __forceinline__ float2 split(double d) {
  const float h = (float)d;
  return make_float2(h, (float)(d - (double)h));
}
__device__ __forceinline__ double join(float2 a) { return (double)a.x + (double)a.y; }

// c a - s b for double-floats (products exact in their leading parts, cross terms added).
__device__ __forceinline__ float2 rot(float2 c, float2 a, float2 s, float2 b) {
  const float p1 = c.x * a.x;
  float e1 = fmaf(c.x, a.x, -p1);
  e1 = fmaf(c.x, a.y, fmaf(c.y, a.x, e1));
  const float p2 = s.x * b.x;
  float e2 = fmaf(s.x, b.x, -p2);
  e2 = fmaf(s.x, b.y, fmaf(s.y, b.x, e2));
  float h, l;
  slc::two_sum(p1, -p2, h, l);
  l = l + (e1 - e2);
  const float r = h + l;
  return make_float2(r, l - (r - h));
}

// Rotation (c, s) of the symmetric 2 x 2 Schur decomposition (Golub & Van Loan, Alg. 8.4.1)
// that annihilates apq in [[app, apq], [apq, aqq]], as double-floats without FP64: the
// tangent t comes from FP32 arithmetic on the leading words (an angle off by ~1e-7 leaves
// a residual of ~1e-7 apq, which the next sweep removes like any other entry), then
// c = (1 + t^2)^(-1/2) by one double-float Newton step from rsqrtf and s = t c, so that
// c^2 + s^2 = 1 to ~2^-46 for whatever t: the rotation stays orthogonal.
__device__ __forceinline__ void angle_df(float2 app, float2 aqq, float2 apq, float2& c,
                                         float2& s) {
  if (apq.x == 0.f) {
    c = make_float2(1.f, 0.f);
    s = make_float2(0.f, 0.f);
    return;
  }
  const float d = (aqq.x - app.x) + (aqq.y - app.y);
  const float tau = d / (2.f * apq.x);
  const float at = fabsf(tau);
  const float t = at > 1e18f ? 0.5f / tau
                             : copysignf(1.f, tau) / (at + sqrtf(fmaf(tau, tau, 1.f)));
  float xh, xl;                                     // x = 1 + t^2 as a double-float
  const float p = t * t;
  slc::two_sum(1.f, p, xh, xl);
  xl += fmaf(t, t, -p);
  const float r0 = rsqrtf(xh);
  const float q = r0 * r0, qe = fmaf(r0, r0, -q);   // r0^2 = q + qe exactly
  const float y = fmaf(xh, q, -1.f) + fmaf(xh, qe, xl * q);   // x r0^2 - 1
  float ch, cl;
  slc::two_sum(r0, -0.5f * r0 * y, ch, cl);         // r0 (1 - y / 2)
  c = make_float2(ch, cl);
  float sh, sl;
  slc::two_sum(t * ch, fmaf(t, ch, -(t * ch)) + t * cl, sh, sl);
  s = make_float2(sh, sl);
}

// Eigendecomposition of the symmetric m x m matrix A (double-floats, ld m, global) in place:
// on return A's diagonal holds the eigenvalues and V (ld m) the eigenvectors (columns).
// pair_s: 2*ceil(m/2) ints, cs_s: 4*ceil(m/2) floats (shared), red_s: kRedDoubles doubles.
// Returns the sweeps used, or -1 if A holds a non-finite value.
static __device__ int jacobi_eig_df(float2* __restrict__ A, float2* __restrict__ V, int m,
                                    int* pair_s, float* cs_s, double* red_s) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < m * m; e += blockDim.x)
    V[e] = make_float2((e / m == e % m) ? 1.f : 0.f, 0.f);
  __syncthreads();
  const int mm = m + (m & 1);
  const int np = mm / 2;
  int sweep = 0;
  double prev = 1.7e308;
  for (; sweep < kMaxSweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = tid; e < m * m; e += blockDim.x) {
      const double v = (double)A[e].x;
      tot += v * v;
      if (e / m != e % m) off += v * v;
    }
    off = warp_sum(off);
    tot = warp_sum(tot);
    if (lane == 0) { red_s[warp] = off; red_s[kMaxWarps + warp] = tot; }
    __syncthreads();
    double so = 0.0, st = 0.0;
    for (int w = 0; w < nwarps(); ++w) { so += red_s[w]; st += red_s[kMaxWarps + w]; }
    __syncthreads();
    if (!(st <= 1.7e308)) return -1;     // NaN or infinity somewhere in A
    if (m == 1 || !(so > 1e-24 * st)) break;       // off(A) <= 1e-12 ||A||_F
    // at double-float rounding level (about 2^-44 ||A|| per entry, so for larger m the
    // bound above is out of reach) a sweep no longer shrinks off(A) quadratically
    if (so <= 1e-18 * st && so > 0.25 * prev) break;
    prev = so;
    for (int s = 0; s < mm - 1; ++s) {
      for (int k = tid; k < np; k += blockDim.x) {
        int p, q;
        if (k == 0) { p = s; q = mm - 1; }
        else { p = (s + k) % (mm - 1); q = (s - k + mm - 1) % (mm - 1); }
        if (p > q) { const int t = p; p = q; q = t; }
        float2 cd = make_float2(1.f, 0.f), sd = make_float2(0.f, 0.f);
        if (q < m) angle_df(A[p * m + p], A[q * m + q], A[p * m + q], cd, sd);
        pair_s[2 * k] = p;
        pair_s[2 * k + 1] = q;
        cs_s[4 * k] = cd.x;
        cs_s[4 * k + 1] = cd.y;
        cs_s[4 * k + 2] = sd.x;
        cs_s[4 * k + 3] = sd.y;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int e = tid; e < np * m; e += blockDim.x) {
        const int k = e / m, i = e % m;
        const int p = pair_s[2 * k], q = pair_s[2 * k + 1];
        if (q >= m) continue;
        const float2 c = make_float2(cs_s[4 * k], cs_s[4 * k + 1]);
        const float2 sn = make_float2(cs_s[4 * k + 2], cs_s[4 * k + 3]);
        if (sn.x == 0.f) continue;
        const float2 nc = make_float2(-c.x, -c.y);
        const float2 ap = A[i * m + p], aq = A[i * m + q];
        A[i * m + p] = rot(c, ap, sn, aq);
        A[i * m + q] = rot(sn, ap, nc, aq);              // s ap + c aq
        const float2 vp = V[i * m + p], vq = V[i * m + q];
        V[i * m + p] = rot(c, vp, sn, vq);
        V[i * m + q] = rot(sn, vp, nc, vq);
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int e = tid; e < np * m; e += blockDim.x) {
        const int k = e / m, i = e % m;
        const int p = pair_s[2 * k], q = pair_s[2 * k + 1];
        if (q >= m) continue;
        const float2 c = make_float2(cs_s[4 * k], cs_s[4 * k + 1]);
        const float2 sn = make_float2(cs_s[4 * k + 2], cs_s[4 * k + 3]);
        if (sn.x == 0.f) continue;
        const float2 nc = make_float2(-c.x, -c.y);
        const float2 ap = A[p * m + i], aq = A[q * m + i];
        A[p * m + i] = rot(c, ap, sn, aq);
        A[q * m + i] = rot(sn, ap, nc, aq);
      }
      __syncthreads();
    }
  }
  return sweep;
}

// Index of (r, c), r <= c, in the row-packed upper triangle of an m x m symmetric matrix.
__device__ __forceinline__ int pidx(int r, int c, int m) { return r * m - (r * (r - 1)) / 2 + (c - r); }
__device__ __forceinline__ int pidx_sym(int a, int b, int m) {
  return a <= b ? pidx(a, b, m) : pidx(b, a, m);
}

// The same decomposition with A's upper triangle packed in shared memory (P, m(m+1)/2
// double-floats) and the eigenvectors transposed in global memory (Vt, ld m: row k = the
// k-th eigenvector), so every step touches only shared memory and coalesced rows.  A step's
// disjoint rotations act on 2 x 2 blocks of A: block (k, l), rows of pair k and columns of
// pair l, becomes J_k^T B J_l, J = [[c, s], [-s, c]] (one thread per block of the upper block
// triangle, so every packed entry has one writer).  On return P's diagonal holds the
// eigenvalues.  Same returns as jacobi_eig_df.
static __device__ int jacobi_eig_df_packed(float2* __restrict__ P, float2* __restrict__ Vt,
                                           int m, int* pair_s, float* cs_s, double* red_s) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < m * m; e += blockDim.x)
    Vt[e] = make_float2((e / m == e % m) ? 1.f : 0.f, 0.f);
  __syncthreads();
  const int mm = m + (m & 1);
  const int np = mm / 2;
  int sweep = 0;
  double prev = 1.7e308;
  for (; sweep < kMaxSweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = tid; e < m * m; e += blockDim.x) {
      const int r = e / m, c = e - r * m;
      if (r > c) continue;
      const double v = (double)P[pidx(r, c, m)].x;
      tot += (r == c ? 1.0 : 2.0) * v * v;
      if (r != c) off += 2.0 * v * v;
    }
    off = warp_sum(off);
    tot = warp_sum(tot);
    if (lane == 0) { red_s[warp] = off; red_s[kMaxWarps + warp] = tot; }
    __syncthreads();
    double so = 0.0, st = 0.0;
    for (int w = 0; w < nwarps(); ++w) { so += red_s[w]; st += red_s[kMaxWarps + w]; }
    __syncthreads();
    if (!(st <= 1.7e308)) return -1;     // NaN or infinity somewhere in A
    if (m == 1 || !(so > 1e-24 * st)) break;       // off(A) <= 1e-12 ||A||_F
    // at double-float rounding level (about 2^-44 ||A|| per entry, so for larger m the
    // bound above is out of reach) a sweep no longer shrinks off(A) quadratically
    if (so <= 1e-18 * st && so > 0.25 * prev) break;
    prev = so;
    for (int s = 0; s < mm - 1; ++s) {
      for (int k = tid; k < np; k += blockDim.x) {
        int p, q;
        if (k == 0) { p = s; q = mm - 1; }
        else { p = (s + k) % (mm - 1); q = (s - k + mm - 1) % (mm - 1); }
        if (p > q) { const int t = p; p = q; q = t; }
        float2 cd = make_float2(1.f, 0.f), sd = make_float2(0.f, 0.f);
        if (q < m) angle_df(P[pidx(p, p, m)], P[pidx(q, q, m)], P[pidx(p, q, m)], cd, sd);
        pair_s[2 * k] = p;
        pair_s[2 * k + 1] = q;
        cs_s[4 * k] = cd.x;
        cs_s[4 * k + 1] = cd.y;
        cs_s[4 * k + 2] = sd.x;
        cs_s[4 * k + 3] = sd.y;
      }
      __syncthreads();
      // blocks (k, l), k <= l, of the upper block triangle, folded into rows of np + 1:
      // folded row r holds block row r (np - r blocks) followed by block row np - 1 - r
      // (r + 1 blocks); for odd np the middle row holds only its own blocks.  A thread's
      // blocks advance by blockDim.x, i.e. by dr folded rows and dc places (no division)
      const int np1 = np + 1;
      const int nblk = (np / 2) * np1 + ((np & 1) ? np1 / 2 : 0);   // np (np + 1) / 2
      const int dr = blockDim.x / np1, dc = blockDim.x - dr * np1;
      int r_nx = tid / np1, c_nx = tid - r_nx * np1;
      for (int e = tid; e < nblk; e += blockDim.x) {
        const int r = r_nx, cc = c_nx;
        r_nx += dr;
        c_nx += dc;
        if (c_nx >= np1) { c_nx -= np1; ++r_nx; }
        const bool first = cc < np - r;
        const int k = first ? r : np - 1 - r;
        const int l = first ? r + cc : k + (cc - (np - r));
        const int pk = pair_s[2 * k], qk = pair_s[2 * k + 1];
        const int pl = pair_s[2 * l], ql = pair_s[2 * l + 1];
        const bool hk = qk < m, hl = ql < m;            // pair has its second index
        const float2 ck = make_float2(cs_s[4 * k], cs_s[4 * k + 1]);
        const float2 sk = make_float2(cs_s[4 * k + 2], cs_s[4 * k + 3]);
        const float2 cl = make_float2(cs_s[4 * l], cs_s[4 * l + 1]);
        const float2 sl = make_float2(cs_s[4 * l + 2], cs_s[4 * l + 3]);
        const float2 z = make_float2(0.f, 0.f);
        const float2 nck = make_float2(-ck.x, -ck.y), ncl = make_float2(-cl.x, -cl.y);
        if (k == l) {
          if (!hk || sk.x == 0.f) continue;               // no rotation
          const float2 b00 = P[pidx(pk, pk, m)], b01 = P[pidx(pk, qk, m)], b11 = P[pidx(qk, qk, m)];
          // C = B J, then B' = J^T C (symmetric)
          const float2 c00 = rot(ck, b00, sk, b01), c01 = rot(sk, b00, nck, b01);
          const float2 c10 = rot(ck, b01, sk, b11), c11 = rot(sk, b01, nck, b11);
          P[pidx(pk, pk, m)] = rot(ck, c00, sk, c10);
          P[pidx(pk, qk, m)] = rot(ck, c01, sk, c11);
          P[pidx(qk, qk, m)] = rot(sk, c01, nck, c11);
          continue;
        }
        const bool rk = hk && sk.x != 0.f, rl = hl && sl.x != 0.f;   // rotations applied
        if (!rk && !rl) continue;
        const int i00 = pidx_sym(pk, pl, m);
        const int i01 = hl ? pidx_sym(pk, ql, m) : 0;
        const int i10 = hk ? pidx_sym(qk, pl, m) : 0;
        const int i11 = (hk && hl) ? pidx_sym(qk, ql, m) : 0;
        float2 b00 = P[i00];
        float2 b01 = hl ? P[i01] : z;
        float2 b10 = hk ? P[i10] : z;
        float2 b11 = (hk && hl) ? P[i11] : z;
        if (rl) {                                          // columns: B J_l
          const float2 t00 = rot(cl, b00, sl, b01), t01 = rot(sl, b00, ncl, b01);
          const float2 t10 = rot(cl, b10, sl, b11), t11 = rot(sl, b10, ncl, b11);
          b00 = t00; b01 = t01; b10 = t10; b11 = t11;
        }
        if (rk) {                                          // rows: J_k^T B
          const float2 t00 = rot(ck, b00, sk, b10), t10 = rot(sk, b00, nck, b10);
          const float2 t01 = rot(ck, b01, sk, b11), t11 = rot(sk, b01, nck, b11);
          b00 = t00; b01 = t01; b10 = t10; b11 = t11;
        }
        P[i00] = b00;
        if (hl) P[i01] = b01;
        if (hk) P[i10] = b10;
        if (hk && hl) P[i11] = b11;
      }
      // eigenvectors: rows p, q of Vt, kVtU elements per thread loaded before any is
      // stored (the rows live in global memory: one round trip per kVtU elements)
      // element e = k m + i of the loop is pair k, row entry i; a thread's elements advance by
      // blockDim.x, i.e. by dk pairs and di entries (no division per element)
      const int dk = blockDim.x / m, di = blockDim.x - dk * m;
      int k_nx = tid / m, i_nx = tid - k_nx * m;
      for (int e0 = tid; e0 < np * m; e0 += kVtU * blockDim.x) {
        float2 vp[kVtU], vq[kVtU];
        int ip[kVtU], iq[kVtU], kk[kVtU];
#pragma unroll
        for (int u = 0; u < kVtU; ++u) {
          const int e = e0 + u * blockDim.x;
          const int k = k_nx, i = i_nx;
          k_nx += dk;
          i_nx += di;
          if (i_nx >= m) { i_nx -= m; ++k_nx; }
          kk[u] = -1;
          if (e < np * m) {
            const int p = pair_s[2 * k], q = pair_s[2 * k + 1];
            if (q < m && cs_s[4 * k + 2] != 0.f) {
              kk[u] = k;
              ip[u] = p * m + i;
              iq[u] = q * m + i;
              vp[u] = Vt[ip[u]];
              vq[u] = Vt[iq[u]];
            }
          }
        }
#pragma unroll
        for (int u = 0; u < kVtU; ++u) {
          if (kk[u] < 0) continue;
          const int k = kk[u];
          const float2 c = make_float2(cs_s[4 * k], cs_s[4 * k + 1]);
          const float2 sn = make_float2(cs_s[4 * k + 2], cs_s[4 * k + 3]);
          const float2 nc = make_float2(-c.x, -c.y);
          Vt[ip[u]] = rot(c, vp[u], sn, vq[u]);
          Vt[iq[u]] = rot(sn, vp[u], nc, vq[u]);
        }
      }
      __syncthreads();
    }
  }
  return sweep;
}

// C = A op(B) for m x m FP64 matrices in global memory (row-major, ld m; op(B) = B, or B^T
// with TB), accumulated as double-floats on the FP32 units: the leading products error-free
// through FMA, the cross terms in FP32, the pair renormalised after every product (about 46
// bits).  64 x 64 output tiles over 16-wide k-slices staged in shared memory as (hi, lo)
// pairs; 512 threads, 2 x 4 outputs each.  sm: (16 * 65 + 16 * 64) float2 of shared memory.
// C must not overlap A or B.
constexpr int kGdTile = 64, kGdK = 16, kGdLdA = kGdTile + 1;
template <bool TB>
__device__ void gemm_df(const double* __restrict__ A, const double* __restrict__ B,
                        double* __restrict__ C, int m, float2* sm) {
  float2* As = sm;                                  // [kGdK][kGdLdA]: As[kk][ii] = A(i0+ii, k0+kk)
  float2* Bs = sm + kGdK * kGdLdA;                  // [kGdK][kGdTile]: Bs[kk][jj] = op(B)(k0+kk, j0+jj)
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;   // ty in 0..31
  const int nt = (m + kGdTile - 1) / kGdTile;
  for (int t = 0; t < nt * nt; ++t) {
    const int i0 = (t / nt) * kGdTile, j0 = (t % nt) * kGdTile;
    float hi[2][4], lo[2][4];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) hi[r][c] = lo[r][c] = 0.f;
    for (int k0 = 0; k0 < m; k0 += kGdK) {
      for (int q = tid; q < kGdK * kGdTile; q += blockDim.x) {
        {   // A: consecutive threads along k (contiguous in memory)
          const int ii = q / kGdK, kk = q - ii * kGdK;
          const int i = i0 + ii, k = k0 + kk;
          As[kk * kGdLdA + ii] = split(i < m && k < m ? A[(size_t)i * m + k] : 0.0);
        }
        if (TB) {   // B^T(k, j) = B(j, k): consecutive threads along k
          const int jj = q / kGdK, kk = q - jj * kGdK;
          const int j = j0 + jj, k = k0 + kk;
          Bs[kk * kGdTile + jj] = split(j < m && k < m ? B[(size_t)j * m + k] : 0.0);
        } else {    // B(k, j): consecutive threads along j
          const int kk = q / kGdTile, jj = q - kk * kGdTile;
          const int j = j0 + jj, k = k0 + kk;
          Bs[kk * kGdTile + jj] = split(j < m && k < m ? B[(size_t)k * m + j] : 0.0);
        }
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < kGdK; ++kk) {
        float2 av[2], bv[4];
#pragma unroll
        for (int r = 0; r < 2; ++r) av[r] = As[kk * kGdLdA + ty + 32 * r];
#pragma unroll
        for (int c = 0; c < 4; ++c) bv[c] = Bs[kk * kGdTile + tx + 16 * c];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float pr = av[r].x * bv[c].x;
            float e = fmaf(av[r].x, bv[c].x, -pr);
            e = fmaf(av[r].x, bv[c].y, fmaf(av[r].y, bv[c].x, e));
            float sh, u;
            slc::two_sum(hi[r][c], pr, sh, u);
            u = u + (lo[r][c] + e);
            hi[r][c] = sh + u;
            lo[r][c] = u - (hi[r][c] - sh);
          }
      }
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = i0 + ty + 32 * r, j = j0 + tx + 16 * c;
        if (i < m && j < m) C[(size_t)i * m + j] = (double)hi[r][c] + (double)lo[r][c];
      }
  }
  __syncthreads();
}

}  // namespace jdf
}  // namespace submat
