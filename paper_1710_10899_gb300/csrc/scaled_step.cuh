// Spectrally scaled steps of the coupled iteration (internal header).
//
// The coupled iteration X_{k+1} = X_k T_k, M_{k+1} = T_k^p M_k keeps M_k = X_k^p M_0 for
// any T_k that is a polynomial in M_k (all iterates then commute), so at M = I the iterate
// X is M_0^(-1/p) whatever T_k was used.  Newton's choice T = ((p+1) I - M)/p maps an
// eigenvalue x of M to x ((p+1-x)/p)^p: small eigenvalues grow by only ((p+1)/p)^p per step,
// which is where most steps of a badly scaled start go.
//
// Scaled step: with the spectrum of M_k in [lo, 1], take T = c (alpha I - M).  It maps x to
// c^p g(x), g(x) = x (alpha - x)^p, which rises to its peak at alpha/(p+1) and falls after.
// alpha in (1, p+1) is chosen so that g(lo) = g(1) (the two ends of the interval land on the
// same value, the peak lies between them) and c so that the peak lands on 1; the next
// interval is [g(lo)/g(peak), 1].  As lo -> 1 this tends to Newton (alpha = p+1, c = 1/p).
// lo only steers the speed: an eigenvalue below the assumed lo still grows (by up to
// (c alpha)^p per step), and the invariant above holds for any c and alpha, so the limit and
// the accuracy are those of the plain iteration.
//
// The starting lo comes from a few power steps on I - M_0 (its largest eigenvalue is
// 1 - lambda_min(M_0)); ||(I - M_0) v|| for a unit v never exceeds that eigenvalue, so the
// estimate errs towards a larger lo, which is the safe side; it is then halved.  An
// interval of [1, 1] gives Newton's step, i.e. the plain iteration.
#pragma once
#include "common.cuh"
#include "refine.cuh"

namespace submat {

// The constants only steer the speed, so they are computed in FP32 (cheap on every GPU
// thread; FP64 units are scarce): c and alpha are then exact FP32 numbers.
struct ScaledStep {
  float c, alpha;      // T = c (alpha I - M)
  float lo_next;       // lower end of the spectrum of the next M (upper end 1)
  float tmax;          // c alpha: bound of T's eigenvalues (M's spectrum lies in (0, 1])
  bool newton;         // c = 1/p, alpha = p+1 (to be taken exactly in higher precision)
};

__host__ __device__ inline float step_map(float x, float alpha, int p) {   // x (alpha-x)^p
  float r = x;
  const float t = alpha - x;
  for (int i = 0; i < p; ++i) r *= t;
  return r;
}

constexpr float kLoMin = 1e-4f;     // lower ends below this are treated as this
constexpr float kLoNewton = 1e-3f;  // intervals [lo, 1] with 1 - lo below this take Newton
constexpr int kStartLoSteps = 8;    // power steps for the starting lower end

// g(lo) = g(1) has the closed form alpha = (r - lo) / (r - 1) with r = lo^(-1/p), i.e.
// alpha = 1 + (1 - lo) / expm1(-ln(lo) / p), evaluated without cancellation near lo = 1.
// With alpha_quantum > 0, alpha is rounded to a multiple of it (an engine that applies
// alpha I as an exact integer operand needs that) and c and the next lower end are taken for
// the rounded alpha, so the peak still lands on 1; any alpha keeps the iteration's invariant.
__host__ __device__ inline ScaledStep scaled_step(float lo, int p, float alpha_quantum = 0.f) {
  ScaledStep s;
  if (!(lo >= kLoMin)) lo = kLoMin;
  const float d = 1.f - lo;
  if (d <= kLoNewton) {
    s.newton = true;
    s.c = 1.f / (float)p;
    s.alpha = (float)(p + 1);
    s.tmax = (float)(p + 1) / (float)p;
    // Newton maps [lo, 1] to [lo (1 + d/p)^p, 1]
    float g = lo;
    for (int i = 0; i < p; ++i) g *= 1.f + d / (float)p;
    s.lo_next = fminf(g, 1.f);
    return s;
  }
  s.newton = false;
  const float em = expm1f(-log1pf(-d) / (float)p);
  float alpha = 1.f + d / em;
  if (alpha_quantum > 0.f)     // (alpha stays above 1, where g(1) would vanish)
    alpha = fmaxf(rintf(alpha / alpha_quantum), 1.f / alpha_quantum + 1.f) * alpha_quantum;
  const float peak = step_map(alpha / (float)(p + 1), alpha, p);
  s.alpha = alpha;
  s.c = powf(peak, -1.f / (float)p);
  // g(lo) = g(1) unless alpha was rounded: the lower of the two ends
  s.lo_next = fminf(fminf(step_map(lo, alpha, p), step_map(1.f, alpha, p)) / peak, 1.f);
  s.tmax = s.c * alpha;
  return s;
}

// Bound of the eigenvalues of T^i M (1 <= i < p) for M's spectrum in (0, 1]:
// max over x in (0, 1] of c^i x (alpha - x)^i.
__host__ __device__ inline float partial_bound(const ScaledStep& s, int i) {
  const float x = fminf(s.alpha / (float)(i + 1), 1.f);
  float r = x;
  const float t = s.c * (s.alpha - x);
  for (int k = 0; k < i; ++k) r *= t;
  return r;
}

// Lower end of M_0 = S / lam's spectrum: power steps on I - M_0 from a fixed +-1 vector
// (the raw estimate; callers steer with half of it).
// S: FP64 m x m (ld m).  a_s, b_s: shared vectors of m doubles.  All threads call it.
__device__ inline float start_lo(const double* S, int m, double inv_lam, double* a_s,
                                  double* b_s, double* red_s, int steps) {
  const int tid = threadIdx.x;
  for (int i = tid; i < m; i += blockDim.x) a_s[i] = (i % 3 == 0) ? 1.0 : -1.0;
  __syncthreads();
  double nv = block_norm2(a_s, m, red_s);
  for (int i = tid; i < m; i += blockDim.x) a_s[i] /= nv;
  __syncthreads();
  DenseLoad Sl{S, m};
  double nb = 1.0;
  for (int t = 0; t < steps; ++t) {
    matvec_rows(Sl, inv_lam, a_s, b_s, m);                    // b = M_0 a
    for (int i = tid; i < m; i += blockDim.x) b_s[i] = a_s[i] - b_s[i];
    __syncthreads();
    nb = block_norm2(b_s, m, red_s);                           // ||(I - M_0) a||
    if (nb == 0.0) return 1.f;     // a lies in M_0's eigenvalue 1 (m = 1): plain Newton steps
    if (!(nb > 0.0)) break;
    for (int i = tid; i < m; i += blockDim.x) a_s[i] = b_s[i] / nb;
    __syncthreads();
  }
  double lo = 1.0 - nb;
  if (!(lo == lo)) lo = kLoMin;
  return (float)lo;
}

}  // namespace submat
