// Device helpers shared by the dense and the compressed (HODLR) kernels:
// indexing, Appendix A integration rule, warp reductions, small solves.
#pragma once
#include "common.cuh"
#include "state.h"

namespace hk {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ long long tri(int T) { return (long long)T * (T + 1) / 2; }

// First uncompressed row of instance n.  An instance whose last step comes
// before N_t - 1 stops taking part in the compression once its rows end: its
// front freezes at the last whole leaf of rows older than k + 1 steps, and
// the rows after it stay in their ring slots, which no later kernel writes.
__device__ __forceinline__ int front_of(const Dev& d, int n) {
  const int lk = d.last[n] - d.k;
  const int fz = lk >= d.L ? (lk / d.L) * d.L : 0;
  return d.cdir < fz ? d.cdir : fz;
}

__device__ __forceinline__ void* ringX(const Dev& d, int X) {
  return X == 0 ? d.GR : X == 1 ? d.GL : X == 2 ? d.SR : d.SL;
}

// Row T of a two-time component: the dense lower triangle, or (compressed
// storage) the ring of uncompressed rows, slot T mod ring.
// S is the storage element type (double2 or float2).
template <int NO, typename S>
__device__ __forceinline__ S* el(void* base, const Dev& d, int n, int T, int t) {
  S* b = static_cast<S*>(base);
  if (d.ring) return b + (((long long)n * d.ring + (T % d.ring)) * d.nt + t) * (NO * NO);
  return b + ((long long)n * d.ntri + tri(T) + t) * (NO * NO);
}
// FP64 copy of element (T, t) of component X (complex64 compressed form).
template <int NO>
__device__ __forceinline__ double2* el64(const Dev& d, int X, int n, int T, int t) {
  return d.ring64[X] + (((long long)n * d.ring + (T % d.ring)) * d.nt + t) * (NO * NO);
}
// Entry q of element (T, t) of component X in FP64: from the FP64 copy when
// there is one (and it is seeded), else from the storage.
template <int NO, typename S>
__device__ __forceinline__ zd ldx(const Dev& d, int X, int n, int T, int t, int q) {
  if (d.ring64[X] && d.use64) return ld(el64<NO>(d, X, n, T, t) + q);
  return ld(el<NO, S>(ringX(d, X), d, n, T, t) + q);
}
// Write entry q of element (T, t) of component X: the storage (rounded in the
// complex64 form) and the FP64 copy.
template <int NO, typename S>
__device__ __forceinline__ void stx(const Dev& d, int X, int n, int T, int t, int q, const zd& v) {
  st(el<NO, S>(ringX(d, X), d, n, T, t) + q, v);
  if (d.ring64[X]) st(el64<NO>(d, X, n, T, t) + q, v);
}

// Mixed components G^tv, Sigma^tv: complex128 in both precision forms (their
// DLR convolution is ill-conditioned; they are r/T times smaller than a row set).
template <int NO>
__device__ __forceinline__ double2* tv(void* base, const Dev& d, int n, int T, int i) {
  return static_cast<double2*>(base) + (((long long)n * d.nt + T) * d.r + i) * (NO * NO);
}
template <int NO>
__device__ __forceinline__ double2* epsp(const Dev& d, int n, int t) {  // eps(t), t >= -1
  return d.eps + ((long long)n * (d.nt + 1) + (t + 1)) * (NO * NO);
}

__device__ __forceinline__ double rule_w(const DevW& w, int n, int l) {
  const int k = w.k;
  if (n <= 0) return 0.0;
  if (n <= k) return (l >= 0 && l <= k) ? w.I0[n][l] : 0.0;
  if (n < 2 * k + 1) {
    double s = 0.0;
    if (l >= 0 && l <= k) s += w.I0[n - k][l];
    if (l >= n - k && l <= n) s += w.I0[k][l - (n - k)];
    return s;
  }
  if (l < 0 || l > n) return 0.0;
  if (l <= k) return w.omega[l];
  if (l >= n - k) return w.omega[n - l];
  return 1.0;
}

// The same rule in the arithmetic R of the bulk sums (float tables for float).
template <typename R>
__device__ __forceinline__ R rule_wr(const DevW& w, int n, int l) {
  if constexpr (sizeof(R) == sizeof(double)) {
    return rule_w(w, n, l);
  } else {
    const int k = w.k;
    if (n <= 0) return 0.0f;
    if (n <= k) return (l >= 0 && l <= k) ? w.I0f[n][l] : 0.0f;
    if (n < 2 * k + 1) {
      float s = 0.0f;
      if (l >= 0 && l <= k) s += w.I0f[n - k][l];
      if (l >= n - k && l <= n) s += w.I0f[k][l - (n - k)];
      return s;
    }
    if (l < 0 || l > n) return 0.0f;
    if (l <= k) return w.omegaf[l];
    if (l >= n - k) return w.omegaf[n - l];
    return 1.0f;
  }
}

constexpr int FOLD = 8;  // terms summed in R before they enter the compensated accumulator

__device__ __forceinline__ zd wshfl(zd v, int off) {
  return zd(__shfl_xor_sync(FULL, v.re, off), __shfl_xor_sync(FULL, v.im, off));
}
template <int L>
__device__ __forceinline__ void warp_sum(zd (&v)[L]) {
#pragma unroll
  for (int off = 16; off; off >>= 1)
#pragma unroll
    for (int i = 0; i < L; ++i) v[i] += wshfl(v[i], off);
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int off = 16; off; off >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, off));
  return v;
}

// Sigma^R(a, b) continued above the diagonal: -[Sigma^R(b, a)]^dagger for a < b.
template <int NO, typename S>
__device__ __forceinline__ zd srx(const Dev& d, int n, int a, int b, int x, int y) {
  if (a >= b) return ld(el<NO, S>(d.SR, d, n, a, b) + x * NO + y);
  return -ld(el<NO, S>(d.SR, d, n, b, a) + y * NO + x).conj();
}
// Sigma^<(t, l) anywhere (Eq. GLantiHerm)
template <int NO, typename S>
__device__ __forceinline__ zd sless(const Dev& d, int n, int t, int l, int x, int y) {
  if (t <= l) return ld(el<NO, S>(d.SL, d, n, l, t) + x * NO + y);
  return -ld(el<NO, S>(d.SL, d, n, t, l) + y * NO + x).conj();
}

// ---------------------------------------------------------------------------
// Warp-parallel dense solve A X = B (n <= 32, nrhs <= 32), A and B in shared
// memory, LU with partial pivoting; lane r owns row r during elimination.
// With nrhs = 0 it only factors (L below the diagonal, row swaps in piv).
// ---------------------------------------------------------------------------
static __device__ __noinline__ void warp_lu_solve(int n, zd* A, zd* B, int nrhs, int* piv) {
  const int lane = threadIdx.x & 31;
  for (int c = 0; c < n; ++c) {
    double v = (lane >= c && lane < n) ? A[lane * n + c].abs2() : -1.0;
    int p = lane;
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      double v2 = __shfl_xor_sync(FULL, v, off);
      int p2 = __shfl_xor_sync(FULL, p, off);
      if (v2 > v || (v2 == v && p2 < p)) { v = v2; p = p2; }
    }
    if (piv && lane == 0) piv[c] = p;
    if (p != c) {
      for (int j = lane; j < n; j += 32) { zd t = A[c * n + j]; A[c * n + j] = A[p * n + j]; A[p * n + j] = t; }
      for (int j = lane; j < nrhs; j += 32) { zd t = B[c * nrhs + j]; B[c * nrhs + j] = B[p * nrhs + j]; B[p * nrhs + j] = t; }
    }
    __syncwarp();
    if (lane > c && lane < n) {
      zd f = cdiv(A[lane * n + c], A[c * n + c]);
      A[lane * n + c] = f;
      for (int j = c + 1; j < n; ++j) A[lane * n + j] -= f * A[c * n + j];
      for (int j = 0; j < nrhs; ++j) B[lane * nrhs + j] -= f * B[c * nrhs + j];
    }
    __syncwarp();
  }
  for (int j = lane; j < nrhs; j += 32)
    for (int c = n - 1; c >= 0; --c) {
      zd s = B[c * nrhs + j];
      for (int m = c + 1; m < n; ++m) s -= A[c * n + m] * B[m * nrhs + j];
      B[c * nrhs + j] = cdiv(s, A[c * n + c]);
    }
  __syncwarp();
}
// Solve with a factor from warp_lu_solve(nrhs = 0) for one right-hand side b.
__device__ __forceinline__ void lu_apply(int n, const zd* A, const int* piv, zd* b) {
  for (int c = 0; c < n; ++c)
    if (piv[c] != c) { zd t = b[c]; b[c] = b[piv[c]]; b[piv[c]] = t; }
  for (int c = 0; c < n; ++c)
    for (int r = c + 1; r < n; ++r) b[r] -= A[r * n + c] * b[c];
  for (int c = n - 1; c >= 0; --c) {
    zd s = b[c];
    for (int m = c + 1; m < n; ++m) s -= A[c * n + m] * b[m];
    b[c] = cdiv(s, A[c * n + c]);
  }
}

// small vector solves: y M = r (row vector) and M x = r (column vector)
template <int NO>
__device__ void solve_row(const M<NO>& Mm, const zd* r, zd* y) {
  M<NO> B = M<NO>::zero();
#pragma unroll
  for (int j = 0; j < NO; ++j) B.a[0][j] = r[j];
  M<NO> X = solve_right<NO>(Mm, B);
#pragma unroll
  for (int j = 0; j < NO; ++j) y[j] = X.a[0][j];
}
template <int NO>
__device__ void solve_col(const M<NO>& Mm, const zd* r, zd* x) {
  M<NO> B = M<NO>::zero();
#pragma unroll
  for (int j = 0; j < NO; ++j) B.a[j][0] = r[j];
  M<NO> X = solve_left<NO>(Mm, B);
#pragma unroll
  for (int j = 0; j < NO; ++j) x[j] = X.a[j][0];
}

__device__ __forceinline__ double fermi(double e, double beta) { return 0.5 * (1.0 - tanh(0.5 * beta * e)); }

}  // namespace hk
