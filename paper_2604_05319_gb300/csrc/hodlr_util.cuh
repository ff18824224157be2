// Accessors of the compressed (HODLR) storage: block factors, leaf triangles,
// the near-diagonal band, projection slots, and Sigma^R from whichever
// storage holds an element.
#pragma once
#include "dev_util.cuh"

namespace hk {

constexpr int CHH = 32;     // sweep sub-chunk (the leaf size is a multiple)
constexpr int NWH = 8;      // warps per sweep CTA

template <int NO, typename S>
__device__ __forceinline__ S* Up(const Dev& d, int X, int n, int b, int p) {
  const long long rows = d.b_r1[b] - d.b_r0[b];
  return static_cast<S*>(d.hod[X].U) + ((long long)n * d.utot + d.b_uoff[b] + p * rows) * d.rmax;
}
template <int NO, typename S>
__device__ __forceinline__ S* Vp(const Dev& d, int X, int n, int b, int p) {
  const long long cols = d.b_c1[b] - d.b_c0[b];
  return static_cast<S*>(d.hod[X].V) + ((long long)n * d.vtot + d.b_voff[b] + p * cols) * d.rmax;
}
template <int NO>
__device__ __forceinline__ double* Sp(const Dev& d, int X, int n, int b, int p) {
  return d.hod[X].S + (((long long)n * d.nblk + b) * (NO * NO) + p) * d.rmax;
}
template <int NO>
__device__ __forceinline__ int* Rk(const Dev& d, int X, int n, int b, int p) {
  return d.hod[X].rank + ((long long)n * d.nblk + b) * (NO * NO) + p;
}
// element (t, l) of leaf j of component X (t, l inside the leaf, l <= t)
template <int NO, typename S>
__device__ __forceinline__ S* Lf(const Dev& d, int X, int n, int j, int t, int l) {
  const int A = j * d.L;
  return static_cast<S*>(d.hod[X].leaf) + ((long long)n * d.leaftot + d.leafoff[j] + tri(t - A) + (l - A)) * (NO * NO);
}
template <int NO, typename S>
__device__ __forceinline__ S* Bd(const Dev& d, int n, int t, int dd) {
  return static_cast<S*>(d.band) + (((long long)n * d.nt + t) * d.k + (dd - 1)) * (NO * NO);
}
// sweep projection slots: [n][row/col][maxl][no2][rmax]
template <int NO>
__device__ __forceinline__ double2* Pj(const Dev& d, int n, int which, int lv, int p) {
  return d.proj + ((((long long)n * NO + which) * d.maxl + lv) * (NO * NO) + p) * d.rmax;
}

// Sigma^R(t, l), l <= t, from whichever storage holds it.
template <int NO, typename S>
__device__ __forceinline__ zd sr_any(const Dev& d, int n, int t, int l, int x, int y) {
  if (t >= d.cdir) return ld(el<NO, S>(d.SR, d, n, t, l) + x * NO + y);
  const int jt = t / d.L, jl = l / d.L;
  if (jt == jl) return ld(Lf<NO, S>(d, 2, n, jt, t, l) + x * NO + y);
  for (int lv = 0; lv < d.maxl; ++lv) {
    const int b = d.rowblk[jt * d.maxl + lv];
    if (b < 0 || l < d.b_c0[b] || l >= d.b_c1[b]) continue;
    const int p = x * NO + y, rk = *Rk<NO>(d, 2, n, b, p);
    const S* U = Up<NO, S>(d, 2, n, b, p) + (long long)(t - d.b_r0[b]) * d.rmax;
    const S* V = Vp<NO, S>(d, 2, n, b, p) + (long long)(l - d.b_c0[b]) * d.rmax;
    const double* S = Sp<NO>(d, 2, n, b, p);
    zd s = zd();
    for (int q = 0; q < rk; ++q) s += ld(U + q) * ld(V + q).conj() * S[q];
    return s;
  }
  return zd();
}
template <int NO, typename S>
__device__ __forceinline__ zd srx_any(const Dev& d, int n, int a, int b, int x, int y) {
  if (a >= b) return sr_any<NO, S>(d, n, a, b, x, y);
  return -sr_any<NO, S>(d, n, b, a, y, x).conj();
}


}  // namespace hk
