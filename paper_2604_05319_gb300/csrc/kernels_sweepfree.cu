// The sweep-free variant of a time step's retarded row and lesser column
// (dense FP64 storage).  Not the paper's discretisation: every point of the
// row or column is an independent small solve or a quadrature over stored
// history, so no point waits for its neighbour.
//
// Retarded row T:
//   t' = T-1 .. T-k: the start block of Eq. KBER (k N_o unknowns of the row
//     solved together per orbital row, as in the paper's scheme);
//   t' = T - n, n > k: the retarded Dyson equation in its first time
//     argument at t = T, BDF over the rows T - j,
//     (i/h) sum_j a_j G^R(T-j,t') = eps(T) G^R(T,t') + h sum_{l<=n} w^(n)_l Sigma^R(T,t'+l) G^R(t'+l,t'),
//     the unknown entering through a_0 and l = n: one N_o x N_o solve per t'.
// Lesser column T (the resolvent form of Eq. KBEL's Volterra equation in its
// first argument):
//   G^<(t,T) = i G^R(t,0) G^<(0,T) + h sum_l w^(t)_l G^R_x(t,l) q_l,  t = 1..T
//   (T - 1 with the diagonal density-matrix scheme), q the lesser source,
//   G^R_x(t,l) = -[G^R(l,t)]^dagger above the diagonal (start weights, t < k).
#include <cuda_runtime.h>

#include "hodlr_util.cuh"
#include "sweepfree.h"

namespace hk {
namespace {

// Start block: one warp per (orbital row irow, instance), y_s = G^R(T, T-s)
// for s = 1..k from the k N_o x k N_o system with the weights D and I_{0,s,l}
// of Appendix A, and y_0 = G^R(T,T) = -i.
template <int NO>
__global__ void __launch_bounds__(32) k_ret_sf_start(Dev d, int T) {
  using S = double2;
  const int irow = blockIdx.x, n = blockIdx.y, lane = threadIdx.x;
  if (!d.active[n]) return;
  const int k = d.k, ns = k * NO;
  const double h = d.h;
  const DevW& W = d.w;
  __shared__ zd sA[20 * 20];
  __shared__ zd sB[20];
  for (int e = lane; e < ns * ns; e += 32) {
    const int row = e / ns, col = e % ns;
    const int s = row / NO + 1, j = row % NO, l = col / NO + 1, m = col % NO;
    zd v = srx_any<NO, S>(d, n, T - l, T - s, m, j) * (-h * W.I0[s][l]);
    if (m == j) v += zd(0, W.D[s][l] / h);
    if (l == s) v -= ld(epsp<NO>(d, n, T - s) + m * NO + j);
    sA[row * ns + col] = v;
  }
  for (int row = lane; row < ns; row += 32) {
    const int s = row / NO + 1, j = row % NO;
    zd c = srx_any<NO, S>(d, n, T, T - s, irow, j) * (-h * W.I0[s][0]);
    if (irow == j) c += zd(0, W.D[s][0] / h);
    sB[row] = zd(0, 1) * c;
  }
  __syncwarp();
  warp_lu_solve(ns, sA, sB, 1, nullptr);
  double err = 0.0;
  for (int row = lane; row < ns; row += 32) {
    const int s = row / NO + 1, j = row % NO;
    double2* p = el<NO, S>(d.GR, d, n, T, T - s) + irow * NO + j;
    err = fmax(err, sqrt((sB[row] - ld(p)).abs2()));
    st(p, sB[row]);
  }
  if (lane < NO) {
    double2* p = el<NO, S>(d.GR, d, n, T, T) + irow * NO + lane;
    const zd v = lane == irow ? zd(0, -1) : zd();
    err = fmax(err, sqrt((v - ld(p)).abs2()));
    st(p, v);
  }
  err = warp_max(err);
  if (lane == 0 && err > 0) atomic_max_nonneg(d.err + n, err);
}

// t' = T - n, n > k: one thread per (t', instance).  The threads of a block
// walk the rows s from the block's first t' upward together, so at each s they
// read the adjacent entries G^R(s, t') of one stored row and one broadcast
// Sigma^R(T, s); a thread adds its terms from s = t' on.
template <int NO>
__global__ void __launch_bounds__(128) k_ret_sf_far(Dev d, int T) {
  using S = double2;
  constexpr int NO2 = NO * NO;
  const int n = blockIdx.y;
  if (!d.active[n]) return;
  const int k = d.k, tp0 = blockIdx.x * blockDim.x, tp = tp0 + threadIdx.x;
  const int last = T - k - 1;                    // t' <= T - k - 1, i.e. n > k
  if (tp0 > last) return;
  const double h = d.h;
  const DevW& W = d.w;
  const bool mine = tp <= last;
  const int nn = T - tp;
  M<NO> acc = M<NO>::zero();
  if (mine) {
    for (int j = 1; j <= k; ++j) {               // -(i a_j / h) G^R(T-j, t')
      const M<NO> g = load<NO>(el<NO, S>(d.GR, d, n, T - j, tp));
      const double c = W.ah[j];
#pragma unroll
      for (int q = 0; q < NO2; ++q) {
        zd& a = acc.a[q / NO][q % NO];
        const zd& v = g.a[q / NO][q % NO];
        a = zd(fma(c, v.im, a.re), fma(-c, v.re, a.im));
      }
    }
  }
  for (int s = tp0; s < T; ++s) {                 // h sum_{l<n} w^(n)_l Sigma^R(T,s) G^R(s,t'), s = t'+l
    if (!mine || s < tp) continue;
    const M<NO> sg = load<NO>(el<NO, S>(d.SR, d, n, T, s));
    const M<NO> g = load<NO>(el<NO, S>(d.GR, d, n, s, tp));
    mac<NO>(acc, sg, g, zd(h * rule_w(W, nn, s - tp)));
  }
  if (!mine) return;
  const M<NO> st_ = load<NO>(el<NO, S>(d.SR, d, n, T, T));
  const double2* ep = epsp<NO>(d, n, T);
  const double wn = h * rule_w(W, nn, nn);
  M<NO> Mm;
#pragma unroll
  for (int x = 0; x < NO; ++x)
#pragma unroll
    for (int y = 0; y < NO; ++y)
      Mm.a[x][y] = (x == y ? zd(0, W.ah[0]) : zd()) - ld(ep + x * NO + y) - st_.a[x][y] * wn;
  const M<NO> X = solve_left<NO>(Mm, acc);
  double2* p = el<NO, S>(d.GR, d, n, T, tp);
  const M<NO> old = load<NO>(p);
  store<NO>(p, X);
  atomic_max_nonneg(d.err + n, maxabs_diff<NO>(X, old));
}

// Lesser column: one warp per (t, instance), lanes over the quadrature points l.
template <int NO>
__global__ void __launch_bounds__(128) k_les_sf(Dev d, int T, int last) {
  using S = double2;
  constexpr int NO2 = NO * NO;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int n = blockIdx.y, t = gw;
  if (t > last || !d.active[n]) return;
  const int k = d.k;
  const double h = d.h;
  const DevW& W = d.w;
  const M<NO> x0 = load<NO>(d.x0 + (long long)n * NO2);   // G^<(0, T) = -[G^tv(T, 0+)]^dagger
  M<NO> X;
  if (t == 0) {
    X = x0;
  } else {
    const double2* q = d.qsrc + (long long)n * d.nt * NO2;
    const int nl = max(t, k) + 1;
    zd acc[NO2];
#pragma unroll
    for (int e = 0; e < NO2; ++e) acc[e] = zd();
    for (int l = lane; l < nl; l += 32) {
      M<NO> g;
      if (l <= t) {
        g = load<NO>(el<NO, S>(d.GR, d, n, t, l));
      } else {                                     // -[G^R(l, t)]^dagger
        const M<NO> u = load<NO>(el<NO, S>(d.GR, d, n, l, t));
#pragma unroll
        for (int x = 0; x < NO; ++x)
#pragma unroll
          for (int y = 0; y < NO; ++y) g.a[x][y] = -u.a[y][x].conj();
      }
      const M<NO> ql = load<NO>(q + (long long)l * NO2);
      const double wl = h * rule_w(W, t, l);
#pragma unroll
      for (int x = 0; x < NO; ++x)
#pragma unroll
        for (int z = 0; z < NO; ++z) {
          const zd gx = g.a[x][z] * wl;
#pragma unroll
          for (int y = 0; y < NO; ++y) acc[x * NO + y] = cfma(gx, ql.a[z][y], acc[x * NO + y]);
        }
    }
    warp_sum<NO2>(acc);
    if (lane != 0) return;
    const M<NO> g0 = load<NO>(el<NO, S>(d.GR, d, n, t, 0));   // + i G^R(t, 0) x_0
#pragma unroll
    for (int x = 0; x < NO; ++x)
#pragma unroll
      for (int y = 0; y < NO; ++y) {
        zd s = zd();
#pragma unroll
        for (int z = 0; z < NO; ++z) s = cfma(g0.a[x][z], x0.a[z][y], s);
        X.a[x][y] = acc[x * NO + y] + zd(-s.im, s.re);
      }
  }
  if (lane != 0) return;
  double2* p = el<NO, S>(d.GL, d, n, T, t);
  const M<NO> old = load<NO>(p);
  store<NO>(p, X);
  atomic_max_nonneg(d.err + n, maxabs_diff<NO>(X, old));
}

#define SF_DISPATCH(CALL)                                  \
  switch (d.no) {                                          \
    case 1: { constexpr int NO = 1; CALL; break; }         \
    case 2: { constexpr int NO = 2; CALL; break; }         \
    case 3: { constexpr int NO = 3; CALL; break; }         \
    case 4: { constexpr int NO = 4; CALL; break; }         \
    default: return cudaErrorInvalidValue;                 \
  }

}  // namespace

cudaError_t launch_ret_sf(const Dev& d, int T, cudaStream_t s) {
  if (d.ring || d.prec || d.k * d.no > 20 || T <= d.k) return cudaErrorInvalidValue;
  SF_DISPATCH((k_ret_sf_start<NO><<<dim3(d.no, d.n_inst), 32, 0, s>>>(d, T)));
  const int nfar = T - d.k;                       // t' = 0 .. T - k - 1
  if (nfar > 0) SF_DISPATCH((k_ret_sf_far<NO><<<dim3((nfar + 127) / 128, d.n_inst), 128, 0, s>>>(d, T)));
  return cudaGetLastError();
}

cudaError_t launch_les_sf(const Dev& d, int T, cudaStream_t s) {
  if (d.ring || d.prec || T <= d.k) return cudaErrorInvalidValue;
  const int last = d.rho_mode == 1 ? T - 1 : T;
  const int warps = last + 1;                     // t = 0 .. last
  SF_DISPATCH((k_les_sf<NO><<<dim3((warps * 32 + 127) / 128, d.n_inst), 128, 0, s>>>(d, T, last)));
  return cudaGetLastError();
}

}  // namespace hk
