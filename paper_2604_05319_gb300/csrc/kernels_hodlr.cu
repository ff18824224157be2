// Compressed (HODLR) form of the time step (Sec. 2.2, Fig. 2): the two-time
// components are stored as dense leaf triangles on the diagonal, U S V^dagger
// blocks below them (one scalar TSVD per orbital pair, Sec. 2.3), and a ring
// of the most recent uncompressed rows (the red and green regions: the
// current row and the rows not yet old enough to compress).
//
// History integrals over compressed rows use block projections:
//   retarded row (columns t' of Sigma^R):  pi_B = sum_s y(s) U_B(s,:) S_B,
//     contribution to t' = pi_B . conj(V_B(t',:))
//   lesser column (rows t of Sigma^R):     rho_B = S_B sum_l w_l conj(V_B(l,:)) x(l),
//     contribution to t = U_B(t,:) . rho_B
//   lesser source (Sigma^<, both triangles): each block is used as B and -B^dagger.
// Gregory weights differ from 1 only near the ends (App. A): lower-end weights
// omega_l, l <= k, are folded into the projections; near-diagonal block entries
// (|t - t'| <= k) get an explicit (w - 1) correction from a dense band copy.
//
// update_blocks (Sec. 3.1): whenever a whole leaf of rows is older than k+1
// steps, its rows are appended to every block containing them by a batched
// Brand update: P = R V, E = R - P V^dagger (projected twice), an orthonormal
// basis Q of E's rows by two-pass Gram-Schmidt, the core
// K = [[S, 0], [P, C]] (C = E Q^dagger), its SVD by one-sided Jacobi, truncation
// of singular values below the SVD tolerance (Sec. 2.2), and rotation of U, V.
#include "hodlr_util.cuh"
#include "lattice.cuh"

namespace hk {


// ---------------------------------------------------------------------------
// Lesser source with compressed Sigma^< (two-sided HODLR matvec).
// Stored S[r][c] = Sigma^<(c, r), c <= r.  q(t) = h sum_l w_l Sigma^<(t,l) g_l,
// g_l = [G^R(T,l)]^dagger:  l >= t uses S[l][t] (column t), l < t uses
// -S[t][l]^dagger (row t).
// Projections per (block, pair (x,z), y):
//   P1 = S o sum_{rows l} w_l g_l[z][y] U(l,:),  q(t in cols) += P1 . conj(V(t,:))
//   P2 = S o sum_{cols l} w_l g_l[z][y] V(l,:),  q(t in rows) -= conj(U(t,:)) . P2
// ---------------------------------------------------------------------------
// Slot of P1 (which = 0) or P2 (which = 1), rmax complex values in the bulk
// arithmetic R of the form (FP32 in the complex64 form: the products with the
// factor rows need no conversion), inside a complex128-sized slot.
template <int NO, typename R>
__device__ __forceinline__ cx<R>* Psrc(const Dev& d, int n, int b, int p, int y, int which) {
  return reinterpret_cast<cx<R>*>(d.proj + (long long)d.n_inst * NO * d.maxl * NO * NO * d.rmax +
                                  (((((long long)n * d.nblk + b) * (NO * NO) + p) * NO + y) * 2 + which) * d.rmax);
}

// sum_{q < rk} P[q] conj(F[q]) for one thread: P (bulk type, shared by the
// CTA, cached) and F (a factor row in global memory) with eight loads of F in
// flight rather than one load per term.
template <typename R, typename S>
__device__ __forceinline__ cx<R> lr_dot_conj(const cx<R>* P, const S* F, int rk) {
  cx<R> acc = cx<R>(0);
  for (int q0 = 0; q0 < rk; q0 += 8) {
    cx<R> f[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) f[u] = q0 + u < rk ? ldr<R>(F + q0 + u) : cx<R>(0);
#pragma unroll
    for (int u = 0; u < 8; ++u) acc = cfma(P[q0 + u < rk ? q0 + u : 0], f[u].conj(), acc);
  }
  return acc;
}

template <int NO, typename S>
__global__ void __launch_bounds__(256) k_src_proj(Dev d, int T) {
  constexpr int NO2 = NO * NO;
  using R = typename Bulk<S>::R;
  const int b = blockIdx.x, n = blockIdx.y;
  if (!d.active[n]) return;
  const int c = d.cdir;
  if (d.b_r0[b] >= c) return;
  const int r0 = d.b_r0[b], rl = min(d.b_r1[b], c), c0 = d.b_c0[b], c1 = d.b_c1[b];
  const DevW& W = d.w;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // YB values of y per pass over a factor row (N_o <= 2: all of them), so each
  // factor row is read once per pair and side.
  constexpr int YB = NO <= 2 ? NO : 1;
  // A job is one (side, pair, y-block); it runs on a group of wpj warps (one
  // warp per job when there are at least 8 jobs), the group splitting the
  // job's rows.  Within a warp, lpr = 8, 16 or 32 lanes cover the rank of a
  // factor row (with up to 4 entries per lane: ranks up to 128), so a small
  // rank keeps every lane loading (32 / lpr rows per step).  P1 serves pair p = (x, z) (uses g[z]); P2 serves pair p = (z, x)
  // (uses g[z]); g_l[z][y] = conj(G^R(T,l)[y][z]).
  constexpr int NJOB = NO2 * 2 * (NO / YB);
  constexpr int WPJ = NJOB >= 8 ? 1 : 8 / NJOB;
  constexpr int NGRP = 8 / WPJ;
  __shared__ zd pbuf[WPJ > 1 ? 8 : 1][YB * 128];  // a group's per-warp partial sums
  const int grp = warp / WPJ, wig = warp % WPJ;
  for (int job0 = 0; job0 < NJOB; job0 += NGRP) {
    const int job = job0 + grp;
    const bool act = job < NJOB;
    const int which = job & 1, rest = job >> 1;
    const int yb = (rest % (NO / YB)) * YB, p = act ? rest / (NO / YB) : 0;
    const int z = which == 0 ? p % NO : p / NO;
    const int rk = act ? *Rk<NO>(d, 3, n, b, p) : 0;
    const S* F = which == 0 ? Up<NO, S>(d, 3, n, b, p) : Vp<NO, S>(d, 3, n, b, p);
    const int lo = which == 0 ? r0 : c0, hi = act ? (which == 0 ? rl : c1) : lo;
    const int lpr = rk <= 8 ? 8 : rk <= 16 ? 16 : 32;
    const int rps = 32 / lpr, sub = lane / lpr, q0 = lane % lpr;
    const int stride = WPJ * rps;
    KAcc<R> part[YB][4];   // compensated FP32 sums in the complex64 form
    for (int l0 = lo + wig * rps + sub; l0 < hi; l0 += stride * FOLD) {
      cx<R> pp[YB][4];
#pragma unroll
      for (int yy = 0; yy < YB; ++yy)
#pragma unroll
        for (int u = 0; u < 4; ++u) pp[yy][u] = cx<R>(0);
#pragma unroll
      for (int jj = 0; jj < FOLD; ++jj) {
        const int l = l0 + stride * jj;
        if (l < hi) {
          const R wl = rule_wr<R>(W, T, l);
          const S* gp = el<NO, S>(d.GR, d, n, T, l);
          cx<R> g[YB];
#pragma unroll
          for (int yy = 0; yy < YB; ++yy) g[yy] = ldr<R>(gp + (yb + yy) * NO + z).conj() * wl;
          const S* fr = F + (long long)(l - lo) * d.rmax;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int q = q0 + lpr * u;
            if (q < rk) {
              const cx<R> f = ldr<R>(fr + q);
#pragma unroll
              for (int yy = 0; yy < YB; ++yy) pp[yy][u] = cfma(g[yy], f, pp[yy][u]);
            }
          }
        }
      }
#pragma unroll
      for (int yy = 0; yy < YB; ++yy)
#pragma unroll
        for (int u = 0; u < 4; ++u) part[yy][u].add(pp[yy][u]);
    }
    // the warp's rows combined (every lane calls the shuffles)
#pragma unroll
    for (int yy = 0; yy < YB; ++yy)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const auto r = kacc_lanes(part[yy][u], lpr, 32);
        const int q = q0 + lpr * u;   // < 128
        if (sub == 0 && q < rk) {
          if (WPJ == 1) {
            const zd v = val_of(r) * Sp<NO>(d, 3, n, b, p)[q];
            Psrc<NO, R>(d, n, b, p, yb + yy, which)[q] = cx<R>((R)v.re, (R)v.im);
          } else {
            pbuf[warp][yy * 128 + q] = val_of(r);
          }
        }
      }
    if (WPJ > 1) {   // the group's warps combined: at most one job per group here (NJOB <= 8)
      __syncthreads();
      if (act && wig == 0)
        for (int e = lane; e < YB * rk; e += 32) {
          const int yy = e / rk, q = e % rk;
          zd acc = zd();
          for (int w2 = 0; w2 < WPJ; ++w2) acc += pbuf[grp * WPJ + w2][yy * 128 + q];
          const zd v = acc * Sp<NO>(d, 3, n, b, p)[q];
          Psrc<NO, R>(d, n, b, p, yb + yy, which)[q] = cx<R>((R)v.re, (R)v.im);
        }
      __syncthreads();
    }
  }
}

// q(t) for the compressed columns t < c, one thread per t (adjacent threads
// read adjacent elements of every row).  The weighted G^A(l, T) of the
// uncompressed rows l in [c, T] (at most a leaf plus k+1 rows) is staged in
// shared memory once per block.
constexpr int kSrcRing = 80;   // >= leaf + k + 1 uncompressed rows
template <int NO, typename S>
__global__ void __launch_bounds__(128) k_src_c(Dev d, int T) {
  constexpr int NO2 = NO * NO;
  using R = typename Bulk<S>::R;
  const int n = blockIdx.y;
  if (!d.active[n]) return;
  const int c = d.cdir, L = d.L;
  const DevW& W = d.w;
  __shared__ cx<R> gs[kSrcRing][NO2];  // gs[l - c][z][y] = w_l conj(G^R(T, l)[y][z])
  const int nr = T + 1 - c;
  for (int e = threadIdx.x; e < nr * NO2; e += blockDim.x) {
    const int li = e / NO2, q = e % NO2, z = q / NO, y = q % NO, l = c + li;
    gs[li][q] = ldr<R>(el<NO, S>(d.GR, d, n, T, l) + y * NO + z).conj() * rule_wr<R>(W, T, l);
  }
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= c) return;
  const int jt = t / L, A = jt * L, E = min(A + L, c);
  zd acc[NO2];
#pragma unroll
  for (int q = 0; q < NO2; ++q) acc[q] = zd();
  KAcc<R> ka[NO2];   // the history sums: compensated FP32 in the complex64 form
  cx<R> pa[NO2];
  auto zero = [&]() {
#pragma unroll
    for (int q = 0; q < NO2; ++q) pa[q] = cx<R>(0);
  };
  auto fold = [&]() {
#pragma unroll
    for (int q = 0; q < NO2; ++q) ka[q].add(pa[q]);
    zero();
  };
  // pa[x][y] += sum_z Sx[x][z] g[z][y], Sx = S or S^dagger
  auto mac_g = [&](const S* sp, bool dagS, const cx<R>* g) {
#pragma unroll
    for (int x = 0; x < NO; ++x)
#pragma unroll
      for (int z = 0; z < NO; ++z) {
        const cx<R> sxz = dagS ? ldr<R>(sp + z * NO + x).conj() : ldr<R>(sp + x * NO + z);
#pragma unroll
        for (int y = 0; y < NO; ++y) pa[x * NO + y] = cfma(sxz, g[z * NO + y], pa[x * NO + y]);
      }
  };
  auto gload = [&](int l, cx<R>* g) {  // g[z][y] = w_l conj(G^R(T,l)[y][z])
    const R wl = rule_wr<R>(W, T, l);
    const S* gp = el<NO, S>(d.GR, d, n, T, l);
#pragma unroll
    for (int z = 0; z < NO; ++z)
#pragma unroll
      for (int y = 0; y < NO; ++y) g[z * NO + y] = ldr<R>(gp + y * NO + z).conj() * wl;
  };
  zero();
  // l >= t: Sigma^<(t, l) = S[l][t]; the uncompressed rows [c, T] (coalesced over t)
  for (int l0 = 0; l0 < nr; l0 += FOLD) {
#pragma unroll
    for (int jj = 0; jj < FOLD; ++jj)
      if (l0 + jj < nr) mac_g(el<NO, S>(d.SL, d, n, c + l0 + jj, t), false, gs[l0 + jj]);
    fold();
  }
  // the same leaf, l in [t, E)
  cx<R> g[NO2];
  for (int l0 = t; l0 < E; l0 += FOLD) {
#pragma unroll
    for (int jj = 0; jj < FOLD; ++jj) {
      const int l = l0 + jj;
      if (l < E) {
        gload(l, g);
        mac_g(Lf<NO, S>(d, 3, n, jt, l, t), false, g);
      }
    }
    fold();
  }
  // l < t in the same leaf: -S[t][l]^dagger
  for (int l0 = A; l0 < t; l0 += FOLD) {
#pragma unroll
    for (int jj = 0; jj < FOLD; ++jj) {
      const int l = l0 + jj;
      if (l < t) {
        gload(l, g);
#pragma unroll
        for (int q = 0; q < NO2; ++q) g[q] = -g[q];
        mac_g(Lf<NO, S>(d, 3, n, jt, t, l), true, g);
      }
    }
    fold();
  }
  // blocks with t in their columns (P1 . conj V) and in their rows (-conj U . P2)
  for (int lv = 0; lv < d.maxl; ++lv) {
    const int b = d.colblk[jt * d.maxl + lv];
    if (b < 0 || d.b_r0[b] >= c) continue;
    const int c0 = d.b_c0[b];
#pragma unroll
    for (int p = 0; p < NO2; ++p) {
      const int x = p / NO;
      const int rk = *Rk<NO>(d, 3, n, b, p);
      const S* V = Vp<NO, S>(d, 3, n, b, p) + (long long)(t - c0) * d.rmax;
#pragma unroll
      for (int y = 0; y < NO; ++y) {
        ka[x * NO + y].add(lr_dot_conj<R, S>(Psrc<NO, R>(d, n, b, p, y, 0), V, rk));
      }
    }
  }
  for (int lv = 0; lv < d.maxl; ++lv) {
    const int b = d.rowblk[jt * d.maxl + lv];
    if (b < 0) continue;
    const int r0 = d.b_r0[b];
#pragma unroll
    for (int p = 0; p < NO2; ++p) {  // p = (z, x)
      const int x = p % NO;
      const int rk = *Rk<NO>(d, 3, n, b, p);
      const S* U = Up<NO, S>(d, 3, n, b, p) + (long long)(t - r0) * d.rmax;
#pragma unroll
      for (int y = 0; y < NO; ++y) {
        ka[x * NO + y].add(-lr_dot_conj<R, S>(Psrc<NO, R>(d, n, b, p, y, 1), U, rk));
      }
    }
  }
#pragma unroll
#pragma unroll
  for (int q = 0; q < NO2; ++q) acc[q] += ka[q].get();
  for (int q = 0; q < NO2; ++q) acc[q] = acc[q] * d.h;
  for (int a = 0; a < d.r; ++a) {  // -i sum_a Sigma^tv(t, tau_a) v_a
    const double2* sv = tv<NO>(d.STV, d, n, t, a);
    const double2* vv = d.vvec + ((long long)n * d.r + a) * NO2;
#pragma unroll
    for (int x = 0; x < NO; ++x)
#pragma unroll
      for (int z = 0; z < NO; ++z) {
        const zd sxz = ld(sv + x * NO + z) * zd(0, -1);
#pragma unroll
        for (int y = 0; y < NO; ++y) acc[x * NO + y] = cfma(sxz, ld(vv + z * NO + y), acc[x * NO + y]);
      }
  }
  double2* qp = d.qsrc + ((long long)n * d.nt + t) * NO2;
#pragma unroll
  for (int q = 0; q < NO2; ++q) st(qp + q, acc[q]);
}

// q(t) for the uncompressed rows t in [c, T]: one warp per t (lanes along the row).
template <int NO, typename S>
__global__ void k_src_h(Dev d, int T) {
  constexpr int NO2 = NO * NO;
  using R = typename Bulk<S>::R;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int nrow = T + 1 - d.cdir;
  const int n = gw / nrow, t = d.cdir + gw % nrow;
  if (n >= d.n_inst || !d.active[n]) return;
  const int c = d.cdir, L = d.L;
  const double h = d.h;
  const DevW& W = d.w;
  zd acc[NO2];
#pragma unroll
  for (int q = 0; q < NO2; ++q) acc[q] = zd();
  KAcc<R> ka[NO2];   // the history sums: compensated FP32 in the complex64 form
  const int jt = t / L, A = jt * L, E = min(A + L, d.nt);
  // pa[x][y] += wl sum_z Sx[x][z] conj(G^R(T,l)[y][z]), Sx = S or S^dagger (in R)
  auto sg = [&](cx<R>* pa, const S* sp, bool dagS, const S* gp, R wl) {
#pragma unroll
    for (int x = 0; x < NO; ++x)
#pragma unroll
      for (int z = 0; z < NO; ++z) {
        const cx<R> sxz = (dagS ? ldr<R>(sp + z * NO + x).conj() : ldr<R>(sp + x * NO + z)) * wl;
#pragma unroll
        for (int y = 0; y < NO; ++y) pa[x * NO + y] = cfma(sxz, ldr<R>(gp + y * NO + z).conj(), pa[x * NO + y]);
      }
  };
  auto fold = [&](cx<R>* pa) {
#pragma unroll
    for (int q = 0; q < NO2; ++q) { ka[q].add(pa[q]); pa[q] = cx<R>(0); }
  };
  cx<R> pa[NO2];
#pragma unroll
  for (int q = 0; q < NO2; ++q) pa[q] = cx<R>(0);
  // part 1, l >= t: S[l][t]
  for (int l = max(t, c) + lane; l <= T; l += 32)  // uncompressed rows (at most a leaf and k+8)
    sg(pa, el<NO, S>(d.SL, d, n, l, t), false, el<NO, S>(d.GR, d, n, T, l), rule_wr<R>(W, T, l));
  if (t < c) {
    for (int l = t + lane; l < min(E, c); l += 32)  // same leaf
      sg(pa, Lf<NO, S>(d, 3, n, jt, l, t), false, el<NO, S>(d.GR, d, n, T, l), rule_wr<R>(W, T, l));
  }
  fold(pa);
  for (int lv = 0; lv < d.maxl; ++lv) {  // blocks with t in their columns
    const int b = d.colblk[jt * d.maxl + lv];
    if (b < 0 || d.b_r0[b] >= c) continue;
    const int c0 = d.b_c0[b];
#pragma unroll
    for (int p = 0; p < NO2; ++p) {
      const int x = p / NO;
      const int rk = *Rk<NO>(d, 3, n, b, p);
      const S* V = Vp<NO, S>(d, 3, n, b, p) + (long long)(t - c0) * d.rmax;
#pragma unroll
      for (int y = 0; y < NO; ++y) {
        const cx<R>* P = Psrc<NO, R>(d, n, b, p, y, 0);
        cx<R> sb = cx<R>(0);
        for (int q = lane; q < rk; q += 32) sb = cfma(P[q], ldr<R>(V + q).conj(), sb);
        ka[x * NO + y].add(sb);
      }
    }
  }
  // part 2, l < t: -S[t][l]^dagger
  if (t >= c) {
    for (int l0 = lane; l0 < t; l0 += 32 * FOLD) {  // the whole (uncompressed) row t
#pragma unroll
      for (int jj = 0; jj < FOLD; ++jj) {
        const int l = l0 + 32 * jj;
        if (l < t) sg(pa, el<NO, S>(d.SL, d, n, t, l), true, el<NO, S>(d.GR, d, n, T, l), -rule_wr<R>(W, T, l));
      }
      fold(pa);
    }
  } else {
    for (int l = A + lane; l < t; l += 32)
      sg(pa, Lf<NO, S>(d, 3, n, jt, t, l), true, el<NO, S>(d.GR, d, n, T, l), -rule_wr<R>(W, T, l));
    fold(pa);
    for (int lv = 0; lv < d.maxl; ++lv) {  // blocks with t in their rows
      const int b = d.rowblk[jt * d.maxl + lv];
      if (b < 0) continue;
      const int r0 = d.b_r0[b];
#pragma unroll
      for (int p = 0; p < NO2; ++p) {  // p = (z, x): conj(U^{zx}(t,:)) . P2^{(zx), y} -> q_xy
        const int x = p % NO;
        const int rk = *Rk<NO>(d, 3, n, b, p);
        const S* U = Up<NO, S>(d, 3, n, b, p) + (long long)(t - r0) * d.rmax;
#pragma unroll
        for (int y = 0; y < NO; ++y) {
          const cx<R>* P = Psrc<NO, R>(d, n, b, p, y, 1);
          cx<R> sb = cx<R>(0);
          for (int q = lane; q < rk; q += 32) sb = cfma(ldr<R>(U + q).conj(), P[q], sb);
          ka[x * NO + y].add(-sb);
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NO2; ++q) acc[q] += ka[q].get();
#pragma unroll
  for (int q = 0; q < NO2; ++q) acc[q] = acc[q] * h;
  for (int a = lane; a < d.r; a += 32) {
    M<NO> Sm = load<NO>(tv<NO>(d.STV, d, n, t, a));
    M<NO> V = load<NO>(d.vvec + ((long long)n * d.r + a) * NO2);
    mac<NO>(*reinterpret_cast<M<NO>*>(acc), Sm, V, zd(0, -1));
  }
  warp_sum<NO2>(acc);
  if (lane == 0) {
    double2* p = d.qsrc + ((long long)n * d.nt + t) * NO2;
#pragma unroll
    for (int q = 0; q < NO2; ++q) st(p + q, acc[q]);
  }
}

// ---------------------------------------------------------------------------
// update_blocks: compress the rows [A, A+nb) of every component
// ---------------------------------------------------------------------------
template <int NO, typename S>
__global__ void k_comp_copy(Dev d, int A, int nb) {
  constexpr int NO2 = NO * NO;
  const int n = blockIdx.y;
  if (A + nb + d.k > d.last[n]) return;   // the instance's rows end before this leaf is final
  const int j = A / d.L;
  const long long ntr = (long long)nb * (nb + 1) / 2;
  const long long total = 4 * ntr + (long long)nb * d.k;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    if (idx < 4 * ntr) {
      const int X = (int)(idx / ntr);
      long long e = idx % ntr;
      int i = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
      while ((long long)i * (i + 1) / 2 > e) --i;
      while ((long long)(i + 1) * (i + 2) / 2 <= e) ++i;
      const int l = (int)(e - (long long)i * (i + 1) / 2);
      const int t = A + i, col = A + l;
      const S* src = el<NO, S>(ringX(d, X), d, n, t, col);
      S* dst = Lf<NO, S>(d, X, n, j, t, col);
#pragma unroll
      for (int q = 0; q < NO2; ++q) dst[q] = src[q];
    } else {
      const long long e = idx - 4 * ntr;
      const int t = A + (int)(e / d.k), dd = (int)(e % d.k) + 1;
      S* dst = Bd<NO, S>(d, n, t, dd);
      if (t - dd >= 0) {
        const S* src = el<NO, S>(d.SR, d, n, t, t - dd);
#pragma unroll
        for (int q = 0; q < NO2; ++q) dst[q] = src[q];
      } else {
#pragma unroll
        for (int q = 0; q < NO2; ++q) st(dst + q, zd());
      }
    }
  }
}

// One CTA per (component X, level slot, pair p) x instance.  Workspace per
// CTA (complex doubles): E [nb][ncol], Q [nb][ncol], P [nb][rmax], C [nb][nb],
// K [(rmax+nb)][(rmax+nb)] column-major, Vh [(rmax+nb)][(rmax+nb)] column-major.
//
// FP64 throughout, in both storage forms.  The complex64 form truncates at
// the rounding floor of its stored rows (below), so every step must round
// well below that floor; measured on the C4 batch, FP32 variants of the
// projections (even with FP64 folds), of the residual rows, of the rotation
// of V, or of the core Jacobi each put rounding directions above it and the
// ranks grew to r_max within a few hundred steps.
constexpr double kF32Unit = 5.9604644775390625e-8;  // 2^-24, complex64 unit roundoff

template <int NO, typename S>
__global__ void __launch_bounds__(256) k_tsvd(Dev d, int A, int nb, int n0) {
  constexpr int NO2 = NO * NO;
  const int n = n0 + blockIdx.y;   // instances n0 .. n0 + gridDim.y - 1 share the workspace
  const int X = blockIdx.x / (d.maxl * NO2);
  const int lv = (blockIdx.x / NO2) % d.maxl;
  const int p = blockIdx.x % NO2;
  const int j = A / d.L;
  const int b = d.rowblk[j * d.maxl + lv];
  if (b < 0 || A + nb + d.k > d.last[n]) return;   // the instance's rows end before this leaf is final
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int r0 = d.b_r0[b], c0 = d.b_c0[b];
  const int ncol = d.b_c1[b] - c0;
  const int rmax = d.rmax;
  const int ld_k = rmax + d.L;  // leading dimension of K and Vh
  double2* ws = d.tsvd_ws + (((long long)blockIdx.y * 4 + X) * NO2 + p) * d.tsvd_ws_per + d.ws_lvoff[lv];
  double2* Em = ws;                                   // [nb][ncol]
  double2* Qm = Em + (long long)d.L * ncol;           // [nb][ncol]
  double2* Pm = Qm + (long long)d.L * ncol;           // [nb][rmax]
  double2* Cm = Pm + (long long)d.L * rmax;           // [nb][nb]
  double2* Km = Cm + (long long)d.L * d.L;            // [ld_k cols][ld_k rows]
  double2* Vh = Km + (long long)ld_k * ld_k;          // [ld_k cols][ld_k rows]
  __shared__ int s_rnew;
  __shared__ double s_wpart[32];
  __shared__ double s_sig[256];
  __shared__ int s_ord[256];
  int* rkp = Rk<NO>(d, X, n, b, p);
  const int r = *rkp;
  S* U = Up<NO, S>(d, X, n, b, p);
  S* V = Vp<NO, S>(d, X, n, b, p);
  double* Sv = Sp<NO>(d, X, n, b, p);
  void* ring = ringX(d, X);
  // E <- new rows (and max |E| for the complex64 rounding floor below).  The
  // complex64 form reads them from its FP64 copies: rows free of storage
  // rounding, whose residuals against V hold real directions only.
  double emax = 0.0;
  for (long long e = tid; e < (long long)nb * ncol; e += blockDim.x) {
    const int i = (int)(e / ncol), l = (int)(e % ncol);
    const zd v = d.ring64[X] ? ld(el64<NO>(d, X, n, A + i, c0 + l) + p) : ld(el<NO, S>(ring, d, n, A + i, c0 + l) + p);
    emax = fmax(emax, v.abs2());
    st(Em + (long long)i * ncol + l, v);
  }
  emax = warp_max(emax);
  if (lane == 0) s_wpart[warp] = emax;
  __syncthreads();
  for (int w2 = 0; w2 < nw; ++w2) emax = fmax(emax, s_wpart[w2]);
  emax = sqrt(emax);
  __syncthreads();
  // Truncation threshold: eps_SVD, raised in the complex64 storage form to
  // the rounding floor of the appended rows.  Their rounding is a matrix of
  // independent entries below 2^-24 max|E|, whose largest singular value
  // stays below 2^-24 max|E| (sqrt(nb) + sqrt(ncol)); directions under that
  // level are storage noise, and keeping them would let the rank grow by the
  // leaf size at every append.
  double tol = d.svd_tol;
  if (sizeof(S) == sizeof(float2)) tol = fmax(tol, kF32Unit * emax * (sqrt((double)nb) + sqrt((double)ncol)));
  // P = E V, E -= P V^dagger, twice (the second pass restores orthogonality
  // to V lost to rounding).  The per-pass coefficients are staged in Q's
  // storage (r <= ncol), which is free until the Gram-Schmidt below.
  for (long long e = tid; e < (long long)nb * rmax; e += blockDim.x) Pm[e] = make_double2(0, 0);
  __syncthreads();
  for (int pass = 0; pass < 2 && r > 0; ++pass) {
    for (int e = tid; e < nb * r; e += blockDim.x) {
      const int i = e / r, q = e % r;
      zd sacc = zd();
      for (int l = 0; l < ncol; ++l) sacc = cfma(ld(Em + (long long)i * ncol + l), ld(V + (long long)l * rmax + q), sacc);
      st(Pm + (long long)i * rmax + q, ld(Pm + (long long)i * rmax + q) + sacc);
      st(Qm + (long long)i * ncol + q, sacc);
    }
    __syncthreads();
    for (long long e = tid; e < (long long)nb * ncol; e += blockDim.x) {
      const int i = (int)(e / ncol), l = (int)(e % ncol);
      zd sacc = ld(Em + e);
      for (int q = 0; q < r; ++q) sacc -= ld(Qm + (long long)i * ncol + q) * ld(V + (long long)l * rmax + q).conj();
      st(Em + e, sacc);
    }
    __syncthreads();
  }
  for (long long e = tid; e < (long long)d.L * d.L; e += blockDim.x) Cm[e] = make_double2(0, 0);
  __syncthreads();
  // Two-pass Gram-Schmidt on the rows of E: E = C Q, rows of Q orthonormal.
  // residual rows below a quarter of the threshold add no basis direction
  // (a higher floor, the rounding level of one stored row, rejects rows that
  // are each at noise level but together carry a direction above the
  // threshold: measured on the C4 batch, the ranks then grew about threefold)
  const double delta = 0.25 * tol;
  __shared__ zd s_coef[64];

  // ke, the number of accepted basis rows, is kept in a register: every thread
  // takes the same accept decision from the same (fixed-order) norm.
  int ke = 0;
  for (int i = 0; i < nb; ++i) {
    double2* v = Em + (long long)i * ncol;
    for (int pass = 0; pass < 2; ++pass) {
      for (int e = warp; e < ke; e += nw) {  // coef_e = <Q_e, v>
        const double2* qe = Qm + (long long)e * ncol;
        zd s = zd();
        for (int l = lane; l < ncol; l += 32) s = cfma(ld(qe + l).conj(), ld(v + l), s);
        zd tmp[1] = {s};
        warp_sum<1>(tmp);
        if (lane == 0) s_coef[e] = tmp[0];
      }
      __syncthreads();
      for (int l = tid; l < ncol; l += blockDim.x) {
        zd s = ld(v + l);
        for (int e = 0; e < ke; ++e) s -= s_coef[e] * ld(Qm + (long long)e * ncol + l);
        st(v + l, s);
      }
      if (tid < ke) st(Cm + (long long)i * d.L + tid, ld(Cm + (long long)i * d.L + tid) + s_coef[tid]);
      __syncthreads();
    }
    // norm of the residual
    double part = 0.0;
    for (int l = tid; l < ncol; l += blockDim.x) part += ld(v + l).abs2();
#pragma unroll
    for (int off = 16; off; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if (lane == 0) s_wpart[warp] = part;
    __syncthreads();
    double nsq = 0.0;  // fixed summation order: reproducible bit for bit
    for (int w2 = 0; w2 < nw; ++w2) nsq += s_wpart[w2];
    const double nrm = sqrt(nsq);
    if (nrm > delta) {
      for (int l = tid; l < ncol; l += blockDim.x) st(Qm + (long long)ke * ncol + l, ld(v + l) * (1.0 / nrm));
      if (tid == 0) st(Cm + (long long)i * d.L + ke, zd(nrm));
      ++ke;
    }
    __syncthreads();
  }
  const int m = r + nb, nk = r + ke;  // core rows, columns
  // K = [[diag(S), 0], [P, C]] column-major; Vh = I
  for (long long e = tid; e < (long long)ld_k * ld_k; e += blockDim.x) {
    Km[e] = make_double2(0, 0);
    Vh[e] = make_double2(0, 0);
  }
  __syncthreads();
  for (int e = tid; e < nk * m; e += blockDim.x) {
    const int col = e / m, row = e % m;
    zd v = zd();
    if (row < r) v = (col == row) ? zd(Sv[row]) : zd();
    else if (col < r) v = ld(Pm + (long long)(row - r) * rmax + col);
    else v = ld(Cm + (long long)(row - r) * d.L + (col - r));
    st(Km + (long long)col * ld_k + row, v);
  }
  for (int e = tid; e < nk; e += blockDim.x) st(Vh + (long long)e * ld_k + e, zd(1.0));
  __syncthreads();
  // one-sided Jacobi (Hestenes) on the columns of K, round-robin pairing
  const int npad = nk + (nk & 1);
  __shared__ int s_rot;
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < npad - 1; ++round) {
      for (int pr = warp; pr < npad / 2; pr += nw) {
        // round-robin tournament: position 0 fixed, positions 1..npad-1 rotate
        auto at = [&](int i) { return i == 0 ? 0 : ((i - 1 + round) % (npad - 1)) + 1; };
        int a = at(pr), bq = at(npad - 1 - pr);
        if (a > bq) { const int t2 = a; a = bq; bq = t2; }
        if (bq >= nk) continue;
        double2* ka = Km + (long long)a * ld_k;
        double2* kb = Km + (long long)bq * ld_k;
        double al = 0, be = 0;
        zd ga = zd();
        for (int i = lane; i < m; i += 32) {
          const zd x = ld(ka + i), y = ld(kb + i);
          al += x.abs2();
          be += y.abs2();
          ga = cfma(x.conj(), y, ga);
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, off);
          be += __shfl_xor_sync(0xffffffffu, be, off);
          ga.re += __shfl_xor_sync(0xffffffffu, ga.re, off);
          ga.im += __shfl_xor_sync(0xffffffffu, ga.im, off);
        }
        const double g = sqrt(ga.abs2());
        if (g <= 1e-14 * sqrt(al * be) || g == 0.0) continue;
        if (lane == 0) s_rot = 1;
        const zd ph(ga.re / g, -ga.im / g);  // e^{-i phi}
        const double zeta = (be - al) / (2.0 * g);
        const double tt = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
        for (int i = lane; i < m; i += 32) {
          const zd x = ld(ka + i), y = ld(kb + i) * ph;
          st(ka + i, x * cs - y * sn);
          st(kb + i, x * sn + y * cs);
        }
        double2* va = Vh + (long long)a * ld_k;
        double2* vb = Vh + (long long)bq * ld_k;
        for (int i = lane; i < nk; i += 32) {
          const zd x = ld(va + i), y = ld(vb + i) * ph;
          st(va + i, x * cs - y * sn);
          st(vb + i, x * sn + y * cs);
        }
      }
      __syncthreads();
    }
    if (!s_rot) break;
    if (sweep == 39 && tid == 0) atomicAdd(d.status + 1, 1);
    __syncthreads();
  }
  // singular values, sorted, truncated
  for (int col = warp; col < nk; col += nw) {
    double s2 = 0;
    for (int i = lane; i < m; i += 32) s2 += ld(Km + (long long)col * ld_k + i).abs2();
#pragma unroll
    for (int off = 16; off; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    if (lane == 0) s_sig[col] = sqrt(s2);
  }
  __syncthreads();
  if (tid == 0) {
    for (int i = 0; i < nk; ++i) s_ord[i] = i;
    for (int i = 0; i < nk; ++i) {  // selection sort, descending
      int best = i;
      for (int q = i + 1; q < nk; ++q)
        if (s_sig[s_ord[q]] > s_sig[s_ord[best]]) best = q;
      int t2 = s_ord[i]; s_ord[i] = s_ord[best]; s_ord[best] = t2;
    }
    int rn = 0;
    while (rn < nk && s_sig[s_ord[rn]] > tol) ++rn;
    if (rn > rmax) { atomicAdd(d.status, 1); rn = rmax; }
    s_rnew = rn;
  }
  __syncthreads();
  const int rn = s_rnew;
  // U' = [[U, 0], [0, I]] Uhat : old rows r0..A-1, new rows A..A+nb-1
  const int nold = A - r0;
  for (int row = warp; row < nold + nb; row += nw) {
    S* urow = U + (long long)row * rmax;
    // compute U'[row][j] for j = lane, lane+32, ...
    zd res[4];
    for (int t2 = 0; t2 < 4; ++t2) res[t2] = zd();
    for (int t2 = 0; t2 < 4; ++t2) {
      const int jj = lane + 32 * t2;
      if (jj >= rn) continue;
      const int col = s_ord[jj];
      const double inv = 1.0 / s_sig[col];
      zd s = zd();
      if (row < nold) {
        for (int q = 0; q < r; ++q) s = cfma(ld(urow + q), ld(Km + (long long)col * ld_k + q), s);
      } else {
        s = ld(Km + (long long)col * ld_k + r + (row - nold));
      }
      res[t2] = s * inv;
    }
    __syncwarp();
    for (int t2 = 0; t2 < 4; ++t2) {
      const int jj = lane + 32 * t2;
      if (jj < rmax) st(urow + jj, jj < rn ? res[t2] : zd());
    }
    __syncwarp();
  }
  // V' = [V, Q^H] Vhat
  for (int l = warp; l < ncol; l += nw) {
    S* vrow = V + (long long)l * rmax;
    zd res[4];
    for (int t2 = 0; t2 < 4; ++t2) {
      res[t2] = zd();
      const int jj = lane + 32 * t2;
      if (jj >= rn) continue;
      const int col = s_ord[jj];
      const double2* vh = Vh + (long long)col * ld_k;
      zd s = zd();
      for (int q = 0; q < r; ++q) s = cfma(ld(vrow + q), ld(vh + q), s);
      for (int e = 0; e < ke; ++e) s = cfma(ld(Qm + (long long)e * ncol + l).conj(), ld(vh + r + e), s);
      res[t2] = s;
    }
    __syncwarp();
    for (int t2 = 0; t2 < 4; ++t2) {
      const int jj = lane + 32 * t2;
      if (jj < rmax) st(vrow + jj, jj < rn ? res[t2] : zd());
    }
    __syncwarp();
  }
  __syncthreads();
  for (int q = tid; q < rmax; q += blockDim.x) Sv[q] = (q < rn) ? s_sig[s_ord[q]] : 0.0;
  if (tid == 0) *rkp = rn;
}

// Reconstruct row T of G^R and G^< (any T <= current) into out_r, out_l
// ([T+1][no2] each), from the ring, the leaves or the blocks.
template <int NO, typename S>
__global__ void k_row_out(Dev d, int n, int T, double2* out_r, double2* out_l) {
  constexpr int NO2 = NO * NO;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t > T) return;
  for (int X = 0; X < 2; ++X) {
    double2* out = (X == 0) ? out_r : out_l;
    if (!out) continue;
    for (int p = 0; p < NO2; ++p) {
      zd v;
      if (T >= front_of(d, n)) {
        v = ld(el<NO, S>(ringX(d, X), d, n, T, t) + p);
      } else {
        const int jT = T / d.L, jt = t / d.L;
        if (jT == jt) {
          v = ld(Lf<NO, S>(d, X, n, jT, T, t) + p);
        } else {
          v = zd();
          for (int lv = 0; lv < d.maxl; ++lv) {
            const int b = d.rowblk[jT * d.maxl + lv];
            if (b < 0 || t < d.b_c0[b] || t >= d.b_c1[b]) continue;
            const int rk = *Rk<NO>(d, X, n, b, p);
            const S* U = Up<NO, S>(d, X, n, b, p) + (long long)(T - d.b_r0[b]) * d.rmax;
            const S* V = Vp<NO, S>(d, X, n, b, p) + (long long)(t - d.b_c0[b]) * d.rmax;
            const double* Sv = Sp<NO>(d, X, n, b, p);
            for (int q = 0; q < rk; ++q) v += ld(U + q) * ld(V + q).conj() * Sv[q];
          }
        }
      }
      st(out + (long long)t * NO2 + p, v);
    }
  }
}

// rho(t) = xi i G^<(t, t) of every instance, from a row (dense or ring) or a leaf.
template <int NO, typename S>
__global__ void k_density_at(Dev d, int t, double2* out) {
  constexpr int NO2 = NO * NO;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.n_inst * NO2) return;
  const int n = e / NO2, q = e % NO2;
  if (t > d.last[n]) {   // past the instance's last step
    st(out + e, zd());
    return;
  }
  const S* p = (!d.ring || t >= front_of(d, n)) ? el<NO, S>(d.GL, d, n, t, t) : Lf<NO, S>(d, 1, n, t / d.L, t, t);
  st(out + e, ld(p + q) * zd(0, (double)d.xi));
}


// ---------------------------------------------------------------------------
// 2D Hubbard lattice, second Born (Sec. 4.2), N_o = 1, one instance per
// k = 2 pi (m_x, m_y)/L (instance m_x L + m_y), or, with the reflection
// k_y -> -k_y of a drive along x (Sec. 4.2, the L(L/2+1) k-set), one
// instance per m_y <= L/2 (instance m_x (L/2+1) + m_y; k-point (m_x, L - m_y)
// reads instance (m_x, m_y)).  One CTA per time t of the current row (and
// per DLR node for the mixed row); thread q owns grid point q = m_x L + m_y
// and real-space point r = (q / L, q % L):
//   X_r = (1/N_k) sum_k e^{+i k.r} X_k,  Y_{-r} = (1/N_k) sum_k e^{-i k.r} Y_k,
//   Sigma^>_r = U(T)U(t) G^>_r(T,t)^2 G^<_{-r}(t,T),
//   Sigma^<_r = U(T)U(t) G^<_r(T,t)^2 G^>_{-r}(t,T),
//   Sigma_k = sum_r e^{-i k.r} Sigma_r,  Sigma^R = Sigma^> - Sigma^<;
// mixed: Sigma^tv_r = U(T)U(0_|) G^tv_r(T,tau)^2 G^vt_{-r}(tau,T).
// The 2D transforms are done as two passes of L-point sums (rows, columns).
// ---------------------------------------------------------------------------
template <typename S>
__global__ void __launch_bounds__(kLatMaxK) k_sigma_lattice(Dev d, int T) {
  __shared__ zd X1[kLatMaxK], X2[kLatMaxK], Y1[kLatMaxK], Y2[kLatMaxK], tmp[kLatMaxK], tw[16];
  const int L = (int)d.mpar[0], ys = (int)d.mpar[1], N = L * L, q = threadIdx.x;
  const int nq = lat_inst(q, L, ys);
  lat_twiddles(tw, L);
  const double* U = d.drU;   // U(t) of instance 0 (the same for every k)
  const double invN = 1.0 / N;
  const int b = blockIdx.x;
  __syncthreads();
  if (b <= T) {
    const int t = b;
    if (q < N) {
      const zd gr = ldx<1, S>(d, 0, nq, T, t, 0);
      const zd glc = ldx<1, S>(d, 1, nq, T, t, 0);        // G^<(t, T)
      const zd glr = -glc.conj();                         // G^<(T, t)
      const zd ggr = gr + glr;                            // G^>(T, t)
      X1[q] = ggr; X2[q] = glr; Y1[q] = glc; Y2[q] = -ggr.conj();
    }
    __syncthreads();
    lat_dft2(X1, tmp, tw, L, +1, invN);
    lat_dft2(X2, tmp, tw, L, +1, invN);
    lat_dft2(Y1, tmp, tw, L, -1, invN);
    lat_dft2(Y2, tmp, tw, L, -1, invN);
    const double uu = U[T + 1] * U[t + 1];
    if (q < N) {
      X1[q] = X1[q] * X1[q] * Y1[q] * uu;    // Sigma^>_r
      X2[q] = X2[q] * X2[q] * Y2[q] * uu;    // Sigma^<_r
    }
    __syncthreads();
    lat_dft2(X1, tmp, tw, L, -1, 1.0);
    lat_dft2(X2, tmp, tw, L, -1, 1.0);
    if (q < N && lat_owner(q, L, ys)) {
      stx<1, S>(d, 2, nq, T, t, 0, X1[q] - X2[q]);
      stx<1, S>(d, 3, nq, T, t, 0, -X2[q].conj());
    }
  } else {
    const int i = b - (T + 1), r = d.r;
    if (q < N) {
      X1[q] = ld(tv<1>(d.GTV, d, nq, T, i));
      zd gb = zd();                                        // G^tv(T, beta - tau_i)
      for (int c = 0; c < r; ++c) gb += ld(tv<1>(d.GTV, d, nq, T, c)) * d.rev[i * r + c];
      Y1[q] = gb.conj() * (-(double)d.xi);                 // G^vt(tau_i, T)
    }
    __syncthreads();
    lat_dft2(X1, tmp, tw, L, +1, invN);
    lat_dft2(Y1, tmp, tw, L, -1, invN);
    if (q < N) X1[q] = X1[q] * X1[q] * Y1[q] * (U[T + 1] * U[0]);
    __syncthreads();
    lat_dft2(X1, tmp, tw, L, -1, 1.0);
    if (q < N && lat_owner(q, L, ys)) st(tv<1>(d.STV, d, nq, T, i), X1[q]);
  }
}

// Lattice observables at time t (Sec. 4.2): n = -(i/N) sum_k G^<_k(t,t),
// E_kin = -(2i/N) sum_k eps_k G^<_k(t,t), eps_k = -2(cos k_x + cos k_y),
// j = -(2i/N) sum_k 2 sin(k_x - A(t)) G^<_k(t,t); out = (n, E_kin, j).  The
// sums run over the whole L x L grid (a reflected k-point reads its mirror).
template <typename S>
__global__ void __launch_bounds__(kLatMaxK) k_lattice_obs(Dev d, int t, double* out) {
  __shared__ double red[3][kLatMaxK];
  const int L = (int)d.mpar[0], ys = (int)d.mpar[1], N = L * L, q = threadIdx.x;
  double v[3] = {0, 0, 0};
  if (q < N) {
    const int nq = lat_inst(q, L, ys);
    const S* p = (!d.ring || t >= d.cdir) ? el<1, S>(d.GL, d, nq, t, t) : Lf<1, S>(d, 1, nq, t / d.L, t, t);
    const double mi = (-ld(p) * zd(0, 1)).re;            // Re(-i G^<(t,t))
    const double kx = 2.0 * M_PI * (q / L) / L, ky = 2.0 * M_PI * (q % L) / L;
    const double A = d.drA[t + 1];
    v[0] = mi / N;
    v[1] = 2.0 * (-2.0 * (cos(kx) + cos(ky))) * mi / N;
    v[2] = 2.0 * 2.0 * sin(kx - A) * mi / N;
  }
  for (int c = 0; c < 3; ++c) red[c][q] = v[c];
  __syncthreads();
  if (q == 0) {
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int e = 0; e < N; ++e) s += red[c][e];   // fixed order
      out[c] = s;
    }
  }
}

#define HK_DISPATCH(NOV, CALL)                                                  \
  switch ((NOV) * 2 + d.prec) {                                                 \
    case 2: { constexpr int NO = 1; using S = double2; CALL; break; }           \
    case 3: { constexpr int NO = 1; using S = float2; CALL; break; }            \
    case 4: { constexpr int NO = 2; using S = double2; CALL; break; }           \
    case 5: { constexpr int NO = 2; using S = float2; CALL; break; }            \
    case 6: { constexpr int NO = 3; using S = double2; CALL; break; }           \
    case 7: { constexpr int NO = 3; using S = float2; CALL; break; }            \
    case 8: { constexpr int NO = 4; using S = double2; CALL; break; }           \
    case 9: { constexpr int NO = 4; using S = float2; CALL; break; }            \
    default: return cudaErrorInvalidValue;                                      \
  }

cudaError_t launch_src_h(const Dev& d, int T, cudaStream_t s) {
  if (d.cdir > 0) {
    dim3 g(d.nblk, d.n_inst);
    HK_DISPATCH(d.no, (k_src_proj<NO, S><<<g, 256, 0, s>>>(d, T)));
  }
  if (d.cdir > 0) {
    if (T + 1 - d.cdir > kSrcRing) return cudaErrorInvalidValue;
    dim3 g((d.cdir + 127) / 128, d.n_inst);
    HK_DISPATCH(d.no, (k_src_c<NO, S><<<g, 128, 0, s>>>(d, T)));
  }
  const long long warps = (long long)d.n_inst * (T + 1 - d.cdir);
  HK_DISPATCH(d.no, (k_src_h<NO, S><<<(unsigned)((warps * 32 + 127) / 128), 128, 0, s>>>(d, T)));
  return cudaGetLastError();
}
cudaError_t launch_compress(const Dev& d, int A, int nb, cudaStream_t s) {
  {
    dim3 g(64, d.n_inst);
    HK_DISPATCH(d.no, (k_comp_copy<NO, S><<<g, 256, 0, s>>>(d, A, nb)));
  }
  for (int n0 = 0; n0 < d.n_inst; n0 += d.tsvd_group) {
    dim3 g(4 * d.maxl * d.no * d.no, min(d.tsvd_group, d.n_inst - n0));
    HK_DISPATCH(d.no, (k_tsvd<NO, S><<<g, 256, 0, s>>>(d, A, nb, n0)));
  }
  return cudaGetLastError();
}
cudaError_t launch_density_at(const Dev& d, int t, double2* out, cudaStream_t s) {
  HK_DISPATCH(d.no, (k_density_at<NO, S><<<(d.n_inst * d.no * d.no + 127) / 128, 128, 0, s>>>(d, t, out)));
  return cudaGetLastError();
}
cudaError_t launch_sigma_lattice(const Dev& d, int T, cudaStream_t s) {
  if (d.no != 1 || d.n_inst > kLatMaxK) return cudaErrorInvalidValue;
  if (d.prec) k_sigma_lattice<float2><<<T + 1 + d.r, kLatMaxK, 0, s>>>(d, T);
  else k_sigma_lattice<double2><<<T + 1 + d.r, kLatMaxK, 0, s>>>(d, T);
  return cudaGetLastError();
}
cudaError_t launch_lattice_obs(const Dev& d, int t, double* out, cudaStream_t s) {
  if (d.no != 1 || d.n_inst > kLatMaxK) return cudaErrorInvalidValue;
  if (d.prec) k_lattice_obs<float2><<<1, kLatMaxK, 0, s>>>(d, t, out);
  else k_lattice_obs<double2><<<1, kLatMaxK, 0, s>>>(d, t, out);
  return cudaGetLastError();
}
cudaError_t launch_row_out(const Dev& d, int n, int T, double2* out_r, double2* out_l, cudaStream_t s) {
  HK_DISPATCH(d.no, (k_row_out<NO, S><<<(T + 128) / 128, 128, 0, s>>>(d, n, T, out_r, out_l)));
  return cudaGetLastError();
}

}  // namespace hk
