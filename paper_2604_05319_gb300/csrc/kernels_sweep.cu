// The two Volterra sweeps of a time step (Eq. KBER retarded row, Eq. KBEL
// lesser column) for both storage forms (dense triangles, or HODLR with a
// ring of uncompressed rows), organised in 32-point chunks at fixed absolute
// positions.
//
// Within one chunk the unknowns couple through the near-diagonal part of the
// discretised equation: the BDF stencil, eps, and Sigma^R entries inside the
// chunk with their Gregory weights.  Once every coefficient of that local
// system is final and its weights no longer depend on T, the system is frozen
// and its inverse is computed once (k_chunk_inv) and reused at every later
// iteration and step:
//   retarded chunk [a, a+32): frozen when a + 32 + 2k <= T (all points see the
//     standard Gregory weights at their end of the integral, and no row of the
//     chunk is within k of T);
//   lesser chunk [a, a+32): frozen when a + 32 <= T (its rows are final; the
//     lesser weights depend on the row and column only).  Chunk 0 holds rows
//     1..31 including the start block.
// A chunk's solve is then F times the inverse (retarded, row vector) or the
// inverse times F (lesser), where F holds everything outside the chunk (the
// far field).  Only the chunks near T are solved point by point in one warp.
#include "bulk_copy.cuh"
#include "hodlr_util.cuh"

namespace hk {

namespace {

constexpr int CK = 32;   // chunk length
using Y = double2;       // element type of the row / column being solved
template <int NO> constexpr bool kStage = NO <= 2;   // hot-chunk coefficients staged in shared memory
template <int NO> constexpr size_t kStageBytes = kStage<NO> ? sizeof(zd) * CK * CK * NO * NO : 0;
// Bytes of a frozen chunk inverse that are staged in shared memory (the
// dynamic buffer of the hot-chunk coefficients, free while a frozen chunk is
// solved) by a bulk copy issued before the chunk's far field, so the copy
// overlaps that phase: the whole inverse (FP64, or the hi and lo matrices of
// the complex64 form, 16 bytes per entry either way); 0 (read from global
// memory) for N_o > 2.
template <int NO, typename S>
constexpr uint32_t kInvStage = kStage<NO> ? (uint32_t)(CK * NO * CK * NO * sizeof(double2)) : 0u;
static_assert(kInvStage<2, double2> <= kStageBytes<2> && kInvStage<1, double2> <= kStageBytes<1>,
              "a staged inverse must fit the hot-chunk buffer");
constexpr int kCopyWaitPolls = 1 << 20;   // bound of the wait for a staged inverse

// Sum over the 8 lanes of an aligned lane group of their history
// accumulators (every lane receives it).  Complex64 form: the compensated
// FP32 sums are combined in float-float, so the reduction runs on the FP32
// pipes; FP64 form: plain FP64.  val_of converts to FP64 (once, by the lane
// that uses the sum).
template <typename R>
__device__ __forceinline__ auto reduce8(const KAcc<R>& k) { return kacc_lanes(k, 1, 8); }

// Where a sweep keeps the row it solves: in place (FP64 storage), or in FP64
// next to the complex64 storage: the row's slot of the FP64 ring copies of the
// compressed form (which the TSVD later compresses), else the buffer
// row64[n][which] of the dense form.
template <int NO, typename S>
struct Row64 {
  static constexpr bool separate = true;
  __device__ static Y* get(const Dev& d, int n, int which, int T, S*) {
    if (d.ring64[which]) return el64<NO>(d, which, n, T, 0);
    return d.row64 + ((long long)n * 2 + which) * d.nt * (NO * NO);
  }
};
template <int NO>
struct Row64<NO, double2> {
  static constexpr bool separate = false;
  __device__ static Y* get(const Dev&, int, int, int, double2* p) { return p; }
};

// Inverse of frozen chunk cc of sweep `which`, (32 N_o)^2 entries.  FP64
// storage form: complex128.  Complex64 form: the same 16 bytes per entry
// hold a complex64 pair hi + lo (hi = the inverse rounded to complex64, lo =
// the rounding of hi), [hi matrix][lo matrix].  The chunk's right-hand side
// splits into the far field (history sums, lesser source), whose image under
// the inverse is about h / a_0 times smaller than the row and needs FP32 only,
// and the BDF terms reaching across the chunk edge (k rows), which carry the
// implicit recursion and get hi + lo in float-float (about 48 bits); a plain
// complex64 inverse would put 2^-24 times the BDF amplitude a_j / h into
// every chunk and accumulate.
template <int NO>
__device__ __forceinline__ double2* Cinv(const Dev& d, int n, int cc, int which) {
  const long long nn = (long long)(CK * NO) * (CK * NO);
  return d.cinv + (((long long)n * d.nchunk + cc) * 2 + which) * nn;
}

// Projections of one block of Sigma^R for all N_o^2 orbital pairs in one pass
// (complex64 form, N_o <= 2, rank <= 64): out_p[q] = S_p[q] sum_{l in [l0, l1)}
// v_p(l) F_p(l, q) for q < rank_p, with F = U (ROWS: the retarded sweep, v_p =
// y_m, m = p / N_o) or F = conj(V) (the lesser sweep, v_p = w_l x_nn, nn =
// p % N_o); vf(l, i) returns the vector's component i at l.  A warp covers
// 32 / lpr rows per step, lpr = 8, 16 or 32 lanes per row (the smallest that
// holds the largest rank), so small ranks keep every lane loading; warps split
// the rows, and the pairs share the vector loads.  Partial sums (compensated
// FP32) are combined across a warp's rows in float-float and across warps in
// red ([8][N_o^2][64], shared memory).  Every thread calls it.
template <int NO, typename S, bool ROWS, typename VF>
__device__ __forceinline__ void proj_block(const Dev& d, int n, int blk, int lv, int slot, int l0, int l1, VF vf,
                                           zd* red) {
  constexpr int NO2 = NO * NO;
  using R = typename Bulk<S>::R;
  static_assert(sizeof(R) == sizeof(float), "the one-pass projections serve the complex64 form");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int rk[NO2];
  const S* F[NO2];
  int rkmax = 0;
#pragma unroll
  for (int p = 0; p < NO2; ++p) {
    rk[p] = *Rk<NO>(d, 2, n, blk, p);
    F[p] = ROWS ? Up<NO, S>(d, 2, n, blk, p) : Vp<NO, S>(d, 2, n, blk, p);
    rkmax = max(rkmax, rk[p]);
  }
  const int base = ROWS ? d.b_r0[blk] : d.b_c0[blk];
  const int lpr = rkmax <= 8 ? 8 : rkmax <= 16 ? 16 : 32;   // lanes per row
  const int rps = 32 / lpr, sub = lane / lpr, q0 = lane % lpr;
  const int stride = 8 * rps;                               // rows per CTA step
  KAcc<R> part[NO2][2];
  for (int sb = l0 + warp * rps + sub; sb < l1; sb += stride * FOLD) {
    cx<R> pp[NO2][2];
#pragma unroll
    for (int p = 0; p < NO2; ++p) pp[p][0] = pp[p][1] = cx<R>(0);
#pragma unroll
    for (int jj = 0; jj < FOLD; ++jj) {
      const int l = sb + stride * jj;
      if (l < l1) {
        cx<R> v[NO];
#pragma unroll
        for (int i = 0; i < NO; ++i) v[i] = vf(l, i);
#pragma unroll
        for (int p = 0; p < NO2; ++p) {
          const S* fr = F[p] + (long long)(l - base) * d.rmax;
          const cx<R> vp = v[ROWS ? p / NO : p % NO];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int q = q0 + lpr * u;
            if (q < rk[p]) {
              const cx<R> f = ROWS ? ldr<R>(fr + q) : ldr<R>(fr + q).conj();
              pp[p][u] = cfma(vp, f, pp[p][u]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int p = 0; p < NO2; ++p) {
      part[p][0].add(pp[p][0]);
      part[p][1].add(pp[p][1]);
    }
  }
#pragma unroll
  for (int p = 0; p < NO2; ++p)
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const cff r = kacc_lanes(part[p][u], lpr, 32);
      const int q = q0 + lpr * u;
      if (sub == 0 && q < 64) red[(warp * NO2 + p) * 64 + q] = cff_val(r);
    }
  __syncthreads();
  for (int e = tid; e < NO2 * d.rmax; e += blockDim.x) {
    const int p = e / d.rmax, q = e % d.rmax;
    int rkp = 0;
#pragma unroll
    for (int pp2 = 0; pp2 < NO2; ++pp2)
      if (pp2 == p) rkp = rk[pp2];
    zd acc = zd();
    if (q < rkp)   // entries q >= the pair's rank are not written by every warp
      for (int w2 = 0; w2 < 8; ++w2) acc += red[(w2 * NO2 + p) * 64 + q];
    st(Pj<NO>(d, n, slot, lv, p) + q, q < rkp ? acc * Sp<NO>(d, 2, n, blk, p)[q] : zd());
  }
  __syncthreads();
}

// Sum over q < rk of P[q] * F[q] (or P[q] * conj(F[q])): the far field of one
// compressed block at one row or column, P its projection vector staged in
// shared memory, F the block's factor row in global memory.  Four threads
// share an output (q = sl, sl + 4, ...) and each keeps eight loads of F in
// flight, so the row streams instead of waiting on one load per term.
template <typename R, typename S, bool CONJ>
__device__ __forceinline__ cx<R> lr_dot4(const cx<R>* P, const S* F, int rk, int sl) {
  cx<R> acc = cx<R>(0);
  for (int q0 = sl; q0 < rk; q0 += 32) {
    cx<R> f[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = q0 + 4 * u;
      f[u] = q < rk ? ldr<R>(F + q) : cx<R>(0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) acc = cfma(P[q0 + 4 * u < rk ? q0 + 4 * u : 0], CONJ ? f[u].conj() : f[u], acc);
  }
  return acc;
}

}  // namespace

// ---------------------------------------------------------------------------
// Retarded row, Eq. KBER: unknown y(t') = G^R(T, t') (row irow), solved for
// t' = T-1 .. 0; the start block t' >= T-k is solved together.
// ---------------------------------------------------------------------------
template <int NO, typename S>
__global__ void __launch_bounds__(256, (NO <= 2) ? 2 : 1) k_ret2(Dev d, int T, int staged) {
  constexpr int NO2 = NO * NO;
  using R = typename Bulk<S>::R;
  const int n = blockIdx.y, irow = blockIdx.x;
  if (!d.active[n]) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = d.k, c = d.cdir, L = d.L;
  const double h = d.h;
  const DevW& W = d.w;
  __shared__ zd sA[20 * 20];
  __shared__ zd sB[20];
  __shared__ zd FB[64][NO];
  __shared__ zd pbuf[8][128];
  __shared__ zd Fs[CK][NO];
  __shared__ zd Fb[CK][NO];      // the BDF part of Fs (rows at the chunk edge; zero elsewhere)
  __shared__ zd Old[CK][NO];     // the chunk's previous iterate (convergence measure)
  __shared__ zf Ff[CK][NO];      // complex64 form: the far field (Fs - Fb) rounded to complex64
  __shared__ cff FbF[CK][NO];    // complex64 form: Fb in float-float
  __shared__ double serr;
  extern __shared__ __align__(16) zd ctile[];  // [CK][CK][NO2] hot-chunk coefficients (N_o <= 2);
                                 // at leaf entry (staged != 0) the block projections
                                 // [maxl][NO2][rmax]; for a frozen chunk its staged inverse
  __shared__ __align__(8) uint64_t cbar;   // completion of the inverse's bulk copy
  __shared__ int s_stage;                  // 0 once a wait for a copy has timed out
  uint32_t cphase = 0;
  if (tid == 0) {
    serr = 0.0;
    s_stage = 1;
    if (kInvStage<NO, S>) mbar_init(&cbar);
  }
  // The row being solved lives in FP64 during the sweep (in the complex64
  // storage form a separate buffer), so the point-to-point recursion of the
  // sweep (BDF terms, point solves) does not accumulate storage rounding.
  // yp: the FP64 row; sp: its storage, written at the same time (rounded in
  // the complex64 form), which the FP32 bulk sums read; it holds the previous
  // iterate until an element is overwritten (the convergence measure).
  S* rowp = el<NO, S>(d.GR, d, n, T, 0);
  Y* rowy = Row64<NO, S>::get(d, n, 0, T, rowp);
  auto yp = [&](int tp) { return rowy + (long long)tp * NO2 + irow * NO; };
  auto sp = [&](int tp) { return rowp + (long long)tp * NO2 + irow * NO; };
  double myerr = 0.0;
  // ---- start block t' = T-k .. T-1 (s = 1..k), and y(T) = -i ----
  const int ns = k * NO;
  if (warp == 0) {
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
      zd cc = srx_any<NO, S>(d, n, T, T - s, irow, j) * (-h * W.I0[s][0]);
      if (irow == j) cc += zd(0, W.D[s][0] / h);
      sB[row] = zd(0, 1) * cc;
    }
    __syncwarp();
    warp_lu_solve(ns, sA, sB, 1, nullptr);
    for (int row = lane; row < ns; row += 32) {
      const int s = row / NO + 1, j = row % NO;
      myerr = fmax(myerr, (sB[row] - ld(sp(T - s) + j)).abs2());
      st(yp(T - s) + j, sB[row]);
      if constexpr (Row64<NO, S>::separate) st(sp(T - s) + j, sB[row]);
    }
    if (lane == 0) {
      for (int j = 0; j < NO; ++j) {
        zd v = (j == irow) ? zd(0, -1) : zd();
        myerr = fmax(myerr, (ld(sp(T) + j) - v).abs2());
        st(yp(T) + j, v);
        if constexpr (Row64<NO, S>::separate) st(sp(T) + j, v);
      }
    }
  }
  __syncthreads();
  const int top = T - k - 1;
  for (int cc = top / CK; cc >= 0; --cc) {
    const int a = cc * CK, b = min(a + CK, top + 1), cn = b - a;
    const bool comp = (c > 0 && b <= c);
    const int jl = comp ? a / L : 0, A = jl * L, E = comp ? (jl + 1) * L : 0;
    if (comp && b == E) {
      // Entering leaf jl from above.  (1) projections pi_B = sum_s y(s) U_B(s,:) S_B
      // of the blocks whose columns end at E, rows summed in 4 slices.
      for (int lv = 0; lv < d.maxl; ++lv) {
        const int blk = d.colblk[jl * d.maxl + lv];
        if (blk < 0 || d.b_c1[blk] != E) continue;
        const int r0 = d.b_r0[blk], rl = min(d.b_r1[blk], c);
        if constexpr (kStage<NO> && Row64<NO, S>::separate) {   // complex64 form: all pairs in one
          if (d.rmax <= 64) {                                     // pass (ctile is free here)
            proj_block<NO, S, true>(d, n, blk, lv, irow, r0, rl,
                                    [&](int s2, int m) { return ldr<R>(sp(s2) + m); }, ctile);
            continue;
          }
        }
        for (int p = 0; p < NO2; ++p) {
          const int m = p / NO;
          const int rk = *Rk<NO>(d, 2, n, blk, p);
          const S* U = Up<NO, S>(d, 2, n, blk, p);
          KAcc<R> part[4];
          for (int s0 = r0 + warp; s0 < rl; s0 += 8 * FOLD) {  // warps over rows, lanes over rank
            cx<R> pp[4] = {cx<R>(0), cx<R>(0), cx<R>(0), cx<R>(0)};
#pragma unroll
            for (int jj = 0; jj < FOLD; ++jj) {
              const int s2 = s0 + 8 * jj;
              if (s2 < rl) {
                const cx<R> yv = ldr<R>(sp(s2) + m);
                const S* ur = U + (long long)(s2 - r0) * d.rmax;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  const int q = lane + 32 * u;
                  if (q < rk) pp[u] = cfma(yv, ldr<R>(ur + q), pp[u]);
                }
              }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) part[u].add(pp[u]);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) pbuf[warp][lane + 32 * u] = part[u].get();
          __syncthreads();
          if (tid < d.rmax) {
            zd acc = zd();
            for (int w2 = 0; w2 < 8; ++w2) acc += pbuf[w2][tid];
            st(Pj<NO>(d, n, irow, lv, p) + tid, tid < rk ? acc * Sp<NO>(d, 2, n, blk, p)[tid] : zd());
          }
          __syncthreads();
        }
      }
      __syncthreads();
      // projections of every block over this leaf's columns, staged in shared
      // memory for the far-field loop below (the buffer of the hot-chunk
      // coefficients, which the chunk solves fill only after it)
      cx<R>* Ps = reinterpret_cast<cx<R>*>(ctile);
      if (staged) {
        const int per = NO2 * d.rmax;
        for (int e = tid; e < d.maxl * per; e += blockDim.x) {
          const int lv = e / per, p = (e / d.rmax) % NO2, q = e % d.rmax;
          const int blk = d.colblk[jl * d.maxl + lv];
          Ps[e] = (blk >= 0 && d.b_r0[blk] < c) ? ldr<R>(Pj<NO>(d, n, irow, lv, p) + q) : cx<R>(0);
        }
        __syncthreads();
      }
      // (2) for every column of the leaf: uncompressed rows s in [c, T], the
      // blocks below the leaf (weight 1) and the near-diagonal corrections;
      // 4 threads per column.
      {
        const int col = tid >> 2, sl = tid & 3;
        zd acc[NO];
#pragma unroll
        for (int j = 0; j < NO; ++j) acc[j] = zd();
        KAcc<R> ka[NO];   // FP32 history sums, compensated (FP64 in the FP64 form)
        const int tp = A + col;
        if (col < L) {
          for (int s0 = c + sl; s0 <= T; s0 += 4 * FOLD) {
            cx<R> pa[NO];
#pragma unroll
            for (int j = 0; j < NO; ++j) pa[j] = cx<R>(0);
#pragma unroll
            for (int jj = 0; jj < FOLD; ++jj) {
              const int s2 = s0 + 4 * jj;
              if (s2 <= T) {
                const R ws = rule_wr<R>(W, T - tp, T - s2);
                const S* yl = sp(s2);
                const S* sr = el<NO, S>(d.SR, d, n, s2, tp);
#pragma unroll
                for (int m = 0; m < NO; ++m) {
                  const cx<R> ym = ldr<R>(yl + m) * ws;
#pragma unroll
                  for (int j = 0; j < NO; ++j) pa[j] = cfma(ym, ldr<R>(sr + m * NO + j), pa[j]);
                }
              }
            }
#pragma unroll
            for (int j = 0; j < NO; ++j) ka[j].add(pa[j]);
          }
          for (int lv = 0; lv < d.maxl; ++lv) {
            const int blk = d.colblk[jl * d.maxl + lv];
            if (blk < 0 || d.b_r0[blk] >= c) continue;
            const int c0 = d.b_c0[blk];
#pragma unroll
            for (int p = 0; p < NO2; ++p) {
              const int j = p % NO;
              const int rk = *Rk<NO>(d, 2, n, blk, p);
              const S* V = Vp<NO, S>(d, 2, n, blk, p) + (long long)(tp - c0) * d.rmax;
              cx<R> pb = cx<R>(0);
              if (staged) {
                pb = lr_dot4<R, S, true>(Ps + (lv * NO2 + p) * d.rmax, V, rk, sl);
              } else {
                const double2* P = Pj<NO>(d, n, irow, lv, p);
                for (int q = sl; q < rk; q += 4) pb = cfma(ldr<R>(P + q), ldr<R>(V + q).conj(), pb);
              }
              ka[j].add(pb);
            }
          }
          for (int s2 = E + sl; s2 <= tp + k && s2 < c; s2 += 4) {
            const double ws = rule_w(W, T - tp, T - s2) - 1.0;
            const S* bd = Bd<NO, S>(d, n, s2, s2 - tp);
            const Y* yl = yp(s2);
#pragma unroll
            for (int m = 0; m < NO; ++m) {
              const zd ym = ld(yl + m) * ws;
#pragma unroll
              for (int j = 0; j < NO; ++j) acc[j] = cfma(ym, ld(bd + m * NO + j), acc[j]);
            }
          }
        }
#pragma unroll
        for (int j = 0; j < NO; ++j) acc[j] += ka[j].get();
#pragma unroll
        for (int j = 0; j < NO; ++j) {
          acc[j] += zd(__shfl_xor_sync(FULL, acc[j].re, 1), __shfl_xor_sync(FULL, acc[j].im, 1));
          acc[j] += zd(__shfl_xor_sync(FULL, acc[j].re, 2), __shfl_xor_sync(FULL, acc[j].im, 2));
        }
        if (sl == 0 && col < L)
#pragma unroll
          for (int j = 0; j < NO; ++j) FB[col][j] = acc[j];
      }
      __syncthreads();
    }
    // the frozen inverse of this chunk into shared memory, overlapping the far field
    const bool stage_now = kInvStage<NO, S> && cc < d.nfrozR && s_stage;
    if (stage_now && tid == 0) bulk_g2s(ctile, Cinv<NO>(d, n, cc, 0), kInvStage<NO, S>, &cbar);
    // ---- far field of the chunk: rows s >= b not covered above; 8 threads per column ----
    {
      const int col = tid >> 3, sl = tid & 7;
      const int tp = a + col;
      zd acc[NO];
#pragma unroll
      for (int j = 0; j < NO; ++j) acc[j] = zd();
        KAcc<R> ka[NO];   // FP32 history sums, compensated (FP64 in the FP64 form)
      if (col < cn) {
        const int s_end = comp ? E : T + 1;   // compressed: the rest of the leaf; else every later row
        for (int s0 = b + sl; s0 < s_end; s0 += 8 * FOLD) {
          cx<R> pa[NO];
#pragma unroll
          for (int j = 0; j < NO; ++j) pa[j] = cx<R>(0);
#pragma unroll
          for (int jj = 0; jj < FOLD; ++jj) {
            const int s2 = s0 + 8 * jj;
            if (s2 < s_end) {
              const R ws = rule_wr<R>(W, T - tp, T - s2);
              const S* yl = sp(s2);
              const S* sr = comp ? Lf<NO, S>(d, 2, n, jl, s2, tp) : el<NO, S>(d.SR, d, n, s2, tp);
#pragma unroll
              for (int m = 0; m < NO; ++m) {
                const cx<R> ym = ldr<R>(yl + m) * ws;
#pragma unroll
                for (int j = 0; j < NO; ++j) pa[j] = cfma(ym, ldr<R>(sr + m * NO + j), pa[j]);
              }
            }
          }
#pragma unroll
          for (int j = 0; j < NO; ++j) ka[j].add(pa[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < NO; ++j) {
        const auto r = reduce8(ka[j]);
        if (sl == 0) acc[j] = val_of(r);
      }
      if (sl == 0 && col < cn) {
        zd F[NO];
        zd Fbd[NO];
#pragma unroll
        for (int j = 0; j < NO; ++j) {
          F[j] = (acc[j] + (comp ? FB[tp - A][j] : zd())) * h;
          Fbd[j] = zd();
        }
        for (int jj = 1; jj <= k; ++jj) {  // BDF terms reaching above the chunk: (-i a_j / h) y(s2)
          const int s2 = tp + jj;
          if (s2 < b) continue;
          const double cj = W.ah[jj];
#pragma unroll
          for (int m = 0; m < NO; ++m) {
            const zd y = ld(yp(s2) + m);
            Fbd[m] = zd(fma(cj, y.im, Fbd[m].re), fma(-cj, y.re, Fbd[m].im));
          }
        }
#pragma unroll
        for (int j = 0; j < NO; ++j) {
          Fs[col][j] = F[j] + Fbd[j];
          Fb[col][j] = Fbd[j];
          Ff[col][j] = zf((float)F[j].re, (float)F[j].im);
          FbF[col][j] = cff_of(Fbd[j]);
        }
      }
      if (sl == 1 && col < cn)
#pragma unroll
        for (int j = 0; j < NO; ++j) Old[col][j] = ld(sp(tp) + j);
    }
    __syncthreads();
    if (cc < d.nfrozR) {
      // frozen chunk: y = F C^-1 (row vector times the precomputed inverse),
      // 8 threads per output element
      const double2* Mi = Cinv<NO>(d, n, cc, 0);
      bool smem_inv = false;
      if (stage_now) {
        smem_inv = mbar_wait(&cbar, cphase, kCopyWaitPolls);
        cphase ^= 1u;
        if (!smem_inv) {
          s_stage = 0;
          atomicAdd(d.status + 2, 1);
        }
      }
      const double2* Mg = smem_inv ? reinterpret_cast<const double2*>(ctile) : Mi;
      constexpr int LD = CK * NO;
      for (int o8 = tid; o8 < CK * NO * 8; o8 += blockDim.x) {
        const int o = o8 >> 3, sl = o8 & 7, ti = o / NO, j = o % NO;
        zd sacc = zd();
        if constexpr (Row64<NO, S>::separate) {
          // complex64 form: far field x hi in FP32, the k edge rows x (hi + lo)
          // in float-float, reduced over the 8 lanes in float-float
          const float2* Mh = reinterpret_cast<const float2*>(Mg);
          const float2* Ml = Mh + LD * LD;
          zf s32 = zf(0);
          for (int si = sl; si < CK; si += 8)
#pragma unroll
            for (int m = 0; m < NO; ++m)
              s32 = cfma(Ff[si][m], ldr<float>(Mh + (long long)(si * NO + m) * LD + ti * NO + j), s32);
          cff sf = cff_of(s32);
          for (int si = CK - k + sl; si < CK; si += 8)
#pragma unroll
            for (int m = 0; m < NO; ++m) {
              const long long e = (long long)(si * NO + m) * LD + ti * NO + j;
              const float2 hv = Mh[e], lv = Ml[e];
              sf = cff_add(sf, cff_mul(FbF[si][m], cff{{hv.x, lv.x}, {hv.y, lv.y}}));
            }
#pragma unroll
          for (int off = 1; off < 8; off <<= 1) sf = cff_add(sf, cff_shfl_xor(sf, off));
          if (sl == 0) sacc = cff_val(sf);
        } else {
          for (int si = sl; si < CK; si += 8)
#pragma unroll
            for (int m = 0; m < NO; ++m) sacc = cfma(Fs[si][m], ld(Mg + (long long)(si * NO + m) * LD + ti * NO + j), sacc);
#pragma unroll
          for (int off = 1; off < 8; off <<= 1)
            sacc += zd(__shfl_xor_sync(FULL, sacc.re, off), __shfl_xor_sync(FULL, sacc.im, off));
        }
        if (sl == 0) {
          myerr = fmax(myerr, (sacc - Old[ti][j]).abs2());
          st(yp(a + ti) + j, sacc);
          if constexpr (Row64<NO, S>::separate) st(sp(a + ti) + j, sacc);
        }
      }
    } else {
      // chunk near T: right-looking triangular solve in one warp.  Lane L owns
      // t'' = a + L; after point s is solved every lane with t'' < s removes
      // y(s) C(s, t'') from its right-hand side.  The coefficients C(s, t'')
      // are first staged in shared memory by the whole block (N_o <= 2), so
      // the 32 dependent steps of the solve wait on no global load.
      auto coef = [&](int i, int L0, zd* cf) {
        const int spt = a + i, tq = a + L0;
        const double wl = -h * rule_w(W, T - tq, T - spt);
        const S* sr = comp ? Lf<NO, S>(d, 2, n, jl, spt, tq) : el<NO, S>(d.SR, d, n, spt, tq);
        const int dd = spt - tq;
#pragma unroll
        for (int q = 0; q < NO2; ++q) {
          cf[q] = ld(sr + q) * wl;
          if (dd <= k && (q / NO) == (q % NO)) cf[q] += zd(0, W.a[dd] / h);
        }
      };
      if constexpr (kStage<NO>) {
        for (int e = tid; e < CK * CK; e += blockDim.x) {
          const int i = e / CK, L0 = e % CK;
          if (L0 < i && i < cn) coef(i, L0, ctile + (long long)e * NO2);
        }
        __syncthreads();
      }
      if (warp == 0) {
      const int L0 = lane, tq = a + L0;
      M<NO> Dinv;
      zd f[NO];
      if (L0 < cn) {
        const double ws = h * rule_w(W, T - tq, T - tq);
        const S* sd = comp ? Lf<NO, S>(d, 2, n, jl, tq, tq) : el<NO, S>(d.SR, d, n, tq, tq);
        const double2* ep = epsp<NO>(d, n, tq);
        M<NO> Mm;
#pragma unroll
        for (int x = 0; x < NO; ++x)
#pragma unroll
          for (int y2 = 0; y2 < NO; ++y2)
            Mm.a[x][y2] = (x == y2 ? zd(0, W.a[0] / h) : zd()) - ld(ep + x * NO + y2) - ld(sd + x * NO + y2) * ws;
        Dinv = solve_left<NO>(Mm, M<NO>::eye(zd(1.0)));
#pragma unroll
        for (int j = 0; j < NO; ++j) f[j] = Fs[L0][j];
      }
      for (int i = cn - 1; i >= 0; --i) {
        const int spt = a + i;
        // coefficient C(spt, tq) for this lane (only lanes with tq < spt use it)
        zd cf[NO2];
        if (L0 < i) {
          if constexpr (kStage<NO>) {
#pragma unroll
            for (int q = 0; q < NO2; ++q) cf[q] = ctile[(long long)(i * CK + L0) * NO2 + q];
          } else {
            coef(i, L0, cf);
          }
        }
        zd y[NO];
        if (L0 == i) {
#pragma unroll
          for (int j = 0; j < NO; ++j) {
            y[j] = zd();
#pragma unroll
            for (int m = 0; m < NO; ++m) y[j] = cfma(f[m], Dinv.a[m][j], y[j]);
          }
#pragma unroll
          for (int j = 0; j < NO; ++j) {
            myerr = fmax(myerr, (y[j] - ld(sp(spt) + j)).abs2());
            st(yp(spt) + j, y[j]);
            if constexpr (Row64<NO, S>::separate) st(sp(spt) + j, y[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < NO; ++j) y[j] = zd(__shfl_sync(FULL, y[j].re, i), __shfl_sync(FULL, y[j].im, i));
        if (L0 < i) {
#pragma unroll
          for (int m = 0; m < NO; ++m)
#pragma unroll
            for (int j = 0; j < NO; ++j) f[j] -= y[m] * cf[m * NO + j];
        }
      }
      }
    }
    __syncthreads();
  }
  myerr = sqrt(warp_max(myerr));
  if (lane == 0 && myerr > 0) atomic_max_nonneg(&serr, myerr);
  __syncthreads();
  if (tid == 0) atomic_max_nonneg(d.err + n, serr);
  // after a timed-out wait, a copy may still be in flight into this CTA's
  // shared memory: wait for it (bounded) before the CTA exits
  if (kInvStage<NO, S> && tid == 0 && !s_stage) mbar_wait(&cbar, cphase ^ 1u, kCopyWaitPolls);
}

// ---------------------------------------------------------------------------
// Lesser column, Eq. KBEL: unknown x(t) = G^<(t, T) (column jc), t = 0..T.
// ---------------------------------------------------------------------------
template <int NO, typename S>
__global__ void __launch_bounds__(256, (NO <= 2) ? 2 : 1) k_les2(Dev d, int T, int staged) {
  constexpr int NO2 = NO * NO;
  using R = typename Bulk<S>::R;
  const int n = blockIdx.y, jc = blockIdx.x;
  if (!d.active[n]) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = d.k, c = d.cdir, L = d.L;
  const double h = d.h;
  const DevW& W = d.w;
  __shared__ zd sA[20 * 20];
  __shared__ zd sB[20];
  __shared__ zd FB[64][NO];
  __shared__ zd pbuf[8][128];
  __shared__ zd Fs[CK][NO];
  __shared__ zd Fb[CK][NO];      // the BDF part of Fs (rows at the chunk edge; zero elsewhere)
  __shared__ zd Old[CK][NO];     // the chunk's previous iterate (convergence measure)
  __shared__ zf Ff[CK][NO];      // complex64 form: the far field (Fs - Fb) rounded to complex64
  __shared__ cff FbF[CK][NO];    // complex64 form: Fb in float-float
  __shared__ double serr;
  extern __shared__ __align__(16) zd ctile[];  // [CK][CK][NO2] hot-chunk coefficients (N_o <= 2);
                                 // at leaf entry (staged != 0) the block projections
                                 // [maxl][NO2][rmax]; for a frozen chunk its staged inverse
  __shared__ __align__(8) uint64_t cbar;   // completion of the inverse's bulk copy
  __shared__ int s_stage;                  // 0 once a wait for a copy has timed out
  uint32_t cphase = 0;
  if (tid == 0) {
    serr = 0.0;
    s_stage = 1;
    if (kInvStage<NO, S>) mbar_init(&cbar);
  }
  // FP64 column during the sweep (see k_ret2); xp: as solved, sp: storage
  S* colp = el<NO, S>(d.GL, d, n, T, 0);
  Y* coly = Row64<NO, S>::get(d, n, 1, T, colp);
  auto xp = [&](int t) { return coly + (long long)t * NO2; };  // element [m*NO + jc]
  auto sp = [&](int t) { return colp + (long long)t * NO2; };
  const double2* qs = d.qsrc + (long long)n * d.nt * NO2;
  double myerr = 0.0;
  const int last = (d.rho_mode == 1) ? T - 1 : T;
  if (warp == 0 && lane < NO) {  // x(0) = -[G^tv(T, 0+)]^dagger
    const int m = lane;
    zd v = ld(d.x0 + (long long)n * NO2 + m * NO + jc);
    myerr = fmax(myerr, (v - ld(sp(0) + m * NO + jc)).abs2());
    st(xp(0) + m * NO + jc, v);
    if constexpr (Row64<NO, S>::separate) st(sp(0) + m * NO + jc, v);
  }
  __syncthreads();
  for (int cc = 0; cc * CK <= last; ++cc) {
    const int a = (cc == 0) ? 1 : cc * CK, b = min((cc + 1) * CK, last + 1), cn = b - a;
    if (cn <= 0) break;
    const bool comp = (c > 0 && b <= c);
    const int jl = comp ? a / L : 0, A = jl * L;
    if (comp && cc * CK == A) {
      // Entering leaf jl.  (1) rho_B = S_B sum_l w_l conj(V_B(l,:)) x(l) for the
      // blocks whose rows start at A (w_l = omega_l for l <= k, else 1).
      for (int lv = 0; lv < d.maxl && jl > 0; ++lv) {
        const int blk = d.rowblk[jl * d.maxl + lv];
        if (blk < 0 || d.b_r0[blk] != A) continue;
        const int c0 = d.b_c0[blk], c1 = d.b_c1[blk];
        if constexpr (kStage<NO> && Row64<NO, S>::separate) {   // complex64 form: all pairs in one
          if (d.rmax <= 64) {                                     // pass (ctile is free here)
            proj_block<NO, S, false>(d, n, blk, lv, jc, c0, c1, [&](int l, int nn) {
              const R wl = (l <= k) ? (R)W.omega[l] : (R)1;
              return ldr<R>(sp(l) + nn * NO + jc) * wl;
            }, ctile);
            continue;
          }
        }
        for (int p = 0; p < NO2; ++p) {
          const int nn = p % NO;
          const int rk = *Rk<NO>(d, 2, n, blk, p);
          const S* V = Vp<NO, S>(d, 2, n, blk, p);
          KAcc<R> part[4];
          for (int l0 = c0 + warp; l0 < c1; l0 += 8 * FOLD) {  // warps over columns, lanes over rank
            cx<R> pp[4] = {cx<R>(0), cx<R>(0), cx<R>(0), cx<R>(0)};
#pragma unroll
            for (int jj = 0; jj < FOLD; ++jj) {
              const int l = l0 + 8 * jj;
              if (l < c1) {
                const R wl = (l <= k) ? (R)W.omega[l] : (R)1;
                const cx<R> xv = ldr<R>(sp(l) + nn * NO + jc) * wl;
                const S* vr = V + (long long)(l - c0) * d.rmax;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  const int q = lane + 32 * u;
                  if (q < rk) pp[u] = cfma(ldr<R>(vr + q).conj(), xv, pp[u]);
                }
              }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) part[u].add(pp[u]);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) pbuf[warp][lane + 32 * u] = part[u].get();
          __syncthreads();
          if (tid < d.rmax) {
            zd acc = zd();
            for (int w2 = 0; w2 < 8; ++w2) acc += pbuf[w2][tid];
            st(Pj<NO>(d, n, jc, lv, p) + tid, tid < rk ? acc * Sp<NO>(d, 2, n, blk, p)[tid] : zd());
          }
          __syncthreads();
        }
      }
      __syncthreads();
      // projections of every block left of this leaf's rows, staged in shared
      // memory for the loop below (the buffer of the hot-chunk coefficients,
      // which the chunk solves fill only after it)
      cx<R>* Ps = reinterpret_cast<cx<R>*>(ctile);
      if (staged) {
        const int per = NO2 * d.rmax;
        for (int e = tid; e < d.maxl * per; e += blockDim.x) {
          const int lv = e / per, p = (e / d.rmax) % NO2, q = e % d.rmax;
          const int blk = d.rowblk[jl * d.maxl + lv];
          Ps[e] = blk >= 0 ? ldr<R>(Pj<NO>(d, n, jc, lv, p) + q) : cx<R>(0);
        }
        __syncthreads();
      }
      // (2) every row of the leaf: blocks left of it and near-diagonal corrections
      {
        const int row = tid >> 2, sl = tid & 3;
        const int t = A + row;
        zd acc[NO];
#pragma unroll
        for (int m = 0; m < NO; ++m) acc[m] = zd();
        KAcc<R> ka[NO];   // FP32 history sums, compensated (FP64 in the FP64 form)
        if (row < L) {
          for (int lv = 0; lv < d.maxl; ++lv) {
            const int blk = d.rowblk[jl * d.maxl + lv];
            if (blk < 0) continue;
            const int r0 = d.b_r0[blk];
#pragma unroll
            for (int p = 0; p < NO2; ++p) {
              const int m = p / NO;
              const int rk = *Rk<NO>(d, 2, n, blk, p);
              const S* U = Up<NO, S>(d, 2, n, blk, p) + (long long)(t - r0) * d.rmax;
              cx<R> pb = cx<R>(0);
              if (staged) {
                pb = lr_dot4<R, S, false>(Ps + (lv * NO2 + p) * d.rmax, U, rk, sl);
              } else {
                const double2* P = Pj<NO>(d, n, jc, lv, p);
                for (int q = sl; q < rk; q += 4) pb = cfma(ldr<R>(U + q), ldr<R>(P + q), pb);
              }
              ka[m].add(pb);
            }
          }
          for (int l = max(t - k, 0) + sl; l < A; l += 4) {
            const double wl = rule_w(W, t, l) - 1.0;
            const S* bd = Bd<NO, S>(d, n, t, t - l);
#pragma unroll
            for (int y = 0; y < NO; ++y) {
              const zd xy = ld(xp(l) + y * NO + jc) * wl;
#pragma unroll
              for (int m = 0; m < NO; ++m) acc[m] = cfma(ld(bd + m * NO + y), xy, acc[m]);
            }
          }
        }
#pragma unroll
        for (int m = 0; m < NO; ++m) acc[m] += ka[m].get();
#pragma unroll
        for (int m = 0; m < NO; ++m) {
          acc[m] += zd(__shfl_xor_sync(FULL, acc[m].re, 1), __shfl_xor_sync(FULL, acc[m].im, 1));
          acc[m] += zd(__shfl_xor_sync(FULL, acc[m].re, 2), __shfl_xor_sync(FULL, acc[m].im, 2));
        }
        if (sl == 0 && row < L)
#pragma unroll
          for (int m = 0; m < NO; ++m) FB[row][m] = acc[m];
      }
      __syncthreads();
    }
    const bool frozen = (cc < d.nfrozL) && (b - a == ((cc == 0) ? CK - 1 : CK));
    // the frozen inverse of this chunk into shared memory, overlapping the far field
    const bool stage_now = kInvStage<NO, S> && frozen && s_stage;
    if (stage_now && tid == 0) bulk_g2s(ctile, Cinv<NO>(d, n, cc, 1), kInvStage<NO, S>, &cbar);
    // ---- far field F(t) = q(t) - sum_{l < a} C(t,l) x(l); 8 threads per row ----
    {
      const int row = tid >> 3, sl = tid & 7;
      const int t = a + row;
      zd acc[NO], fbo[NO];   // fbo: this lane's BDF part (only the owner lane's is nonzero)
#pragma unroll
      for (int m = 0; m < NO; ++m) acc[m] = fbo[m] = zd();
        KAcc<R> ka[NO];   // FP32 history sums, compensated (FP64 in the FP64 form)
      if (row < cn) {
        if (t <= k) {
          if (sl == 0) {  // start rows: only l = 0 lies left of chunk 0 (a derivative term: kept in Fb)
            zd fb[NO];
#pragma unroll
            for (int m = 0; m < NO; ++m) fb[m] = zd();
            for (int y = 0; y < NO; ++y) {
              const zd xv = ld(xp(0) + y * NO + jc);
#pragma unroll
              for (int m = 0; m < NO; ++m) {
                zd cf = srx_any<NO, S>(d, n, t, 0, m, y) * (-h * W.I0[t][0]);
                if (m == y) cf += zd(0, W.D[t][0] / h);
                fb[m] -= cf * xv;
              }
            }
#pragma unroll
            for (int m = 0; m < NO; ++m) {
              fbo[m] = fb[m];
              Fb[row][m] = fb[m];
            }
          }
        } else {
          const int l0 = comp ? A : 0;
          const S* srow = comp ? nullptr : el<NO, S>(d.SR, d, n, t, 0);
          const R hr = (R)h;
          for (int lb = l0 + sl; lb < a; lb += 8 * FOLD) {
            cx<R> pa[NO];
#pragma unroll
            for (int m = 0; m < NO; ++m) pa[m] = cx<R>(0);
#pragma unroll
            for (int jj = 0; jj < FOLD; ++jj) {
              const int l = lb + 8 * jj;
              if (l < a) {
                const R wl = hr * rule_wr<R>(W, t, l);
                const S* sr = comp ? Lf<NO, S>(d, 2, n, jl, t, l) : srow + (long long)l * NO2;
#pragma unroll
                for (int y = 0; y < NO; ++y) {
                  const cx<R> xy = ldr<R>(sp(l) + y * NO + jc) * wl;
#pragma unroll
                  for (int m = 0; m < NO; ++m) pa[m] = cfma(ldr<R>(sr + m * NO + y), xy, pa[m]);
                }
              }
            }
#pragma unroll
            for (int m = 0; m < NO; ++m) ka[m].add(pa[m]);
          }
          if (sl == 1) {  // BDF terms reaching left of the chunk, kept apart in Fb
            zd fb[NO];
#pragma unroll
            for (int m = 0; m < NO; ++m) fb[m] = zd();
            for (int jj = 1; jj <= k; ++jj) {   // (-i a_j / h) x(t - j)
              if (t - jj >= a) continue;
              const double cj = W.ah[jj];
#pragma unroll
              for (int m = 0; m < NO; ++m) {
                const zd x = ld(xp(t - jj) + m * NO + jc);
                fb[m] = zd(fma(cj, x.im, fb[m].re), fma(-cj, x.re, fb[m].im));
              }
            }
#pragma unroll
            for (int m = 0; m < NO; ++m) {
              fbo[m] = fb[m];
              Fb[row][m] = fb[m];
            }
          }
        }
      }
      // the BDF part from its owner lane (sl 0 for the start rows, else sl 1)
      const int owner = (lane & ~7) | (t <= k ? 0 : 1);
#pragma unroll
      for (int m = 0; m < NO; ++m) {
        const auto r = reduce8(ka[m]);
        const zd fbm(__shfl_sync(FULL, fbo[m].re, owner), __shfl_sync(FULL, fbo[m].im, owner));
        if (sl == 0 && row < cn) {
          const zd far = val_of(r) + (comp && t > k ? FB[t - A][m] * h : zd()) +
                         ld(qs + (long long)t * NO2 + m * NO + jc);
          Fs[row][m] = far + fbm;
          Ff[row][m] = zf((float)far.re, (float)far.im);
          FbF[row][m] = cff_of(fbm);
        }
      }
      (void)acc;
      if (sl == 1 && row < cn)
#pragma unroll
        for (int m = 0; m < NO; ++m) Old[row][m] = ld(sp(t) + m * NO + jc);
    }
    __syncthreads();
    if (frozen) {
      const double2* Mi = Cinv<NO>(d, n, cc, 1);
      bool smem_inv = false;
      if (stage_now) {
        smem_inv = mbar_wait(&cbar, cphase, kCopyWaitPolls);
        cphase ^= 1u;
        if (!smem_inv) {
          s_stage = 0;
          atomicAdd(d.status + 2, 1);
        }
      }
      const double2* Mg = smem_inv ? reinterpret_cast<const double2*>(ctile) : Mi;
      constexpr int LD = CK * NO;
      for (int o8 = tid; o8 < CK * NO * 8; o8 += blockDim.x) {
        const int o = o8 >> 3, sl = o8 & 7, ti = o / NO, m = o % NO;
        zd sacc = zd();
        if constexpr (Row64<NO, S>::separate) {
          // complex64 form: far field x hi in FP32, the k edge rows x (hi + lo) in
          // float-float, reduced over the 8 lanes in float-float
          const float2* Mh = reinterpret_cast<const float2*>(Mg);
          const float2* Ml = Mh + LD * LD;
          cff sf = cff_of(zf(0));
          if (ti < cn) {
            zf s32 = zf(0);
            for (int li = sl; li < cn; li += 8)
#pragma unroll
              for (int y = 0; y < NO; ++y)
                s32 = cfma(ldr<float>(Mh + (long long)(ti * NO + m) * LD + li * NO + y), Ff[li][y], s32);
            sf = cff_of(s32);
            for (int li = sl; li < k && li < cn; li += 8)
#pragma unroll
              for (int y = 0; y < NO; ++y) {
                const long long e = (long long)(ti * NO + m) * LD + li * NO + y;
                const float2 hv = Mh[e], lv = Ml[e];
                sf = cff_add(sf, cff_mul(cff{{hv.x, lv.x}, {hv.y, lv.y}}, FbF[li][y]));
              }
          }
#pragma unroll
          for (int off = 1; off < 8; off <<= 1) sf = cff_add(sf, cff_shfl_xor(sf, off));
          if (sl == 0) sacc = cff_val(sf);
        } else {
          if (ti < cn)
            for (int li = sl; li < cn; li += 8)
#pragma unroll
              for (int y = 0; y < NO; ++y)
                sacc = cfma(ld(Mg + (long long)(ti * NO + m) * LD + li * NO + y), Fs[li][y], sacc);
#pragma unroll
          for (int off = 1; off < 8; off <<= 1)
            sacc += zd(__shfl_xor_sync(FULL, sacc.re, off), __shfl_xor_sync(FULL, sacc.im, off));
        }
        if (sl == 0 && ti < cn) {
          myerr = fmax(myerr, (sacc - Old[ti][m]).abs2());
          st(xp(a + ti) + m * NO + jc, sacc);
          if constexpr (Row64<NO, S>::separate) st(sp(a + ti) + m * NO + jc, sacc);
        }
      }
    } else {
      // chunk near T: right-looking triangular solve in one warp; lane L owns
      // row t'' = a + L.  Chunk 0 first solves its start block t = 1..k.  The
      // coefficients C(t'', tp) are staged in shared memory first (N_o <= 2).
      auto coef = [&](int L0, int i, zd* cf) {
        const int tq = a + L0, tp = a + i;
        const double wl = -h * rule_w(W, tq, tp);
        const S* sr = comp ? Lf<NO, S>(d, 2, n, jl, tq, tp) : el<NO, S>(d.SR, d, n, tq, tp);
        const int dd = tq - tp;
#pragma unroll
        for (int q = 0; q < NO2; ++q) {
          cf[q] = ld(sr + q) * wl;
          if (dd <= k && (q / NO) == (q % NO)) cf[q] += zd(0, W.a[dd] / h);
        }
      };
      if constexpr (kStage<NO>) {
        const int i0s = (cc == 0) ? k : 0;
        for (int e = tid; e < CK * CK; e += blockDim.x) {
          const int L0 = e / CK, i = e % CK;
          if (i >= i0s && i < L0 && L0 < cn) coef(L0, i, ctile + (long long)e * NO2);
        }
        __syncthreads();
      }
      if (warp == 0) {
      const int L0 = lane, tq = a + L0;
      int i0 = 0;
      zd f[NO];
      if (L0 < cn)
#pragma unroll
        for (int m = 0; m < NO; ++m) f[m] = Fs[L0][m];
      if (cc == 0) {
        const int nsb = k * NO;
        for (int e = lane; e < nsb * nsb; e += 32) {
          const int row = e / nsb, col = e % nsb;
          const int t = row / NO + 1, m = row % NO, l = col / NO + 1, y = col % NO;
          zd v = srx_any<NO, S>(d, n, t, l, m, y) * (-h * W.I0[t][l]);
          if (m == y) v += zd(0, W.D[t][l] / h);
          if (l == t) v -= ld(epsp<NO>(d, n, t) + m * NO + y);
          sA[row * nsb + col] = v;
        }
        for (int row = lane; row < nsb; row += 32) sB[row] = Fs[row / NO][row % NO];
        __syncwarp();
        warp_lu_solve(nsb, sA, sB, 1, nullptr);
        for (int row = lane; row < nsb; row += 32) {
          const int t = row / NO + 1, m = row % NO;
          if (t <= last) {
            myerr = fmax(myerr, (sB[row] - ld(sp(t) + m * NO + jc)).abs2());
            st(xp(t) + m * NO + jc, sB[row]);
            if constexpr (Row64<NO, S>::separate) st(sp(t) + m * NO + jc, sB[row]);
          }
        }
        __syncwarp();
        if (L0 < cn && tq > k) {  // rows below the start block remove its contribution
          for (int l = 1; l <= k; ++l) {
            const double wl = -h * rule_w(W, tq, l);
            const S* sr = comp ? Lf<NO, S>(d, 2, n, jl, tq, l) : el<NO, S>(d.SR, d, n, tq, l);
            const int dd = tq - l;
#pragma unroll
            for (int m = 0; m < NO; ++m)
#pragma unroll
              for (int y = 0; y < NO; ++y) {
                zd cfv = ld(sr + m * NO + y) * wl;
                if (dd <= k && m == y) cfv += zd(0, W.a[dd] / h);
                f[m] -= cfv * sB[(l - 1) * NO + y];
              }
          }
        }
        i0 = k;  // rows a..k (a = 1) are done
      }
      M<NO> Dinv;
      if (L0 < cn && L0 >= i0) {
        const double wt = h * rule_w(W, tq, tq);
        const S* sd = comp ? Lf<NO, S>(d, 2, n, jl, tq, tq) : el<NO, S>(d.SR, d, n, tq, tq);
        const double2* ep = epsp<NO>(d, n, tq);
        M<NO> Mm;
#pragma unroll
        for (int x2 = 0; x2 < NO; ++x2)
#pragma unroll
          for (int y = 0; y < NO; ++y)
            Mm.a[x2][y] = (x2 == y ? zd(0, W.a[0] / h) : zd()) - ld(ep + x2 * NO + y) - ld(sd + x2 * NO + y) * wt;
        Dinv = solve_left<NO>(Mm, M<NO>::eye(zd(1.0)));
      }
      for (int i = i0; i < cn; ++i) {
        const int tp = a + i;
        zd cf[NO2];
        if (L0 > i && L0 < cn) {
          if constexpr (kStage<NO>) {
#pragma unroll
            for (int q = 0; q < NO2; ++q) cf[q] = ctile[(long long)(L0 * CK + i) * NO2 + q];
          } else {
            coef(L0, i, cf);
          }
        }
        zd x[NO];
        if (L0 == i) {
#pragma unroll
          for (int m = 0; m < NO; ++m) {
            x[m] = zd();
#pragma unroll
            for (int y = 0; y < NO; ++y) x[m] = cfma(Dinv.a[m][y], f[y], x[m]);
          }
#pragma unroll
          for (int m = 0; m < NO; ++m) {
            myerr = fmax(myerr, (x[m] - ld(sp(tp) + m * NO + jc)).abs2());
            st(xp(tp) + m * NO + jc, x[m]);
            if constexpr (Row64<NO, S>::separate) st(sp(tp) + m * NO + jc, x[m]);
          }
        }
#pragma unroll
        for (int m = 0; m < NO; ++m) x[m] = zd(__shfl_sync(FULL, x[m].re, i), __shfl_sync(FULL, x[m].im, i));
        if (L0 > i && L0 < cn) {
#pragma unroll
          for (int m = 0; m < NO; ++m)
#pragma unroll
            for (int y = 0; y < NO; ++y) f[m] -= cf[m * NO + y] * x[y];
        }
      }
      }
    }
    __syncthreads();
  }
  myerr = sqrt(warp_max(myerr));
  if (lane == 0 && myerr > 0) atomic_max_nonneg(&serr, myerr);
  __syncthreads();
  if (tid == 0) atomic_max_nonneg(d.err + n, serr);
  // after a timed-out wait, a copy may still be in flight into this CTA's
  // shared memory: wait for it (bounded) before the CTA exits
  if (kInvStage<NO, S> && tid == 0 && !s_stage) mbar_wait(&cbar, cphase ^ 1u, kCopyWaitPolls);
}

// ---------------------------------------------------------------------------
// Inverse of a frozen chunk's local system, by Gauss-Jordan with partial
// pivoting (FP64), one CTA per instance.  Retarded (which 0): unknowns
// y(t'), t' in [a, a+32), matrix C[(s,m),(t',j)] = (i/h) a_{s-t'} [0 <= s-t' <= k]
// delta_mj - delta_{s t'} eps(t')_mj - h w(s-t') Sigma^R(s,t')_mj with the
// standard Gregory end weight w(d) = omega_d (d <= k) else 1.  Lesser (which 1):
// unknowns x(t), rows t of the chunk; rows t <= k are the start equations with
// D and I_{0,t,.}, other rows the BDF/Gregory equation with the weights w^(t)_l.
// ---------------------------------------------------------------------------
template <int NO, typename S>
__global__ void __launch_bounds__(256) k_chunk_inv(Dev d, int which, int cc, double2* ws) {
  const int n = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = d.k;
  const double h = d.h;
  const DevW& W = d.w;
  const int a = (which == 1 && cc == 0) ? 1 : cc * CK;
  const int cnt = (which == 1 && cc == 0) ? CK - 1 : CK;
  if (cc * CK + CK + (which == 0 ? 2 * k : 0) > d.last[n]) return;   // frozen only after the instance ends
  const int nn = cnt * NO;
  constexpr int LD = CK * NO;
  double2* Bout = Cinv<NO>(d, n, cc, which);
  double2* Am = ws + (long long)n * 2 * LD * LD;   // FP64 work matrix
  double2* B = Am + (long long)LD * LD;            // FP64 inverse under construction
  __shared__ zd fcol[CK * 4];
  __shared__ int s_piv;
  __shared__ zd s_inv;
  for (int e = tid; e < nn * nn; e += blockDim.x) {
    const int r = e / nn, col = e % nn;
    const int ri = r / NO, m = r % NO, ci = col / NO, j = col % NO;
    zd v = zd();
    if (which == 0) {
      const int s = a + ri, tp = a + ci, dd = s - tp;
      if (dd >= 0) {
        const double wf = (dd <= k) ? W.omega[dd] : 1.0;
        v = sr_any<NO, S>(d, n, s, tp, m, j) * (-h * wf);
        if (dd <= k && m == j) v += zd(0, W.a[dd] / h);
        if (dd == 0) v -= ld(epsp<NO>(d, n, tp) + m * NO + j);
      }
    } else {
      const int t = a + ri, l = a + ci;
      if (t <= k) {
        if (l <= k) {
          v = srx_any<NO, S>(d, n, t, l, m, j) * (-h * W.I0[t][l]);
          if (m == j) v += zd(0, W.D[t][l] / h);
          if (l == t) v -= ld(epsp<NO>(d, n, t) + m * NO + j);
        }
      } else if (l <= t) {
        v = sr_any<NO, S>(d, n, t, l, m, j) * (-h * rule_w(W, t, l));
        if (t - l <= k && m == j) v += zd(0, W.a[t - l] / h);
        if (l == t) v -= ld(epsp<NO>(d, n, t) + m * NO + j);
      }
    }
    st(Am + (long long)r * LD + col, v);
    st(B + (long long)r * LD + col, (r == col) ? zd(1.0) : zd());
  }
  __syncthreads();
  for (int piv = 0; piv < nn; ++piv) {
    if (warp == 0) {
      double best = -1.0;
      int arg = piv;
      for (int r = piv + lane; r < nn; r += 32) {
        const double v = ld(Am + (long long)r * LD + piv).abs2();
        if (v > best) { best = v; arg = r; }
      }
#pragma unroll
      for (int off = 16; off; off >>= 1) {
        const double b2 = __shfl_xor_sync(0xffffffffu, best, off);
        const int a2 = __shfl_xor_sync(0xffffffffu, arg, off);
        if (b2 > best || (b2 == best && a2 < arg)) { best = b2; arg = a2; }
      }
      if (lane == 0) s_piv = arg;
    }
    __syncthreads();
    const int p = s_piv;
    if (p != piv) {
      for (int j = tid; j < nn; j += blockDim.x) {
        double2 t1 = Am[(long long)piv * LD + j]; Am[(long long)piv * LD + j] = Am[(long long)p * LD + j]; Am[(long long)p * LD + j] = t1;
        double2 t2 = B[(long long)piv * LD + j]; B[(long long)piv * LD + j] = B[(long long)p * LD + j]; B[(long long)p * LD + j] = t2;
      }
    }
    __syncthreads();
    if (tid == 0) s_inv = cdiv(zd(1.0), ld(Am + (long long)piv * LD + piv));
    __syncthreads();
    for (int j = tid; j < nn; j += blockDim.x) {
      st(Am + (long long)piv * LD + j, ld(Am + (long long)piv * LD + j) * s_inv);
      st(B + (long long)piv * LD + j, ld(B + (long long)piv * LD + j) * s_inv);
    }
    for (int r = tid; r < nn; r += blockDim.x) fcol[r] = ld(Am + (long long)r * LD + piv);
    __syncthreads();
    for (int e = tid; e < nn * nn; e += blockDim.x) {
      const int r = e / nn, j = e % nn;
      if (r == piv) continue;
      const zd f = fcol[r];
      st(Am + (long long)r * LD + j, ld(Am + (long long)r * LD + j) - f * ld(Am + (long long)piv * LD + j));
      st(B + (long long)r * LD + j, ld(B + (long long)r * LD + j) - f * ld(B + (long long)piv * LD + j));
    }
    __syncthreads();
  }
  for (int e = tid; e < nn * nn; e += blockDim.x) {
    const int r = e / nn, col = e % nn;
    const zd v = ld(B + (long long)r * LD + col);
    if constexpr (sizeof(S) == sizeof(float2)) {   // complex64 form: hi and lo matrices (see Cinv)
      float2* Oh = reinterpret_cast<float2*>(Bout);
      const float2 hi = make_float2((float)v.re, (float)v.im);
      Oh[(long long)r * LD + col] = hi;
      Oh[(long long)LD * LD + (long long)r * LD + col] = make_float2((float)(v.re - (double)hi.x), (float)(v.im - (double)hi.y));
    } else {
      st(Bout + (long long)r * LD + col, v);
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

// Static plus dynamic shared memory above the 48 KB default needs an opt-in
// per kernel (the static arrays of the sweeps take 24-31 KB).
template <typename K>
static cudaError_t allow_smem(K kern, size_t bytes) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, kern);
  if (e != cudaSuccess) return e;
  if (a.sharedSizeBytes + bytes <= 48 * 1024) return cudaSuccess;
  if (a.sharedSizeBytes + bytes > 227 * 1024) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
// Dynamic shared memory of a sweep: the hot-chunk coefficients (N_o <= 2)
// and, in the compressed form, the staged block projections, which share one
// buffer; staging is used when it fits in 64 KiB.
template <int NO, typename S>
static size_t sweep_smem(const Dev& d, int* staged) {
  using R = typename Bulk<S>::R;
  const size_t ps = d.ring ? (size_t)d.maxl * NO * NO * d.rmax * sizeof(cx<R>) : 0;
  *staged = (d.ring && ps <= 65536) ? 1 : 0;
  return std::max(kStageBytes<NO>, *staged ? ps : (size_t)0);
}
template <int NO, typename S>
static cudaError_t sweep_ret(const Dev& d, int T, cudaStream_t s) {
  int staged = 0;
  const size_t bytes = sweep_smem<NO, S>(d, &staged);
  cudaError_t e = allow_smem(k_ret2<NO, S>, bytes);
  if (e != cudaSuccess) return e;
  k_ret2<NO, S><<<dim3(d.no, d.n_inst), 256, bytes, s>>>(d, T, staged);
  return cudaGetLastError();
}
template <int NO, typename S>
static cudaError_t sweep_les(const Dev& d, int T, cudaStream_t s) {
  int staged = 0;
  const size_t bytes = sweep_smem<NO, S>(d, &staged);
  cudaError_t e = allow_smem(k_les2<NO, S>, bytes);
  if (e != cudaSuccess) return e;
  k_les2<NO, S><<<dim3(d.no, d.n_inst), 256, bytes, s>>>(d, T, staged);
  return cudaGetLastError();
}
cudaError_t launch_ret_h(const Dev& d, int T, cudaStream_t s) {
  HK_DISPATCH(d.no, return (sweep_ret<NO, S>(d, T, s)));
  return cudaSuccess;
}
cudaError_t launch_les_h(const Dev& d, int T, cudaStream_t s) {
  HK_DISPATCH(d.no, return (sweep_les<NO, S>(d, T, s)));
  return cudaSuccess;
}
cudaError_t launch_chunk_inv(const Dev& d, int which, int c0, int c1, cudaStream_t s) {
  for (int cc = c0; cc < c1; ++cc) {
    HK_DISPATCH(d.no, (k_chunk_inv<NO, S><<<d.n_inst, 256, 0, s>>>(d, which, cc, d.cinv_ws)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace hk
