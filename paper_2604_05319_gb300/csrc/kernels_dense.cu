// Dense FP64 kernels of one Kadanoff-Baym time step (Eqs. KBER, KBET, KBEL,
// Appendix A weights) and of the bootstrap square (Sec. 3.3).
//
// Storage is lower-triangular per instance: element (T, t), t <= T, of the
// N_o x N_o matrices lives at ((n*ntri + T(T+1)/2 + t) * N_o^2).  GL(T, t)
// holds G^<(t, T) (the paper's G^<_{t1 t2} = G^<(t2, t1)).
//
// Per self-consistency iteration at step T the launches are
//   k_sigma  Sigma^R(T, .), Sigma^<(., T), Sigma^tv(T, .) from the current G
//   (the retarded row, Eq. KBER, is solved by k_ret2 in kernels_sweep.cu)
//   k_mixed  G^tv(T, tau_i) (Eq. KBET), one warp per (instance, node)
//   k_vt     v_a = sum_b Q_ab G^vt(tau_b, T) and x_0 = -[G^tv(T, 0)]^dagger
//   k_src    lesser source q(t), t = 0..T, one warp per (instance, t)
//   k_les    lesser column x_t = G^<(t, T) (Eq. KBEL), one CTA per
//            (instance, orbital column): start block t <= k solved together,
//            then chunks of 32 points: far-field history sums in parallel over
//            the CTA, near field + point solve sequentially in one warp.  The
//            stepper uses the chunked sweep k_les2 (kernels_sweep.cu); k_les
//            serves the allocation-free entry point
//   k_rho    diagonal density-matrix update (Sec. 3.3), when selected
// Each kernel folds max |new - old| of what it writes into err[instance].
#include "dev_util.cuh"

namespace hk {

// ---------------------------------------------------------------------------
// Self-energy functionals (Sec. 3 / Eq. Hybrid; bath level model)
// ---------------------------------------------------------------------------

template <int NO>
__device__ void bath_sigma(const double* mp, zd g0, double eb_dt_sign, int which, const Dev& d,
                           double tphase, double tauv, zd* out) {
  // which: 0 retarded (-i e^{-i eb dt}), 1 lesser (i n_b e^{-i eb dt}),
  //        2 mixed (-xi i n_b e^{-i eb t} e^{eb tau});  dt passed in tphase
  const int nb = (int)mp[0];
  for (int x = 0; x < NO; ++x)
    for (int y = 0; y < NO; ++y) out[x * NO + y] = zd();
  for (int b = 0; b < nb; ++b) {
    const double eb = mp[1 + b];
    zd g;
    double s, c;
    sincos(-eb * tphase, &s, &c);
    zd ph(c, s);
    if (which == 0) g = zd(0, -1) * ph;
    else if (which == 1) g = zd(0, fermi(eb, d.beta)) * ph;
    else g = zd(0, -(double)d.xi * fermi(eb, d.beta)) * ph * exp(eb * tauv);
    const double* V = mp + 1 + nb;  // V[x][b] interleaved
    for (int x = 0; x < NO; ++x) {
      zd vx(V[2 * (x * nb + b)], V[2 * (x * nb + b) + 1]);
      for (int y = 0; y < NO; ++y) {
        zd vy(V[2 * (y * nb + b)], V[2 * (y * nb + b) + 1]);
        out[x * NO + y] += vx * g * vy.conj();
      }
    }
  }
  (void)g0; (void)eb_dt_sign;
}

// Nambu DMFT self-energy (N_o = 2): driven hybridisation of Eq. Hybrid plus
// the second-Born bubble and exchange of Eq. Sigma2B, element by element
//   Delta_ij(t,t') = v^2 s_i s_j G_ij(t,t') cos(s_i A(t) - s_j A(t')), s = (1,-1),
//   Sigma^>(T,t)_ij = U(T)U(t) [X_ij X_{bi bj} - X_{bi j} X_{i bj}] Y_{bj bi},
//   X = G^>(T,t), Y = G^<(t,T); Sigma^< likewise with X = G^<(T,t), Y = G^>(t,T);
// Sigma^R = Sigma^> - Sigma^< for t <= T.  bar i = 1 - i.
__device__ __forceinline__ void nambu_bar(const zd* X, const zd* Y, double u, zd* out) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int bi = 1 - i, bj = 1 - j;
      out[i * 2 + j] = (X[i * 2 + j] * X[bi * 2 + bj] - X[bi * 2 + j] * X[i * 2 + bj]) * Y[bj * 2 + bi] * u;
    }
}
template <typename S>
__device__ void nambu_sigma(const Dev& d, int n, int T, int idx) {
  const double* mp = d.mpar + (long long)n * MP;
  const double v2 = mp[0] * mp[0];
  const double* A = d.drA + (long long)n * (d.nt + 1);
  const double* U = d.drU + (long long)n * (d.nt + 1);
  const double s[2] = {1.0, -1.0};
  if (idx <= T) {
    const int t = idx;
    zd GR[4], GLc[4], GLr[4], GGr[4], GGc[4], Sg[4], Sl[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) { GR[q] = ldx<2, S>(d, 0, n, T, t, q); GLc[q] = ldx<2, S>(d, 1, n, T, t, q); }  // GLc: G^<(t, T)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) GLr[i * 2 + j] = -GLc[j * 2 + i].conj();     // G^<(T, t)
#pragma unroll
    for (int q = 0; q < 4; ++q) GGr[q] = GR[q] + GLr[q];                       // G^>(T, t)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) GGc[i * 2 + j] = -GGr[j * 2 + i].conj();     // G^>(t, T)
    const double uu = U[T + 1] * U[t + 1];
    nambu_bar(GGr, GLc, uu, Sg);
    nambu_bar(GLr, GGc, uu, Sl);
    // optional Holstein coupling (unrenormalised Migdal, free phonon of w0):
    // Sigma^≷ += i g^2 D0^≷(T,t) s_i s_j G^≷_ij(T,t)
    const double g = mp[1], w0 = mp[2];
    zd dg = zd(), dl = zd();
    if (g != 0.0) {
      const double nb = 1.0 / expm1(d.beta * w0), x = w0 * (T - t) * d.h;
      double sx, cx;
      sincos(x, &sx, &cx);
      dg = zd(0, -1) * (zd(cx, -sx) * (nb + 1.0) + zd(cx, sx) * nb) * zd(0, g * g);
      dl = zd(0, -1) * (zd(cx, sx) * (nb + 1.0) + zd(cx, -sx) * nb) * zd(0, g * g);
    }
    zd slr[4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const double w = v2 * s[i] * s[j] * cos(s[i] * A[T + 1] - s[j] * A[t + 1]);
        const double ssij = s[i] * s[j];
        const zd mg = dg * GGr[i * 2 + j] * ssij, ml = dl * GLr[i * 2 + j] * ssij;
        stx<2, S>(d, 2, n, T, t, i * 2 + j, Sg[i * 2 + j] - Sl[i * 2 + j] + GR[i * 2 + j] * w + mg - ml);
        slr[i * 2 + j] = Sl[i * 2 + j] + GLr[i * 2 + j] * w + ml;               // Sigma^<(T, t)
      }
#pragma unroll
    for (int i = 0; i < 2; ++i)                                                  // stores Sigma^<(t, T)
#pragma unroll
      for (int j = 0; j < 2; ++j) stx<2, S>(d, 3, n, T, t, i * 2 + j, -slr[j * 2 + i].conj());
    if (t == T) {  // Fock term of Eq. SigmaF, Sigma^F_ij = -U(T) rho_ij [i = bar j], rho = xi i G^<(T,T)
      const zd rxi(0, (double)d.xi);
      const double2* ee = d.eps_ext + ((long long)n * (d.nt + 1) + T + 1) * 4;
      double2* e = d.eps + ((long long)n * (d.nt + 1) + T + 1) * 4;
      st(e + 0, ld(ee + 0));
      st(e + 3, ld(ee + 3));
      st(e + 1, ld(ee + 1) - GLc[1] * rxi * U[T + 1]);
      st(e + 2, ld(ee + 2) - GLc[2] * rxi * U[T + 1]);
    }
  } else if (idx > 2 * T + 1) {
    const int i = idx - 2 * (T + 1), r = d.r;
    zd Gtv[4], Gvt[4], Sb[4];
    const double2* pt = tv<2>(d.GTV, d, n, T, i);
#pragma unroll
    for (int q = 0; q < 4; ++q) Gtv[q] = ld(pt + q);
    zd gb[4] = {zd(), zd(), zd(), zd()};          // G^tv(T, beta - tau_i)
    for (int c = 0; c < r; ++c) {
      const double rv = d.rev[i * r + c];
      const double2* pc = tv<2>(d.GTV, d, n, T, c);
#pragma unroll
      for (int q = 0; q < 4; ++q) gb[q] += ld(pc + q) * rv;
    }
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
      for (int y = 0; y < 2; ++y) Gvt[x * 2 + y] = gb[y * 2 + x].conj() * (-(double)d.xi);  // G^vt(tau_i, T)
    nambu_bar(Gtv, Gvt, U[T + 1] * U[0], Sb);
    const double g = mp[1], w0 = mp[2];
    zd dtv = zd();
    if (g != 0.0) {  // i g^2 D0^tv(T, tau_i)
      const double nb = 1.0 / expm1(d.beta * w0), tT = T * d.h, ta = d.tau[i];
      double sx, cx;
      sincos(w0 * tT, &sx, &cx);
      dtv = zd(0, -1) * (zd(cx, sx) * ((nb + 1.0) * exp(-w0 * ta)) + zd(cx, -sx) * (nb * exp(w0 * ta))) * zd(0, g * g);
    }
    double2* so = tv<2>(d.STV, d, n, T, i);
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
      for (int y = 0; y < 2; ++y)
        st(so + x * 2 + y, Sb[x * 2 + y] + Gtv[x * 2 + y] * (v2 * s[x] * s[y] * cos(s[x] * A[T + 1] - s[y] * A[0])) +
                               dtv * Gtv[x * 2 + y] * (s[x] * s[y]));
  }
}

template <int NO, typename S>
__global__ void k_sigma(Dev d, int T) {
  constexpr int NO2 = NO * NO;
  const int n = blockIdx.y;
  if (!d.active[n]) return;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int total = 2 * (T + 1) + d.r;
  if (idx >= total) return;
  if constexpr (NO == 2) {
    if (d.model == 3) {
      nambu_sigma<S>(d, n, T, idx);
      return;
    }
  }
  const double* mp = d.mpar + (long long)n * MP;
  // src / dst are S* for the two-time rows, double2* for the mixed row
  auto apply = [&](const auto* src, auto* dst, int which, double tph, double tauv) {
    if (d.model == 1) {  // Bethe: Sigma = v^2 G
      const double v2 = mp[0] * mp[0];
#pragma unroll
      for (int e = 0; e < NO2; ++e) st(dst + e, ld(src + e) * v2);
    } else if (d.model == 2) {
      zd out[NO2];
      bath_sigma<NO>(mp, zd(), 0.0, which, d, tph, tauv, out);
#pragma unroll
      for (int e = 0; e < NO2; ++e) st(dst + e, out[e]);
    } else {
#pragma unroll
      for (int e = 0; e < NO2; ++e) st(dst + e, zd());
    }
  };
  if (idx <= 2 * T + 1) {   // two-time rows: read G and write Sigma in FP64 where the form keeps FP64 copies
    const int X = idx <= T ? 0 : 1, t = idx <= T ? idx : idx - (T + 1);
    zd out[NO2];
    if (d.model == 1) {  // Bethe: Sigma = v^2 G
      const double v2 = mp[0] * mp[0];
#pragma unroll
      for (int e = 0; e < NO2; ++e) out[e] = ldx<NO, S>(d, X, n, T, t, e) * v2;
    } else if (d.model == 2) {
      bath_sigma<NO>(mp, zd(), 0.0, X, d, X == 0 ? (T - t) * d.h : (t - T) * d.h, 0.0, out);
    } else {
#pragma unroll
      for (int e = 0; e < NO2; ++e) out[e] = zd();
    }
#pragma unroll
    for (int e = 0; e < NO2; ++e) stx<NO, S>(d, X + 2, n, T, t, e, out[e]);
  } else {
    const int i = idx - 2 * (T + 1);
    apply(tv<NO>(d.GTV, d, n, T, i), tv<NO>(d.STV, d, n, T, i), 2, T * d.h, d.tau[i]);
  }
}

// ---------------------------------------------------------------------------
// Extrapolated initial guess for step T (Sec. 3.4): degree-k polynomial along
// the diagonal through the previous k+1 points, e_l = (-1)^l C(k+1, l+1).
// ---------------------------------------------------------------------------
template <int NO, typename S>
__global__ void k_extrap(Dev d, int T) {
  constexpr int NO2 = NO * NO;
  const int n = blockIdx.y;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = d.k;
  if (idx >= 2 * (T + 1) + d.r || T > d.last[n]) return;
  double e[6];
  {
    double c = 1.0;  // C(k+1, l+1) built incrementally
    for (int l = 0; l <= k; ++l) {
      c = (l == 0) ? (double)(k + 1) : c * (double)(k + 1 - l) / (double)(l + 1);
      e[l] = (l & 1) ? -c : c;
    }
  }
  zd acc[NO2];
  for (int q = 0; q < NO2; ++q) acc[q] = zd();
  if (idx <= 2 * T + 1) {   // G^R row (X = 0) or G^< column (X = 1), from the FP64 copies where kept
    const int X = idx <= T ? 0 : 1, tp = idx <= T ? idx : idx - (T + 1);
    if (X == 0 && tp == T) {
      for (int x = 0; x < NO; ++x) acc[x * NO + x] = zd(0, -1);
    } else if (tp >= k + 1 || tp == 0) {
      for (int l = 0; l <= k; ++l) {
        const int c = (tp == 0) ? 0 : tp - 1 - l;
        for (int q = 0; q < NO2; ++q) acc[q] += ldx<NO, S>(d, X, n, T - 1 - l, c, q) * e[l];
      }
    } else {
      for (int q = 0; q < NO2; ++q) acc[q] = ldx<NO, S>(d, X, n, T - 1, tp - 1, q);
    }
    for (int q = 0; q < NO2; ++q) stx<NO, S>(d, X, n, T, tp, q, acc[q]);
    return;
  } else {
    const int i = idx - 2 * (T + 1);
    for (int l = 0; l <= k; ++l) {
      const double2* s = tv<NO>(d.GTV, d, n, T - 1 - l, i);
      for (int q = 0; q < NO2; ++q) acc[q] += ld(s + q) * e[l];
    }
    double2* dtv = tv<NO>(d.GTV, d, n, T, i);
    for (int q = 0; q < NO2; ++q) st(dtv + q, acc[q]);
  }
}

constexpr int CH = 32;     // chunk of the sequential sweeps
constexpr int NWARP = 8;   // warps per sweep CTA

// ---------------------------------------------------------------------------
// Mixed component at step T, Eq. KBET (one warp per (instance, node)).
// ---------------------------------------------------------------------------
template <int NO, typename S>
__global__ void k_mixed(Dev d, int T) {
  constexpr int NO2 = NO * NO;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int n = gw / d.r, i = gw % d.r;
  if (n >= d.n_inst || !d.active[n]) return;
  const int k = d.k;
  const double h = d.h;
  const DevW& W = d.w;
  zd acc[NO2];
#pragma unroll
  for (int q = 0; q < NO2; ++q) acc[q] = zd();
  if constexpr (sizeof(S) == sizeof(float2)) {
    // complex64 form: h sum_l w_l Sigma^R(T,l) G^tv(l, tau_i) with FP32 products
    // (G^tv truncated to FP32 on the integer pipes) in compensated FP32 sums
    KAcc<float> ka[NO2];
    const float hf = (float)h;
    for (int l0 = lane; l0 < T; l0 += 32 * 4) {
      zf pa[NO2];
#pragma unroll
      for (int q = 0; q < NO2; ++q) pa[q] = zf(0.f);
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int l = l0 + 32 * jj;
        if (l < T) {
          const float wl = hf * rule_wr<float>(W, T, l);
          const S* sp = el<NO, S>(d.SR, d, n, T, l);
          const double2* gp = tv<NO>(d.GTV, d, n, l, i);
          zf g[NO2];
#pragma unroll
          for (int q = 0; q < NO2; ++q) g[q] = ld_f32(gp + q);
#pragma unroll
          for (int x = 0; x < NO; ++x)
#pragma unroll
            for (int z = 0; z < NO; ++z) {
              const zf sx = ldr<float>(sp + x * NO + z) * wl;
#pragma unroll
              for (int y = 0; y < NO; ++y) pa[x * NO + y] = cfma(sx, g[z * NO + y], pa[x * NO + y]);
            }
        }
      }
#pragma unroll
      for (int q = 0; q < NO2; ++q) ka[q].add(pa[q]);
    }
#pragma unroll
    for (int q = 0; q < NO2; ++q) acc[q] = ka[q].get();
  } else {
    for (int l = lane; l < T; l += 32) {  // h sum_l w_l Sigma^R(T,l) G^tv(l, tau_i)
      const double wl = h * rule_w(W, T, l);
      M<NO> Sm = load<NO>(el<NO, S>(d.SR, d, n, T, l));
      M<NO> G = load<NO>(tv<NO>(d.GTV, d, n, l, i));
#pragma unroll
      for (int x = 0; x < NO; ++x)
#pragma unroll
        for (int z = 0; z < NO; ++z) {
          zd sx = Sm.a[x][z] * wl;
#pragma unroll
          for (int y = 0; y < NO; ++y) acc[x * NO + y] = cfma(sx, G.a[z][y], acc[x * NO + y]);
        }
    }
  }
  for (int a = lane; a < d.r; a += 32) {  // sum_a Sigma^tv(T, tau_a) W[a][i]
    M<NO> Sm = load<NO>(tv<NO>(d.STV, d, n, T, a));
    M<NO> C = load<NO>(d.wconv + (((long long)n * d.r + a) * d.r + i) * NO2);
    mac<NO>(*reinterpret_cast<M<NO>*>(acc), Sm, C, zd(1.0));
  }
  if (lane >= 1 && lane <= k) {
    M<NO> G = load<NO>(tv<NO>(d.GTV, d, n, T - lane, i));
    const zd c(0, -W.a[lane] / h);
#pragma unroll
    for (int q = 0; q < NO2; ++q) acc[q] += c * G.a[q / NO][q % NO];
  }
  warp_sum<NO2>(acc);
  if (lane == 0) {
    const double wt = h * rule_w(W, T, T);
    M<NO> Mm, R;
    const S* sd = el<NO, S>(d.SR, d, n, T, T);
    const double2* ep = epsp<NO>(d, n, T);
#pragma unroll
    for (int x = 0; x < NO; ++x)
#pragma unroll
      for (int y = 0; y < NO; ++y) {
        Mm.a[x][y] = (x == y ? zd(0, W.a[0] / h) : zd()) - ld(ep + x * NO + y) - ld(sd + x * NO + y) * wt;
        R.a[x][y] = acc[x * NO + y];
      }
    M<NO> X = solve_left<NO>(Mm, R);
    double2* p = tv<NO>(d.GTV, d, n, T, i);
    M<NO> old = load<NO>(p);
    store<NO>(p, X);
    atomic_max_nonneg(d.err + n, maxabs_diff<NO>(X, old));
  }
}

// v_a = sum_b Q_ab G^vt(tau_b, T), G^vt(tau_b, T) = -xi [G^tv(T, beta - tau_b)]^dagger,
// x_0 = -[G^tv(T, 0+)]^dagger.  One CTA per instance, thread per node.
template <int NO, typename S>
__global__ void k_vt(Dev d, int T) {
  constexpr int NO2 = NO * NO;
  const int n = blockIdx.x;
  if (!d.active[n]) return;
  extern __shared__ zd gvt[];  // [r][NO2]
  const int r = d.r;
  for (int b = threadIdx.x; b < r; b += blockDim.x) {
    M<NO> acc = M<NO>::zero();
    for (int c = 0; c < r; ++c) {
      M<NO> G = load<NO>(tv<NO>(d.GTV, d, n, T, c));
      const double rv = d.rev[b * r + c];
#pragma unroll
      for (int q = 0; q < NO2; ++q) acc.a[q / NO][q % NO] += G.a[q / NO][q % NO] * rv;
    }
    M<NO> g = scale<NO>(dag<NO>(acc), zd(-(double)d.xi));
#pragma unroll
    for (int q = 0; q < NO2; ++q) gvt[b * NO2 + q] = g.a[q / NO][q % NO];
  }
  __syncthreads();
  for (int a = threadIdx.x; a < r; a += blockDim.x) {
    zd acc[NO2];
#pragma unroll
    for (int q = 0; q < NO2; ++q) acc[q] = zd();
    for (int b = 0; b < r; ++b) {
      const double qv = d.q[a * r + b];
#pragma unroll
      for (int q = 0; q < NO2; ++q) acc[q] += gvt[b * NO2 + q] * qv;
    }
    double2* p = d.vvec + ((long long)n * r + a) * NO2;
#pragma unroll
    for (int q = 0; q < NO2; ++q) st(p + q, acc[q]);
  }
  if (threadIdx.x == 0) {
    M<NO> acc = M<NO>::zero();
    for (int c = 0; c < r; ++c) {
      M<NO> G = load<NO>(tv<NO>(d.GTV, d, n, T, c));
#pragma unroll
      for (int q = 0; q < NO2; ++q) acc.a[q / NO][q % NO] += G.a[q / NO][q % NO] * d.e0[c];
    }
    store<NO>(d.x0 + (long long)n * NO2, scale<NO>(dag<NO>(acc), zd(-1.0)));
  }
}

// Lesser source q(t) = h sum_l w^(T)_l Sigma^<(t,l) G^A(l,T) - i sum_a Sigma^tv(t,tau_a) v_a
template <int NO, typename S>
__global__ void k_src(Dev d, int T) {
  constexpr int NO2 = NO * NO;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int n = gw / (T + 1), t = gw % (T + 1);
  if (n >= d.n_inst || !d.active[n]) return;
  const double h = d.h;
  zd acc[NO2];
#pragma unroll
  for (int q = 0; q < NO2; ++q) acc[q] = zd();
  for (int l = lane; l <= T; l += 32) {
    const double wl = h * rule_w(d.w, T, l);
    M<NO> Sm;
#pragma unroll
    for (int x = 0; x < NO; ++x)
#pragma unroll
      for (int y = 0; y < NO; ++y) Sm.a[x][y] = sless<NO, S>(d, n, t, l, x, y);
    M<NO> GA = dag<NO>(load<NO>(el<NO, S>(d.GR, d, n, T, l)));
    mac<NO>(*reinterpret_cast<M<NO>*>(acc), Sm, GA, zd(wl));
  }
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
// Lesser column, Eq. KBEL: x_t = G^<(t, T), left-multiplying VIDE in t.
// ---------------------------------------------------------------------------
template <int NO, typename S>
__global__ void __launch_bounds__(256) k_les(Dev d, int T) {
  constexpr int NO2 = NO * NO;
  const int n = blockIdx.y, jc = blockIdx.x;
  if (!d.active[n]) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = d.k;
  const double h = d.h;
  const DevW& W = d.w;
  __shared__ zd sA[20 * 20];
  __shared__ zd sB[20];
  __shared__ zd farsh[CH][NO];
  __shared__ zd xch[CH][NO];
  __shared__ double serr;
  if (tid == 0) serr = 0.0;
  S* colp = el<NO, S>(d.GL, d, n, T, 0);  // G^<(t, T) at colp + t NO2
  auto xptr = [&](int t) { return colp + (long long)t * NO2; };   // element [m][jc] at + m*NO + jc
  const double2* qs = d.qsrc + (long long)n * d.nt * NO2;
  double myerr = 0.0;
  const int last = (d.rho_mode == 1) ? T - 1 : T;
  if (warp == 0) {
    // x_0
    if (lane < NO) {
      const int m = lane;
      zd v = ld(d.x0 + (long long)n * NO2 + m * NO + jc);
      S* p = xptr(0) + m * NO + jc;
      myerr = fmax(myerr, sqrt((v - ld(p)).abs2()));
      st(p, v);
    }
    __syncwarp();
    const int ns = k * NO;
    for (int e = lane; e < ns * ns; e += 32) {
      const int row = e / ns, col = e % ns;       // row (t, m), col (l, y)
      const int t = row / NO + 1, m = row % NO, l = col / NO + 1, y = col % NO;
      zd v = srx<NO, S>(d, n, t, l, m, y) * (-h * W.I0[t][l]);
      if (m == y) v += zd(0, W.D[t][l] / h);
      if (l == t) v -= ld(epsp<NO>(d, n, t) + m * NO + y);
      sA[row * ns + col] = v;
    }
    for (int row = lane; row < ns; row += 32) {
      const int t = row / NO + 1, m = row % NO;
      zd b = ld(qs + t * NO2 + m * NO + jc);
      for (int y = 0; y < NO; ++y) {
        zd c = srx<NO, S>(d, n, t, 0, m, y) * (-h * W.I0[t][0]);
        if (m == y) c += zd(0, W.D[t][0] / h);
        if (t == 0) c -= ld(epsp<NO>(d, n, t) + m * NO + y);
        b -= c * ld(xptr(0) + y * NO + jc);
      }
      sB[row] = b;
    }
    __syncwarp();
    warp_lu_solve(ns, sA, sB, 1, nullptr);
    for (int row = lane; row < ns; row += 32) {
      const int t = row / NO + 1, m = row % NO;
      if (t > last) continue;
      S* p = xptr(t) + m * NO + jc;
      myerr = fmax(myerr, sqrt((sB[row] - ld(p)).abs2()));
      st(p, sB[row]);
    }
  }
  __syncthreads();
  for (int t0 = k + 1; t0 <= last; t0 += CH) {
    const int cn = min(CH, last + 1 - t0);
    // far field: warp w handles rows t = t0 + w + 8 i, lanes over l < t0
    for (int tl = warp; tl < cn; tl += NWARP) {
      const int t = t0 + tl;
      zd acc[NO];
#pragma unroll
      for (int m = 0; m < NO; ++m) acc[m] = zd();
      const S* srow = el<NO, S>(d.SR, d, n, t, 0);
      for (int l = lane; l < t0; l += 32) {
        const double wl = rule_w(W, t, l);
        const S* sr = srow + (long long)l * NO2;
        const S* xl = xptr(l);
#pragma unroll
        for (int y = 0; y < NO; ++y) {
          const zd xy = ld(xl + y * NO + jc) * wl;
#pragma unroll
          for (int m = 0; m < NO; ++m) acc[m] = cfma(ld(sr + m * NO + y), xy, acc[m]);
        }
      }
      warp_sum<NO>(acc);
      if (lane == 0)
#pragma unroll
        for (int m = 0; m < NO; ++m) farsh[tl][m] = acc[m] * h;
    }
    __syncthreads();
    if (warp == 0) {
      for (int tl = 0; tl < cn; ++tl) {
        const int t = t0 + tl;
        zd part[NO];
#pragma unroll
        for (int m = 0; m < NO; ++m) part[m] = zd();
        if (lane < tl) {
          const int l = t0 + lane;
          const double wl = h * rule_w(W, t, l);
          const S* sr = el<NO, S>(d.SR, d, n, t, l);
#pragma unroll
          for (int y = 0; y < NO; ++y) {
            const zd xy = xch[lane][y] * wl;
#pragma unroll
            for (int m = 0; m < NO; ++m) part[m] = cfma(ld(sr + m * NO + y), xy, part[m]);
          }
        }
        if (lane >= 1 && lane <= k) {
          const int tj = t - lane;
          const zd c = zd(0, -W.a[lane] / h);
#pragma unroll
          for (int m = 0; m < NO; ++m) {
            const zd xm = (tj >= t0) ? xch[tj - t0][m] : ld(xptr(tj) + m * NO + jc);
            part[m] += c * xm;
          }
        }
        warp_sum<NO>(part);
        if (lane == 0) {
          zd rhs[NO], x[NO];
#pragma unroll
          for (int m = 0; m < NO; ++m) rhs[m] = part[m] + farsh[tl][m] + ld(qs + (long long)t * NO2 + m * NO + jc);
          const double wt = h * rule_w(W, t, t);
          const S* sd = el<NO, S>(d.SR, d, n, t, t);
          const double2* ep = epsp<NO>(d, n, t);
          M<NO> Mm;
#pragma unroll
          for (int x2 = 0; x2 < NO; ++x2)
#pragma unroll
            for (int y = 0; y < NO; ++y)
              Mm.a[x2][y] = (x2 == y ? zd(0, W.a[0] / h) : zd()) - ld(ep + x2 * NO + y) - ld(sd + x2 * NO + y) * wt;
          solve_col<NO>(Mm, rhs, x);
#pragma unroll
          for (int m = 0; m < NO; ++m) {
            S* p = xptr(t) + m * NO + jc;
            myerr = fmax(myerr, sqrt((x[m] - ld(p)).abs2()));
            st(p, x[m]);
            xch[tl][m] = x[m];
          }
        }
        __syncwarp();
      }
    }
    __syncthreads();
  }
  myerr = warp_max(myerr);
  if (lane == 0 && myerr > 0) atomic_max_nonneg(&serr, myerr);
  __syncthreads();
  if (tid == 0) atomic_max_nonneg(d.err + n, serr);
}

// ---------------------------------------------------------------------------
// Diagonal density matrix (Sec. 3.3): (a_0/h) rho + i (A rho - rho A^dag) =
//   -(1/h) sum_{j>=1} a_j rho(T-j) + xi (r0 + r0^dag),
// A = eps(T) + h w_T Sigma^R(T,T), r0 = h sum_{l<T} w_l Sigma^R(T,l) x_l + q(T).
// ---------------------------------------------------------------------------
template <int NO, typename S>
__global__ void k_rho(Dev d, int T) {
  constexpr int NO2 = NO * NO;
  const int n = blockIdx.x;
  if (!d.active[n]) return;
  const double h = d.h;
  __shared__ zd part[8][NO2];
  zd acc[NO2];
#pragma unroll
  for (int q = 0; q < NO2; ++q) acc[q] = zd();
  for (int l = threadIdx.x; l < T; l += blockDim.x) {
    const double wl = h * rule_w(d.w, T, l);
    M<NO> Sm = load<NO>(el<NO, S>(d.SR, d, n, T, l));
    M<NO> X = load<NO>(el<NO, S>(d.GL, d, n, T, l));
    mac<NO>(*reinterpret_cast<M<NO>*>(acc), Sm, X, zd(wl));
  }
  warp_sum<NO2>(acc);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
    for (int q = 0; q < NO2; ++q) part[warp][q] = acc[q];
  __syncthreads();
  if (threadIdx.x != 0) return;
  zd r0[NO2];
  for (int q = 0; q < NO2; ++q) {
    r0[q] = ld(d.qsrc + ((long long)n * d.nt + T) * NO2 + q);
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) r0[q] += part[w2][q];
  }
  const double xi = d.xi;
  const double wt = h * rule_w(d.w, T, T);
  M<NO> A, rhs;
  const S* sd = el<NO, S>(d.SR, d, n, T, T);
  const double2* ep = epsp<NO>(d, n, T);
  for (int x = 0; x < NO; ++x)
    for (int y = 0; y < NO; ++y) {
      A.a[x][y] = ld(ep + x * NO + y) + ld(sd + x * NO + y) * wt;
      rhs.a[x][y] = (r0[x * NO + y] + r0[y * NO + x].conj()) * xi;
    }
  constexpr bool f64 = sizeof(S) == sizeof(double2);  // else: FP64 diagonal history in diag64
  for (int j = 1; j <= d.k; ++j) {
    const M<NO> gd = f64 ? load<NO>(el<NO, S>(d.GL, d, n, T - j, T - j))
                         : load<NO>(d.diag64 + ((long long)n * d.nt + T - j) * NO2);
    M<NO> rho = scale<NO>(gd, zd(0, xi));
    rhs = rhs - scale<NO>(rho, zd(d.w.a[j] / h));
  }
  // L vec(rho) = vec(rhs), vec row-major, L[(x,y),(u,v)]
  zd L[NO2 * NO2], b[NO2];
  for (int p = 0; p < NO2; ++p) {
    const int u = p / NO, v = p % NO;
    for (int q = 0; q < NO2; ++q) {
      const int x = q / NO, y = q % NO;
      // (a0/h) E + i (A E - E A^dag) with E = e_u e_v^T
      zd val = (x == u && y == v) ? zd(d.w.a[0] / h) : zd();
      if (y == v) val += zd(0, 1) * A.a[x][u];
      if (x == u) val -= zd(0, 1) * A.a[y][v].conj();
      L[q * NO2 + p] = val;
    }
    b[p] = rhs.a[u][v];
  }
  for (int c = 0; c < NO2; ++c) {  // Gaussian elimination with pivoting
    int pv = c;
    for (int r = c + 1; r < NO2; ++r)
      if (L[r * NO2 + c].abs2() > L[pv * NO2 + c].abs2()) pv = r;
    if (pv != c) {
      for (int j = 0; j < NO2; ++j) { zd t = L[c * NO2 + j]; L[c * NO2 + j] = L[pv * NO2 + j]; L[pv * NO2 + j] = t; }
      zd t = b[c]; b[c] = b[pv]; b[pv] = t;
    }
    for (int r = c + 1; r < NO2; ++r) {
      zd f = cdiv(L[r * NO2 + c], L[c * NO2 + c]);
      for (int j = c; j < NO2; ++j) L[r * NO2 + j] -= f * L[c * NO2 + j];
      b[r] -= f * b[c];
    }
  }
  for (int c = NO2 - 1; c >= 0; --c) {
    zd s = b[c];
    for (int j = c + 1; j < NO2; ++j) s -= L[c * NO2 + j] * b[j];
    b[c] = cdiv(s, L[c * NO2 + c]);
  }
  S* p = el<NO, S>(d.GL, d, n, T, T);
  double e = 0.0;
  for (int q = 0; q < NO2; ++q) {
    zd x = b[q] * zd(0, -xi);  // G^<(T,T) = -i xi rho
    e = fmax(e, sqrt((x - ld(p + q)).abs2()));
    st(p + q, x);
    if (d.ring64[1]) st(el64<NO>(d, 1, n, T, T) + q, x);
    if (!f64) st(d.diag64 + ((long long)n * d.nt + T) * NO2 + q, x);
  }
  atomic_max_nonneg(d.err + n, e);
}

template <int NO, typename S>
__global__ void k_diag_seed(Dev d) {
  constexpr int NO2 = NO * NO;
  const int n = blockIdx.x;
  for (int e = threadIdx.x; e < (d.k + 1) * NO2; e += blockDim.x) {
    const int t = e / NO2, q = e % NO2;
    st(d.diag64 + ((long long)n * d.nt + t) * NO2 + q, ld(el<NO, S>(d.GL, d, n, t, t) + q));
  }
  // FP64 copies of the start square's G^R and G^< rows (complex64 compressed form)
  const int sq = (d.k + 1) * (d.k + 2) / 2;
  for (int X = 0; X < 2; ++X) {
    if (!d.ring64[X]) continue;
    for (int e = threadIdx.x; e < sq * NO2; e += blockDim.x) {
      const int el_ = e / NO2, q = e % NO2;
      int T = 0;
      while ((T + 1) * (T + 2) / 2 <= el_) ++T;
      const int t = el_ - T * (T + 1) / 2;
      st(el64<NO>(d, X, n, T, t) + q, ld(el<NO, S>(ringX(d, X), d, n, T, t) + q));
    }
  }
}

// ---------------------------------------------------------------------------
// Bootstrap square t <= k (Sec. 3.3, polynomial weights of Appendix A).
// ---------------------------------------------------------------------------
template <int NO, typename S>
__global__ void __launch_bounds__(256) k_boot_mixed(Dev d) {
  constexpr int NO2 = NO * NO;
  const int n = blockIdx.x;
  if (!d.active[n]) return;
  const int k = d.k, r = d.r, ns = k * NO;
  const double h = d.h;
  const DevW& W = d.w;
  __shared__ zd sA[20 * 20];
  __shared__ int piv[20];
  // G^tv(0, tau_i) = i xi G^M(beta - tau_i)
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    M<NO> acc = M<NO>::zero();
    for (int c = 0; c < r; ++c) {
      M<NO> G = load<NO>(d.gm + ((long long)n * r + c) * NO2);
      const double rv = d.rev[i * r + c];
#pragma unroll
      for (int q = 0; q < NO2; ++q) acc.a[q / NO][q % NO] += G.a[q / NO][q % NO] * rv;
    }
    double2* p = tv<NO>(d.GTV, d, n, 0, i);
    M<NO> v = scale<NO>(acc, zd(0, (double)d.xi));
    atomic_max_nonneg(d.err + n, maxabs_diff<NO>(v, load<NO>(p)));
    store<NO>(p, v);
  }
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int e = lane; e < ns * ns; e += 32) {
      const int row = e / ns, col = e % ns;
      const int m = row / NO + 1, x = row % NO, l = col / NO + 1, y = col % NO;
      zd v = srx<NO, S>(d, n, m, l, x, y) * (-h * W.I0[m][l]);
      if (x == y) v += zd(0, W.D[m][l] / h);
      if (l == m) v -= ld(epsp<NO>(d, n, m) + x * NO + y);
      sA[row * ns + col] = v;
    }
    __syncwarp();
    warp_lu_solve(ns, sA, nullptr, 0, piv);
  }
  __syncthreads();
  // one right-hand side per (node i, column y)
  for (int col = threadIdx.x; col < r * NO; col += blockDim.x) {
    const int i = col / NO, y = col % NO;
    zd b[20];
    for (int m = 1; m <= k; ++m)
      for (int x = 0; x < NO; ++x) {
        zd s = zd();
        for (int a = 0; a < r; ++a) {  // C(m, tau_i) = sum_a Sigma^tv(m, a) W[a][i]
          const double2* Sa = tv<NO>(d.STV, d, n, m, a);
          const double2* C = d.wconv + (((long long)n * r + a) * r + i) * NO2;
          for (int z = 0; z < NO; ++z) s += ld(Sa + x * NO + z) * ld(C + z * NO + y);
        }
        for (int z = 0; z < NO; ++z) {
          zd c0 = srx<NO, S>(d, n, m, 0, x, z) * (-h * W.I0[m][0]);
          if (x == z) c0 += zd(0, W.D[m][0] / h);
          s -= c0 * ld(tv<NO>(d.GTV, d, n, 0, i) + z * NO + y);
        }
        b[(m - 1) * NO + x] = s;
      }
    lu_apply(ns, sA, piv, b);
    double e = 0.0;
    for (int m = 1; m <= k; ++m)
      for (int x = 0; x < NO; ++x) {
        double2* p = tv<NO>(d.GTV, d, n, m, i) + x * NO + y;
        e = fmax(e, sqrt((b[(m - 1) * NO + x] - ld(p)).abs2()));
        st(p, b[(m - 1) * NO + x]);
      }
    atomic_max_nonneg(d.err + n, e);
  }
}

template <int NO, typename S>
__global__ void k_boot_ret(Dev d) {
  constexpr int NO2 = NO * NO;
  const int n = blockIdx.x;
  if (!d.active[n]) return;
  const int k = d.k, lane = threadIdx.x;
  const double h = d.h;
  const DevW& W = d.w;
  __shared__ zd sA[20 * 20];
  __shared__ zd sB[20 * 4];
  for (int m = 0; m <= k; ++m)
    if (lane < NO2) st(el<NO, S>(d.GR, d, n, m, m) + lane, (lane / NO == lane % NO) ? zd(0, -1) : zd());
  __syncwarp();
  double e = 0.0;
  for (int c = 0; c < k; ++c) {  // column n' = c
    const int nu = (k - c) * NO;
    for (int idx = lane; idx < nu * nu; idx += 32) {
      const int row = idx / nu, col = idx % nu;
      const int m = row / NO + c + 1, x = row % NO, l = col / NO + c + 1, y = col % NO;
      zd v = srx<NO, S>(d, n, m, l, x, y) * (-h * (W.I0[m][l] - W.I0[c][l]));
      if (x == y) v += zd(0, W.D[m][l] / h);
      if (l == m) v -= ld(epsp<NO>(d, n, m) + x * NO + y);
      sA[row * nu + col] = v;
    }
    for (int idx = lane; idx < nu * NO; idx += 32) {
      const int row = idx / NO, y = idx % NO;
      const int m = row / NO + c + 1, x = row % NO;
      zd s = zd();
      for (int l = 0; l <= c; ++l)
        for (int z = 0; z < NO; ++z) {
          zd blk = srx<NO, S>(d, n, m, l, x, z) * (-h * (W.I0[m][l] - W.I0[c][l]));
          if (x == z) blk += zd(0, W.D[m][l] / h);
          // gx(l) = G^R(l, c) for l >= c, -[G^R(c, l)]^dagger for l < c
          zd g = (l >= c) ? ld(el<NO, S>(d.GR, d, n, l, c) + z * NO + y)
                          : -ld(el<NO, S>(d.GR, d, n, c, l) + y * NO + z).conj();
          s -= blk * g;
        }
      sB[row * NO + y] = s;
    }
    __syncwarp();
    warp_lu_solve(nu, sA, sB, NO, nullptr);
    for (int idx = lane; idx < nu * NO; idx += 32) {
      const int row = idx / NO, y = idx % NO;
      const int m = row / NO + c + 1, x = row % NO;
      S* p = el<NO, S>(d.GR, d, n, m, c) + x * NO + y;
      e = fmax(e, sqrt((sB[row * NO + y] - ld(p)).abs2()));
      st(p, sB[row * NO + y]);
    }
    __syncwarp();
  }
  e = warp_max(e);
  if (lane == 0) atomic_max_nonneg(d.err + n, e);
}

template <int NO, typename S>
__global__ void k_boot_les(Dev d) {
  constexpr int NO2 = NO * NO;
  const int n = blockIdx.x;
  if (!d.active[n]) return;
  const int k = d.k, r = d.r, lane = threadIdx.x;
  const double h = d.h, xi = d.xi;
  const DevW& W = d.w;
  __shared__ zd sA[20 * 20];
  __shared__ zd sB[20 * 4];
  __shared__ zd x0s[NO2];
  double2* vv = d.vvec + (long long)n * r * NO2;
  double e = 0.0;
  for (int m = 0; m <= k; ++m) {
    // x_0 = -[G^tv(m, 0)]^dagger ; v_a = sum_b Q_ab (-xi) [sum_c Rev_bc G^tv(m, c)]^dagger
    if (lane < NO2) {
      const int x = lane / NO, y = lane % NO;
      zd s = zd();
      for (int c = 0; c < r; ++c) s += ld(tv<NO>(d.GTV, d, n, m, c) + y * NO + x) * d.e0[c];
      x0s[lane] = -s.conj();
      S* p = el<NO, S>(d.GL, d, n, m, 0) + lane;
      e = fmax(e, sqrt((x0s[lane] - ld(p)).abs2()));
      st(p, x0s[lane]);
    }
    for (int idx = lane; idx < r * NO2; idx += 32) {
      const int a = idx / NO2, q = idx % NO2, x = q / NO, y = q % NO;
      zd s = zd();
      for (int b = 0; b < r; ++b) {
        zd g = zd();
        for (int c = 0; c < r; ++c) g += ld(tv<NO>(d.GTV, d, n, m, c) + y * NO + x) * d.rev[b * r + c];
        s += g.conj() * (-xi * d.q[a * r + b]);
      }
      st(vv + idx, s);
    }
    __syncwarp();
    if (m == 0) continue;
    // column m solves the start block t = 1..k for every x(t) = G^<(t, m) and
    // keeps t <= m (entries t > m belong to the lower triangle of column t)
    const int nu = k * NO;
    for (int idx = lane; idx < nu * nu; idx += 32) {
      const int row = idx / nu, col = idx % nu;
      const int t = row / NO + 1, x = row % NO, l = col / NO + 1, y = col % NO;
      zd v = srx<NO, S>(d, n, t, l, x, y) * (-h * W.I0[t][l]);
      if (x == y) v += zd(0, W.D[t][l] / h);
      if (l == t) v -= ld(epsp<NO>(d, n, t) + x * NO + y);
      sA[row * nu + col] = v;
    }
    for (int idx = lane; idx < nu * NO; idx += 32) {
      const int row = idx / NO, y = idx % NO;
      const int t = row / NO + 1, x = row % NO;
      zd s = zd();
      // q_m(t) = h sum_{l=0}^{k} I_{0,m,l} Sigma^<(t,l) G^A_x(l,m) - i sum_a Sigma^tv(t,a) v_a
      for (int l = 0; l <= k; ++l) {
        const double wl = h * W.I0[m][l];
        for (int z = 0; z < NO; ++z) {
          zd ga = (l <= m) ? ld(el<NO, S>(d.GR, d, n, m, l) + y * NO + z).conj()
                           : -ld(el<NO, S>(d.GR, d, n, l, m) + z * NO + y);
          s += sless<NO, S>(d, n, t, l, x, z) * ga * wl;
        }
      }
      for (int a = 0; a < r; ++a)
        for (int z = 0; z < NO; ++z)
          s += ld(tv<NO>(d.STV, d, n, t, a) + x * NO + z) * ld(vv + a * NO2 + z * NO + y) * zd(0, -1);
      for (int z = 0; z < NO; ++z) {  // known point l = 0
        zd blk = srx<NO, S>(d, n, t, 0, x, z) * (-h * W.I0[t][0]);
        if (x == z) blk += zd(0, W.D[t][0] / h);
        s -= blk * x0s[z * NO + y];
      }
      sB[row * NO + y] = s;
    }
    __syncwarp();
    warp_lu_solve(nu, sA, sB, NO, nullptr);
    for (int idx = lane; idx < nu * NO; idx += 32) {
      const int row = idx / NO, y = idx % NO;
      const int t = row / NO + 1, x = row % NO;
      if (t > m) continue;
      S* p = el<NO, S>(d.GL, d, n, m, t) + x * NO + y;
      e = fmax(e, sqrt((sB[row * NO + y] - ld(p)).abs2()));
      st(p, sB[row * NO + y]);
    }
    __syncwarp();
  }
  e = warp_max(e);
  if (lane == 0) atomic_max_nonneg(d.err + n, e);
}

// Per-instance convergence bookkeeping after an iteration.
__global__ void k_set_active(Dev d, double tol, int iter, int min_iter, int* any) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= d.n_inst) return;
  if (!d.active[n]) return;
  const double e = d.err[n];
  if ((e < tol && iter >= min_iter) || !(e == e)) d.active[n] = 0;
  else atomicOr(any, 1);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
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

cudaError_t launch_extrapolate(const Dev& d, int T, cudaStream_t s) {
  dim3 g((2 * (T + 1) + d.r + 127) / 128, d.n_inst);
  HK_DISPATCH(d.no, (k_extrap<NO, S><<<g, 128, 0, s>>>(d, T)));
  return cudaGetLastError();
}
cudaError_t launch_sigma(const Dev& d, int T, cudaStream_t s) {
  if (d.model == 4) return launch_sigma_lattice(d, T, s);
  dim3 g((2 * (T + 1) + d.r + 127) / 128, d.n_inst);
  HK_DISPATCH(d.no, (k_sigma<NO, S><<<g, 128, 0, s>>>(d, T)));
  return cudaGetLastError();
}
cudaError_t launch_mixed(const Dev& d, int T, cudaStream_t s) {
  const long long warps = (long long)d.n_inst * d.r;
  HK_DISPATCH(d.no, (k_mixed<NO, S><<<(unsigned)((warps * 32 + 127) / 128), 128, 0, s>>>(d, T)));
  return cudaGetLastError();
}
cudaError_t launch_vt(const Dev& d, int T, cudaStream_t s) {
  HK_DISPATCH(d.no, (k_vt<NO, S><<<d.n_inst, 128, d.r * NO * NO * sizeof(zd), s>>>(d, T)));
  return cudaGetLastError();
}
cudaError_t launch_src(const Dev& d, int T, cudaStream_t s) {
  const long long warps = (long long)d.n_inst * (T + 1);
  HK_DISPATCH(d.no, (k_src<NO, S><<<(unsigned)((warps * 32 + 127) / 128), 128, 0, s>>>(d, T)));
  return cudaGetLastError();
}
cudaError_t launch_les(const Dev& d, int T, cudaStream_t s) {
  dim3 g(d.no, d.n_inst);
  HK_DISPATCH(d.no, (k_les<NO, S><<<g, 256, 0, s>>>(d, T)));
  return cudaGetLastError();
}
cudaError_t launch_rho(const Dev& d, int T, cudaStream_t s) {
  HK_DISPATCH(d.no, (k_rho<NO, S><<<d.n_inst, 256, 0, s>>>(d, T)));
  return cudaGetLastError();
}
cudaError_t launch_diag_seed(const Dev& d, cudaStream_t s) {
  if (!d.diag64) return cudaSuccess;
  HK_DISPATCH(d.no, (k_diag_seed<NO, S><<<d.n_inst, 128, 0, s>>>(d)));
  return cudaGetLastError();
}
cudaError_t launch_boot(const Dev& d, cudaStream_t s) {
  for (int t = 0; t <= d.k; ++t) {
    cudaError_t e = launch_sigma(d, t, s);
    if (e != cudaSuccess) return e;
  }
  HK_DISPATCH(d.no, (k_boot_mixed<NO, S><<<d.n_inst, 256, 0, s>>>(d)));
  HK_DISPATCH(d.no, (k_boot_ret<NO, S><<<d.n_inst, 32, 0, s>>>(d)));
  HK_DISPATCH(d.no, (k_boot_les<NO, S><<<d.n_inst, 32, 0, s>>>(d)));
  return cudaGetLastError();
}
cudaError_t launch_set_active(const Dev& d, double tol, int iter, int min_iter, int* any, cudaStream_t s) {
  k_set_active<<<(d.n_inst + 127) / 128, 128, 0, s>>>(d, tol, iter, min_iter, any);
  return cudaGetLastError();
}

}  // namespace hk
