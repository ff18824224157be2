// Equilibrium (Matsubara) Dyson equation on the DLR grid, Eq. KBEM, solved
// self-consistently on the host (declared in include/hkbe.h).  It prepares
// interacting initial states; nothing here runs per time step.
//
// Representation: G^M(tau) = -sum_l c_l K(tau, w_l), K(tau, w) =
// e^{-tau w}/(1 + e^{-beta w}), whose Fourier series is sum_l c_l/(i nu - w_l)
// at fermionic nu = (2n+1) pi/beta.  Dyson, G(i nu) = [i nu - eps -
// Sigma(i nu)]^{-1}, is imposed at r frequencies chosen greedily (pivoted
// Gram-Schmidt on the rows 1/(i nu_n - w_l), |n| < n_max), where values and
// coefficients determine each other.  Sigma^M(tau) on the nodes from the
// contour functionals restricted to the imaginary branch (G^M = -i G(-i tau,0)):
//   BETHE      v^2 G
//   NAMBU      v^2 s_z G s_z  -U^2 [G_ij G_{bi bj} - G_{bi j} G_{i bj}](tau) G_{bj bi}(-tau)
//              + g^2 [(n_B+1) e^{-w0 tau} + n_B e^{w0 tau}] s_z G s_z,
//              Fock -U rho_ij [i = bar j] (rho = -G^M(beta^-)) added to eps
//   LATTICE2B  Sigma_r(tau) = -U^2 G_r(tau)^2 G_{-r}(-tau) over an L x L k-grid
// with G(-tau) = xi G(beta - tau) from the DLR reversal.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/hkbe.h"
#include "host_numerics.h"

namespace {

using zc = std::complex<double>;

// Dense LU with partial pivoting, complex, row-major n x n; solves in place
// for m right-hand sides stored row-major [n][m].  Returns false if singular.
bool zsolve(int n, std::vector<zc> A, zc* B, int m) {
  std::vector<int> piv(n);
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::abs(A[(size_t)r * n + c]) > std::abs(A[(size_t)p * n + c])) p = r;
    if (A[(size_t)p * n + c] == zc(0)) return false;
    if (p != c) {
      for (int j = 0; j < n; ++j) std::swap(A[(size_t)c * n + j], A[(size_t)p * n + j]);
      for (int j = 0; j < m; ++j) std::swap(B[(size_t)c * m + j], B[(size_t)p * m + j]);
    }
    for (int r = c + 1; r < n; ++r) {
      const zc f = A[(size_t)r * n + c] / A[(size_t)c * n + c];
      if (f == zc(0)) continue;
      for (int j = c; j < n; ++j) A[(size_t)r * n + j] -= f * A[(size_t)c * n + j];
      for (int j = 0; j < m; ++j) B[(size_t)r * m + j] -= f * B[(size_t)c * m + j];
    }
  }
  for (int j = 0; j < m; ++j)
    for (int c = n - 1; c >= 0; --c) {
      zc s = B[(size_t)c * m + j];
      for (int k = c + 1; k < n; ++k) s -= A[(size_t)c * n + k] * B[(size_t)k * m + j];
      B[(size_t)c * m + j] = s / A[(size_t)c * n + c];
    }
  return true;
}

bool zinv(int n, const zc* A, zc* out) {
  std::vector<zc> M(A, A + (size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) out[i * n + j] = (i == j) ? 1.0 : 0.0;
  return zsolve(n, M, out, n);
}

struct Solver {
  int r, no, n2;
  double beta;
  int xi;
  std::vector<double> tau, om;
  std::vector<zc> Kt, Kn;        // [r][r]
  std::vector<double> nu;        // r chosen frequencies
  hk::DLRMats dm;

  bool init(int r_, const double* tau_, const double* om_, double beta_, int no_) {
    r = r_; no = no_; n2 = no * no; beta = beta_; xi = -1;
    tau.assign(tau_, tau_ + r); om.assign(om_, om_ + r);
    Kt.resize((size_t)r * r);
    for (int i = 0; i < r; ++i)
      for (int l = 0; l < r; ++l) Kt[(size_t)i * r + l] = hk::dlr_kernel(tau[i], om[l], beta);
    if (!hk::dlr_build(r, tau_, om_, beta, xi, &dm)) return false;
    // frequency nodes: greedy pivoted Gram-Schmidt on the rows 1/(i nu_n - w_l)
    double wmax = 0.0;
    for (double w : om) wmax = std::max(wmax, std::abs(w));
    const int nmax = (int)(beta * wmax / M_PI) + 100;
    const int nrow = 2 * nmax;
    std::vector<zc> rows((size_t)nrow * r);
    std::vector<double> nuall(nrow), nrm(nrow);
    for (int q = 0; q < nrow; ++q) {
      const int n = q - nmax;
      nuall[q] = (2 * n + 1) * M_PI / beta;
      for (int l = 0; l < r; ++l) rows[(size_t)q * r + l] = 1.0 / (zc(0, nuall[q]) - om[l]);
    }
    std::vector<char> used(nrow, 0);
    for (int s = 0; s < r; ++s) {
      int best = -1;
      double bn = -1.0;
      for (int q = 0; q < nrow; ++q) {
        if (used[q]) continue;
        double v = 0.0;
        for (int l = 0; l < r; ++l) v += std::norm(rows[(size_t)q * r + l]);
        if (v > bn) { bn = v; best = q; }
      }
      if (best < 0 || bn <= 0.0) return false;
      used[best] = 1;
      nu.push_back(nuall[best]);
      const double inv = 1.0 / std::sqrt(bn);
      std::vector<zc> e(r);
      for (int l = 0; l < r; ++l) e[l] = rows[(size_t)best * r + l] * inv;
      for (int q = 0; q < nrow; ++q) {
        if (used[q]) continue;
        zc dot = 0;
        for (int l = 0; l < r; ++l) dot += std::conj(e[l]) * rows[(size_t)q * r + l];
        for (int l = 0; l < r; ++l) rows[(size_t)q * r + l] -= dot * e[l];
      }
    }
    std::sort(nu.begin(), nu.end());
    Kn.resize((size_t)r * r);
    for (int k = 0; k < r; ++k)
      for (int l = 0; l < r; ++l) Kn[(size_t)k * r + l] = 1.0 / (zc(0, nu[k]) - om[l]);
    return true;
  }
  // values on the tau nodes [r][n2] -> values at the frequency nodes [r][n2]
  bool to_freq(const zc* g, zc* gn) const {
    std::vector<zc> c(g, g + (size_t)r * n2);
    for (auto& x : c) x = -x;
    if (!zsolve(r, Kt, c.data(), n2)) return false;
    for (int k = 0; k < r; ++k)
      for (int q = 0; q < n2; ++q) {
        zc s = 0;
        for (int l = 0; l < r; ++l) s += Kn[(size_t)k * r + l] * c[(size_t)l * n2 + q];
        gn[(size_t)k * n2 + q] = s;
      }
    return true;
  }
  bool to_tau(const zc* gn, zc* g) const {
    std::vector<zc> c(gn, gn + (size_t)r * n2);
    if (!zsolve(r, Kn, c.data(), n2)) return false;
    for (int i = 0; i < r; ++i)
      for (int q = 0; q < n2; ++q) {
        zc s = 0;
        for (int l = 0; l < r; ++l) s += Kt[(size_t)i * r + l] * c[(size_t)l * n2 + q];
        g[(size_t)i * n2 + q] = -s;
      }
    return true;
  }
  void reversed(const zc* g, zc* out) const {  // g(beta - tau_i), [r][n2]
    for (int i = 0; i < r; ++i)
      for (int q = 0; q < n2; ++q) {
        zc s = 0;
        for (int c = 0; c < r; ++c) s += dm.rev[(size_t)i * r + c] * g[(size_t)c * n2 + q];
        out[(size_t)i * n2 + q] = s;
      }
  }
  bool dyson(const zc* eps, const zc* sig, zc* g) const {   // one instance
    std::vector<zc> sn((size_t)r * n2), gn((size_t)r * n2);
    if (!to_freq(sig, sn.data())) return false;
    std::vector<zc> M(n2);
    for (int k = 0; k < r; ++k) {
      for (int x = 0; x < no; ++x)
        for (int y = 0; y < no; ++y)
          M[x * no + y] = (x == y ? zc(0, nu[k]) : zc(0)) - eps[x * no + y] - sn[(size_t)k * n2 + x * no + y];
      if (!zinv(no, M.data(), &gn[(size_t)k * n2])) return false;
    }
    return to_tau(gn.data(), g);
  }
};

}  // namespace

// F = -Kn Kt^{-1} (to_freq) and B = -Kt Kn^{-1} (to_tau), each from one LU
// solve of the transposed system: Kt^T X = Kn^T gives F = -X^T, and
// Kn^T Y = Kt^T gives B = -Y^T.
bool hk::mats_maps(int r, const double* tau, const double* om, double beta, std::vector<zc>* F,
                   std::vector<zc>* B, std::vector<double>* nu) {
  Solver sv;
  if (!sv.init(r, tau, om, beta, 1)) return false;
  auto tr = [r](const std::vector<zc>& M) {
    std::vector<zc> T((size_t)r * r);
    for (int i = 0; i < r; ++i)
      for (int j = 0; j < r; ++j) T[(size_t)j * r + i] = M[(size_t)i * r + j];
    return T;
  };
  std::vector<zc> X = tr(sv.Kn), Y = tr(sv.Kt);
  if (!zsolve(r, tr(sv.Kt), X.data(), r) || !zsolve(r, tr(sv.Kn), Y.data(), r)) return false;
  F->assign((size_t)r * r, zc(0));
  B->assign((size_t)r * r, zc(0));
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < r; ++j) {
      (*F)[(size_t)i * r + j] = -X[(size_t)j * r + i];
      (*B)[(size_t)i * r + j] = -Y[(size_t)j * r + i];
    }
  *nu = sv.nu;
  return true;
}

extern "C" int hkbe_matsubara_solve(int r, const double* tau, const double* omega, double beta, int model,
                                    int n_inst, int nao, const double* eps, const double* params, int nparams,
                                    double U_eq, double eta, int n_eta, double mix, double tol, int max_iter,
                                    double* gm_out, double* eps_out, int32_t* iters, double* err_out) {
  if (!tau || !omega || !eps || !gm_out || r < 1 || r > 128 || n_inst < 1 || nao < 1 || nao > 4 || !(beta > 0) ||
      !(mix > 0 && mix <= 1) || max_iter < 1)
    return HKBE_ERR_ARG;
  if (model == HKBE_MODEL_NAMBU && nao != 2) return HKBE_ERR_ARG;
  if (model == HKBE_MODEL_LATTICE2B && nao != 1) return HKBE_ERR_ARG;
  if (model != HKBE_MODEL_NONE && model != HKBE_MODEL_BETHE && model != HKBE_MODEL_NAMBU &&
      model != HKBE_MODEL_LATTICE2B)
    return HKBE_ERR_ARG;
  if (model != HKBE_MODEL_NONE && (!params || nparams < 1)) return HKBE_ERR_ARG;
  int L = 0, ys = 0;
  if (model == HKBE_MODEL_LATTICE2B) {   // params [L] or [L, ysymm] (reflection-reduced k-set)
    L = (int)params[0];
    ys = nparams >= 2 && params[1] != 0.0;
    if (L < 1 || L > 16 || (ys && L % 2) || (ys ? L * (L / 2 + 1) : L * L) != n_inst) return HKBE_ERR_ARG;
  }
  Solver sv;
  if (!sv.init(r, tau, omega, beta, nao)) return HKBE_ERR_ARG;
  const int n2 = nao * nao;
  const size_t per = (size_t)r * n2;
  std::vector<zc> e0((size_t)n_inst * n2), G((size_t)n_inst * per), Gn(G.size()), S(G.size()), e_eff(e0.size());
  for (size_t i = 0; i < e0.size(); ++i) e0[i] = zc(eps[2 * i], eps[2 * i + 1]);
  const double s[2] = {1.0, -1.0};
  auto sigma = [&](const std::vector<zc>& Gx, std::vector<zc>& Sx) {
    std::fill(Sx.begin(), Sx.end(), zc(0));
    if (model == HKBE_MODEL_BETHE) {
      for (int n = 0; n < n_inst; ++n) {
        const double v = params[(size_t)n * nparams];
        for (size_t e = 0; e < per; ++e) Sx[n * per + e] = v * v * Gx[n * per + e];
      }
    } else if (model == HKBE_MODEL_NAMBU) {
      std::vector<zc> gm(per);
      for (int n = 0; n < n_inst; ++n) {
        const double* p = params + (size_t)n * nparams;
        const double v = p[0], g = nparams >= 3 ? p[1] : 0.0, w0 = nparams >= 3 ? p[2] : 1.0;
        const zc* Gi = &Gx[n * per];
        zc* Si = &Sx[n * per];
        sv.reversed(Gi, gm.data());
        for (auto& x : gm) x *= (double)sv.xi;    // G(-tau)
        const double nb = g != 0.0 ? 1.0 / std::expm1(beta * w0) : 0.0;
        for (int i = 0; i < r; ++i) {
          const zc* a = Gi + (size_t)i * 4;
          const zc* b = gm.data() + (size_t)i * 4;
          const double dph = g != 0.0 ? g * g * ((nb + 1) * std::exp(-w0 * tau[i]) + nb * std::exp(w0 * tau[i])) : 0.0;
          for (int x = 0; x < 2; ++x)
            for (int y = 0; y < 2; ++y) {
              const int bx = 1 - x, by = 1 - y;
              zc val = (v * v + dph) * s[x] * s[y] * a[x * 2 + y];
              val += -U_eq * U_eq * (a[x * 2 + y] * a[bx * 2 + by] - a[bx * 2 + y] * a[x * 2 + by]) * b[by * 2 + bx];
              Si[(size_t)i * 4 + x * 2 + y] = val;
            }
        }
      }
    } else if (model == HKBE_MODEL_LATTICE2B) {
      // grid point q = m_x L + m_y lives in instance kin(q); with ysymm the
      // point (m_x, L - m_y) is the mirror of (m_x, m_y) and shares its instance
      const int N = L * L;
      auto kin = [&](int q) { const int y = q % L; return ys ? (q / L) * (L / 2 + 1) + std::min(y, L - y) : q; };
      std::vector<zc> gr((size_t)N * r), gmr((size_t)N * r), sr((size_t)N * r), gmk((size_t)n_inst * r), tmp(r);
      for (int q = 0; q < n_inst; ++q) {   // G_k(-tau)
        sv.reversed(&Gx[(size_t)q * r], tmp.data());
        for (int i = 0; i < r; ++i) gmk[(size_t)q * r + i] = (double)sv.xi * tmp[i];
      }
      // G_r = (1/N) sum_k e^{ikr} G_k,  G_{-r}(-tau) = (1/N) sum_k e^{-ikr} G_k(-tau)
      for (int rr = 0; rr < N; ++rr) {
        const int rx = rr / L, ry = rr % L;
        for (int q = 0; q < N; ++q) {
          const int mx = q / L, my = q % L, nq = kin(q);
          const double ph = 2.0 * M_PI * (double)(mx * rx + my * ry) / L;
          const zc e(std::cos(ph), std::sin(ph));
          for (int i = 0; i < r; ++i) {
            gr[(size_t)rr * r + i] += e * Gx[(size_t)nq * r + i] / (double)N;
            gmr[(size_t)rr * r + i] += std::conj(e) * gmk[(size_t)nq * r + i] / (double)N;
          }
        }
        for (int i = 0; i < r; ++i)
          sr[(size_t)rr * r + i] = -U_eq * U_eq * gr[(size_t)rr * r + i] * gr[(size_t)rr * r + i] * gmr[(size_t)rr * r + i];
      }
      for (int q = 0; q < N; ++q) {    // Sigma_k = sum_r e^{-ikr} Sigma_r
        const int mx = q / L, my = q % L;
        if (ys && my > L / 2) continue;   // a mirror point: its instance is filled by (m_x, L - m_y)
        for (int rr = 0; rr < N; ++rr) {
          const int rx = rr / L, ry = rr % L;
          const double ph = 2.0 * M_PI * (double)(mx * rx + my * ry) / L;
          const zc e(std::cos(ph), -std::sin(ph));
          for (int i = 0; i < r; ++i) Sx[(size_t)kin(q) * r + i] += e * sr[(size_t)rr * r + i];
        }
      }
    }
  };
  auto update_eps = [&](int it) {
    e_eff = e0;
    if (model != HKBE_MODEL_NAMBU) return;
    for (int n = 0; n < n_inst; ++n) {
      zc rho[4] = {0, 0, 0, 0};   // rho = -G^M(beta^-) = -sum_c ebeta_c G(tau_c)
      for (int c = 0; c < r; ++c)
        for (int q = 0; q < 4; ++q) rho[q] -= sv.dm.ebeta[c] * G[n * per + (size_t)c * 4 + q];
      e_eff[(size_t)n * 4 + 1] += -U_eq * rho[1] + (it <= n_eta ? eta : 0.0);
      e_eff[(size_t)n * 4 + 2] += -U_eq * rho[2] + (it <= n_eta ? eta : 0.0);
    }
  };
  // start: the non-interacting G^M of eps
  std::fill(S.begin(), S.end(), zc(0));
  for (int n = 0; n < n_inst; ++n)
    if (!sv.dyson(&e0[(size_t)n * n2], &S[n * per], &G[n * per])) return HKBE_ERR_NAN;
  int it = 0;
  double err = INFINITY;
  for (it = 1; it <= max_iter; ++it) {
    update_eps(it);
    sigma(G, S);
    for (int n = 0; n < n_inst; ++n)
      if (!sv.dyson(&e_eff[(size_t)n * n2], &S[n * per], &Gn[n * per])) return HKBE_ERR_NAN;
    err = 0.0;
    for (size_t e = 0; e < G.size(); ++e) err = std::max(err, std::abs(Gn[e] - G[e]));
    if (!std::isfinite(err)) return HKBE_ERR_NAN;
    if (err < tol && it > n_eta) {
      G = Gn;
      break;
    }
    for (size_t e = 0; e < G.size(); ++e) G[e] = (it > 1 ? mix : 1.0) * Gn[e] + (it > 1 ? 1.0 - mix : 0.0) * G[e];
  }
  for (size_t e = 0; e < G.size(); ++e) {
    gm_out[2 * e] = G[e].real();
    gm_out[2 * e + 1] = G[e].imag();
  }
  if (eps_out)
    for (size_t e = 0; e < e_eff.size(); ++e) {
      eps_out[2 * e] = e_eff[e].real();
      eps_out[2 * e + 1] = e_eff[e].imag();
    }
  if (iters) *iters = it > max_iter ? max_iter : it;
  if (err_out) *err_out = err;
  return (it > max_iter) ? HKBE_ERR_NOCONV : HKBE_OK;
}
