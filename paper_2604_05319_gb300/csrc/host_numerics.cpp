// Host-side numerics of the library: Appendix A weights and the DLR matrices.
// Everything here runs once at set-up time; the per-step path is on the GPU.
#include "host_numerics.h"

#include <cmath>
#include <cstring>
#include <vector>

namespace hk {

// ---------------------------------------------------------------------------
// Appendix A weights.  P = M^-1 with M_ja = j^a is formed by Gauss-Jordan in
// long double; D_ml = sum_{a>=1} P_al a m^(a-1); I_mnl = sum_a P_al
// (n^(a+1) - m^(a+1))/(a+1); a_j = -D_0j.  Gregory end weights omega_i are the
// partial sums of the (k+1)-step Adams-Moulton weights, b_j = int_k^{k+1} of
// the Lagrange basis polynomial of node k+1-j on nodes 0..k+1.
// ---------------------------------------------------------------------------
static void vandermonde_inverse(int k, long double* P /*(k+1)^2, P[a*(k+1)+l]*/) {
  const int n = k + 1;
  long double A[6][12];
  for (int j = 0; j < n; ++j) {
    for (int a = 0; a < n; ++a) A[j][a] = std::pow((long double)j, (long double)a);
    for (int c = 0; c < n; ++c) A[j][n + c] = (j == c) ? 1.0L : 0.0L;
  }
  if (n >= 1) A[0][0] = 1.0L;  // 0^0 = 1
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r][c]) > std::fabs(A[p][c])) p = r;
    if (p != c)
      for (int j = 0; j < 2 * n; ++j) std::swap(A[c][j], A[p][j]);
    long double d = A[c][c];
    for (int j = 0; j < 2 * n; ++j) A[c][j] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      long double f = A[r][c];
      for (int j = 0; j < 2 * n; ++j) A[r][j] -= f * A[c][j];
    }
  }
  // M P = I  ->  rows of A's right half are M^-1 rows indexed [j][c]; M^-1 is (a, l)
  for (int a = 0; a < n; ++a)
    for (int l = 0; l < n; ++l) P[a * n + l] = A[a][n + l];
}

static long double lagrange_integral(int npts, int j, long double lo, long double hi) {
  // integral over [lo, hi] of prod_{m != j} (x - m)/(j - m), nodes 0..npts-1
  long double coef[8] = {1.0L};
  int deg = 0;
  long double den = 1.0L;
  for (int m = 0; m < npts; ++m) {
    if (m == j) continue;
    den *= (long double)(j - m);
    long double nc[8] = {0};
    for (int p = 0; p <= deg; ++p) {
      nc[p + 1] += coef[p];
      nc[p] -= coef[p] * (long double)m;
    }
    ++deg;
    for (int p = 0; p <= deg; ++p) coef[p] = nc[p];
  }
  long double s = 0;
  for (int p = 0; p <= deg; ++p)
    s += coef[p] * (std::pow(hi, (long double)(p + 1)) - std::pow(lo, (long double)(p + 1))) / (p + 1);
  return s / den;
}

void weights_build(int k, Weights* w) {
  std::memset(w, 0, sizeof(Weights));
  w->k = k;
  const int n = k + 1;
  long double P[36];
  vandermonde_inverse(k, P);
  for (int m = 0; m < n; ++m)
    for (int l = 0; l < n; ++l) {
      long double d = 0;
      for (int a = 1; a < n; ++a) d += P[a * n + l] * a * std::pow((long double)m, (long double)(a - 1));
      w->D[m][l] = (double)d;
    }
  for (int nn = 0; nn < n; ++nn)
    for (int l = 0; l < n; ++l) {
      long double s = 0;
      for (int a = 0; a < n; ++a) s += P[a * n + l] * std::pow((long double)nn, (long double)(a + 1)) / (a + 1);
      w->I0[nn][l] = (double)s;
    }
  for (int j = 0; j < n; ++j) {
    long double d = 0;
    for (int a = 1; a < n; ++a) d += P[a * n + j] * a * (a == 1 ? 1.0L : 0.0L);  // m = 0
    w->a[j] = (double)(-d);
  }
  long double acc = 0;
  for (int i = 0; i < n; ++i) {
    acc += lagrange_integral(k + 2, k + 1 - i, (long double)k, (long double)(k + 1));
    w->omega[i] = (double)acc;
  }
}

double rule_weight(const Weights& w, int n, int l) {
  const int k = w.k;
  if (n <= 0) return 0.0;
  if (n <= k) return (l <= k) ? w.I0[n][l] : 0.0;
  if (n < 2 * k + 1) {
    double s = 0;
    if (l <= k) s += w.I0[n - k][l];
    if (l >= n - k && l <= n) s += w.I0[k][l - (n - k)];
    return s;
  }
  if (l < 0 || l > n) return 0.0;
  if (l <= k) return w.omega[l];
  if (l >= n - k) return w.omega[n - l];
  return 1.0;
}

// I_{m,n,l} = I_{0,n,l} - I_{0,m,l}
double integ_weight(const Weights& w, int m, int n, int l) { return w.I0[n][l] - w.I0[m][l]; }

// ---------------------------------------------------------------------------
// DLR matrices.  Fermionic kernel K(x, w) = c(w) exp(-x w),
// c(w) = 1/(1+exp(-beta w)), evaluated in log form (no overflow for |beta w|
// up to ~700).  Cardinal functions l(x) = K^-T k(x) by LU solves.
// ---------------------------------------------------------------------------
static double softplus(double x) { return x > 0 ? x + std::log1p(std::exp(-x)) : std::log1p(std::exp(x)); }
static double log_c(double w, double beta) { return -softplus(-beta * w); }
static double log_K(double x, double w, double beta) { return -x * w + log_c(w, beta); }
double dlr_kernel(double x, double w, double beta) { return std::exp(log_K(x, w, beta)); }

// LU with partial pivoting (row-major n x n), in place
static bool lu_factor(int n, std::vector<double>& A, std::vector<int>& piv) {
  piv.resize(n);
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[p * n + c])) p = r;
    piv[c] = p;
    if (A[p * n + c] == 0.0) return false;
    if (p != c)
      for (int j = 0; j < n; ++j) std::swap(A[c * n + j], A[p * n + j]);
    for (int r = c + 1; r < n; ++r) {
      A[r * n + c] /= A[c * n + c];
      double f = A[r * n + c];
      for (int j = c + 1; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
    }
  }
  return true;
}
// solve A^T x = b for each of nrhs columns of B (B is n x nrhs row-major)
static void lu_solve_T(int n, const std::vector<double>& LU, const std::vector<int>& piv,
                       double* B, int nrhs) {
  // A = P^T L U  (row swaps recorded in piv) ; A^T = U^T L^T P
  // solve U^T y = b, L^T z = y, x = P^T z
  for (int c = 0; c < nrhs; ++c) {
    for (int i = 0; i < n; ++i) {
      double s = B[i * nrhs + c];
      for (int j = 0; j < i; ++j) s -= LU[j * n + i] * B[j * nrhs + c];
      B[i * nrhs + c] = s / LU[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = B[i * nrhs + c];
      for (int j = i + 1; j < n; ++j) s -= LU[j * n + i] * B[j * nrhs + c];
      B[i * nrhs + c] = s;
    }
    for (int i = n - 1; i >= 0; --i)
      if (piv[i] != i) std::swap(B[i * nrhs + c], B[piv[i] * nrhs + c]);
  }
}

bool dlr_build(int r, const double* tau, const double* om, double beta, int xi, DLRMats* out) {
  out->r = r;
  std::vector<double> K(r * r);
  for (int i = 0; i < r; ++i)
    for (int l = 0; l < r; ++l) K[i * r + l] = dlr_kernel(tau[i], om[l], beta);
  std::vector<int> piv;
  std::vector<double> LU = K;
  if (!lu_factor(r, LU, piv)) return false;
  // cardinal row at x: l(x) K = k(x)  ->  K^T l^T = k(x)^T
  auto cardinal = [&](double x, double* row) {
    for (int l = 0; l < r; ++l) row[l] = dlr_kernel(x, om[l], beta);
    lu_solve_T(r, LU, piv, row, 1);
  };
  out->e0.resize(r);
  out->ebeta.resize(r);
  out->rev.resize(r * r);
  cardinal(0.0, out->e0.data());
  cardinal(beta, out->ebeta.data());
  for (int i = 0; i < r; ++i) cardinal(beta - tau[i], &out->rev[i * r]);
  // Q and Phi integrate products of cardinal functions.  The cardinal
  // functions are bounded (they interpolate), but their DLR coefficients are
  // not (|K^-1| grows like cond(K)), so the integrals are taken in node space:
  // each l(x) comes from one LU solve and the integral uses tanh-sinh
  // quadrature, whose nodes cluster doubly exponentially at both interval
  // ends where exp(-x w) has its boundary layers.
  auto tanh_sinh = [](double a, double b, std::vector<double>& xs, std::vector<double>& ws) {
    xs.clear();
    ws.clear();
    const double hstep = 1.0 / 48.0, half = 0.5 * (b - a), mid = 0.5 * (a + b);
    for (int j = -6 * 48; j <= 6 * 48; ++j) {
      const double t = j * hstep;
      const double u = 0.5 * M_PI * std::sinh(t);
      const double ch = std::cosh(u);
      const double w = hstep * 0.5 * M_PI * std::cosh(t) / (ch * ch);
      if (w * half < 1e-300) continue;
      // x = mid + half tanh(u), written to keep the distance to the nearer end exact
      const double e = std::exp(-2.0 * std::fabs(u));
      const double dist = half * 2.0 * e / (1.0 + e);   // half (1 - |tanh u|)
      const double x = (u < 0) ? a + dist : b - dist;
      xs.push_back(x);
      ws.push_back(w * half);
    }
  };
  std::vector<double> xs, ws, La((size_t)r), Lc((size_t)r);
  out->q.assign((size_t)r * r, 0.0);
  tanh_sinh(0.0, beta, xs, ws);
  for (size_t p = 0; p < xs.size(); ++p) {
    cardinal(xs[p], La.data());
    for (int a = 0; a < r; ++a)
      for (int b = 0; b < r; ++b) out->q[a * r + b] += ws[p] * La[a] * La[b];
  }
  // phi[a][c][i] = int_0^beta l_a(u) l_c^ext(u - tau_i) du, split at u = tau_i
  out->phi.assign((size_t)r * r * r, 0.0);
  for (int i = 0; i < r; ++i) {
    const double t = tau[i];
    for (int part = 0; part < 2; ++part) {
      if (part == 0) tanh_sinh(0.0, t, xs, ws);
      else tanh_sinh(t, beta, xs, ws);
      for (size_t p = 0; p < xs.size(); ++p) {
        cardinal(xs[p], La.data());
        const double arg = (part == 0) ? xs[p] - t + beta : xs[p] - t;
        cardinal(arg, Lc.data());
        const double f = ws[p] * ((part == 0) ? (double)xi : 1.0);
        for (int a = 0; a < r; ++a) {
          const double fa = f * La[a];
          double* row = &out->phi[(size_t)a * r * r];
          for (int c = 0; c < r; ++c) row[(size_t)c * r + i] += fa * Lc[c];
        }
      }
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// Hermitian eigen-decomposition of a small matrix (cyclic complex Jacobi),
// used for the mean-field guess of the bootstrap (green_from_H).
// ---------------------------------------------------------------------------
void herm_eig(int n, const std::complex<double>* A, double* E, std::complex<double>* U) {
  using zc = std::complex<double>;
  zc a[4][4], v[4][4];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      a[i][j] = 0.5 * (A[i * n + j] + std::conj(A[j * n + i]));
      v[i][j] = (i == j) ? 1.0 : 0.0;
    }
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += std::norm(a[p][q]);
    if (off < 1e-30) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double g = std::abs(a[p][q]);
        if (g < 1e-300) continue;
        zc ph = a[p][q] / g;  // a_pq = g e^{i phi}
        double app = a[p][p].real(), aqq = a[q][q].real();
        double theta = 0.5 * std::atan2(2 * g, aqq - app);
        double c = std::cos(theta), s = std::sin(theta);
        // rotation R acting on columns p, q: [c, s*ph; -s*conj(ph), c]
        for (int k2 = 0; k2 < n; ++k2) {
          zc akp = a[k2][p], akq = a[k2][q];
          a[k2][p] = c * akp - s * std::conj(ph) * akq;
          a[k2][q] = s * ph * akp + c * akq;
        }
        for (int k2 = 0; k2 < n; ++k2) {
          zc apk = a[p][k2], aqk = a[q][k2];
          a[p][k2] = c * apk - s * ph * aqk;
          a[q][k2] = s * std::conj(ph) * apk + c * aqk;
        }
        for (int k2 = 0; k2 < n; ++k2) {
          zc vkp = v[k2][p], vkq = v[k2][q];
          v[k2][p] = c * vkp - s * std::conj(ph) * vkq;
          v[k2][q] = s * ph * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) {
    E[i] = a[i][i].real();
    for (int j = 0; j < n; ++j) U[i * n + j] = v[i][j];
  }
}

}  // namespace hk
