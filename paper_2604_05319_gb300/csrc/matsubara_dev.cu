// Equilibrium Dyson equation on the DLR grid (Eq. KBEM, Sec. 2.5, 3.2) solved
// by kernels: the iteration of hkbe_matsubara_solve (matsubara.cpp) with every
// step on the device.  One iteration:
//   Sigma^M(tau_i) from the current G^M (the contour functionals restricted
//     to the imaginary branch: v^2 G for BETHE; hybridisation, Holstein and
//     second-Born bubble/exchange for NAMBU; -U^2 G_r(tau)^2 G_{-r}(-tau) for
//     LATTICE2B through the real-space grid), with G(-tau) = xi G(beta - tau)
//     from the DLR reversal;
//   Dyson at r fermionic frequencies nu_k: Sigma(i nu_k) = F Sigma(tau),
//     G(i nu_k) = [i nu_k - eps - Sigma(i nu_k)]^{-1} (N_o x N_o, Gauss-Jordan
//     with partial pivoting), G_new(tau_i) = B G(i nu);
//   err = max |G_new - G|, then linear mixing (host decides from err).
// F and B are the fixed r x r maps of the DLR representation (host set-up).
#include <cuda_runtime.h>

#include "common.cuh"
#include "lattice.cuh"
#include "matsubara_dev.h"

namespace hk {

// ---- Sigma^M(tau_i), one CTA per instance (BETHE, NAMBU, NONE) ----------
template <int NO>
__global__ void __launch_bounds__(128) k_mats_sigma(MatsDev m) {
  constexpr int N2 = NO * NO;
  __shared__ zd gneg[128 * N2];   // G(-tau_i) = xi sum_c rev[i][c] G(tau_c)
  const int n = blockIdx.x, r = m.r;
  const double2* G = m.G + (size_t)n * r * N2;
  double2* S = m.S + (size_t)n * r * N2;
  const double* p = m.mpar + (size_t)n * MP;
  if (m.model == kMatsNambu) {
    for (int e = threadIdx.x; e < r * N2; e += blockDim.x) {
      const int i = e / N2, q = e % N2;
      zd s = zd();
      for (int c = 0; c < r; ++c) s += ld(G + (size_t)c * N2 + q) * m.rev[i * r + c];
      gneg[e] = s * (double)m.xi;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < r * N2; e += blockDim.x) {
    const int i = e / N2, q = e % N2;
    zd val = zd();
    if (m.model == kMatsBethe) {
      val = ld(G + e) * (p[0] * p[0]);
    } else if (m.model == kMatsNambu) {
      // Nambu (N_o = 2): s = diag(1, -1); hybridisation v^2 s G s, Holstein
      // g^2 [(n_B + 1) e^{-w0 tau} + n_B e^{w0 tau}] s G s, and the second-Born
      // bubble and exchange -U^2 [G_xy G_bxby - G_bxy G_xby](tau) G_byx(-tau)
      const int x = q / 2, y = q % 2, bx = 1 - x, by = 1 - y;
      const double v = p[0], g = p[1], w0 = p[2];   // [v] or [v, g, w0]; unset entries are 0
      double dph = 0.0;
      if (g != 0.0) {
        const double nb = 1.0 / expm1(m.beta * w0);
        dph = g * g * ((nb + 1.0) * exp(-w0 * m.tau[i]) + nb * exp(w0 * m.tau[i]));
      }
      const double sx = x ? -1.0 : 1.0, sy = y ? -1.0 : 1.0;
      const double2* a = G + (size_t)i * 4;
      const zd* b = gneg + i * 4;
      val = ld(a + x * 2 + y) * ((v * v + dph) * sx * sy);
      val += (ld(a + x * 2 + y) * ld(a + bx * 2 + by) - ld(a + bx * 2 + y) * ld(a + x * 2 + by)) * b[by * 2 + bx] *
             (-m.U * m.U);
    }
    st(S + e, val);
  }
}

// ---- Sigma^M(tau_i) of LATTICE2B, one CTA per DLR node ------------------
// thread q owns grid point q = m_x L + m_y (instance lat_inst(q)) and the
// real-space point (q / L, q % L):
//   G_r(tau) = (1/N) sum_k e^{ikr} G_k(tau),  G_{-r}(-tau) = (1/N) sum_k e^{-ikr} G_k(-tau),
//   Sigma_r = -U^2 G_r^2 G_{-r}(-tau),  Sigma_k = sum_r e^{-ikr} Sigma_r.
__global__ void __launch_bounds__(kLatMaxK) k_mats_sigma_lattice(MatsDev m) {
  __shared__ zd X[kLatMaxK], Y[kLatMaxK], tmp[kLatMaxK], tw[16];
  const int L = m.L, N = L * L, q = threadIdx.x, i = blockIdx.x, r = m.r;
  const int nq = lat_inst(q, L, m.ys);
  lat_twiddles(tw, L);
  if (q < N) {
    const double2* G = m.G + (size_t)nq * r;
    X[q] = ld(G + i);
    zd s = zd();
    for (int c = 0; c < r; ++c) s += ld(G + c) * m.rev[i * r + c];
    Y[q] = s * (double)m.xi;
  }
  __syncthreads();
  lat_dft2(X, tmp, tw, L, +1, 1.0 / N);
  lat_dft2(Y, tmp, tw, L, -1, 1.0 / N);
  if (q < N) X[q] = X[q] * X[q] * Y[q] * (-m.U * m.U);
  __syncthreads();
  lat_dft2(X, tmp, tw, L, -1, 1.0);
  if (q < N && lat_owner(q, L, m.ys)) st(m.S + (size_t)nq * r + i, X[q]);
}

// in-place inverse of an N x N complex matrix in registers (Gauss-Jordan,
// partial pivoting); false if a pivot is exactly zero
template <int N>
__device__ bool small_inv(zd* A, zd* Inv) {
#pragma unroll
  for (int i = 0; i < N * N; ++i) Inv[i] = zd(i / N == i % N ? 1.0 : 0.0);
#pragma unroll
  for (int c = 0; c < N; ++c) {
    int p = c;
    double best = A[c * N + c].abs2();
#pragma unroll
    for (int rr = c + 1; rr < N; ++rr)
      if (A[rr * N + c].abs2() > best) { best = A[rr * N + c].abs2(); p = rr; }
    if (best == 0.0) return false;
    if (p != c) {
#pragma unroll
      for (int j = 0; j < N; ++j) {
        zd t = A[c * N + j]; A[c * N + j] = A[p * N + j]; A[p * N + j] = t;
        t = Inv[c * N + j]; Inv[c * N + j] = Inv[p * N + j]; Inv[p * N + j] = t;
      }
    }
    const zd pv = A[c * N + c];
    const zd ip = pv.conj() * (1.0 / pv.abs2());
#pragma unroll
    for (int j = 0; j < N; ++j) { A[c * N + j] = A[c * N + j] * ip; Inv[c * N + j] = Inv[c * N + j] * ip; }
#pragma unroll
    for (int rr = 0; rr < N; ++rr) {
      if (rr == c) continue;
      const zd f = A[rr * N + c];
#pragma unroll
      for (int j = 0; j < N; ++j) { A[rr * N + j] -= f * A[c * N + j]; Inv[rr * N + j] -= f * Inv[c * N + j]; }
    }
  }
  return true;
}

// ---- Dyson step, one CTA per instance ----------------------------------
// out = B [i nu - e_eff - F S]^{-1}; err[n] = max |out - G| (NaN for a
// singular Dyson matrix).  e_eff = eps(0_|) plus, for NAMBU, the Fock term
// -U rho_ij (i != j, rho = -G(beta^-) = -sum_c ebeta_c G(tau_c)) and the
// pairing field eta (while it <= n_eta).
template <int NO>
__global__ void __launch_bounds__(128) k_mats_dyson(MatsDev m, int it, double2* out) {
  constexpr int N2 = NO * NO;
  extern __shared__ zd sm[];
  zd* Sn = sm;                      // [r][N2]: Sigma(i nu_k), then G(i nu_k)
  __shared__ zd ee[N2];
  __shared__ double red[128];
  __shared__ int bad;
  const int n = blockIdx.x, r = m.r, tid = threadIdx.x;
  const double2* G = m.G + (size_t)n * r * N2;
  const double2* S = m.S + (size_t)n * r * N2;
  if (tid == 0) bad = 0;
  if (tid < N2) {
    zd e = ld(m.e0 + (size_t)n * m.e0_stride + tid);
    if (m.model == kMatsNambu && it > 0 && (tid == 1 || tid == 2)) {
      zd rho = zd();
      for (int c = 0; c < r; ++c) rho -= ld(G + (size_t)c * N2 + tid) * m.ebeta[c];
      e += rho * (-m.U) + zd(it <= m.n_eta ? m.eta : 0.0);
    }
    ee[tid] = e;
  }
  for (int e = tid; e < r * N2; e += blockDim.x) {
    const int k = e / N2, q = e % N2;
    zd s = zd();
    for (int l = 0; l < r; ++l) s += ld(m.F + (size_t)k * r + l) * ld(S + (size_t)l * N2 + q);
    Sn[e] = s;
  }
  __syncthreads();
  for (int k = tid; k < r; k += blockDim.x) {
    zd A[N2], Inv[N2];
#pragma unroll
    for (int q = 0; q < N2; ++q) A[q] = zd(q / NO == q % NO ? 1.0 : 0.0) * zd(0.0, m.nu[k]) - ee[q] - Sn[k * N2 + q];
    if (!small_inv<NO>(A, Inv)) bad = 1;
#pragma unroll
    for (int q = 0; q < N2; ++q) Sn[k * N2 + q] = Inv[q];
  }
  __syncthreads();
  double e_max = 0.0;
  bool nonfinite = bad != 0;
  for (int e = tid; e < r * N2; e += blockDim.x) {
    const int i = e / N2, q = e % N2;
    zd s = zd();
    for (int k = 0; k < r; ++k) s += ld(m.B + (size_t)i * r + k) * Sn[k * N2 + q];
    if (!isfinite(s.re) || !isfinite(s.im)) nonfinite = true;
    if (out != m.G) e_max = fmax(e_max, sqrt((s - ld(G + e)).abs2()));
    st(out + (size_t)n * r * N2 + e, s);
  }
  red[tid] = nonfinite ? NAN : e_max;
  __syncthreads();
  if (tid == 0) {
    double mx = 0.0;
    bool nan = false;
    for (int j = 0; j < blockDim.x; ++j) {
      if (red[j] != red[j]) nan = true;
      mx = fmax(mx, red[j]);
    }
    m.err[n] = (nan || bad) ? NAN : mx;
  }
}

// G = a Gn + (1 - a) G
__global__ void k_mats_mix(MatsDev m, double a) {
  const size_t cnt = (size_t)m.n_inst * m.r * m.no * m.no;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < cnt; e += (size_t)gridDim.x * blockDim.x)
    st(m.G + e, ld(m.Gn + e) * a + ld(m.G + e) * (1.0 - a));
}

// W[n][a][i] = sum_c phi[a][c][i] G(tau_c), the convolution tensor of the
// mixed component (Eq. KBET); one CTA per (instance, a)
__global__ void k_mats_wconv(MatsDev m, const double* phi, double2* W) {
  const int n = blockIdx.y, a = blockIdx.x, r = m.r, n2 = m.no * m.no;
  for (int e = threadIdx.x; e < r * n2; e += blockDim.x) {
    const int i = e / n2, q = e % n2;
    zd s = zd();
    for (int c = 0; c < r; ++c) s += ld(m.G + ((size_t)n * r + c) * n2 + q) * phi[((size_t)a * r + c) * r + i];
    st(W + (((size_t)n * r + a) * r + i) * n2 + q, s);
  }
}

#define MATS_DISPATCH(CALL)                                  \
  switch (m.no) {                                            \
    case 1: { constexpr int NO = 1; CALL; break; }           \
    case 2: { constexpr int NO = 2; CALL; break; }           \
    case 3: { constexpr int NO = 3; CALL; break; }           \
    case 4: { constexpr int NO = 4; CALL; break; }           \
    default: return cudaErrorInvalidValue;                   \
  }

cudaError_t launch_mats_sigma(const MatsDev& m, cudaStream_t s) {
  if (m.r > 128) return cudaErrorInvalidValue;
  if (m.model == kMatsLattice) {
    if (m.no != 1 || m.L * m.L > kLatMaxK) return cudaErrorInvalidValue;
    k_mats_sigma_lattice<<<m.r, kLatMaxK, 0, s>>>(m);
  } else {
    MATS_DISPATCH((k_mats_sigma<NO><<<m.n_inst, 128, 0, s>>>(m)));
  }
  return cudaGetLastError();
}
cudaError_t launch_mats_dyson(const MatsDev& m, int it, double2* out, cudaStream_t s) {
  const size_t smem = (size_t)m.r * m.no * m.no * sizeof(zd);
  MATS_DISPATCH((k_mats_dyson<NO><<<m.n_inst, 128, smem, s>>>(m, it, out)));
  return cudaGetLastError();
}
cudaError_t launch_mats_mix(const MatsDev& m, double a, cudaStream_t s) {
  k_mats_mix<<<152 * 4, 256, 0, s>>>(m, a);
  return cudaGetLastError();
}
cudaError_t launch_mats_wconv(const MatsDev& m, const double* phi, double2* W, cudaStream_t s) {
  k_mats_wconv<<<dim3(m.r, m.n_inst), 128, 0, s>>>(m, phi, W);
  return cudaGetLastError();
}

}  // namespace hk
