// Host-side set-up numerics of the library (weights, DLR matrices, small
// Hermitian eigen-decomposition).  None of it runs per time step.
#pragma once
#include <complex>
#include <vector>

namespace hk {

struct Weights {
  int k;
  double a[6];        // BDF a_j = -D_0j
  double omega[6];    // Gregory end weights
  double D[6][6];     // D_ml
  double I0[6][6];    // I_{0,n,l}
};

void weights_build(int k, Weights* w);
double rule_weight(const Weights& w, int n, int l);     // w^(n)_l
double integ_weight(const Weights& w, int m, int n, int l);  // I_{m,n,l}

struct DLRMats {
  int r;
  std::vector<double> e0, ebeta, rev, q, phi;
};
double dlr_kernel(double x, double w, double beta);
bool dlr_build(int r, const double* tau, const double* om, double beta, int xi, DLRMats* out);

void herm_eig(int n, const std::complex<double>* A, double* E, std::complex<double>* U);

// Linear maps of the Matsubara solve as r x r row-major matrices: values on
// the DLR nodes tau_i -> values at the r chosen fermionic frequencies nu_k
// (F), and back (B), with the frequencies nu[r] (the same nodes and maps as
// hkbe_matsubara_solve).  False if a DLR kernel matrix is singular.
bool mats_maps(int r, const double* tau, const double* om, double beta, std::vector<std::complex<double>>* F,
               std::vector<std::complex<double>>* B, std::vector<double>* nu);

}  // namespace hk
