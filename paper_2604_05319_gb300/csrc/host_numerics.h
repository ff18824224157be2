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

}  // namespace hk
