// Device-resident state of one stepper handle and the launch entry points of
// the kernels (defined in kernels_dense.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hk {

// Appendix A weights passed to kernels by value.
struct DevW {
  int k;
  double a[6], omega[6], D[6][6], I0[6][6];
};

constexpr int MP = 64;  // doubles of model parameters per instance

// Lower-triangular storage: element (T, t), t <= T, of instance n lives at
// ((n * ntri + T*(T+1)/2 + t) * no*no).  Mixed arrays are [n][T][i][no*no].
struct Dev {
  int nt, k, no, r, n_inst, xi, rho_mode, model;
  long long ntri;  // nt*(nt+1)/2
  double h, beta;
  DevW w;
  double2 *GR, *GL, *SR, *SL;  // lower-triangular, GL(T,t) = G^<(t,T)
  double2 *GTV, *STV;          // [n][nt][r][no2]
  double2 *eps;                // [n][nt+1][no2], index t+1
  double2 *gm;                 // [n][r][no2]
  double2 *wconv;              // [n][r(a)][r(i)][no2]
  double *tau, *e0, *ebeta, *rev, *q;  // [r], [r], [r], [r*r], [r*r]
  double *mpar;                // [n][MP]
  double2 *qsrc;               // [n][nt][no2]   lesser source q(t)
  double2 *vvec;               // [n][r][no2]    v_a = sum_b Q_ab G^vt(tau_b, T)
  double2 *x0;                 // [n][no2]       -[G^tv(T,0)]^dagger
  double2 *scratch;            // [n][scratch_per_inst]  start-block right-hand sides
  long long scratch_per_inst;
  double *err;                 // [n]
  int *active;                 // [n]
};

// ---- launchers (all on `s`) ----
cudaError_t launch_extrapolate(const Dev& d, int T, cudaStream_t s);
cudaError_t launch_sigma(const Dev& d, int T, cudaStream_t s);
cudaError_t launch_ret(const Dev& d, int T, cudaStream_t s);
cudaError_t launch_mixed(const Dev& d, int T, cudaStream_t s);
cudaError_t launch_vt(const Dev& d, int T, cudaStream_t s);
cudaError_t launch_src(const Dev& d, int T, cudaStream_t s);
cudaError_t launch_les(const Dev& d, int T, cudaStream_t s);
cudaError_t launch_rho(const Dev& d, int T, cudaStream_t s);
cudaError_t launch_boot(const Dev& d, cudaStream_t s);   // one bootstrap pass (Sigma + R/mixed/lesser)
cudaError_t launch_set_active(const Dev& d, double tol, int iter, int min_iter, int* any_active_dev, cudaStream_t s);

}  // namespace hk
