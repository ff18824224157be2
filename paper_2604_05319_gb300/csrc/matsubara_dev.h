// Device form of the equilibrium (Matsubara) Dyson iteration: the arguments
// of its kernels (matsubara_dev.cu) and their launchers.
#pragma once
#include <cuda_runtime.h>

#include "state.h"

namespace hk {

enum { kMatsNone = 0, kMatsBethe = 1, kMatsNambu = 2, kMatsLattice = 3 };

struct MatsDev {
  int r, no, n_inst, model, L, ys, xi, n_eta;
  double beta, U, eta;
  const double2 *F, *B;          // [r][r]: tau -> nu and nu -> tau maps of the DLR representation
  const double *nu, *rev, *ebeta, *tau;  // [r], [r][r], [r], [r]
  const double* mpar;            // [n][MP] model parameters (as set by hkbe_set_model)
  const double2* e0;             // eps(0_|) of instance n at e0 + n * e0_stride, [no][no]
  long long e0_stride;
  double2 *G, *Gn, *S;           // [n][r][no][no]: iterate, Dyson output, Sigma^M(tau)
  double* err;                   // [n] max |G_new - G| of the last Dyson step
};

cudaError_t launch_mats_sigma(const MatsDev& m, cudaStream_t s);
// out = Dyson(G, S); it = 0: the non-interacting start written into G (S = 0)
cudaError_t launch_mats_dyson(const MatsDev& m, int it, double2* out, cudaStream_t s);
cudaError_t launch_mats_mix(const MatsDev& m, double a, cudaStream_t s);
cudaError_t launch_mats_wconv(const MatsDev& m, const double* phi, double2* W, cudaStream_t s);

}  // namespace hk
