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
  float omegaf[6], I0f[6][6];   // float copies for the bulk sums of the complex64 form
  double ah[6];                  // a_j / h (the BDF coefficients of the time derivative)
};

constexpr int MP = 64;  // doubles of model parameters per instance

// Lower-triangular storage: element (T, t), t <= T, of instance n lives at
// ((n * ntri + T*(T+1)/2 + t) * no*no).  Mixed arrays are [n][T][i][no*no].
// Compressed (HODLR) storage of one two-time component (Sec. 2.2): dense
// leaf triangles plus U S V^dagger blocks, one scalar TSVD per orbital pair.
// Element type of the two-time storage (U, V, leaves, band, ring or triangle
// rows): double2 in the FP64 form, float2 in the mixed form.  Mixed
// components, chunk inverses, singular values and projections are FP64 in both.
struct Hod {
  void* U;       // [n][utot][rmax]   U of block b, pair p at (uoff[b] + p*rows_b) * rmax
  void* V;       // [n][vtot][rmax]   V of block b, pair p at (voff[b] + p*cols_b) * rmax
  double* S;     // [n][nblk][no2][rmax]
  int* rank;     // [n][nblk][no2]
  void* leaf;    // [n][leaftot][no2] lower triangles of the diagonal leaves
};

struct Dev {
  int nt, k, no, r, n_inst, xi, rho_mode, model;
  // ---- compressed storage (ring == 0: dense triangles, no compression) ----
  int ring;            // rows kept uncompressed in a ring of this many slots
  int cdir;            // first uncompressed row (multiple of the leaf size)
  int L, nleaf, nblk, rmax, maxl;
  double svd_tol;
  const int *b_r0, *b_r1, *b_c0, *b_c1, *b_lvl;   // block geometry
  const long long *b_uoff, *b_voff, *leafoff;     // factor / leaf offsets
  const int *rowblk, *colblk;                     // [nleaf][maxl] block ids or -1
  long long utot, vtot, leaftot;
  Hod hod[4];          // 0 G^R, 1 G^<, 2 Sigma^R, 3 Sigma^<
  void* band;          // [n][nt][k][no2] Sigma^R(t, t-d), d = 1..k
  double2* proj;       // sweep projections [n][no][maxl][no2][rmax] (+ source: see kernels)
  double2* tsvd_ws;    // TSVD workspace: [tsvd_group][4][no2] slots of tsvd_ws_per entries,
  long long tsvd_ws_per;  // level lv of a slot at offset ws_lvoff[lv]; the compression
  int tsvd_group;         // runs tsvd_group instances at a time on one shared workspace
  const long long* ws_lvoff;
  int* status;         // [0] rank overflow count, [1] Jacobi non-convergence count
  // frozen 32-point chunk inverses of the two sweeps (FP64): [n][nchunk][2][(32 no)^2]
  double2* cinv;
  double2* cinv_ws;    // [n][(32 no)^2] Gauss-Jordan workspace
  int nchunk;          // ceil(nt / 32)
  int nfrozR, nfrozL;  // chunks [0, nfroz) of each sweep have a valid inverse
  long long ntri;  // nt*(nt+1)/2
  double h, beta;
  DevW w;
  int prec;                    // 0: double2 storage, 1: float2 storage (mixed form)
  void *GR, *GL, *SR, *SL;     // lower-triangular (or ring), GL(T,t) = G^<(t,T)
  void *GTV, *STV;             // [n][nt][r][no2], complex128 in both forms
  double2 *eps;                // [n][nt+1][no2], index t+1 (external eps plus any Fock term)
  double2 *eps_ext;            // [n][nt+1][no2] external eps as set by the caller
  double *drA, *drU;           // [n][nt+1] drive: vector potential A(t), interaction U(t)
  double2 *gm;                 // [n][r][no2]
  double2 *wconv;              // [n][r(a)][r(i)][no2]
  double *tau, *e0, *ebeta, *rev, *q;  // [r], [r], [r], [r*r], [r*r]
  double *mpar;                // [n][MP]
  double2 *qsrc;               // [n][nt][no2]   lesser source q(t)
  double2 *vvec;               // [n][r][no2]    v_a = sum_b Q_ab G^vt(tau_b, T)
  double2 *x0;                 // [n][no2]       -[G^tv(T,0)]^dagger
  double2 *scratch;            // [n][scratch_per_inst]  start-block right-hand sides
  long long scratch_per_inst;
  // complex64 storage form only (null otherwise):
  double2 *row64;              // [n][2][nt][no2] FP64 row of G^R / column of G^< being solved
                               // (dense storage; the compressed form solves in ring64)
  // complex64 compressed form only: FP64 copies of the ring rows of G^R, G^<,
  // Sigma^R, Sigma^< ([n][ring][nt][no2], the storage ring's slots).  The
  // sweeps solve into them, the self-energy and the extrapolation read them,
  // and the TSVD compresses from them, so appended rows carry no complex64
  // rounding noise (null otherwise).
  double2 *ring64[4];
  int use64;                   // 1 once the start square's copies are seeded
  double2 *diag64;             // [n][nt][no2]    FP64 history of G^<(t, t) (diagonal scheme)
  double *err;                 // [n]
  int *active;                 // [n]
  const int *last;             // [n] last time step of each instance (N_t of the instance - 1)
};

// ---- launchers (all on `s`) ----
cudaError_t launch_extrapolate(const Dev& d, int T, cudaStream_t s);
cudaError_t launch_sigma(const Dev& d, int T, cudaStream_t s);
cudaError_t launch_mixed(const Dev& d, int T, cudaStream_t s);
cudaError_t launch_vt(const Dev& d, int T, cudaStream_t s);
cudaError_t launch_src(const Dev& d, int T, cudaStream_t s);
cudaError_t launch_les(const Dev& d, int T, cudaStream_t s);
cudaError_t launch_rho(const Dev& d, int T, cudaStream_t s);
cudaError_t launch_boot(const Dev& d, cudaStream_t s);   // one bootstrap pass (Sigma + R/mixed/lesser)
cudaError_t launch_diag_seed(const Dev& d, cudaStream_t s);  // diag64[t] = G^<(t,t), t <= k
cudaError_t launch_set_active(const Dev& d, double tol, int iter, int min_iter, int* any_active_dev, cudaStream_t s);
// compressed (HODLR) form
cudaError_t launch_ret_h(const Dev& d, int T, cudaStream_t s);
cudaError_t launch_les_h(const Dev& d, int T, cudaStream_t s);
cudaError_t launch_src_h(const Dev& d, int T, cudaStream_t s);
cudaError_t launch_compress(const Dev& d, int A, int nb, cudaStream_t s);
cudaError_t launch_density_at(const Dev& d, int t, double2* out, cudaStream_t s);  // rho(t), every instance
cudaError_t launch_sigma_lattice(const Dev& d, int T, cudaStream_t s);   // model 4, all k at once
cudaError_t launch_lattice_obs(const Dev& d, int t, double* out, cudaStream_t s);
cudaError_t launch_row_out(const Dev& d, int n, int T, double2* out_r, double2* out_l, cudaStream_t s);
// inverses of the frozen chunks [c0, c1) of sweep `which` (0 retarded, 1 lesser)
cudaError_t launch_chunk_inv(const Dev& d, int which, int c0, int c1, cudaStream_t s);

}  // namespace hk
