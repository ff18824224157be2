/*
 * hkbe.h -- C ABI of the GB300 Kadanoff-Baym time stepper (HODLR history
 * integrals, high-order Gregory/BDF weights, DLR thermal leg).
 *
 * The calls follow the user workflow of the paper: construct the objects
 * (Sec. 3.1), set the initial thermal state on the DLR grid (Sec. 2.5, 3.2),
 * bootstrap the first k steps (Sec. 2.6 / 3.3), time-step with a
 * self-consistency loop per step (Sec. 3.4), and read G^R, G^<, G^tv and
 * observables (Tables 2-5, Sec. 4.2 observables).
 *
 * Conventions for every call
 *   - Return value: HKBE_OK (0) or a negative HKBE_ERR_* code; the message of
 *     the last failure is returned by hkbe_last_error().
 *   - Complex numbers are interleaved (re, im) pairs of double.  An N_o x N_o
 *     matrix is stored row-major, so one matrix is 2*N_o*N_o doubles.
 *   - Every pointer argument is a HOST pointer owned by the caller; the
 *     library copies in or out before returning (inputs) or after the device
 *     work of the call completed (outputs).  The library owns all device
 *     memory it allocates and frees it in hkbe_destroy().
 *   - Device work is issued on the CUDA stream given to hkbe_create() (NULL
 *     means the legacy default stream).
 *   - A handle is not thread-safe (the paper's dyson/dlr_info objects are not
 *     either, Sec. 4.3); use one handle per host thread.
 *   - Time arguments are step indices t = 0..nt-1; the equilibrium branch
 *     value of one-time functions (eps, drive) is index -1 (Sec. 3.2).
 *   - Fermions only (xi = -1) in this version; HKBE_ERR_ARG otherwise.
 */
#ifndef HKBE_H
#define HKBE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  HKBE_OK = 0,
  HKBE_ERR_ARG = -1,      /* invalid argument, size or call order          */
  HKBE_ERR_CUDA = -2,     /* CUDA runtime failure (message has the detail) */
  HKBE_ERR_NOCONV = -3,   /* self-consistency did not reach tol in max_iter */
  HKBE_ERR_RANGE = -4,    /* time index outside the stored/allowed region   */
  HKBE_ERR_RANK = -5,     /* HODLR block rank exceeded its capacity r_max   */
  HKBE_ERR_NAN = -6,      /* non-finite value met during a step             */
  HKBE_ERR_NOMEM = -7,    /* device or host allocation failed               */
  HKBE_ERR_IO = -8        /* checkpoint file cannot be written, read, or does
                             not match the handle it is loaded into          */
};

/* Self-energy functionals (evaluated on the device at every step). */
enum {
  HKBE_MODEL_NONE = 0,   /* Sigma = 0                                              */
  HKBE_MODEL_BETHE = 1,  /* Bethe-lattice DMFT: Sigma = v^2 G (Eq. Hybrid, N_o=1)  */
  HKBE_MODEL_BATH = 2,   /* fixed bath: Sigma = V g_b V^dagger, bath levels eps_b   */
  HKBE_MODEL_NAMBU = 3,  /* Nambu DMFT (N_o = 2): Eq. Hybrid + Eq. Sigma2B + Eq. SigmaF */
  HKBE_MODEL_LATTICE2B = 4  /* 2D Hubbard, second Born through real space (Sec. 4.2)   */
};

/* Storage / arithmetic of the history integrals. */
enum {
  HKBE_PREC_FP64 = 0,     /* complex128 storage of every two-time and mixed
                             component (dense triangles or HODLR factors); FP64
                             arithmetic throughout                               */
  HKBE_PREC_MIXED = 1,    /* complex64 storage of the two-time components
                             (rows, HODLR factors, leaves, band); FP32 bulk
                             history sums and FP32 TSVD; the row being solved,
                             every point solve, the mixed components, weights
                             and DLR matrices stay FP64.  Expected deviation
                             from the FP64 form: about 1e-6 relative (single-
                             precision rounding of the stored history; a GPU
                             design choice, the paper computes in FP64)          */
  HKBE_PREC_TF32X3 = 2,   /* not provided: rejected by hkbe_create (see there) */
  HKBE_PREC_BF16X3 = 3    /* not provided: rejected by hkbe_create (see there) */
};

typedef struct {
  int32_t nt;         /* number of time steps N_t (>= k + 2)                    */
  int32_t k;          /* integration order, 1..5 (Appendix A)                   */
  int32_t nao;        /* orbitals N_o, 1..4                                     */
  int32_t xi;         /* statistics: -1 fermions                                */
  int32_t n_inst;     /* independent instances stepped together (>= 1)          */
  int32_t rho_mode;   /* 0 horizontal, 1 diagonal density-matrix scheme (Sec. 3.3) */
  int32_t precision;  /* HKBE_PREC_*                                             */
  int32_t max_iter;   /* self-consistency iterations per step (Sec. 3.4)        */
  double h;           /* time step                                              */
  double beta;        /* inverse temperature of the thermal initial state       */
  double tol;         /* self-consistency tolerance on max |G^(i) - G^(i-1)|     */
  double svd_tol;     /* > 0: HODLR storage with TSVD truncation at this absolute
                         singular value (Sec. 2.2); 0: dense triangles          */
  int32_t leaf;       /* HODLR leaf size, 32 or 64 (> 2k); blocks are leaf-aligned */
  int32_t r_max;      /* rank capacity per block and orbital pair, 1..128       */
} hkbe_params;

typedef struct hkbe_s hkbe_t;

/* Create a stepper for p->n_inst instances sharing k, nao, h, beta and the
 * storage form (Sec. 3.1 objects; the Sec. 4 examples construct one per
 * system).  nt_per_inst[n_inst] (or NULL: every instance runs p->nt steps)
 * gives each instance its own number of time steps N_t,n in k+2..p->nt: an
 * instance takes part in the steps T <= N_t,n - 1 and is left untouched after
 * them (its iteration count and error are 0 there), its HODLR compression
 * front freezes at its last whole leaf of rows older than k + 1 steps, and
 * its rows stay readable up to N_t,n - 1.  The lattice model needs one N_t
 * for every k-point (hkbe_set_model refuses otherwise).  `stream` is a
 * cudaStream_t (or NULL).  On success *out receives the handle.  Errors:
 * HKBE_ERR_ARG (bad sizes; precision HKBE_PREC_TF32X3 or HKBE_PREC_BF16X3,
 * whose operand splitting serves dense tensor-core contractions, of which
 * this path has none: every history sum is a per-instance matrix-vector
 * product), HKBE_ERR_NOMEM, HKBE_ERR_CUDA. */
int hkbe_create(const hkbe_params* p, const int32_t* nt_per_inst, void* stream, hkbe_t** out);

/* Equilibrium Dyson equation on the DLR grid (Eq. KBEM, Sec. 2.5, 3.2),
 * solved self-consistently on the host: prepares G^M of an interacting
 * initial state for hkbe_set_matsubara.  No handle and no GPU needed.
 *   r, tau[r], omega[r], beta: the DLR grid (as for hkbe_set_dlr);
 *   model, params[n_inst][nparams]: as for hkbe_set_model (HKBE_MODEL_NONE,
 *     BETHE, NAMBU with optional [v, g, w0], LATTICE2B with [L] or
 *     [L, ysymm], the reduced k-set of hkbe_set_model);
 *   eps[n_inst][nao][nao] complex: the equilibrium-branch level eps(0_|);
 *   U_eq: interaction on the equilibrium branch (second Born and Fock);
 *   eta, n_eta: pairing field eta added to eps_01 and eps_10 for the first
 *     n_eta iterations (symmetry breaking, Sec. 4.1); mix in (0, 1]: linear
 *     mixing of successive iterates; tol, max_iter: stop when
 *     max |G_new - G_old| < tol.
 * Sigma^M follows from the real-time functionals restricted to the imaginary
 * branch (G^M = -i G(-i tau, 0), Table 1): v^2 G (Bethe), v^2 s_z G s_z
 * - U^2 [G G - G G](tau) G(-tau) + Holstein (Nambu), -U^2 G_r^2 G_{-r}(-tau)
 * (lattice).  Dyson is imposed at r fermionic Matsubara frequencies chosen
 * by pivoted Gram-Schmidt on the DLR Fourier rows 1/(i nu - omega_l).
 * Outputs: gm_out[n_inst][r][nao][nao] complex, eps_out[n_inst][nao][nao]
 * complex (eps with the converged Fock shift; may be NULL), iters, err (may
 * be NULL).  Errors: HKBE_ERR_ARG, HKBE_ERR_NAN (singular or non-finite),
 * HKBE_ERR_NOCONV (max_iter reached; outputs hold the last iterate). */
int hkbe_matsubara_solve(int r, const double* tau, const double* omega, double beta, int model, int n_inst,
                         int nao, const double* eps, const double* params, int nparams, double U_eq, double eta,
                         int n_eta, double mix, double tol, int max_iter, double* gm_out, double* eps_out,
                         int32_t* iters, double* err);

/* Equilibrium Dyson equation solved on the device (Eq. KBEM, Sec. 2.5, 3.2):
 * the iteration of hkbe_matsubara_solve (the same Sigma^M functionals, Dyson
 * at the same r Matsubara frequencies, the same mixing and stopping rule) run
 * by kernels on h's stream, for h's model (hkbe_set_model: NONE, BETHE, NAMBU
 * or LATTICE2B, the reduced k-set included), DLR grid (hkbe_set_dlr) and
 * equilibrium-branch level eps(0_|) (index 0 of hkbe_set_hamiltonian; NAMBU
 * adds the Fock term itself).  The converged G^M is installed as by
 * hkbe_set_matsubara, so it replaces that call.  Must precede hkbe_bootstrap.
 *   U_eq, eta, n_eta, mix, tol, max_iter: as for hkbe_matsubara_solve;
 *   gm_out (may be NULL): [n_inst][r][nao][nao] complex, the installed G^M;
 *   iters, err (may be NULL): iterations taken, last max |G_new - G|.
 * Allocates and frees its own device buffers (about 3 n_inst r nao^2 complex
 * values and r^3 doubles).  Errors: HKBE_ERR_ARG (order of calls, argument
 * ranges, BATH model), HKBE_ERR_NAN (singular Dyson matrix or non-finite
 * iterate; nothing installed), HKBE_ERR_NOCONV (max_iter reached: the last
 * iterate is installed), HKBE_ERR_CUDA. */
int hkbe_solve_matsubara(hkbe_t* h, double U_eq, double eta, int n_eta, double mix, double tol, int max_iter,
                         double* gm_out, int32_t* iters, double* err);

/* Time-step scheme of the retarded row and the lesser column (default:
 * HKBE_SCHEME_PAPER, the sweeps of Eqs. KBER and KBEL).
 * HKBE_SCHEME_SWEEP_FREE is a variant that is not in the paper (it differs
 * from the paper's discretisation at O(h^k)):
 *   - retarded row: the k points next to the diagonal are the start block of
 *     Eq. KBER; every t' further away comes from the retarded Dyson equation
 *     in its first time argument (BDF over the rows T - j, the Gregory rule
 *     of Appendix A over [t', T]), one N_o x N_o solve per t';
 *   - lesser column: the resolvent form of Eq. KBEL's equation in its first
 *     argument, G^<(t,T) = i G^R(t,0) G^<(0,T) + h sum_l w^(t)_l G^R(t,l) q_l;
 *   - so no point of either waits for its neighbour.
 * Dense FP64 storage only (compressed or complex64 handles: HKBE_ERR_ARG).
 * Must precede hkbe_bootstrap; hkbe_save refuses a handle of this scheme. */
enum { HKBE_SCHEME_PAPER = 0, HKBE_SCHEME_SWEEP_FREE = 1 };
int hkbe_set_scheme(hkbe_t* h, int scheme);

/* Release every device and host resource of h (NULL is accepted). */
int hkbe_destroy(hkbe_t* h);

/* Message of the last failure on h (or of the last failed hkbe_create when h
 * is NULL).  The pointer stays valid until the next call on h. */
const char* hkbe_last_error(const hkbe_t* h);

/* DLR imaginary-time grid (Sec. 2.5): r nodes tau[r] in (0, beta) and the r
 * DLR real frequencies omega[r] (both produced by the caller's DLR
 * construction for cutoff Lambda and accuracy eps).  The library builds its
 * own evaluation, reversal, product and convolution matrices from them.
 * Must precede hkbe_set_matsubara.  Errors: HKBE_ERR_ARG (r < 1, r > 128,
 * nodes outside (0, beta)). */
int hkbe_set_dlr(hkbe_t* h, int r, const double* tau, const double* omega);

/* Equilibrium Matsubara Green's function on the DLR nodes, G^M(tau_i), for
 * every instance: gm[n_inst][r][N_o][N_o] complex (Table 4, get_mat/set_mat).
 * Also precomputes the convolution tensor of Eq. KBET (initGMConvTensor).
 * Errors: HKBE_ERR_ARG (null, or before hkbe_set_dlr). */
int hkbe_set_matsubara(hkbe_t* h, const double* gm);

/* Mean-field Hamiltonian eps(t) = h0(t) + Sigma^MF(t) - mu (Eq. KBEM-KBEL) for
 * t = -1..nt-1 and every instance: eps[n_inst][nt+1][N_o][N_o] complex, index
 * 0 holding the equilibrium branch eps(0_|).  Errors: HKBE_ERR_ARG (null),
 * HKBE_ERR_NAN (non-finite value). */
int hkbe_set_hamiltonian(hkbe_t* h, const double* eps);

/* The same for one time t only: eps_t[n_inst][N_o][N_o] complex replaces
 * eps(t) of every instance (the per-step update of a time-dependent mean
 * field or drive, Sec. 3.4).  Only times not yet computed may change:
 * HKBE_ERR_RANGE unless current step < t <= nt-1; HKBE_ERR_ARG before
 * hkbe_set_hamiltonian; HKBE_ERR_NAN for non-finite input.  Synchronous. */
int hkbe_set_hamiltonian_at(hkbe_t* h, int t, const double* eps_t);

/* Self-energy functional and its parameters, params[n_inst][nparams]:
 *   HKBE_MODEL_NONE : nparams 0.
 *   HKBE_MODEL_BETHE: nparams >= 1, params[0] = v (Sigma = v^2 G).
 *   HKBE_MODEL_BATH : nparams = 1 + nb + 2*N_o*nb with
 *       params[0] = nb (1..4 bath levels), params[1..nb] = eps_b,
 *       then V[N_o][nb] complex interleaved (Sigma = V g_b V^dagger).
 *   HKBE_MODEL_NAMBU: N_o = 2 (Nambu spinor (d_up, d_dn^dagger), Sec. 4.1),
 *       nparams 1 or 3: params[0] = v (hopping scale, Delta carries v^2),
 *       params[1] = g, params[2] = w0 (optional Holstein coupling: the
 *       unrenormalised Migdal Sigma^≷ += i g^2 D0^≷ sigma_z G^≷ sigma_z with
 *       the free phonon propagator of frequency w0 at beta; the paper names
 *       this approximation without printing it).
 *       Sigma = Delta + Sigma^2B with, element by element and s = (1, -1),
 *       Delta_ij(t,t') = v^2 s_i s_j G_ij(t,t') cos(s_i A(t) - s_j A(t'))
 *       (Eq. Hybrid, Peierls phases diag(e^{iA}, e^{-iA})), the bubble and
 *       exchange diagrams of Eq. Sigma2B with U(t)U(t'), and the Fock term
 *       of Eq. SigmaF added to eps(t) at every evaluation (eps as set by the
 *       caller is kept apart).  A(t), U(t) come from hkbe_set_drive.  With the
       Fock term -U rho_12 and the -U/2 shift of Eq. Model absorbed in eps,
       this is the attractive Hubbard term -U (n_up - 1/2)(n_dn - 1/2) of
       Eq. Model through order U^2.
 *   HKBE_MODEL_LATTICE2B: N_o = 1, one instance per k-point of an L x L grid,
 *       k = 2 pi (m_x, m_y)/L at instance m_x L + m_y, n_inst = L^2, L <= 16;
 *       params[n] = [L] or [L, ysymm].  ysymm = 1 (L even) keeps only the
 *       k-points with m_y <= L/2, instance m_x (L/2+1) + m_y, n_inst =
 *       L(L/2+1) (Sec. 4.2: the reflection k_y -> -k_y of a drive along x);
 *       the grid point (m_x, L - m_y) is taken equal to (m_x, m_y) in every
 *       lattice sum, which is exact when eps_k(t) and the initial state have
 *       that symmetry (the caller's responsibility).  Sigma^≷_k from Sigma^≷_r(T,t) =
 *       U(T)U(t) G^≷_r(T,t)^2 G^≶_{-r}(t,T) (G_r the lattice Fourier
 *       transform over k; the mixed part with the imaginary branch latest),
 *       U(t) from hkbe_set_drive (instance 0; the same for every k).  The
 *       dispersion with its Peierls shift eps_{k-A(t)} is the caller's eps.
 *       The k-points iterate together (all or none).
 * Errors: HKBE_ERR_ARG (unknown model, wrong N_o or parameter count, n_inst
 * not L^2 (L(L/2+1) with ysymm), odd L with ysymm, w0 <= 0 with g != 0). */
int hkbe_set_model(hkbe_t* h, int model, const double* params, int nparams);

/* Drive of the Nambu model: A[n_inst][nt+1] (vector potential) and
 * U[n_inst][nt+1] (interaction), index 0 the equilibrium branch, index t+1
 * time t (Sec. 4.1: A(t) = -int_0^t E, U(t) of the Hamiltonian).  Either may
 * be NULL (zero).  Must precede hkbe_bootstrap.  HKBE_ERR_NAN for non-finite
 * values. */
int hkbe_set_drive(hkbe_t* h, const double* A, const double* U);

/* Bootstrap the first k+1 time steps (Sec. 3.3, dyson_start_ntti): mean-field
 * guess (green_from_H) followed by global iterations of Sigma and the start
 * square with the polynomial weights of Appendix A.  Outputs (may be NULL):
 * iters[n_inst], err[n_inst].  Errors: HKBE_ERR_NOCONV if max_iter is
 * reached without err < tol (state is kept), HKBE_ERR_ARG (call order). */
int hkbe_bootstrap(hkbe_t* h, int max_iter, double tol, int32_t* iters, double* err);

/* Start from given rows 0..k instead of hkbe_bootstrap (the start square of
 * Sec. 3.3 supplied by the caller, e.g. from another solver or a previous
 * run).  Per instance n, packed row by row for t = 0..k, s = 0..t:
 *   gr [n_inst][(k+1)(k+2)/2][N_o][N_o]  G^R(t, s)
 *   gl [n_inst][(k+1)(k+2)/2][N_o][N_o]  G^<(s, t)   (column t, the layout
 *                                                     hkbe_get_row returns)
 *   gtv[n_inst][k+1][r][N_o][N_o]        G^tv(t, tau_i)
 * The library then evaluates Sigma on the square and leaves the handle
 * exactly where hkbe_bootstrap would (current step k, hkbe_rewind returns
 * here).  The mixed form rounds the rows to complex64 storage.  Errors:
 * HKBE_ERR_ARG (null, call order: set_dlr, set_matsubara, set_hamiltonian,
 * set_model first, and no bootstrap yet), HKBE_ERR_NAN (non-finite input). */
int hkbe_set_initial_slices(hkbe_t* h, const double* gr, const double* gl, const double* gtv);

/* Advance every instance by n_steps time steps (Sec. 3.4: extrapolate, then
 * per iteration Sigma, retarded row, mixed, lesser column, density matrix,
 * until max |G^(i) - G^(i-1)| < tol or max_iter).  Outputs (may be NULL):
 * iters[n_inst*n_steps], err[n_inst*n_steps].  Errors: HKBE_ERR_RANGE (past
 * nt-1), HKBE_ERR_NOCONV (state kept; the step counter still advances: the
 * self-consistency loop reached max_iter, or, HODLR form, the Jacobi SVD of a
 * TSVD block core did not converge in 40 sweeps), HKBE_ERR_RANK (a block's
 * epsilon-rank was capped at r_max), HKBE_ERR_CUDA (a CUDA error, or a
 * sweep's bounded wait for the shared-memory copy of a frozen chunk inverse
 * timed out; that chunk was then read from global memory).  The TSVD and
 * copy conditions are counted over the n_steps of this call and reset
 * afterwards. */
int hkbe_step(hkbe_t* h, int n_steps, int32_t* iters, double* err);

/* Current time step T (the last completed step), -1 before the bootstrap. */
int hkbe_current_step(const hkbe_t* h, int32_t* T);

/* G^R(t, t') for 0 <= t' <= t <= T into out[N_o][N_o] (Table 3 get_ret).
 * Errors: HKBE_ERR_RANGE outside the computed triangle. */
int hkbe_get_ret(hkbe_t* h, int inst, int t, int tp, double* out);

/* G^<(t, t') for any 0 <= t, t' <= T (Table 3 get_les; the upper triangle
 * uses G^<(t,t') = -[G^<(t',t)]^dagger, Eq. GLantiHerm).  Errors: HKBE_ERR_ARG
 * (null, bad instance), HKBE_ERR_RANGE (a time outside 0..current step). */
int hkbe_get_les(hkbe_t* h, int inst, int t, int tp, double* out);

/* Mixed row G^tv(t, tau_i), i = 0..r-1, into out[r][N_o][N_o] (Table 4 get_tv).
 * Errors: HKBE_ERR_ARG (null, bad instance, no DLR grid), HKBE_ERR_RANGE
 * (t outside 0..current step). */
int hkbe_get_tv(hkbe_t* h, int inst, int t, double* out);

/* Whole retarded row G^R(T, 0..T) and lesser column G^<(0..T, T) of step T:
 * gr[T+1][N_o][N_o], gl[T+1][N_o][N_o] (either may be NULL).  Errors:
 * HKBE_ERR_ARG (bad instance), HKBE_ERR_RANGE (T outside 0..current step). */
int hkbe_get_row(hkbe_t* h, int inst, int T, double* gr, double* gl);

/* Density matrix rho(t) = xi i G^<(t,t) (Sec. 3.3) for t = 0..T of every
 * instance: rho[n_inst][T+1][N_o][N_o] complex.  Errors: HKBE_ERR_ARG (null),
 * HKBE_ERR_RANGE (before the bootstrap). */
int hkbe_get_density(hkbe_t* h, double* rho);

/* rho(t) of every instance at one time t <= current step:
 * rho_t[n_inst][N_o][N_o] complex, gathered on the device and copied once.
 * HKBE_ERR_RANGE outside 0..current step.  Synchronous. */
int hkbe_get_density_at(hkbe_t* h, int t, double* rho_t);

/* Observables of the LATTICE2B model at time t <= current step (Sec. 4.2,
 * spin summed where the paper does): out[0] = n = -(i/N_k) sum_k G^<_k(t,t)
 * (per spin), out[1] = E_kin = -(2i/N_k) sum_k eps_k G^<_k(t,t) with
 * eps_k = -2(cos k_x + cos k_y), out[2] = j = -(2i/N_k) sum_k
 * 2 sin(k_x - A(t)) G^<_k(t,t), the sums over the whole L x L grid (with
 * ysymm a mirror point counts its instance).  Reduced on the device.  HKBE_ERR_ARG for
 * another model, HKBE_ERR_RANGE for t outside 0..current step. */
int hkbe_get_lattice_observables(hkbe_t* h, int t, double* out);

/* Observables at time t <= current step in one call (Sec. 4.2):
 * rho[n_inst][N_o][N_o] complex as hkbe_get_density_at; ekin[1] and
 * current[1] as out[1] and out[2] of hkbe_get_lattice_observables.  Any
 * output may be NULL.  ekin and current exist for LATTICE2B only: asking for
 * them on another model is HKBE_ERR_ARG.  HKBE_ERR_RANGE for t outside
 * 0..current step.  Synchronous. */
int hkbe_get_observables(hkbe_t* h, int t, double* rho, double* ekin, double* current);

/* Device bytes held by the handle (snapshot copies not included) and, HODLR
 * form, the epsilon-ranks of instance `inst`: ranks[4][nblk][nao*nao] for the
 * components G^R, G^<, Sigma^R, Sigma^< (block order of hkbe_get_blocks; 0 for
 * a block with no row built yet).  Either output may be NULL (ranks must be
 * NULL for a dense handle).  Errors: HKBE_ERR_ARG (null handle, bad instance,
 * ranks on a dense handle), HKBE_ERR_CUDA. */
int hkbe_get_stats(hkbe_t* h, int inst, int32_t* ranks, size_t* device_bytes);

/* HODLR geometry (Sec. 2.2, Fig. 2): *nblk blocks; each of the arrays (may be
 * NULL, length >= *nblk when given) receives rows [r0, r1), columns [c0, c1)
 * and level of every block.  Leaves are [j*leaf, (j+1)*leaf); the recursion
 * splits ranges of leaves in halves.  HKBE_ERR_ARG for a dense handle. */
int hkbe_get_blocks(const hkbe_t* h, int32_t* nblk, int32_t* r0, int32_t* r1, int32_t* c0,
                    int32_t* c1, int32_t* level);

/* Current epsilon-rank of every block and orbital pair of component `comp`
 * (0 G^R, 1 G^<, 2 Sigma^R, 3 Sigma^<) of instance `inst`:
 * ranks[nblk][N_o*N_o].  Also returns in *first_direct the first row not yet
 * compressed (rows below it live in leaves and blocks). */
int hkbe_get_ranks(hkbe_t* h, int inst, int comp, int32_t* ranks, int32_t* first_direct);

/* Return to the state right after hkbe_bootstrap (current step = k), so the
 * time stepping can be run again from the same start (e.g. to time it, or
 * to propagate again after changing eps(t) for t > k with hkbe_set_hamiltonian).
 * Errors: HKBE_ERR_ARG before the bootstrap. */
int hkbe_rewind(hkbe_t* h);

/* In-memory checkpoint of the whole propagation state (Sec. 3.6 keeps the
 * full state in checkpoint files for a restart; this keeps one copy in device
 * memory instead).  hkbe_snapshot_save copies every device buffer of the
 * handle that holds state (all but its scratch workspaces) into a second
 * device allocation made on the first call and reused afterwards, together
 * with the step counter and the compression front.  hkbe_snapshot_restore copies it back: stepping the
 * restored handle repeats the run from the saved step bit for bit.
 * hkbe_snapshot_free releases the copy (hkbe_destroy does too).  Both run on
 * the handle's stream and return after it has finished.  Errors:
 * HKBE_ERR_ARG (null, before the bootstrap, restore without a saved copy),
 * HKBE_ERR_NOMEM (the copy does not fit), HKBE_ERR_CUDA. */
int hkbe_snapshot_save(hkbe_t* h);
int hkbe_snapshot_restore(hkbe_t* h);
int hkbe_snapshot_free(hkbe_t* h);

/* Measured FP64 and FP32 fused multiply-add throughput of the current CUDA
 * device in TFLOP/s (2 flop per FMA; many independent FMA chains, CUDA-event
 * timed, about 50 ms in all): the ALU peaks the FP64 history sums and the
 * FP32 bulk sums are compared with.  No handle; the paper has no
 * counterpart.  Errors: HKBE_ERR_ARG (null), HKBE_ERR_NOMEM, HKBE_ERR_CUDA. */
int hkbe_fma_peaks(double* fp64_tflops, double* fp32_tflops);

/* The device's FP64 -> FP32 conversion of the complex64 form's mixed-component
 * history sums (integer-pipe rounding from the IEEE 754 fields, to nearest
 * with ties away from zero; magnitudes below the normal FP32 range become
 * zero), applied to x[n] (host) into y[n] (host), for checking it against a
 * reference rounding.  No handle.  Errors: HKBE_ERR_ARG, HKBE_ERR_NOMEM,
 * HKBE_ERR_CUDA. */
int hkbe_f32_of(int n, const double* x, float* y);

/* Checkpoint (Sec. 3.6, checkpoint files: the full simulation state, restart
 * through a constructor).  hkbe_save writes to `path` the parameters, the
 * host-side set-up (DLR grid, G^M, eps, model, step counter, compression
 * front, bootstrap snapshot) and every device buffer of the handle byte for
 * byte (about hkbe_get_stats bytes), after finishing the work queued on the
 * handle's stream.  hkbe_load creates a new handle on `stream` from such a
 * file: propagating it continues the saved run bit for bit on the same
 * build and GPU type.  The format is this library's own binary layout
 * (magic "HKBECKP1", version 2: with the checksum trailer and the per-instance N_t), not HDF5, and is read on a machine of the
 * same byte order.  Its last 8 bytes are a checksum of everything before
 * them: FNV-1a 64 over the bytes taken as little-endian 64-bit words, the
 * last word zero-padded (offset basis 14695981039346656037, prime
 * 1099511628211).  hkbe_load verifies it before any device work.  Errors:
 * HKBE_ERR_ARG (null), HKBE_ERR_IO (cannot open, short read or write, bad
 * magic or version, checksum mismatch, or the file's buffers do not match
 * the sizes the parameters give), HKBE_ERR_NOMEM, HKBE_ERR_CUDA.  After
 * a failed hkbe_load, *out is NULL and hkbe_last_error(NULL) holds the
 * message. */
int hkbe_save(hkbe_t* h, const char* path);
int hkbe_load(const char* path, void* stream, hkbe_t** out);

/* ---- instrumentation (Sec. 3.5 write_timing / profiling) ---- */
enum {
  HKBE_PHASE_EXTRAP = 0,  /* initial guess of a step                           */
  HKBE_PHASE_SIGMA = 1,   /* self-energy evaluation                            */
  HKBE_PHASE_RET = 2,     /* retarded row (history integral + VIDE)            */
  HKBE_PHASE_MIXED = 3,   /* mixed component                                   */
  HKBE_PHASE_VT = 4,      /* mixed-product vector and lesser boundary value    */
  HKBE_PHASE_SRC = 5,     /* lesser source (Sigma^< and Sigma^tv histories)     */
  HKBE_PHASE_LES = 6,     /* lesser column (history integral + VIDE)           */
  HKBE_PHASE_RHO = 7,     /* diagonal density matrix                           */
  HKBE_PHASE_BOOT = 8,    /* bootstrap square                                  */
  HKBE_PHASE_CTRL = 9,    /* convergence bookkeeping                           */
  HKBE_PHASE_COMPRESS = 10, /* HODLR leaf copy + TSVD block updates (update_blocks) */
  HKBE_PHASE_CHUNKINV = 11, /* inverses of frozen 32-point sweep chunks           */
  HKBE_NPHASE = 12
};

/* When on (nonzero), every kernel launch is bracketed by CUDA events on the
 * handle's stream and its device time is accumulated per phase. */
int hkbe_set_profiling(hkbe_t* h, int on);

/* Accumulated device milliseconds and launch count of `phase` since the last
 * hkbe_reset_counters (timing only while profiling is on; launches always). */
int hkbe_get_timing(const hkbe_t* h, int phase, double* ms, int64_t* launches);

/* Zero the per-phase times and launch counts. */
int hkbe_reset_counters(hkbe_t* h);

/* ---- host-only numerics, exported for inspection (no device work) ---- */

/* Appendix A weights for order k (1..5): a[k+1] (BDF), omega[k+1] (Gregory),
 * D[(k+1)*(k+1)] (D_ml), I0[(k+1)*(k+1)] (I_{0,n,l}, row n).  Any output may
 * be NULL. */
int hkbe_weights(int k, double* a, double* omega, double* D, double* I0);

/* Integration rule w^(n)_l of int_0^{n h} (unit spacing) into w[max(n,k)+1]. */
int hkbe_rule(int k, int n, double* w);

/* HODLR partition of an nt x nt lower triangle with leaf size `leaf` (Sec. 2.2,
 * Fig. 2), as hkbe_create builds it, without a handle or a device: *nblk
 * blocks, and per block (arrays of length >= *nblk when given, any may be
 * NULL) rows [r0, r1), columns [c0, c1) and level.  Call with all arrays
 * NULL to get *nblk.  HKBE_ERR_ARG for nt < 1 or leaf < 1. */
int hkbe_hodlr_partition(int nt, int leaf, int32_t* nblk, int32_t* r0, int32_t* r1, int32_t* c0,
                         int32_t* c1, int32_t* level);

/* DLR matrices the library builds from the grid (cardinal functions by LU
 * solves, integrals by tanh-sinh quadrature): e0[r] (evaluation at tau=0), ebeta[r] (at beta), rev[r*r]
 * (values at beta - tau_i), q[r*r] (int l_a l_b), phi[r*r*r] (phi[a][c][i] =
 * int l_a(t) l_c^ext(t - tau_i) dt).  Outputs may be NULL. */
int hkbe_dlr_matrices(int r, const double* tau, const double* omega, double beta,
                      int xi, double* e0, double* ebeta, double* rev, double* q,
                      double* phi);

/* ---- allocation-free variant (no counterpart in the paper) ---- */

/* Capacity of the static device scratch array used by
 * hkbe_lesser_column_noalloc, in complex doubles (16 bytes each): 1 MiB. */
#define HKBE_NOALLOC_SCRATCH_CPLX 65536

/* The lesser column of one time step, x_t = G^<(t, T) for t = 0..T (the
 * lesser source followed by the lesser integral equation of a time step,
 * horizontal density matrix), computed from buffers the caller already owns
 * and WITHOUT any device allocation.  It is meant for callers that cannot
 * call cudaMalloc (for example code running inside a memory allocator's
 * callbacks, or in a process whose device memory is all handed to another
 * framework); they cannot use hkbe_create, which allocates the handle's
 * arrays.  It runs the library's point-by-point dense lesser kernels (the
 * source, then one point solve per t); hkbe_step's dense FP64 form computes
 * the same column with its chunked sweep, equal up to rounding.  Their
 * scratch (the mixed-product vector, the boundary value and the lesser
 * source, r*nao^2 + nao^2 + nt*nao^2 + 2 complex doubles) lives in one
 * file-scope device array of HKBE_NOALLOC_SCRATCH_CPLX entries that every
 * GPU loading the library holds until the process exits.  Sizes beyond it
 * are rejected with HKBE_ERR_ARG and a message saying so.
 *
 * All array arguments are DEVICE pointers to one instance in the dense layout
 * of the handle API: lower-triangular arrays of nt(nt+1)/2 N_o x N_o complex
 * matrices where element (T', t) sits at T'(T'+1)/2 + t, holding
 *   d_gr  G^R(T', t)        (row T is read)
 *   d_sr  Sigma^R(T', t)    (rows 0..T read)
 *   d_sl  Sigma^<(t, T')    (rows 0..T read)
 *   d_gl  G^<(t, T')        (row T is written: the output)
 * mixed arrays d_gtv = G^tv(T', tau_i), d_stv = Sigma^tv(T', tau_i) of
 * nt x r matrices (row T of d_gtv and rows 0..T of d_stv read), d_eps the
 * (nt+1) matrices eps(t), t = -1..nt-1, and the DLR matrices e0[r], rev[r*r],
 * q[r*r] of hkbe_dlr_matrices.  k is the integration order, h the step, and
 * T the step with k < T < nt.  Work is queued on `stream` (NULL: legacy
 * default stream); the call returns without waiting for it.
 *
 * The first call on a device does a one-time set-up with that device
 * current: it looks up the scratch array's device address
 * (cudaGetSymbolAddress).  With lazy module loading (the CUDA default) that
 * lookup also loads the library's device code and the array onto the
 * device, which allocates device memory.  So make the first call on each
 * device outside any context that forbids allocation, and before any stream
 * capture; later calls allocate nothing.  The set-up is safe to race from
 * several host threads.  Every call shares the array, which keeps the
 * previous call's contents; calls that overlap on the GPU (other streams,
 * other host threads) race on it, so serialise them.  On failure the
 * message is copied into errbuf[errlen] (may be NULL). */
int hkbe_lesser_column_noalloc(int nt, int k, int nao, int r, double h, int T,
                               const void* d_gr, const void* d_sr, const void* d_sl,
                               const void* d_gtv, const void* d_stv, const void* d_eps,
                               const double* d_e0, const double* d_rev, const double* d_q,
                               void* d_gl, void* stream, char* errbuf, size_t errlen);

#ifdef __cplusplus
}
#endif
#endif /* HKBE_H */
