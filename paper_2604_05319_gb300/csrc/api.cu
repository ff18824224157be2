// C ABI of the Kadanoff-Baym stepper (declared in include/hkbe.h).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "../../include/hkbe.h"
#include "host_numerics.h"
#include "state.h"
#include "matsubara_dev.h"
#include "sweepfree.h"

using hk::Dev;
using zc = std::complex<double>;

struct hkbe_s {
  Dev d{};
  hkbe_params p{};
  cudaStream_t s = nullptr;
  std::string err;
  int cur = -1;
  std::vector<int> last;   // last time step of each instance (its N_t - 1)
  bool have_dlr = false, have_gm = false, have_eps = false, have_model = false;
  bool self_consistent = true;
  int lat_L = 0, lat_ys = 0;   // LATTICE2B grid and reduced-set flag
  int scheme = 0;              // HKBE_SCHEME_PAPER or HKBE_SCHEME_SWEEP_FREE
  std::vector<double> tau, om, gm_host, eps_host;
  hk::DLRMats dm;
  int* any_dev = nullptr;
  size_t bytes = 0;
  std::vector<void*> allocs;
  std::vector<size_t> alloc_bytes;  // bytes of each entry of allocs (checkpoint files)
  // instrumentation
  bool profiling = false;
  double phase_ms[HKBE_NPHASE] = {0};
  int64_t phase_launches[HKBE_NPHASE] = {0};
  struct Pending { int phase; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  // bootstrap snapshot for hkbe_rewind (rows 0..k of every component)
  // (raw bytes of the storage element type)
  std::vector<char> snap_gr, snap_gl, snap_sr, snap_sl, snap_tv, snap_stv;
  // HODLR geometry (host copies) and row read-out buffers
  bool hodlr = false;
  std::vector<int> g_r0, g_r1, g_c0, g_c1, g_lvl, g_rowblk, g_colblk;
  std::vector<long long> g_uoff, g_voff, g_leafoff, g_wslv;
  double2 *rowbuf_r = nullptr, *rowbuf_l = nullptr;
  int* status_dev = nullptr;
  double2* diagbuf = nullptr;  // [n_inst][no2] density matrices of one time
  // device arrays that make up the propagation state, zeroed by hkbe_rewind so
  // that a rewound run starts from exactly the state that followed bootstrap
  std::vector<std::pair<void*, size_t>> state_arrays;
  // in-memory snapshot (hkbe_snapshot_save): a device copy of every buffer in
  // allocs, plus the host-side counters that go with it
  std::vector<void*> snap_dev;     // nullptr for scratch buffers (not part of the state)
  std::vector<const void*> scratch;  // buffers whose contents do not outlive a kernel phase
  size_t snap_bytes = 0;
  int snap_cur = -1, snap_cdir = 0, snap_nfrozR = 0, snap_nfrozL = 0;
};

namespace {
// Device buffers owned by one API call, freed when it returns.
struct CallBufs {
  std::vector<void*> p;
  ~CallBufs() {
    for (void* x : p) cudaFree(x);
  }
  template <typename T>
  cudaError_t get(T** out, size_t n) {
    void* x = nullptr;
    cudaError_t e = cudaMalloc(&x, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) p.push_back(x);
    *out = (T*)x;
    return e;
  }
};

// Launch one phase: counts its kernels and, when profiling, brackets it with
// events whose elapsed time is collected at the next drain().
template <typename F>
cudaError_t run_phase(hkbe_t* h, int phase, int nkernels, F launch) {
  h->phase_launches[phase] += nkernels;
  if (!h->profiling) return launch();
  cudaEvent_t ev[2];
  for (int i = 0; i < 2; ++i) {
    if (!h->event_pool.empty()) {
      ev[i] = h->event_pool.back();
      h->event_pool.pop_back();
    } else {
      cudaError_t e = cudaEventCreate(&ev[i]);
      if (e != cudaSuccess) return e;
    }
  }
  cudaEventRecord(ev[0], h->s);
  cudaError_t e = launch();
  cudaEventRecord(ev[1], h->s);
  h->pending.push_back({phase, ev[0], ev[1]});
  return e;
}
// Collect elapsed times of completed phases (call after a stream sync).
void drain(hkbe_t* h) {
  for (auto& p : h->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) h->phase_ms[p.phase] += ms;
    h->event_pool.push_back(p.a);
    h->event_pool.push_back(p.b);
  }
  h->pending.clear();
}
}  // namespace

static std::string g_create_error;

namespace {

int fail(hkbe_t* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return code;
}

#define HK_CUDA(h, call)                                                            \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail(h, HKBE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
int dalloc(hkbe_t* h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) return fail(h, HKBE_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  h->allocs.push_back(*p);
  h->alloc_bytes.push_back(count * sizeof(T));
  h->bytes += count * sizeof(T);
  cudaMemsetAsync(*p, 0, count * sizeof(T), h->s);
  return HKBE_OK;
}

// untyped allocation of `count` storage elements (double2 or float2)
int dalloc_el(hkbe_t* h, void** p, size_t count) {
  int rc = h->d.prec ? dalloc(h, reinterpret_cast<float2**>(p), count) : dalloc(h, reinterpret_cast<double2**>(p), count);
  if (rc == HKBE_OK) h->state_arrays.push_back({*p, std::max<size_t>(count, 1) * (h->d.prec ? sizeof(float2) : sizeof(double2))});
  return rc;
}

// mixed components: complex128 in both precision forms
int dalloc_tv(hkbe_t* h, void** p, size_t count) {
  int rc = dalloc(h, reinterpret_cast<double2**>(p), count);
  if (rc == HKBE_OK) h->state_arrays.push_back({*p, std::max<size_t>(count, 1) * sizeof(double2)});
  return rc;
}

int no2(const hkbe_t* h) { return h->p.nao * h->p.nao; }

// Last computed step of instance n (an instance stops at its own N_t - 1).
int cur_of(const hkbe_t* h, int n) { return std::min(h->cur, h->last[n]); }
// First uncompressed row of instance n (the device-side front_of).
int front_host(const hkbe_t* h, int n) {
  const int lk = h->last[n] - h->d.k;
  const int fz = lk >= h->d.L ? (lk / h->d.L) * h->d.L : 0;
  return std::min(h->d.cdir, fz);
}

// bytes of one complex storage element
size_t esz(const hkbe_t* h) { return h->d.prec ? sizeof(float2) : sizeof(double2); }
char* elp(const hkbe_t* h, void* base, size_t off) { return static_cast<char*>(base) + off * esz(h); }

// Copy `cnt` complex storage elements device -> host as interleaved doubles
// (converted from float in the mixed form).  Synchronises the stream.
cudaError_t d2h_el(hkbe_t* h, double* out, const char* src, size_t cnt) {
  if (!h->d.prec) {
    cudaError_t e = cudaMemcpyAsync(out, src, cnt * sizeof(double2), cudaMemcpyDeviceToHost, h->s);
    return e != cudaSuccess ? e : cudaStreamSynchronize(h->s);
  }
  std::vector<float> tmp(2 * cnt);
  cudaError_t e = cudaMemcpyAsync(tmp.data(), src, cnt * sizeof(float2), cudaMemcpyDeviceToHost, h->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
  if (e != cudaSuccess) return e;
  for (size_t i = 0; i < 2 * cnt; ++i) out[i] = tmp[i];
  return cudaSuccess;
}
// Copy `cnt` complex values (interleaved doubles) host -> device storage
// (rounded to float in the mixed form).  Synchronises the stream.
cudaError_t h2d_el(hkbe_t* h, char* dst, const double* in, size_t cnt) {
  if (!h->d.prec) {
    cudaError_t e = cudaMemcpyAsync(dst, in, cnt * sizeof(double2), cudaMemcpyHostToDevice, h->s);
    return e != cudaSuccess ? e : cudaStreamSynchronize(h->s);
  }
  std::vector<float> tmp(2 * cnt);
  for (size_t i = 0; i < 2 * cnt; ++i) tmp[i] = (float)in[i];
  cudaError_t e = cudaMemcpyAsync(dst, tmp.data(), cnt * sizeof(float2), cudaMemcpyHostToDevice, h->s);
  return e != cudaSuccess ? e : cudaStreamSynchronize(h->s);
}

// Offset (in matrices) of element (T, 0) of instance n in a two-time array.
size_t row_off(const hkbe_t* h, int n, int T) {
  const hk::Dev& d = h->d;
  if (d.ring) return ((size_t)n * d.ring + (size_t)(T % d.ring)) * d.nt * no2(h);
  return ((size_t)n * d.ntri + (size_t)T * (T + 1) / 2) * no2(h);
}

// HODLR partition (Sec. 2.2): leaves [j L, (j+1) L); a range of leaves [a, b)
// is split at m = a + (b - a)/2 into the block rows [m L, b L) x cols [a L, m L)
// and the two halves, recursively.
void build_geometry(hkbe_t* h) {
  const int nt = h->p.nt, L = h->p.leaf;
  const int nleaf = (nt + L - 1) / L;
  h->g_r0.clear(); h->g_r1.clear(); h->g_c0.clear(); h->g_c1.clear(); h->g_lvl.clear();
  int maxdepth = 0;
  struct Rng { int a, b, depth; };
  std::vector<Rng> stack{{0, nleaf, 0}};
  while (!stack.empty()) {
    Rng g = stack.back();
    stack.pop_back();
    if (g.b - g.a <= 1) continue;
    const int m = g.a + (g.b - g.a) / 2;
    h->g_r0.push_back(m * L);
    h->g_r1.push_back(std::min(g.b * L, nt));
    h->g_c0.push_back(g.a * L);
    h->g_c1.push_back(m * L);
    h->g_lvl.push_back(g.depth);
    maxdepth = std::max(maxdepth, g.depth);
    stack.push_back({m, g.b, g.depth + 1});
    stack.push_back({g.a, m, g.depth + 1});
  }
  const int nblk = (int)h->g_r0.size(), maxl = std::max(1, maxdepth + 1), n2 = no2(h);
  h->g_rowblk.assign((size_t)nleaf * maxl, -1);
  h->g_colblk.assign((size_t)nleaf * maxl, -1);
  h->g_uoff.resize(nblk);
  h->g_voff.resize(nblk);
  long long uo = 0, vo = 0;
  for (int b = 0; b < nblk; ++b) {
    h->g_uoff[b] = uo;
    h->g_voff[b] = vo;
    uo += (long long)(h->g_r1[b] - h->g_r0[b]) * n2;
    vo += (long long)(h->g_c1[b] - h->g_c0[b]) * n2;
    for (int j = h->g_r0[b] / L; j * L < h->g_r1[b]; ++j) h->g_rowblk[(size_t)j * maxl + h->g_lvl[b]] = b;
    for (int j = h->g_c0[b] / L; j * L < h->g_c1[b]; ++j) h->g_colblk[(size_t)j * maxl + h->g_lvl[b]] = b;
  }
  h->g_leafoff.resize(nleaf);
  long long lo = 0;
  for (int j = 0; j < nleaf; ++j) {
    h->g_leafoff[j] = lo;
    const long long nj = std::min(L, nt - j * L);
    lo += nj * (nj + 1) / 2;
  }
  hk::Dev& d = h->d;
  d.L = L; d.nleaf = nleaf; d.nblk = nblk; d.maxl = maxl;
  d.utot = uo; d.vtot = vo; d.leaftot = lo;
}

template <typename T>
int upload(hkbe_t* h, const T** dst, const std::vector<T>& v) {
  T* p = nullptr;
  int rc = dalloc(h, &p, v.size());
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->s);
  if (e != cudaSuccess) return fail(h, HKBE_ERR_CUDA, cudaGetErrorString(e));
  *dst = p;
  return HKBE_OK;
}

}  // namespace

extern "C" {

const char* hkbe_last_error(const hkbe_t* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int hkbe_create(const hkbe_params* p, const int32_t* nt_per_inst, void* stream, hkbe_t** out) {
  if (!p || !out) return fail(nullptr, HKBE_ERR_ARG, "null argument");
  *out = nullptr;
  if (p->precision == HKBE_PREC_TF32X3 || p->precision == HKBE_PREC_BF16X3)
    return fail(nullptr, HKBE_ERR_ARG,
                "precision 2 (FP32 + 3xTF32 split) and 3 (BF16x3 split) are not provided: they split the operands "
                "of a dense contraction for the tensor cores, and every history sum here is a per-instance "
                "matrix-vector product; use HKBE_PREC_MIXED for the reduced-precision form");
  if (p->k < 1 || p->k > 5) return fail(nullptr, HKBE_ERR_ARG, "k must be in 1..5");
  if (p->nt < p->k + 2) return fail(nullptr, HKBE_ERR_ARG, "nt must be >= k + 2");
  if (p->nao < 1 || p->nao > 4) return fail(nullptr, HKBE_ERR_ARG, "nao must be in 1..4");
  if (p->xi != -1) return fail(nullptr, HKBE_ERR_ARG, "only fermions (xi = -1) are supported");
  if (p->n_inst < 1) return fail(nullptr, HKBE_ERR_ARG, "n_inst must be >= 1");
  if (!(p->h > 0) || !(p->beta > 0)) return fail(nullptr, HKBE_ERR_ARG, "h and beta must be > 0");
  if (p->rho_mode != 0 && p->rho_mode != 1) return fail(nullptr, HKBE_ERR_ARG, "rho_mode must be 0 or 1");
  if (p->precision != HKBE_PREC_FP64 && p->precision != HKBE_PREC_MIXED)
    return fail(nullptr, HKBE_ERR_ARG, "precision must be HKBE_PREC_FP64 or HKBE_PREC_MIXED");
  if (p->max_iter < 1) return fail(nullptr, HKBE_ERR_ARG, "max_iter must be >= 1");
  if (p->svd_tol < 0) return fail(nullptr, HKBE_ERR_ARG, "svd_tol must be >= 0");
  if (nt_per_inst)
    for (int n = 0; n < p->n_inst; ++n)
      if (nt_per_inst[n] < p->k + 2 || nt_per_inst[n] > p->nt)
        return fail(nullptr, HKBE_ERR_ARG, "nt_per_inst[" + std::to_string(n) + "] must be in k+2..nt");
  if (p->svd_tol > 0) {
    if (p->leaf != 32 && p->leaf != 64) return fail(nullptr, HKBE_ERR_ARG, "leaf must be 32 or 64");
    if (p->leaf <= 2 * p->k) return fail(nullptr, HKBE_ERR_ARG, "leaf must exceed 2k");
    if (p->r_max < 1 || p->r_max > 128) return fail(nullptr, HKBE_ERR_ARG, "r_max must be in 1..128");
  }
  hkbe_t* h = new hkbe_t();
  h->p = *p;
  h->s = (cudaStream_t)stream;
  h->last.assign(p->n_inst, p->nt - 1);
  if (nt_per_inst)
    for (int n = 0; n < p->n_inst; ++n) h->last[n] = nt_per_inst[n] - 1;
  Dev& d = h->d;
  d.nt = p->nt; d.k = p->k; d.no = p->nao; d.n_inst = p->n_inst; d.xi = p->xi;
  d.rho_mode = p->rho_mode; d.h = p->h; d.beta = p->beta; d.r = 0; d.model = 0;
  d.prec = p->precision == HKBE_PREC_MIXED ? 1 : 0;
  d.ntri = (long long)p->nt * (p->nt + 1) / 2;
  hk::Weights w;
  hk::weights_build(p->k, &w);
  d.w.k = w.k;
  std::memcpy(d.w.a, w.a, sizeof(w.a));
  std::memcpy(d.w.omega, w.omega, sizeof(w.omega));
  std::memcpy(d.w.D, w.D, sizeof(w.D));
  std::memcpy(d.w.I0, w.I0, sizeof(w.I0));
  for (int i = 0; i < 6; ++i) {
    d.w.ah[i] = w.a[i] / p->h;
    d.w.omegaf[i] = (float)w.omega[i];
    for (int j = 0; j < 6; ++j) d.w.I0f[i][j] = (float)w.I0[i][j];
  }
  h->hodlr = p->svd_tol > 0;
  size_t tri = (size_t)d.n_inst * d.ntri * d.no * d.no;
  int rc = HKBE_OK;
  if (h->hodlr) {
    build_geometry(h);
    d.ring = p->leaf + 8;
    d.cdir = 0;
    d.rmax = p->r_max;
    d.svd_tol = p->svd_tol;
    tri = (size_t)d.n_inst * d.ring * d.nt * d.no * d.no;
    const size_t n2 = (size_t)d.no * d.no, N = d.n_inst;
    // TSVD workspace: one slot per (instance, component, orbital pair, level),
    // each sized for the widest block of its level
    const int ldk = d.rmax + d.L;
    h->g_wslv.assign(d.maxl + 1, 0);
    for (int lv = 0; lv < d.maxl; ++lv) {
      int ncl = 1;
      for (size_t b = 0; b < h->g_c0.size(); ++b)
        if (h->g_lvl[b] == lv) ncl = std::max(ncl, h->g_c1[b] - h->g_c0[b]);
      h->g_wslv[lv + 1] = h->g_wslv[lv] + 2LL * d.L * ncl + (long long)d.L * d.rmax + (long long)d.L * d.L + 2LL * ldk * ldk;
    }
    d.tsvd_ws_per = h->g_wslv[d.maxl];
    // instances compressed at a time on one shared workspace: as many as fit
    // in 32 GiB of workspace.  One launch over the whole batch is fastest
    // (the CTAs' FP64 work is uneven, and consecutive launches each wait for
    // their slowest CTA: groups of 12 C4 instances made the compression 2.3
    // times slower); groups only bound the memory of very large batches.
    {
      const double per_inst = 4.0 * n2 * d.tsvd_ws_per * sizeof(double2);
      d.tsvd_group = (int)std::max(1.0, std::min((double)N, std::floor(34359738368.0 / per_inst)));
    }
    const size_t ctas = (size_t)d.tsvd_group * 4 * n2;
    for (int X = 0; X < 4; ++X) {
      if ((rc = dalloc_el(h, &d.hod[X].U, N * d.utot * d.rmax)) || (rc = dalloc_el(h, &d.hod[X].V, N * d.vtot * d.rmax)) ||
          (rc = dalloc(h, &d.hod[X].S, N * d.nblk * n2 * d.rmax)) ||
          ((void)h->state_arrays.push_back({d.hod[X].S, N * d.nblk * n2 * d.rmax * sizeof(double)}), false) ||
          (rc = dalloc(h, &d.hod[X].rank, N * d.nblk * n2)) || (rc = dalloc_el(h, &d.hod[X].leaf, N * d.leaftot * n2))) {
        g_create_error = h->err;
        hkbe_destroy(h);
        return rc;
      }
    }
    if ((rc = dalloc_el(h, &d.band, N * d.nt * d.k * n2)) ||
        (rc = dalloc(h, &d.proj, N * d.no * d.maxl * n2 * d.rmax + N * d.nblk * n2 * d.no * 2 * d.rmax)) ||
        (rc = dalloc(h, &d.tsvd_ws, ctas * d.tsvd_ws_per)) ||
        (rc = dalloc(h, &h->rowbuf_r, (size_t)d.nt * n2)) || (rc = dalloc(h, &h->rowbuf_l, (size_t)d.nt * n2)) ||
        (rc = upload(h, &d.b_r0, h->g_r0)) || (rc = upload(h, &d.b_r1, h->g_r1)) ||
        (rc = upload(h, &d.b_c0, h->g_c0)) || (rc = upload(h, &d.b_c1, h->g_c1)) ||
        (rc = upload(h, &d.b_lvl, h->g_lvl)) || (rc = upload(h, &d.b_uoff, h->g_uoff)) ||
        (rc = upload(h, &d.b_voff, h->g_voff)) || (rc = upload(h, &d.leafoff, h->g_leafoff)) ||
        (rc = upload(h, &d.rowblk, h->g_rowblk)) || (rc = upload(h, &d.colblk, h->g_colblk)) ||
        (rc = upload(h, &d.ws_lvoff, h->g_wslv))) {
      g_create_error = h->err;
      hkbe_destroy(h);
      return rc;
    }
    h->scratch.insert(h->scratch.end(), {d.tsvd_ws, h->rowbuf_r, h->rowbuf_l});
  }
  if (d.prec) {
    const size_t rowsz = (size_t)d.n_inst * 2 * d.nt * d.no * d.no, ringsz = (size_t)d.n_inst * d.ring * d.nt * d.no * d.no;
    if ((!h->hodlr && (rc = dalloc(h, &d.row64, rowsz))) ||
        (rc = dalloc(h, &d.diag64, (size_t)d.n_inst * d.nt * d.no * d.no))) {
      g_create_error = h->err;
      hkbe_destroy(h);
      return rc;
    }
    if (!h->hodlr) h->state_arrays.push_back({d.row64, rowsz * sizeof(double2)});
    h->state_arrays.push_back({d.diag64, (size_t)d.n_inst * d.nt * d.no * d.no * sizeof(double2)});
    // FP64 copies of the ring rows of the four two-time components (compressed form)
    for (int X = 0; h->hodlr && X < 4; ++X) {
      if ((rc = dalloc(h, &d.ring64[X], ringsz))) {
        g_create_error = h->err;
        hkbe_destroy(h);
        return rc;
      }
      h->state_arrays.push_back({d.ring64[X], ringsz * sizeof(double2)});
    }
  }
  d.nchunk = (d.nt + 31) / 32;
  d.nfrozR = d.nfrozL = 0;
  // status words: [0] TSVD ranks capped at r_max, [1] TSVD Jacobi non-convergence,
  // [2] timed-out waits for a staged chunk inverse (sweeps)
  if ((rc = dalloc(h, &h->status_dev, 3))) {
    g_create_error = h->err;
    hkbe_destroy(h);
    return rc;
  }
  d.status = h->status_dev;
  {
    const size_t ld = 32 * (size_t)d.no;
    if ((rc = dalloc(h, &d.cinv, (size_t)d.n_inst * d.nchunk * 2 * ld * ld)) ||
        (rc = dalloc(h, &d.cinv_ws, (size_t)d.n_inst * 2 * ld * ld))) {
      g_create_error = h->err;
      hkbe_destroy(h);
      return rc;
    }
  }
  if ((rc = dalloc_el(h, &d.GR, tri)) || (rc = dalloc_el(h, &d.GL, tri)) || (rc = dalloc_el(h, &d.SR, tri)) ||
      (rc = dalloc_el(h, &d.SL, tri)) ||
      (rc = dalloc(h, &d.eps, (size_t)d.n_inst * (d.nt + 1) * d.no * d.no)) ||
      (rc = dalloc(h, &d.eps_ext, (size_t)d.n_inst * (d.nt + 1) * d.no * d.no)) ||
      (rc = dalloc(h, &d.drA, (size_t)d.n_inst * (d.nt + 1))) || (rc = dalloc(h, &d.drU, (size_t)d.n_inst * (d.nt + 1))) ||
      (rc = dalloc(h, &d.mpar, (size_t)d.n_inst * hk::MP)) ||
      (rc = dalloc(h, &d.qsrc, (size_t)d.n_inst * d.nt * d.no * d.no)) ||
      (rc = dalloc(h, &d.x0, (size_t)d.n_inst * d.no * d.no)) || (rc = dalloc(h, &d.err, (size_t)d.n_inst)) ||
      (rc = dalloc(h, &d.active, (size_t)d.n_inst)) || (rc = dalloc(h, &h->any_dev, 1)) ||
      (rc = dalloc(h, &h->diagbuf, (size_t)d.n_inst * d.no * d.no)) || (rc = upload(h, &d.last, h->last))) {
    g_create_error = h->err;
    hkbe_destroy(h);
    return rc;
  }
  h->scratch.insert(h->scratch.end(), {d.cinv_ws, h->diagbuf});
  cudaError_t e = cudaStreamSynchronize(h->s);
  if (e != cudaSuccess) {
    g_create_error = std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e);
    hkbe_destroy(h);
    return HKBE_ERR_CUDA;
  }
  *out = h;
  return HKBE_OK;
}

int hkbe_destroy(hkbe_t* h) {
  if (!h) return HKBE_OK;
  cudaStreamSynchronize(h->s);
  drain(h);
  for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
  for (void* p : h->allocs) cudaFree(p);
  for (void* p : h->snap_dev)
    if (p) cudaFree(p);
  delete h;
  return HKBE_OK;
}

int hkbe_set_dlr(hkbe_t* h, int r, const double* tau, const double* omega) {
  if (!h || !tau || !omega) return fail(h, HKBE_ERR_ARG, "null argument");
  if (h->have_dlr) return fail(h, HKBE_ERR_ARG, "DLR grid already set");
  if (r < 1 || r > 128) return fail(h, HKBE_ERR_ARG, "r must be in 1..128");
  for (int i = 0; i < r; ++i)
    if (!(tau[i] > 0.0 && tau[i] < h->p.beta)) return fail(h, HKBE_ERR_ARG, "DLR nodes must lie in (0, beta)");
  h->tau.assign(tau, tau + r);
  h->om.assign(omega, omega + r);
  if (!hk::dlr_build(r, tau, omega, h->p.beta, h->p.xi, &h->dm))
    return fail(h, HKBE_ERR_ARG, "singular DLR kernel matrix");
  Dev& d = h->d;
  d.r = r;
  const size_t n2 = (size_t)d.no * d.no;
  int rc;
  if ((rc = dalloc(h, &d.tau, r)) || (rc = dalloc(h, &d.e0, r)) || (rc = dalloc(h, &d.ebeta, r)) ||
      (rc = dalloc(h, &d.rev, (size_t)r * r)) || (rc = dalloc(h, &d.q, (size_t)r * r)) ||
      (rc = dalloc_tv(h, &d.GTV, (size_t)d.n_inst * d.nt * r * n2)) ||
      (rc = dalloc_tv(h, &d.STV, (size_t)d.n_inst * d.nt * r * n2)) ||
      (rc = dalloc(h, &d.gm, (size_t)d.n_inst * r * n2)) ||
      (rc = dalloc(h, &d.wconv, (size_t)d.n_inst * r * r * n2)) ||
      (rc = dalloc(h, &d.vvec, (size_t)d.n_inst * r * n2)))
    return rc;
  HK_CUDA(h, cudaMemcpyAsync(d.tau, tau, r * sizeof(double), cudaMemcpyHostToDevice, h->s));
  HK_CUDA(h, cudaMemcpyAsync(d.e0, h->dm.e0.data(), r * sizeof(double), cudaMemcpyHostToDevice, h->s));
  HK_CUDA(h, cudaMemcpyAsync(d.ebeta, h->dm.ebeta.data(), r * sizeof(double), cudaMemcpyHostToDevice, h->s));
  HK_CUDA(h, cudaMemcpyAsync(d.rev, h->dm.rev.data(), r * r * sizeof(double), cudaMemcpyHostToDevice, h->s));
  HK_CUDA(h, cudaMemcpyAsync(d.q, h->dm.q.data(), r * r * sizeof(double), cudaMemcpyHostToDevice, h->s));
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  h->have_dlr = true;
  return HKBE_OK;
}

int hkbe_set_matsubara(hkbe_t* h, const double* gm) {
  if (!h || !gm) return fail(h, HKBE_ERR_ARG, "null argument");
  if (!h->have_dlr) return fail(h, HKBE_ERR_ARG, "hkbe_set_dlr must precede hkbe_set_matsubara");
  Dev& d = h->d;
  const int r = d.r, n2 = no2(h);
  const size_t cnt = (size_t)d.n_inst * r * n2 * 2;
  h->gm_host.assign(gm, gm + cnt);
  // W[a][i] = sum_c phi[a][c][i] G^M(tau_c)   (convolution tensor of Eq. KBET)
  std::vector<double> W((size_t)d.n_inst * r * r * n2 * 2, 0.0);
  for (int n = 0; n < d.n_inst; ++n)
    for (int a = 0; a < r; ++a)
      for (int i = 0; i < r; ++i) {
        double* w = &W[(((size_t)n * r + a) * r + i) * n2 * 2];
        for (int c = 0; c < r; ++c) {
          const double ph = h->dm.phi[((size_t)a * r + c) * r + i];
          const double* g = gm + ((size_t)n * r + c) * n2 * 2;
          for (int q = 0; q < 2 * n2; ++q) w[q] += ph * g[q];
        }
      }
  HK_CUDA(h, cudaMemcpyAsync(d.gm, gm, cnt * sizeof(double), cudaMemcpyHostToDevice, h->s));
  HK_CUDA(h, cudaMemcpyAsync(d.wconv, W.data(), W.size() * sizeof(double), cudaMemcpyHostToDevice, h->s));
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  h->have_gm = true;
  return HKBE_OK;
}

int hkbe_solve_matsubara(hkbe_t* h, double U_eq, double eta, int n_eta, double mix, double tol, int max_iter,
                         double* gm_out, int32_t* iters, double* err_out) {
  if (!h) return fail(h, HKBE_ERR_ARG, "null handle");
  if (!h->have_dlr || !h->have_eps || !h->have_model)
    return fail(h, HKBE_ERR_ARG, "hkbe_set_dlr, hkbe_set_hamiltonian and hkbe_set_model must precede hkbe_solve_matsubara");
  if (h->cur >= 0) return fail(h, HKBE_ERR_ARG, "hkbe_solve_matsubara must precede hkbe_bootstrap");
  if (!(mix > 0.0 && mix <= 1.0) || max_iter < 1 || n_eta < 0 || !std::isfinite(U_eq) || !std::isfinite(eta) ||
      !(tol >= 0.0))
    return fail(h, HKBE_ERR_ARG, "mix in (0, 1], max_iter >= 1, n_eta >= 0, finite U_eq and eta, tol >= 0");
  Dev& d = h->d;
  hk::MatsDev m{};
  switch (d.model) {
    case HKBE_MODEL_NONE: m.model = hk::kMatsNone; break;
    case HKBE_MODEL_BETHE: m.model = hk::kMatsBethe; break;
    case HKBE_MODEL_NAMBU: m.model = hk::kMatsNambu; break;
    case HKBE_MODEL_LATTICE2B: m.model = hk::kMatsLattice; break;
    default: return fail(h, HKBE_ERR_ARG, "no equilibrium solve for this model (its G^M has a closed form)");
  }
  const int r = d.r, n2 = no2(h), N = d.n_inst;
  std::vector<zc> F, B;
  std::vector<double> nu;
  if (!hk::mats_maps(r, h->tau.data(), h->om.data(), h->p.beta, &F, &B, &nu))
    return fail(h, HKBE_ERR_ARG, "singular DLR kernel matrix");
  CallBufs bufs;   // buffers of this call only (an initialisation step, not the per-step path)
  double2 *dF, *dB, *G, *Gn, *S;
  double *dnu, *dphi, *derr;
  const size_t per = (size_t)N * r * n2;
  HK_CUDA(h, bufs.get(&dF, (size_t)r * r));
  HK_CUDA(h, bufs.get(&dB, (size_t)r * r));
  HK_CUDA(h, bufs.get(&dnu, r));
  HK_CUDA(h, bufs.get(&dphi, (size_t)r * r * r));
  HK_CUDA(h, bufs.get(&derr, N));
  HK_CUDA(h, bufs.get(&G, per));
  HK_CUDA(h, bufs.get(&Gn, per));
  HK_CUDA(h, bufs.get(&S, per));
  HK_CUDA(h, cudaMemcpyAsync(dF, F.data(), F.size() * sizeof(double2), cudaMemcpyHostToDevice, h->s));
  HK_CUDA(h, cudaMemcpyAsync(dB, B.data(), B.size() * sizeof(double2), cudaMemcpyHostToDevice, h->s));
  HK_CUDA(h, cudaMemcpyAsync(dnu, nu.data(), r * sizeof(double), cudaMemcpyHostToDevice, h->s));
  HK_CUDA(h, cudaMemcpyAsync(dphi, h->dm.phi.data(), h->dm.phi.size() * sizeof(double), cudaMemcpyHostToDevice,
                             h->s));
  HK_CUDA(h, cudaMemsetAsync(S, 0, per * sizeof(double2), h->s));
  m.r = r; m.no = d.no; m.n_inst = N; m.L = h->lat_L; m.ys = h->lat_ys; m.xi = d.xi; m.n_eta = n_eta;
  m.beta = h->p.beta; m.U = U_eq; m.eta = eta;
  m.F = dF; m.B = dB; m.nu = dnu; m.rev = d.rev; m.ebeta = d.ebeta; m.tau = d.tau; m.mpar = d.mpar;
  m.e0 = d.eps_ext; m.e0_stride = (long long)(d.nt + 1) * n2;
  m.G = G; m.Gn = Gn; m.S = S; m.err = derr;
  HK_CUDA(h, hk::launch_mats_dyson(m, 0, G, h->s));   // the non-interacting G^M of eps(0_|)
  std::vector<double> e_host(N);
  int it = 0;
  double err = INFINITY;
  for (it = 1; it <= max_iter; ++it) {
    HK_CUDA(h, hk::launch_mats_sigma(m, h->s));
    HK_CUDA(h, hk::launch_mats_dyson(m, it, Gn, h->s));
    HK_CUDA(h, cudaMemcpyAsync(e_host.data(), derr, N * sizeof(double), cudaMemcpyDeviceToHost, h->s));
    HK_CUDA(h, cudaStreamSynchronize(h->s));
    err = 0.0;
    for (double e : e_host) err = std::isfinite(e) ? std::max(err, e) : NAN;
    if (!std::isfinite(err)) return fail(h, HKBE_ERR_NAN, "singular Dyson matrix or non-finite iterate");
    if (err < tol && it > n_eta) {
      HK_CUDA(h, cudaMemcpyAsync(G, Gn, per * sizeof(double2), cudaMemcpyDeviceToDevice, h->s));
      break;
    }
    HK_CUDA(h, hk::launch_mats_mix(m, it > 1 ? mix : 1.0, h->s));
  }
  // install: G^M, the convolution tensor of the mixed component, the host copy
  HK_CUDA(h, cudaMemcpyAsync(d.gm, G, per * sizeof(double2), cudaMemcpyDeviceToDevice, h->s));
  HK_CUDA(h, hk::launch_mats_wconv(m, dphi, d.wconv, h->s));
  h->gm_host.assign(per * 2, 0.0);
  HK_CUDA(h, cudaMemcpyAsync(h->gm_host.data(), G, per * sizeof(double2), cudaMemcpyDeviceToHost, h->s));
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  if (gm_out) std::memcpy(gm_out, h->gm_host.data(), per * sizeof(double2));
  h->have_gm = true;
  if (iters) *iters = it > max_iter ? max_iter : it;
  if (err_out) *err_out = err;
  if (it > max_iter) return fail(h, HKBE_ERR_NOCONV, "equilibrium iteration reached max_iter");
  return HKBE_OK;
}

int hkbe_set_scheme(hkbe_t* h, int scheme) {
  if (!h) return fail(h, HKBE_ERR_ARG, "null handle");
  if (scheme != HKBE_SCHEME_PAPER && scheme != HKBE_SCHEME_SWEEP_FREE)
    return fail(h, HKBE_ERR_ARG, "unknown scheme");
  if (h->cur >= 0) return fail(h, HKBE_ERR_ARG, "hkbe_set_scheme must precede hkbe_bootstrap");
  if (scheme == HKBE_SCHEME_SWEEP_FREE && (h->hodlr || h->d.prec != 0 || h->d.k * h->d.no > 20))
    return fail(h, HKBE_ERR_ARG, "the sweep-free scheme runs in the dense FP64 storage form (k N_o <= 20)");
  h->scheme = scheme;
  return HKBE_OK;
}

int hkbe_set_hamiltonian(hkbe_t* h, const double* eps) {
  if (!h || !eps) return fail(h, HKBE_ERR_ARG, "null argument");
  Dev& d = h->d;
  const size_t cnt = (size_t)d.n_inst * (d.nt + 1) * no2(h) * 2;
  for (size_t i = 0; i < cnt; ++i)
    if (!std::isfinite(eps[i])) return fail(h, HKBE_ERR_NAN, "non-finite value in eps");
  h->eps_host.assign(eps, eps + cnt);
  HK_CUDA(h, cudaMemcpyAsync(d.eps, eps, cnt * sizeof(double), cudaMemcpyHostToDevice, h->s));
  HK_CUDA(h, cudaMemcpyAsync(d.eps_ext, eps, cnt * sizeof(double), cudaMemcpyHostToDevice, h->s));
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  h->have_eps = true;
  return HKBE_OK;
}

int hkbe_set_hamiltonian_at(hkbe_t* h, int t, const double* eps_t) {
  if (!h || !eps_t) return fail(h, HKBE_ERR_ARG, "null argument");
  if (!h->have_eps) return fail(h, HKBE_ERR_ARG, "hkbe_set_hamiltonian must precede hkbe_set_hamiltonian_at");
  Dev& d = h->d;
  if (t <= h->cur || t > d.nt - 1) return fail(h, HKBE_ERR_RANGE, "t must satisfy current step < t <= nt-1");
  const int n2 = no2(h);
  for (int i = 0; i < d.n_inst * n2 * 2; ++i)
    if (!std::isfinite(eps_t[i])) return fail(h, HKBE_ERR_NAN, "non-finite value in eps_t");
  // eps is [n][nt+1][no2], index t+1: one strided copy of n_inst pieces
  for (double2* dst : {d.eps, d.eps_ext})
    HK_CUDA(h, cudaMemcpy2DAsync(dst + (size_t)(t + 1) * n2, (size_t)(d.nt + 1) * n2 * sizeof(double2), eps_t,
                                 (size_t)n2 * sizeof(double2), (size_t)n2 * sizeof(double2), d.n_inst,
                                 cudaMemcpyHostToDevice, h->s));
  for (int n = 0; n < d.n_inst; ++n)
    std::memcpy(&h->eps_host[(((size_t)n * (d.nt + 1)) + t + 1) * n2 * 2], eps_t + (size_t)n * n2 * 2,
                n2 * 2 * sizeof(double));
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  return HKBE_OK;
}

int hkbe_set_drive(hkbe_t* h, const double* A, const double* U) {
  if (!h) return fail(h, HKBE_ERR_ARG, "null handle");
  if (h->cur >= 0) return fail(h, HKBE_ERR_ARG, "hkbe_set_drive must precede hkbe_bootstrap");
  Dev& d = h->d;
  const size_t cnt = (size_t)d.n_inst * (d.nt + 1);
  for (int w = 0; w < 2; ++w) {
    const double* src = w == 0 ? A : U;
    double* dst = w == 0 ? d.drA : d.drU;
    if (!src) {
      HK_CUDA(h, cudaMemsetAsync(dst, 0, cnt * sizeof(double), h->s));
      continue;
    }
    for (size_t i = 0; i < cnt; ++i)
      if (!std::isfinite(src[i])) return fail(h, HKBE_ERR_NAN, "non-finite value in the drive");
    HK_CUDA(h, cudaMemcpyAsync(dst, src, cnt * sizeof(double), cudaMemcpyHostToDevice, h->s));
  }
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  return HKBE_OK;
}

int hkbe_set_model(hkbe_t* h, int model, const double* params, int nparams) {
  if (!h) return fail(h, HKBE_ERR_ARG, "null handle");
  Dev& d = h->d;
  const int no = d.no;
  std::vector<double> mp((size_t)d.n_inst * hk::MP, 0.0);
  if (model == HKBE_MODEL_NONE) {
    h->self_consistent = false;
  } else if (model == HKBE_MODEL_BETHE) {
    if (!params || nparams < 1) return fail(h, HKBE_ERR_ARG, "BETHE needs params[0] = v");
    for (int n = 0; n < d.n_inst; ++n) mp[(size_t)n * hk::MP] = params[(size_t)n * nparams];
    h->self_consistent = true;
  } else if (model == HKBE_MODEL_BATH) {
    if (!params || nparams < 1) return fail(h, HKBE_ERR_ARG, "BATH needs parameters");
    for (int n = 0; n < d.n_inst; ++n) {
      const double* q = params + (size_t)n * nparams;
      const int nb = (int)q[0];
      if (nb < 1 || nb > 4 || nparams != 1 + nb + 2 * no * nb)
        return fail(h, HKBE_ERR_ARG, "BATH params must be [nb, eps_b[nb], V[nao][nb] complex]");
      std::memcpy(&mp[(size_t)n * hk::MP], q, nparams * sizeof(double));
    }
    h->self_consistent = false;
  } else if (model == HKBE_MODEL_LATTICE2B) {
    if (no != 1) return fail(h, HKBE_ERR_ARG, "LATTICE2B needs nao = 1");
    if (!params || nparams < 1 || nparams > 2) return fail(h, HKBE_ERR_ARG, "LATTICE2B needs params [L] or [L, ysymm]");
    const int L = (int)params[0];
    const double ysp = nparams == 2 ? params[1] : 0.0;
    if (ysp != 0.0 && ysp != 1.0) return fail(h, HKBE_ERR_ARG, "LATTICE2B ysymm must be 0 or 1");
    const int ys = ysp != 0.0;
    const int nk = ys ? L * (L / 2 + 1) : L * L;
    if (L < 1 || L > 16 || (double)L != params[0] || (ys && L % 2) || nk != d.n_inst)
      return fail(h, HKBE_ERR_ARG, "LATTICE2B needs an integer L in 1..16 with n_inst = L*L (L*(L/2+1), L even, with ysymm)");
    for (int n = 0; n < d.n_inst; ++n)
      if (h->last[n] != d.nt - 1)
        return fail(h, HKBE_ERR_ARG, "LATTICE2B couples its k-points through Sigma: every k needs the same N_t");
    for (int n = 0; n < d.n_inst; ++n) {
      mp[(size_t)n * hk::MP] = L;
      mp[(size_t)n * hk::MP + 1] = ys;
    }
    h->lat_L = L;
    h->lat_ys = ys;
    h->self_consistent = true;
  } else if (model == HKBE_MODEL_NAMBU) {
    if (no != 2) return fail(h, HKBE_ERR_ARG, "NAMBU needs nao = 2");
    if (!params || (nparams != 1 && nparams != 3)) return fail(h, HKBE_ERR_ARG, "NAMBU needs params [v] or [v, g, w0]");
    for (int n = 0; n < d.n_inst; ++n)
      for (int c = 0; c < nparams; ++c) mp[(size_t)n * hk::MP + c] = params[(size_t)n * nparams + c];
    if (nparams == 3)
      for (int n = 0; n < d.n_inst; ++n)
        if (mp[(size_t)n * hk::MP + 1] != 0.0 && !(mp[(size_t)n * hk::MP + 2] > 0.0))
          return fail(h, HKBE_ERR_ARG, "NAMBU phonon frequency w0 must be > 0");
    h->self_consistent = true;
  } else {
    return fail(h, HKBE_ERR_ARG, "unknown model");
  }
  d.model = model;
  HK_CUDA(h, cudaMemcpyAsync(d.mpar, mp.data(), mp.size() * sizeof(double), cudaMemcpyHostToDevice, h->s));
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  h->have_model = true;
  return HKBE_OK;
}

// Mean-field guess of the start square (Sec. 3.3, green_from_H):
// G^R = -i e^{-i e (t-t')}, G^<(t,t') = i e^{-i e t} rho e^{i e t'},
// G^tv = -xi i e^{-i e t} rho e^{e tau}, e = eps(0_|), rho = -G^M(beta^-).
static int hf_guess(hkbe_t* h) {
  Dev& d = h->d;
  const int no = d.no, n2 = no * no, k = d.k, r = d.r;
  const double hh = d.h;
  std::vector<double> gr((size_t)(k + 1) * (k + 2) / 2 * n2 * 2), gl(gr.size()), gtv((size_t)(k + 1) * r * n2 * 2);
  for (int n = 0; n < d.n_inst; ++n) {
    zc e[16], U[16];
    double E[4];
    const double* ep = &h->eps_host[(size_t)n * (d.nt + 1) * n2 * 2];
    for (int q = 0; q < n2; ++q) e[q] = zc(ep[2 * q], ep[2 * q + 1]);
    hk::herm_eig(no, e, E, U);
    zc rho[16];
    for (int q = 0; q < n2; ++q) {
      zc s = 0;
      for (int c = 0; c < r; ++c) {
        const double* g = &h->gm_host[(((size_t)n * r + c) * n2 + q) * 2];
        s += h->dm.ebeta[c] * zc(g[0], g[1]);
      }
      rho[q] = -s;
    }
    auto fun = [&](auto f, zc* out) {  // U diag(f(E)) U^dagger
      for (int x = 0; x < no; ++x)
        for (int y = 0; y < no; ++y) {
          zc s = 0;
          for (int a = 0; a < no; ++a) s += U[x * no + a] * f(E[a]) * std::conj(U[y * no + a]);
          out[x * no + y] = s;
        }
    };
    auto mm = [&](const zc* A, const zc* B, zc* C) {
      for (int x = 0; x < no; ++x)
        for (int y = 0; y < no; ++y) {
          zc s = 0;
          for (int a = 0; a < no; ++a) s += A[x * no + a] * B[a * no + y];
          C[x * no + y] = s;
        }
    };
    size_t off = 0;
    for (int t = 0; t <= k; ++t)
      for (int tp = 0; tp <= t; ++tp, ++off) {
        zc A[16], B[16], C[16], D[16];
        fun([&](double ee) { return zc(0, -1) * std::exp(zc(0, -ee * (t - tp) * hh)); }, A);
        // GL(t, tp) = G^<(tp, t) = i e^{-i e tp} rho e^{i e t}
        fun([&](double ee) { return std::exp(zc(0, -ee * tp * hh)); }, B);
        fun([&](double ee) { return std::exp(zc(0, ee * t * hh)); }, C);
        mm(B, rho, D);
        mm(D, C, B);
        for (int q = 0; q < n2; ++q) {
          gr[(off * n2 + q) * 2] = A[q].real(); gr[(off * n2 + q) * 2 + 1] = A[q].imag();
          zc v = zc(0, 1) * B[q];
          gl[(off * n2 + q) * 2] = v.real(); gl[(off * n2 + q) * 2 + 1] = v.imag();
        }
      }
    // G^tv(t, tau) = e^{-i e t} G^tv(0, tau) from the exact G^tv(0, tau_i) =
    // i xi G^M(beta - tau_i) (the mean-field form -xi i rho e^{e tau} when G^M
    // is that of e; far closer when G^M is an interacting equilibrium)
    std::vector<zc> g0((size_t)r * n2);
    for (int i = 0; i < r; ++i)
      for (int q = 0; q < n2; ++q) {
        zc sacc = 0;
        for (int c = 0; c < r; ++c) {
          const double* g = &h->gm_host[(((size_t)n * r + c) * n2 + q) * 2];
          sacc += h->dm.rev[(size_t)i * r + c] * zc(g[0], g[1]);
        }
        g0[(size_t)i * n2 + q] = zc(0, (double)d.xi) * sacc;
      }
    for (int t = 0; t <= k; ++t)
      for (int i = 0; i < r; ++i) {
        zc B[16], D[16];
        fun([&](double ee) { return std::exp(zc(0, -ee * t * hh)); }, B);
        mm(B, &g0[(size_t)i * n2], D);
        for (int q = 0; q < n2; ++q) {
          gtv[(((size_t)t * r + i) * n2 + q) * 2] = D[q].real();
          gtv[(((size_t)t * r + i) * n2 + q) * 2 + 1] = D[q].imag();
        }
      }
    const size_t sq = (size_t)(k + 1) * (k + 2) / 2 * n2;
    // rows 0..k, stored row by row (dense triangle or ring slots alike)
    for (int t = 0; t <= k; ++t) {
      const size_t o = (size_t)t * (t + 1) / 2 * n2 * 2, c = (size_t)(t + 1) * n2;
      HK_CUDA(h, h2d_el(h, elp(h, d.GR, row_off(h, n, t)), gr.data() + o, c));
      HK_CUDA(h, h2d_el(h, elp(h, d.GL, row_off(h, n, t)), gl.data() + o, c));
    }
    HK_CUDA(h, cudaMemcpyAsync(static_cast<double2*>(d.GTV) + (size_t)n * d.nt * r * n2, gtv.data(),
                               (size_t)(k + 1) * r * n2 * sizeof(double2), cudaMemcpyHostToDevice, h->s));
    HK_CUDA(h, cudaStreamSynchronize(h->s));
  }
  return HKBE_OK;
}

static int check_ready(hkbe_t* h) {
  if (!h) return fail(h, HKBE_ERR_ARG, "null handle");
  if (!h->have_dlr || !h->have_gm || !h->have_eps || !h->have_model)
    return fail(h, HKBE_ERR_ARG, "set_dlr, set_matsubara, set_hamiltonian and set_model must precede stepping");
  return HKBE_OK;
}

}  // extern "C"

// Run the iteration loop of one bootstrap or one time step; `pass` launches
// one iteration.  Records per-instance iteration counts and final errors.
// Instances with act0[n] == 0 (past their last step) take no part.
template <typename F>
static int iterate(hkbe_t* h, int max_iter, double tol, F pass, int32_t* iters, double* errs, bool* any_failed,
                   const std::vector<int>* act0 = nullptr) {
  Dev& d = h->d;
  const int N = d.n_inst;
  std::vector<int> act(N, 1), it_of(N, 0);
  if (act0) act = *act0;
  std::vector<double> err(N, 0.0);
  HK_CUDA(h, cudaMemcpyAsync(d.active, act.data(), N * sizeof(int), cudaMemcpyHostToDevice, h->s));
  const double tol_eff = h->self_consistent ? tol : INFINITY;
  const int min_iter = h->self_consistent ? 1 : 2;
  int it = 0;
  for (it = 1; it <= max_iter; ++it) {
    HK_CUDA(h, cudaMemsetAsync(d.err, 0, N * sizeof(double), h->s));
    HK_CUDA(h, cudaMemsetAsync(h->any_dev, 0, sizeof(int), h->s));
    HK_CUDA(h, pass());
    HK_CUDA(h, run_phase(h, HKBE_PHASE_CTRL, 1,
                         [&]() { return hk::launch_set_active(d, tol_eff, it, min_iter, h->any_dev, h->s); }));
    int any = 0;
    HK_CUDA(h, cudaMemcpyAsync(err.data(), d.err, N * sizeof(double), cudaMemcpyDeviceToHost, h->s));
    HK_CUDA(h, cudaMemcpyAsync(&any, h->any_dev, sizeof(int), cudaMemcpyDeviceToHost, h->s));
    HK_CUDA(h, cudaStreamSynchronize(h->s));
    for (int n = 0; n < N; ++n)
      if (act[n]) {
        it_of[n] = it;
        if (errs) errs[n] = err[n];
        if (!std::isfinite(err[n])) return fail(h, HKBE_ERR_NAN, "non-finite value during the self-consistency loop");
      }
    HK_CUDA(h, cudaMemcpyAsync(act.data(), d.active, N * sizeof(int), cudaMemcpyDeviceToHost, h->s));
    HK_CUDA(h, cudaStreamSynchronize(h->s));
    drain(h);
    if (!any) break;
    if (d.model == HKBE_MODEL_LATTICE2B) {  // k-points are coupled through Sigma: iterate all or none
      if (act0) act = *act0;
      else std::fill(act.begin(), act.end(), 1);
      HK_CUDA(h, cudaMemcpyAsync(d.active, act.data(), N * sizeof(int), cudaMemcpyHostToDevice, h->s));
    }
  }
  *any_failed = false;
  for (int n = 0; n < N; ++n) {
    if (iters) iters[n] = it_of[n];
    if (act[n] && h->self_consistent) *any_failed = true;
  }
  return HKBE_OK;
}

extern "C" {

// Common end of hkbe_bootstrap and hkbe_set_initial_slices once rows 0..k of
// G^R, G^< and G^tv are in place: Sigma of the start square (all instances),
// the snapshot hkbe_rewind returns to, the diagonal-scheme seed, step k.
static int finish_start(hkbe_t* h) {
  Dev& d = h->d;
  std::vector<int> ones(d.n_inst, 1);
  HK_CUDA(h, cudaMemcpyAsync(d.active, ones.data(), d.n_inst * sizeof(int), cudaMemcpyHostToDevice, h->s));
  for (int t = 0; t <= d.k; ++t) HK_CUDA(h, hk::launch_sigma(d, t, h->s));
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  drain(h);
  // snapshot of the start square for hkbe_rewind (rows 0..k of the two-time
  // components, in either layout, and rows 0..k of the mixed components)
  {
    const int n2 = no2(h), k = d.k;
    const size_t sq = (size_t)(k + 1) * (k + 2) / 2 * n2, tvn = (size_t)(k + 1) * d.r * n2;
    const size_t es = esz(h);
    auto grab = [&](std::vector<char>& dst, void* src) -> cudaError_t {
      dst.resize(sq * d.n_inst * es);
      for (int n = 0; n < d.n_inst; ++n)
        for (int t = 0; t <= k; ++t) {
          cudaError_t e = cudaMemcpyAsync(dst.data() + (sq * n + (size_t)t * (t + 1) / 2 * n2) * es, elp(h, src, row_off(h, n, t)),
                                          (size_t)(t + 1) * n2 * es, cudaMemcpyDeviceToHost, h->s);
          if (e != cudaSuccess) return e;
        }
      return cudaStreamSynchronize(h->s);
    };
    auto grab_tv = [&](std::vector<char>& dst, void* src) -> cudaError_t {
      const size_t et = sizeof(double2);
      dst.resize(tvn * d.n_inst * et);
      for (int n = 0; n < d.n_inst; ++n) {
        cudaError_t e = cudaMemcpyAsync(dst.data() + tvn * n * et, static_cast<char*>(src) + (size_t)n * d.nt * d.r * n2 * et,
                                        tvn * et, cudaMemcpyDeviceToHost, h->s);
        if (e != cudaSuccess) return e;
      }
      return cudaStreamSynchronize(h->s);
    };
    HK_CUDA(h, grab(h->snap_gr, d.GR));
    HK_CUDA(h, grab(h->snap_gl, d.GL));
    HK_CUDA(h, grab(h->snap_sr, d.SR));
    HK_CUDA(h, grab(h->snap_sl, d.SL));
    HK_CUDA(h, grab_tv(h->snap_tv, d.GTV));
    HK_CUDA(h, grab_tv(h->snap_stv, d.STV));
  }
  HK_CUDA(h, hk::launch_diag_seed(d, h->s));   // also seeds the FP64 row copies of the start square
  d.use64 = d.ring64[0] ? 1 : 0;
  h->cur = d.k;
  return HKBE_OK;
}

int hkbe_bootstrap(hkbe_t* h, int max_iter, double tol, int32_t* iters, double* err) {
  int rc = check_ready(h);
  if (rc) return rc;
  if (h->cur >= 0) return fail(h, HKBE_ERR_ARG, "bootstrap already done");
  if (max_iter < 1) return fail(h, HKBE_ERR_ARG, "max_iter must be >= 1");
  if ((rc = hf_guess(h))) return rc;
  Dev& d = h->d;
  bool failed = false;
  rc = iterate(h, max_iter, tol,
               [&]() { return run_phase(h, HKBE_PHASE_BOOT, d.k + 4, [&]() { return hk::launch_boot(d, h->s); }); },
               iters, err, &failed);
  if (rc) return rc;
  if ((rc = finish_start(h))) return rc;
  if (failed) return fail(h, HKBE_ERR_NOCONV, "bootstrap did not converge");
  return HKBE_OK;
}

int hkbe_set_initial_slices(hkbe_t* h, const double* gr, const double* gl, const double* gtv) {
  int rc = check_ready(h);
  if (rc) return rc;
  if (!gr || !gl || !gtv) return fail(h, HKBE_ERR_ARG, "null argument");
  if (h->cur >= 0) return fail(h, HKBE_ERR_ARG, "the start square is already set");
  Dev& d = h->d;
  const int n2 = no2(h), k = d.k, r = d.r;
  const size_t sq = (size_t)(k + 1) * (k + 2) / 2 * n2, tvn = (size_t)(k + 1) * r * n2;
  for (size_t i = 0; i < 2 * sq * d.n_inst; ++i)
    if (!std::isfinite(gr[i]) || !std::isfinite(gl[i])) return fail(h, HKBE_ERR_NAN, "non-finite value in gr or gl");
  for (size_t i = 0; i < 2 * tvn * d.n_inst; ++i)
    if (!std::isfinite(gtv[i])) return fail(h, HKBE_ERR_NAN, "non-finite value in gtv");
  for (int n = 0; n < d.n_inst; ++n) {
    for (int t = 0; t <= k; ++t) {
      const size_t o = (sq * n + (size_t)t * (t + 1) / 2 * n2) * 2, c = (size_t)(t + 1) * n2;
      HK_CUDA(h, h2d_el(h, elp(h, d.GR, row_off(h, n, t)), gr + o, c));
      HK_CUDA(h, h2d_el(h, elp(h, d.GL, row_off(h, n, t)), gl + o, c));
    }
    HK_CUDA(h, cudaMemcpyAsync(static_cast<double2*>(d.GTV) + (size_t)n * d.nt * r * n2, gtv + tvn * n * 2,
                               tvn * sizeof(double2), cudaMemcpyHostToDevice, h->s));
  }
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  return finish_start(h);
}

int hkbe_step(hkbe_t* h, int n_steps, int32_t* iters, double* err) {
  int rc = check_ready(h);
  if (rc) return rc;
  if (h->cur < 0) return fail(h, HKBE_ERR_ARG, "hkbe_bootstrap must precede hkbe_step");
  if (n_steps < 0) return fail(h, HKBE_ERR_ARG, "n_steps must be >= 0");
  Dev& d = h->d;
  if (h->cur + n_steps > d.nt - 1) return fail(h, HKBE_ERR_RANGE, "stepping past nt - 1");
  const int N = d.n_inst;
  bool any_failed = false;
  for (int st = 0; st < n_steps; ++st) {
    const int T = h->cur + 1;
    // inverses of the chunks that became frozen (their rows are final and far enough from T)
    if (h->scheme == HKBE_SCHEME_PAPER) {
      const int tR = std::max(0, (T - 2 * d.k) / 32), tL = std::max(0, T / 32);
      if (tR > d.nfrozR) {
        HK_CUDA(h, run_phase(h, HKBE_PHASE_CHUNKINV, tR - d.nfrozR,
                             [&]() { return hk::launch_chunk_inv(d, 0, d.nfrozR, tR, h->s); }));
        d.nfrozR = tR;
      }
      if (tL > d.nfrozL) {
        HK_CUDA(h, run_phase(h, HKBE_PHASE_CHUNKINV, tL - d.nfrozL,
                             [&]() { return hk::launch_chunk_inv(d, 1, d.nfrozL, tL, h->s); }));
        d.nfrozL = tL;
      }
    }
    HK_CUDA(h, run_phase(h, HKBE_PHASE_EXTRAP, 1, [&]() { return hk::launch_extrapolate(d, T, h->s); }));
    std::vector<int> act0(N);
    for (int n = 0; n < N; ++n) act0[n] = T <= h->last[n] ? 1 : 0;
    bool failed = false;
    rc = iterate(h, h->p.max_iter, h->p.tol,
                 [&]() -> cudaError_t {
                   cudaError_t e;
                   if ((e = run_phase(h, HKBE_PHASE_SIGMA, 1, [&]() { return hk::launch_sigma(d, T, h->s); })))
                     return e;
                   if ((e = run_phase(h, HKBE_PHASE_RET, 1, [&]() {
                          return h->scheme ? hk::launch_ret_sf(d, T, h->s) : hk::launch_ret_h(d, T, h->s);
                        })))
                     return e;
                   if ((e = run_phase(h, HKBE_PHASE_MIXED, 1, [&]() { return hk::launch_mixed(d, T, h->s); })))
                     return e;
                   if ((e = run_phase(h, HKBE_PHASE_VT, 1, [&]() { return hk::launch_vt(d, T, h->s); }))) return e;
                   if ((e = run_phase(h, HKBE_PHASE_SRC, (h->hodlr && d.cdir > 0) ? 3 : 1, [&]() {
                          return h->hodlr ? hk::launch_src_h(d, T, h->s) : hk::launch_src(d, T, h->s);
                        })))
                     return e;
                   if ((e = run_phase(h, HKBE_PHASE_LES, 1, [&]() {
                          return h->scheme ? hk::launch_les_sf(d, T, h->s) : hk::launch_les_h(d, T, h->s);
                        })))
                     return e;
                   if (d.rho_mode == 1 &&
                       (e = run_phase(h, HKBE_PHASE_RHO, 1, [&]() { return hk::launch_rho(d, T, h->s); })))
                     return e;
                   return cudaSuccess;
                 },
                 iters ? iters + (size_t)st * N : nullptr, err ? err + (size_t)st * N : nullptr, &failed, &act0);
    if (rc) return rc;
    any_failed |= failed;
    h->cur = T;
    // update_blocks (Sec. 3.1): compress every whole leaf of rows older than k+1 steps
    while (h->hodlr && d.cdir + d.L <= T - d.k) {
      const int A = d.cdir;
      HK_CUDA(h, run_phase(h, HKBE_PHASE_COMPRESS, 2, [&]() { return hk::launch_compress(d, A, d.L, h->s); }));
      d.cdir += d.L;
    }
  }
  {
    // status of these steps: [0] ranks capped at r_max, [1] block cores whose
    // Jacobi SVD did not converge in 40 sweeps (their factors are the last
    // sweep's, still a factorisation of the block), [2] timed-out waits for a
    // staged chunk inverse (that chunk was read from global memory instead)
    int st[3] = {0, 0, 0};
    HK_CUDA(h, cudaMemcpyAsync(st, h->status_dev, sizeof(st), cudaMemcpyDeviceToHost, h->s));
    HK_CUDA(h, cudaMemsetAsync(h->status_dev, 0, sizeof(st), h->s));
    HK_CUDA(h, cudaStreamSynchronize(h->s));
    drain(h);
    if (st[2] > 0) return fail(h, HKBE_ERR_CUDA, "a bulk copy of a chunk inverse into shared memory timed out");
    if (st[0] > 0) return fail(h, HKBE_ERR_RANK, "a block's epsilon-rank exceeded r_max (truncated to r_max)");
    if (st[1] > 0)
      return fail(h, HKBE_ERR_NOCONV, "the Jacobi SVD of " + std::to_string(st[1]) +
                                           " TSVD block core(s) did not converge in 40 sweeps");
  }
  if (any_failed) return fail(h, HKBE_ERR_NOCONV, "self-consistency did not converge within max_iter");
  return HKBE_OK;
}

int hkbe_current_step(const hkbe_t* h, int32_t* T) {
  if (!h || !T) return HKBE_ERR_ARG;
  *T = h->cur;
  return HKBE_OK;
}

// Copy rows T of G^R and G^< (t = 0..T) of an instance to host buffers
// (either may be NULL); compressed rows are reconstructed on the device.
static int fetch_row(hkbe_t* h, int inst, int T, double* gr, double* gl) {
  const size_t cnt = (size_t)(T + 1) * no2(h);
  hk::Dev& d = h->d;
  if (h->hodlr && T < front_host(h, inst)) {
    HK_CUDA(h, hk::launch_row_out(d, inst, T, gr ? h->rowbuf_r : nullptr, gl ? h->rowbuf_l : nullptr, h->s));
    if (gr) HK_CUDA(h, cudaMemcpyAsync(gr, h->rowbuf_r, cnt * sizeof(double2), cudaMemcpyDeviceToHost, h->s));
    if (gl) HK_CUDA(h, cudaMemcpyAsync(gl, h->rowbuf_l, cnt * sizeof(double2), cudaMemcpyDeviceToHost, h->s));
  } else {
    if (gr) HK_CUDA(h, d2h_el(h, gr, elp(h, d.GR, row_off(h, inst, T)), cnt));
    if (gl) HK_CUDA(h, d2h_el(h, gl, elp(h, d.GL, row_off(h, inst, T)), cnt));
  }
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  return HKBE_OK;
}

static int copy_el(hkbe_t* h, int X, int inst, int T, int t, double* out) {
  const int n2 = no2(h);
  std::vector<double> row((size_t)(T + 1) * n2 * 2);
  int rc = fetch_row(h, inst, T, X == 0 ? row.data() : nullptr, X == 1 ? row.data() : nullptr);
  if (rc) return rc;
  std::memcpy(out, row.data() + (size_t)t * n2 * 2, n2 * 2 * sizeof(double));
  return HKBE_OK;
}

int hkbe_get_ret(hkbe_t* h, int inst, int t, int tp, double* out) {
  if (!h || !out) return fail(h, HKBE_ERR_ARG, "null argument");
  if (inst < 0 || inst >= h->d.n_inst) return fail(h, HKBE_ERR_ARG, "instance out of range");
  if (tp < 0 || tp > t || t > cur_of(h, inst))
    return fail(h, HKBE_ERR_RANGE, "need 0 <= t' <= t <= current step (and the instance's last step)");
  return copy_el(h, 0, inst, t, tp, out);
}

int hkbe_get_les(hkbe_t* h, int inst, int t, int tp, double* out) {
  if (!h || !out) return fail(h, HKBE_ERR_ARG, "null argument");
  if (inst < 0 || inst >= h->d.n_inst) return fail(h, HKBE_ERR_ARG, "instance out of range");
  if (t < 0 || tp < 0 || t > cur_of(h, inst) || tp > cur_of(h, inst))
    return fail(h, HKBE_ERR_RANGE, "times must be in 0..current step (and the instance's last step)");
  if (t <= tp) return copy_el(h, 1, inst, tp, t, out);
  const int no = h->d.no;
  std::vector<double> tmp(2 * no * no);
  int rc = copy_el(h, 1, inst, t, tp, tmp.data());
  if (rc) return rc;
  for (int x = 0; x < no; ++x)
    for (int y = 0; y < no; ++y) {
      out[2 * (x * no + y)] = -tmp[2 * (y * no + x)];
      out[2 * (x * no + y) + 1] = tmp[2 * (y * no + x) + 1];
    }
  return HKBE_OK;
}

int hkbe_get_tv(hkbe_t* h, int inst, int t, double* out) {
  if (!h || !out) return fail(h, HKBE_ERR_ARG, "null argument");
  if (!h->have_dlr) return fail(h, HKBE_ERR_ARG, "no DLR grid");
  if (inst < 0 || inst >= h->d.n_inst) return fail(h, HKBE_ERR_ARG, "instance out of range");
  if (t < 0 || t > cur_of(h, inst))
    return fail(h, HKBE_ERR_RANGE, "t must be in 0..current step (and the instance's last step)");
  const size_t cnt = (size_t)h->d.r * no2(h);
  HK_CUDA(h, cudaMemcpyAsync(out, static_cast<double2*>(h->d.GTV) + ((size_t)inst * h->d.nt + t) * cnt,
                             cnt * sizeof(double2), cudaMemcpyDeviceToHost, h->s));
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  return HKBE_OK;
}

int hkbe_get_row(hkbe_t* h, int inst, int T, double* gr, double* gl) {
  if (!h) return fail(h, HKBE_ERR_ARG, "null handle");
  if (inst < 0 || inst >= h->d.n_inst) return fail(h, HKBE_ERR_ARG, "instance out of range");
  if (T < 0 || T > cur_of(h, inst))
    return fail(h, HKBE_ERR_RANGE, "T must be in 0..current step (and the instance's last step)");
  return fetch_row(h, inst, T, gr, gl);
}

int hkbe_get_blocks(const hkbe_t* h, int32_t* nblk, int32_t* r0, int32_t* r1, int32_t* c0, int32_t* c1,
                    int32_t* level) {
  if (!h || !nblk || !h->hodlr) return HKBE_ERR_ARG;
  *nblk = (int32_t)h->g_r0.size();
  for (size_t b = 0; b < h->g_r0.size(); ++b) {
    if (r0) r0[b] = h->g_r0[b];
    if (r1) r1[b] = h->g_r1[b];
    if (c0) c0[b] = h->g_c0[b];
    if (c1) c1[b] = h->g_c1[b];
    if (level) level[b] = h->g_lvl[b];
  }
  return HKBE_OK;
}

int hkbe_get_ranks(hkbe_t* h, int inst, int comp, int32_t* ranks, int32_t* first_direct) {
  if (!h || !h->hodlr) return fail(h, HKBE_ERR_ARG, "not a HODLR handle");
  if (inst < 0 || inst >= h->d.n_inst || comp < 0 || comp > 3) return fail(h, HKBE_ERR_ARG, "bad instance or component");
  const size_t cnt = (size_t)h->d.nblk * no2(h);
  if (ranks)
    HK_CUDA(h, cudaMemcpyAsync(ranks, h->d.hod[comp].rank + (size_t)inst * cnt, cnt * sizeof(int), cudaMemcpyDeviceToHost, h->s));
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  if (first_direct) *first_direct = front_host(h, inst);
  return HKBE_OK;
}

int hkbe_get_density(hkbe_t* h, double* rho) {
  if (!h || !rho) return fail(h, HKBE_ERR_ARG, "null argument");
  if (h->cur < 0) return fail(h, HKBE_ERR_RANGE, "nothing computed yet");
  const int n2 = no2(h), T = h->cur;
  std::vector<double> tmp(2 * n2);
  for (int n = 0; n < h->d.n_inst; ++n)
    for (int t = 0; t <= T; ++t) {
      if (t > h->last[n]) {   // past the instance's last step: zeros
        std::memset(rho + (((size_t)n * (T + 1) + t) * n2) * 2, 0, sizeof(double) * 2 * n2);
        continue;
      }
      int rc = copy_el(h, 1, n, t, t, tmp.data());
      if (rc) return rc;
      double* o = rho + (((size_t)n * (T + 1) + t) * n2) * 2;
      for (int q = 0; q < n2; ++q) {  // rho = xi i G^<
        const double re = tmp[2 * q], im = tmp[2 * q + 1];
        o[2 * q] = -h->p.xi * im;
        o[2 * q + 1] = h->p.xi * re;
      }
    }
  return HKBE_OK;
}

int hkbe_get_density_at(hkbe_t* h, int t, double* rho_t) {
  if (!h || !rho_t) return fail(h, HKBE_ERR_ARG, "null argument");
  if (t < 0 || t > h->cur) return fail(h, HKBE_ERR_RANGE, "t must be in 0..current step");
  const hk::Dev& d = h->d;
  const size_t cnt = (size_t)d.n_inst * no2(h);
  HK_CUDA(h, hk::launch_density_at(d, t, h->diagbuf, h->s));
  HK_CUDA(h, cudaMemcpyAsync(rho_t, h->diagbuf, cnt * sizeof(double2), cudaMemcpyDeviceToHost, h->s));
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  return HKBE_OK;
}

int hkbe_get_lattice_observables(hkbe_t* h, int t, double* out) {
  if (!h || !out) return fail(h, HKBE_ERR_ARG, "null argument");
  if (h->d.model != HKBE_MODEL_LATTICE2B) return fail(h, HKBE_ERR_ARG, "not a LATTICE2B handle");
  if (t < 0 || t > h->cur) return fail(h, HKBE_ERR_RANGE, "t must be in 0..current step");
  double* dev = reinterpret_cast<double*>(h->diagbuf);   // >= 3 doubles (n_inst >= 1 complex)
  HK_CUDA(h, hk::launch_lattice_obs(h->d, t, dev, h->s));
  HK_CUDA(h, cudaMemcpyAsync(out, dev, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->s));
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  return HKBE_OK;
}

int hkbe_get_observables(hkbe_t* h, int t, double* rho, double* ekin, double* current) {
  if (!h) return fail(h, HKBE_ERR_ARG, "null handle");
  if ((ekin || current) && h->d.model != HKBE_MODEL_LATTICE2B)
    return fail(h, HKBE_ERR_ARG, "ekin and current are defined for LATTICE2B only");
  if (t < 0 || t > h->cur) return fail(h, HKBE_ERR_RANGE, "t must be in 0..current step");
  int rc;
  if (ekin || current) {
    double o[3];
    if ((rc = hkbe_get_lattice_observables(h, t, o))) return rc;
    if (ekin) *ekin = o[1];
    if (current) *current = o[2];
  }
  if (rho && (rc = hkbe_get_density_at(h, t, rho))) return rc;
  return HKBE_OK;
}

int hkbe_get_stats(hkbe_t* h, int inst, int32_t* ranks, size_t* device_bytes) {
  if (!h) return fail(h, HKBE_ERR_ARG, "null handle");
  if (device_bytes) *device_bytes = h->bytes;
  if (!ranks) return HKBE_OK;
  if (!h->hodlr) return fail(h, HKBE_ERR_ARG, "ranks requested from a dense handle");
  if (inst < 0 || inst >= h->d.n_inst) return fail(h, HKBE_ERR_ARG, "instance out of range");
  const size_t cnt = (size_t)h->d.nblk * no2(h);
  for (int X = 0; X < 4; ++X)
    HK_CUDA(h, cudaMemcpyAsync(ranks + X * cnt, h->d.hod[X].rank + (size_t)inst * cnt, cnt * sizeof(int),
                               cudaMemcpyDeviceToHost, h->s));
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  return HKBE_OK;
}

int hkbe_snapshot_free(hkbe_t* h) {
  if (!h) return fail(h, HKBE_ERR_ARG, "null handle");
  for (void* p : h->snap_dev)
    if (p) cudaFree(p);
  h->snap_dev.clear();
  h->snap_bytes = 0;
  h->snap_cur = -1;
  return HKBE_OK;
}

int hkbe_snapshot_save(hkbe_t* h) {
  if (!h) return fail(h, HKBE_ERR_ARG, "null handle");
  if (h->cur < 0) return fail(h, HKBE_ERR_ARG, "hkbe_bootstrap must precede hkbe_snapshot_save");
  if (h->snap_dev.size() != h->allocs.size()) {
    hkbe_snapshot_free(h);
    for (size_t i = 0; i < h->allocs.size(); ++i) {
      void* p = nullptr;
      if (std::find(h->scratch.begin(), h->scratch.end(), h->allocs[i]) != h->scratch.end()) {
        h->snap_dev.push_back(nullptr);   // scratch: nothing to keep
        continue;
      }
      cudaError_t e = cudaMalloc(&p, h->alloc_bytes[i]);
      if (e != cudaSuccess) {
        hkbe_snapshot_free(h);
        return fail(h, HKBE_ERR_NOMEM, std::string("snapshot cudaMalloc: ") + cudaGetErrorString(e));
      }
      h->snap_dev.push_back(p);
      h->snap_bytes += h->alloc_bytes[i];
    }
  }
  for (size_t i = 0; i < h->allocs.size(); ++i)
    if (h->snap_dev[i])
      HK_CUDA(h, cudaMemcpyAsync(h->snap_dev[i], h->allocs[i], h->alloc_bytes[i], cudaMemcpyDeviceToDevice, h->s));
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  h->snap_cur = h->cur;
  h->snap_cdir = h->d.cdir;
  h->snap_nfrozR = h->d.nfrozR;
  h->snap_nfrozL = h->d.nfrozL;
  return HKBE_OK;
}

int hkbe_snapshot_restore(hkbe_t* h) {
  if (!h) return fail(h, HKBE_ERR_ARG, "null handle");
  if (h->snap_cur < 0 || h->snap_dev.size() != h->allocs.size())
    return fail(h, HKBE_ERR_ARG, "no snapshot to restore (hkbe_snapshot_save first)");
  for (size_t i = 0; i < h->allocs.size(); ++i)
    if (h->snap_dev[i])
      HK_CUDA(h, cudaMemcpyAsync(h->allocs[i], h->snap_dev[i], h->alloc_bytes[i], cudaMemcpyDeviceToDevice, h->s));
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  h->cur = h->snap_cur;
  h->d.cdir = h->snap_cdir;
  h->d.nfrozR = h->snap_nfrozR;
  h->d.nfrozL = h->snap_nfrozL;
  return HKBE_OK;
}

int hkbe_rewind(hkbe_t* h) {
  if (!h) return fail(h, HKBE_ERR_ARG, "null handle");
  if (h->cur < 0 || h->snap_gr.empty()) return fail(h, HKBE_ERR_ARG, "hkbe_bootstrap must precede hkbe_rewind");
  Dev& d = h->d;
  const int n2 = no2(h), k = d.k;
  const size_t sq = (size_t)(k + 1) * (k + 2) / 2 * n2, tvn = (size_t)(k + 1) * d.r * n2;
  const size_t es = esz(h);
  auto put = [&](const std::vector<char>& src, void* dst) -> cudaError_t {
    for (int n = 0; n < d.n_inst; ++n)
      for (int t = 0; t <= k; ++t) {
        cudaError_t e = cudaMemcpyAsync(elp(h, dst, row_off(h, n, t)), src.data() + (sq * n + (size_t)t * (t + 1) / 2 * n2) * es,
                                        (size_t)(t + 1) * n2 * es, cudaMemcpyHostToDevice, h->s);
        if (e != cudaSuccess) return e;
      }
    return cudaSuccess;
  };
  auto put_tv = [&](const std::vector<char>& src, void* dst) -> cudaError_t {
    const size_t et = sizeof(double2);
    for (int n = 0; n < d.n_inst; ++n) {
      cudaError_t e = cudaMemcpyAsync(static_cast<char*>(dst) + (size_t)n * d.nt * d.r * n2 * et, src.data() + tvn * n * et,
                                      tvn * et, cudaMemcpyHostToDevice, h->s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  for (auto& a : h->state_arrays) HK_CUDA(h, cudaMemsetAsync(a.first, 0, a.second, h->s));
  HK_CUDA(h, cudaMemcpyAsync(d.eps, d.eps_ext, (size_t)d.n_inst * (d.nt + 1) * n2 * sizeof(double2),
                             cudaMemcpyDeviceToDevice, h->s));
  HK_CUDA(h, put(h->snap_gr, d.GR));
  HK_CUDA(h, put(h->snap_gl, d.GL));
  HK_CUDA(h, put(h->snap_sr, d.SR));
  HK_CUDA(h, put(h->snap_sl, d.SL));
  HK_CUDA(h, put_tv(h->snap_tv, d.GTV));
  HK_CUDA(h, put_tv(h->snap_stv, d.STV));
  HK_CUDA(h, hk::launch_diag_seed(d, h->s));
  d.nfrozR = d.nfrozL = 0;
  if (h->hodlr) {
    d.cdir = 0;
    for (int X = 0; X < 4; ++X)
      HK_CUDA(h, cudaMemsetAsync(d.hod[X].rank, 0, (size_t)d.n_inst * d.nblk * n2 * sizeof(int), h->s));
  }
  HK_CUDA(h, cudaMemsetAsync(h->status_dev, 0, 3 * sizeof(int), h->s));
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  h->cur = k;
  return HKBE_OK;
}

}  // extern "C"

// ---- checkpoint files ----
namespace {
constexpr char kCkpMagic[8] = {'H', 'K', 'B', 'E', 'C', 'K', 'P', '1'};
constexpr uint32_t kCkpVersion = 2;   // 2: checksum trailer and per-instance N_t
constexpr size_t kCkpChunk = size_t(64) << 20;  // host staging of device buffers

struct CkpScalars {
  int32_t cur, have_dlr, have_gm, have_eps, have_model, self_consistent;
  int32_t model, r, cdir, nfrozR, nfrozL, pad;
};

// Checksum of a checkpoint file: FNV-1a over the file's bytes taken as
// little-endian 64-bit words (the last word zero-padded), written as an
// 8-byte trailer after everything it covers.
constexpr uint64_t kFnvOffset = 14695981039346656037ull, kFnvPrime = 1099511628211ull;

uint64_t fnv_words(uint64_t h, const unsigned char* p, size_t n) {
  size_t i = 0;
  for (; i + 8 <= n; i += 8) {
    uint64_t w;
    std::memcpy(&w, p + i, 8);
    h = (h ^ w) * kFnvPrime;
  }
  if (i < n) {
    uint64_t w = 0;
    std::memcpy(&w, p + i, n - i);
    h = (h ^ w) * kFnvPrime;
  }
  return h;
}

// Checksum of the first `len` bytes of f, read from the start in chunks of a
// multiple of 8 bytes (so only the final word can be partial).
bool file_checksum(FILE* f, uint64_t len, uint64_t* out) {
  if (std::fseek(f, 0, SEEK_SET) != 0) return false;
  std::vector<unsigned char> buf((size_t)std::min<uint64_t>(len, kCkpChunk));
  uint64_t h = kFnvOffset;
  for (uint64_t done = 0; done < len;) {
    const size_t c = (size_t)std::min<uint64_t>(kCkpChunk, len - done);
    if (std::fread(buf.data(), 1, c, f) != c) return false;
    h = fnv_words(h, buf.data(), c);
    done += c;
  }
  *out = h;
  return true;
}

bool wr(FILE* f, const void* p, size_t n) { return n == 0 || std::fwrite(p, 1, n, f) == n; }
bool rd(FILE* f, void* p, size_t n) { return n == 0 || std::fread(p, 1, n, f) == n; }
template <typename T>
bool wr_vec(FILE* f, const std::vector<T>& v) {
  const uint64_t n = v.size();
  return wr(f, &n, sizeof n) && wr(f, v.data(), n * sizeof(T));
}
// a vector whose length must be 0 (not set) or `expect`
template <typename T>
bool rd_vec(FILE* f, std::vector<T>& v, uint64_t expect) {
  uint64_t n = 0;
  if (!rd(f, &n, sizeof n) || (n != 0 && n != expect)) return false;
  v.resize(n);
  return rd(f, v.data(), n * sizeof(T));
}
}  // namespace

extern "C" {

int hkbe_save(hkbe_t* h, const char* path) {
  if (!h || !path) return fail(h, HKBE_ERR_ARG, "null argument");
  if (h->scheme != HKBE_SCHEME_PAPER) return fail(h, HKBE_ERR_ARG, "checkpoints hold runs of the paper's scheme only");
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  drain(h);
  FILE* f = std::fopen(path, "w+b");   // read back for the checksum trailer
  if (!f) return fail(h, HKBE_ERR_IO, std::string("cannot open ") + path + " for writing");
  const Dev& d = h->d;
  const CkpScalars sc{h->cur, h->have_dlr, h->have_gm, h->have_eps, h->have_model, h->self_consistent,
                      d.model, d.r, d.cdir, d.nfrozR, d.nfrozL, 0};
  const uint32_t ver = kCkpVersion, psz = sizeof(hkbe_params);
  bool ok = wr(f, kCkpMagic, sizeof kCkpMagic) && wr(f, &ver, sizeof ver) && wr(f, &psz, sizeof psz) &&
            wr(f, &h->p, sizeof(hkbe_params)) && wr(f, &sc, sizeof sc) && wr_vec(f, h->last) &&
            wr_vec(f, h->tau) && wr_vec(f, h->om) &&
            wr_vec(f, h->gm_host) && wr_vec(f, h->eps_host) && wr_vec(f, h->snap_gr) && wr_vec(f, h->snap_gl) &&
            wr_vec(f, h->snap_sr) && wr_vec(f, h->snap_sl) && wr_vec(f, h->snap_tv) && wr_vec(f, h->snap_stv);
  const uint64_t na = h->allocs.size();
  ok = ok && wr(f, &na, sizeof na);
  std::vector<char> buf;
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; ok && i < na; ++i) {
    const uint64_t nb = h->alloc_bytes[i];
    ok = wr(f, &nb, sizeof nb);
    for (size_t o = 0; ok && o < nb; o += kCkpChunk) {
      const size_t c = std::min<size_t>(kCkpChunk, nb - o);
      if (buf.size() < c) buf.resize(c);
      e = cudaMemcpyAsync(buf.data(), static_cast<char*>(h->allocs[i]) + o, c, cudaMemcpyDeviceToHost, h->s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
      if (e != cudaSuccess) break;
      ok = wr(f, buf.data(), c);
    }
    if (e != cudaSuccess) break;
  }
  if (ok && e == cudaSuccess) {
    uint64_t sum = 0;
    const long len = (std::fflush(f) == 0) ? std::ftell(f) : -1;
    ok = len >= 0 && file_checksum(f, (uint64_t)len, &sum) && std::fseek(f, 0, SEEK_END) == 0 &&
         wr(f, &sum, sizeof sum);
  }
  const bool closed = std::fclose(f) == 0;
  if (e != cudaSuccess) return fail(h, HKBE_ERR_CUDA, std::string("checkpoint copy: ") + cudaGetErrorString(e));
  if (!ok || !closed) return fail(h, HKBE_ERR_IO, std::string("short write to ") + path);
  return HKBE_OK;
}

int hkbe_load(const char* path, void* stream, hkbe_t** out) {
  if (!path || !out) return fail(nullptr, HKBE_ERR_ARG, "null argument");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(nullptr, HKBE_ERR_IO, std::string("cannot open ") + path);
  hkbe_t* h = nullptr;
  auto bad = [&](int code, std::string msg) {
    std::fclose(f);
    if (h) hkbe_destroy(h);
    g_create_error = std::move(msg);
    return code;
  };
  char mg[8];
  uint32_t ver = 0, psz = 0;
  hkbe_params p{};
  CkpScalars sc{};
  if (!rd(f, mg, sizeof mg) || std::memcmp(mg, kCkpMagic, sizeof mg) != 0)
    return bad(HKBE_ERR_IO, "not a checkpoint file (bad magic)");
  if (!rd(f, &ver, sizeof ver) || ver != kCkpVersion || !rd(f, &psz, sizeof psz) || psz != sizeof(hkbe_params))
    return bad(HKBE_ERR_IO, "unsupported checkpoint version");
  {  // the whole file against its trailer, before any device work
    uint64_t sum = 0, trailer = 0;
    if (std::fseek(f, 0, SEEK_END) != 0) return bad(HKBE_ERR_IO, "cannot seek in the checkpoint file");
    const long len = std::ftell(f);
    if (len < (long)(sizeof mg + sizeof ver + sizeof psz + sizeof trailer)) return bad(HKBE_ERR_IO, "short checkpoint file");
    if (!file_checksum(f, (uint64_t)len - sizeof trailer, &sum) || !rd(f, &trailer, sizeof trailer))
      return bad(HKBE_ERR_IO, "short read (checksum)");
    if (sum != trailer) return bad(HKBE_ERR_IO, "checksum mismatch: the checkpoint file is damaged");
    if (std::fseek(f, (long)(sizeof mg + sizeof ver + sizeof psz), SEEK_SET) != 0)
      return bad(HKBE_ERR_IO, "cannot seek in the checkpoint file");
  }
  if (!rd(f, &p, sizeof p) || !rd(f, &sc, sizeof sc)) return bad(HKBE_ERR_IO, "short read (header)");
  if (sc.r < 0 || sc.r > 128 || (sc.have_dlr != 0) != (sc.r > 0) || sc.cur < -1 || sc.cur >= p.nt || sc.model < 0 ||
      sc.model > HKBE_MODEL_LATTICE2B || sc.cdir < 0 || sc.cdir > std::max(sc.cur, 0) || sc.nfrozR < 0 ||
      sc.nfrozL < 0 || sc.nfrozR > (p.nt + 31) / 32 || sc.nfrozL > (p.nt + 31) / 32)
    return bad(HKBE_ERR_IO, "inconsistent checkpoint header");
  std::vector<int> last;
  if (p.n_inst < 1 || p.nt < 2 || !rd_vec(f, last, (uint64_t)p.n_inst) || last.size() != (size_t)p.n_inst)
    return bad(HKBE_ERR_IO, "short read (per-instance N_t)");
  std::vector<int32_t> ntn(p.n_inst);
  for (int n = 0; n < p.n_inst; ++n) ntn[n] = last[n] + 1;
  int rc = hkbe_create(&p, ntn.data(), stream, &h);
  if (rc) return bad(rc, g_create_error);
  Dev& d = h->d;
  std::vector<double> tau, om;
  if (!rd_vec(f, tau, sc.r) || !rd_vec(f, om, sc.r) || tau.size() != (size_t)sc.r || om.size() != (size_t)sc.r)
    return bad(HKBE_ERR_IO, "short read (DLR grid)");
  if (sc.have_dlr && (rc = hkbe_set_dlr(h, sc.r, tau.data(), om.data()))) return bad(rc, h->err);
  const size_t n2 = (size_t)no2(h), k = d.k, es = esz(h);
  const uint64_t gm_n = (uint64_t)d.n_inst * sc.r * n2 * 2, eps_n = (uint64_t)d.n_inst * (d.nt + 1) * n2 * 2;
  const uint64_t sq_b = (uint64_t)(k + 1) * (k + 2) / 2 * n2 * d.n_inst * es;
  const uint64_t tv_b = (uint64_t)(k + 1) * sc.r * n2 * d.n_inst * sizeof(double2);
  if (!rd_vec(f, h->gm_host, gm_n) || !rd_vec(f, h->eps_host, eps_n) || !rd_vec(f, h->snap_gr, sq_b) ||
      !rd_vec(f, h->snap_gl, sq_b) || !rd_vec(f, h->snap_sr, sq_b) || !rd_vec(f, h->snap_sl, sq_b) ||
      !rd_vec(f, h->snap_tv, tv_b) || !rd_vec(f, h->snap_stv, tv_b))
    return bad(HKBE_ERR_IO, "short read or wrong size (host set-up)");
  if ((sc.have_gm != 0) != !h->gm_host.empty() || (sc.have_eps != 0) != !h->eps_host.empty())
    return bad(HKBE_ERR_IO, "inconsistent checkpoint header");
  uint64_t na = 0;
  if (!rd(f, &na, sizeof na) || na != h->allocs.size())
    return bad(HKBE_ERR_IO, "the file's device buffers do not match its parameters");
  std::vector<char> buf;
  for (size_t i = 0; i < na; ++i) {
    uint64_t nb = 0;
    if (!rd(f, &nb, sizeof nb) || nb != h->alloc_bytes[i])
      return bad(HKBE_ERR_IO, "the file's device buffers do not match its parameters");
    for (size_t o = 0; o < nb; o += kCkpChunk) {
      const size_t c = std::min<size_t>(kCkpChunk, nb - o);
      if (buf.size() < c) buf.resize(c);
      if (!rd(f, buf.data(), c)) return bad(HKBE_ERR_IO, "short read (device buffers)");
      cudaError_t e = cudaMemcpyAsync(static_cast<char*>(h->allocs[i]) + o, buf.data(), c, cudaMemcpyHostToDevice, h->s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
      if (e != cudaSuccess) return bad(HKBE_ERR_CUDA, std::string("checkpoint copy: ") + cudaGetErrorString(e));
    }
  }
  uint64_t trailer = 0;
  char extra;
  if (!rd(f, &trailer, sizeof trailer) || std::fread(&extra, 1, 1, f) != 0)
    return bad(HKBE_ERR_IO, "trailing bytes after the device buffers");
  std::fclose(f);
  h->have_gm = sc.have_gm != 0;
  h->have_eps = sc.have_eps != 0;
  h->have_model = sc.have_model != 0;
  h->self_consistent = sc.self_consistent != 0;
  h->cur = sc.cur;
  d.use64 = (h->cur >= 0 && d.ring64[0]) ? 1 : 0;
  d.model = sc.model;
  d.cdir = sc.cdir;
  d.nfrozR = sc.nfrozR;
  d.nfrozL = sc.nfrozL;
  *out = h;
  return HKBE_OK;
}

int hkbe_set_profiling(hkbe_t* h, int on) {
  if (!h) return HKBE_ERR_ARG;
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  drain(h);
  h->profiling = (on != 0);
  return HKBE_OK;
}

int hkbe_get_timing(const hkbe_t* h, int phase, double* ms, int64_t* launches) {
  if (!h || phase < 0 || phase >= HKBE_NPHASE) return HKBE_ERR_ARG;
  if (ms) *ms = h->phase_ms[phase];
  if (launches) *launches = h->phase_launches[phase];
  return HKBE_OK;
}

int hkbe_reset_counters(hkbe_t* h) {
  if (!h) return HKBE_ERR_ARG;
  HK_CUDA(h, cudaStreamSynchronize(h->s));
  drain(h);
  for (int i = 0; i < HKBE_NPHASE; ++i) {
    h->phase_ms[i] = 0.0;
    h->phase_launches[i] = 0;
  }
  return HKBE_OK;
}

int hkbe_weights(int k, double* a, double* omega, double* D, double* I0) {
  if (k < 1 || k > 5) return HKBE_ERR_ARG;
  hk::Weights w;
  hk::weights_build(k, &w);
  for (int i = 0; i <= k; ++i) {
    if (a) a[i] = w.a[i];
    if (omega) omega[i] = w.omega[i];
    for (int j = 0; j <= k; ++j) {
      if (D) D[i * (k + 1) + j] = w.D[i][j];
      if (I0) I0[i * (k + 1) + j] = w.I0[i][j];
    }
  }
  return HKBE_OK;
}

int hkbe_rule(int k, int n, double* w) {
  if (k < 1 || k > 5 || n < 0 || !w) return HKBE_ERR_ARG;
  hk::Weights W;
  hk::weights_build(k, &W);
  const int L = (n > k ? n : k) + 1;
  for (int l = 0; l < L; ++l) w[l] = hk::rule_weight(W, n, l);
  return HKBE_OK;
}

int hkbe_hodlr_partition(int nt, int leaf, int32_t* nblk, int32_t* r0, int32_t* r1, int32_t* c0,
                         int32_t* c1, int32_t* level) {
  if (nt < 1 || leaf < 1 || !nblk) return HKBE_ERR_ARG;
  hkbe_s tmp;                    // host-side only: build_geometry makes no device call
  tmp.p.nt = nt;
  tmp.p.leaf = leaf;
  tmp.p.nao = 1;
  build_geometry(&tmp);
  *nblk = (int32_t)tmp.g_r0.size();
  for (size_t b = 0; b < tmp.g_r0.size(); ++b) {
    if (r0) r0[b] = tmp.g_r0[b];
    if (r1) r1[b] = tmp.g_r1[b];
    if (c0) c0[b] = tmp.g_c0[b];
    if (c1) c1[b] = tmp.g_c1[b];
    if (level) level[b] = tmp.g_lvl[b];
  }
  return HKBE_OK;
}

int hkbe_dlr_matrices(int r, const double* tau, const double* omega, double beta, int xi, double* e0,
                      double* ebeta, double* rev, double* q, double* phi) {
  if (r < 1 || r > 128 || !tau || !omega || !(beta > 0) || (xi != -1 && xi != 1)) return HKBE_ERR_ARG;
  hk::DLRMats m;
  if (!hk::dlr_build(r, tau, omega, beta, xi, &m)) return HKBE_ERR_ARG;
  if (e0) std::memcpy(e0, m.e0.data(), r * sizeof(double));
  if (ebeta) std::memcpy(ebeta, m.ebeta.data(), r * sizeof(double));
  if (rev) std::memcpy(rev, m.rev.data(), (size_t)r * r * sizeof(double));
  if (q) std::memcpy(q, m.q.data(), (size_t)r * r * sizeof(double));
  if (phi) std::memcpy(phi, m.phi.data(), (size_t)r * r * r * sizeof(double));
  return HKBE_OK;
}

}  // extern "C"
