// Allocation-free entry point: the lesser column of one time step computed
// from caller-owned device buffers, with the scratch it needs kept in a
// file-scope device array instead of memory obtained from cudaMalloc.
//
// Who needs this: code that runs where device allocation is not allowed or
// not possible — inside a caching allocator's own callbacks, in a host
// process that hands all device memory to a framework up front, or in tools
// that must not change the device's memory footprint.  Such callers cannot
// use hkbe_create (it allocates every per-handle array with cudaMalloc), but
// they can pass in buffers they already own.
//
// The scratch array is a fixed-size module global: every GPU that loads the
// library holds it until the process exits, and every call on a device
// shares it.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/hkbe.h"
#include "host_numerics.h"
#include "state.h"

namespace {

// Scratch capacity in complex doubles: the mixed-product vector (r*N_o^2),
// the boundary value (N_o^2), the lesser source ((T+1)*N_o^2) and two slots
// for the convergence flag and error (kept in the layout the kernels expect).
constexpr long long kScratchCplx = HKBE_NOALLOC_SCRATCH_CPLX;
static __device__ __align__(256) double2 g_scratch[kScratchCplx];

// Device address of g_scratch, looked up once per device (std::call_once:
// host threads may make their first calls at the same time).
constexpr int kMaxDevices = 64;
static std::once_flag g_scratch_once[kMaxDevices];
static double2* g_scratch_ptr[kMaxDevices] = {nullptr};
static cudaError_t g_scratch_err[kMaxDevices] = {cudaSuccess};

int report(char* errbuf, size_t errlen, int code, const char* msg) {
  if (errbuf && errlen) {
    std::strncpy(errbuf, msg, errlen - 1);
    errbuf[errlen - 1] = '\0';
  }
  return code;
}

}  // namespace

extern "C" int hkbe_lesser_column_noalloc(int nt, int k, int nao, int r, double h, int T,
                                          const void* d_gr, const void* d_sr, const void* d_sl,
                                          const void* d_gtv, const void* d_stv, const void* d_eps,
                                          const double* d_e0, const double* d_rev, const double* d_q,
                                          void* d_gl, void* stream, char* errbuf, size_t errlen) {
  if (k < 1 || k > 5 || nao < 1 || nao > 4 || r < 1 || r > 128 || !(h > 0) || nt < k + 2)
    return report(errbuf, errlen, HKBE_ERR_ARG, "invalid nt, k, nao, r or h");
  if (T <= k || T >= nt) return report(errbuf, errlen, HKBE_ERR_RANGE, "need k < T < nt");
  if (!d_gr || !d_sr || !d_sl || !d_gtv || !d_stv || !d_eps || !d_e0 || !d_rev || !d_q || !d_gl)
    return report(errbuf, errlen, HKBE_ERR_ARG, "null device pointer");
  const long long no2 = (long long)nao * nao;
  const long long need = (long long)r * no2 + no2 + (long long)nt * no2 + 2;
  if (need > kScratchCplx) {
    char msg[200];
    std::snprintf(msg, sizeof msg,
                  "scratch needs %lld complex doubles (r*nao^2 + nao^2 + nt*nao^2 + 2) but the "
                  "static array holds %lld; reduce nt or nao",
                  need, kScratchCplx);
    return report(errbuf, errlen, HKBE_ERR_ARG, msg);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report(errbuf, errlen, HKBE_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return report(errbuf, errlen, HKBE_ERR_ARG, "device index too large");
  std::call_once(g_scratch_once[dev], [dev]() {  // set-up, once per device, with that device current
    void* p = nullptr;
    g_scratch_err[dev] = cudaGetSymbolAddress(&p, g_scratch);
    if (g_scratch_err[dev] == cudaSuccess) g_scratch_ptr[dev] = static_cast<double2*>(p);
  });
  if (g_scratch_err[dev] != cudaSuccess) return report(errbuf, errlen, HKBE_ERR_CUDA, cudaGetErrorString(g_scratch_err[dev]));
  double2* base = g_scratch_ptr[dev];
  cudaStream_t s = (cudaStream_t)stream;

  hk::Dev d{};
  d.nt = nt; d.k = k; d.no = nao; d.r = r; d.n_inst = 1; d.xi = -1; d.rho_mode = 0; d.model = 0;
  d.ntri = (long long)nt * (nt + 1) / 2;
  d.h = h; d.beta = 0.0;
  hk::Weights w;
  hk::weights_build(k, &w);
  d.w.k = w.k;
  std::memcpy(d.w.a, w.a, sizeof(w.a));
  std::memcpy(d.w.omega, w.omega, sizeof(w.omega));
  std::memcpy(d.w.D, w.D, sizeof(w.D));
  std::memcpy(d.w.I0, w.I0, sizeof(w.I0));
  for (int i = 0; i < 6; ++i) d.w.ah[i] = w.a[i] / h;
  d.GR = (double2*)d_gr; d.SR = (double2*)d_sr; d.SL = (double2*)d_sl; d.GL = (double2*)d_gl;
  d.GTV = (double2*)d_gtv; d.STV = (double2*)d_stv; d.eps = (double2*)d_eps;
  d.e0 = (double*)d_e0; d.rev = (double*)d_rev; d.q = (double*)d_q;
  d.vvec = base;
  d.x0 = base + r * no2;
  d.qsrc = d.x0 + no2;
  d.err = reinterpret_cast<double*>(d.qsrc + (long long)nt * no2);
  d.active = reinterpret_cast<int*>(d.qsrc + (long long)nt * no2 + 1);
  // The array keeps the previous call's contents: reset the two slots that
  // must start defined (error 0; instance active, where any nonzero byte
  // pattern counts as active); everything else is written before it is read.
  if ((e = cudaMemsetAsync(d.err, 0, sizeof(double), s)) != cudaSuccess ||
      (e = cudaMemsetAsync(d.active, 1, sizeof(int), s)) != cudaSuccess ||
      (e = hk::launch_vt(d, T, s)) != cudaSuccess || (e = hk::launch_src(d, T, s)) != cudaSuccess ||
      (e = hk::launch_les(d, T, s)) != cudaSuccess)
    return report(errbuf, errlen, HKBE_ERR_CUDA, cudaGetErrorString(e));
  return HKBE_OK;
}
