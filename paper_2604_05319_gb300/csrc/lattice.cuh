// Lattice helpers of the 2D Hubbard model (Sec. 4.2) shared by the
// real-time self-energy (kernels_hodlr.cu) and the equilibrium solve
// (matsubara_dev.cu): the k-point of a thread, the reflection-reduced k-set,
// and a 2D discrete Fourier transform over an L x L grid held in shared memory.
#pragma once
#include "common.cuh"

namespace hk {

constexpr int kLatMaxK = 256;
// instance holding grid point q = m_x L + m_y (ys: reflection-reduced k-set)
__device__ __forceinline__ int lat_inst(int q, int L, int ys) {
  if (!ys) return q;
  const int y = q % L;
  return (q / L) * (L / 2 + 1) + min(y, L - y);
}
// grid point q is the instance's own k-point (not a reflected copy)
__device__ __forceinline__ bool lat_owner(int q, int L, int ys) { return !ys || q % L <= L / 2; }
// in-place 2D DFT of a[N] (N = L*L, index m_x L + m_y) with sign sg (+1: e^{+i}),
// scaled by sc; tw[m] = e^{2 pi i m / L}; every thread of the CTA must call it
__device__ __forceinline__ void lat_dft2(zd* a, zd* tmp, const zd* tw, int L, int sg, double sc) {
  const int N = L * L, q = threadIdx.x;
  const int x = q / L, y = q % L;
  if (q < N) {  // along m_y: tmp[x][y] = sum_m a[x][m] e^{sg i 2pi m y / L}
    zd s = zd();
    for (int m = 0; m < L; ++m) {
      const zd w = tw[(m * y) % L];
      s += a[x * L + m] * (sg > 0 ? w : w.conj());
    }
    tmp[q] = s;
  }
  __syncthreads();
  if (q < N) {  // along m_x
    zd s = zd();
    for (int m = 0; m < L; ++m) {
      const zd w = tw[(m * x) % L];
      s += tmp[m * L + y] * (sg > 0 ? w : w.conj());
    }
    a[q] = s * sc;
  }
  __syncthreads();
}

// tw[m] = e^{2 pi i m / L}, m < L, written by the first L threads (the
// caller synchronises before use)
__device__ __forceinline__ void lat_twiddles(zd* tw, int L) {
  const int q = threadIdx.x;
  if (q < L) {
    double sn, cs;
    sincospi(2.0 * q / L, &sn, &cs);
    tw[q] = zd(cs, sn);
  }
}

}  // namespace hk
