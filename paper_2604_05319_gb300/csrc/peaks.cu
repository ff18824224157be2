// FP64 and FP32 fused multiply-add throughput of the current device, measured
// with CUDA events: the ALU denominators of the roofline of the FP64 storage
// form (whose history sums run on the FP64 pipe) and of the FP32 bulk sums.
#include <cuda_runtime.h>

#include "../../include/hkbe.h"
#include "common.cuh"

namespace {

// Eight independent FMA chains per thread; one store per thread keeps the
// chains live.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T* out, int iters, T a, T b) {
  T x0 = (T)threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T>
int time_fma(int blocks, int iters, double* tflops) {
  const int threads = 256, reps = 5;
  T* out = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  int rc = HKBE_OK;
  if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads) != cudaSuccess) return HKBE_ERR_NOMEM;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) rc = HKBE_ERR_CUDA;
  float ms = 0.f;
  if (rc == HKBE_OK) {
    k_fma_chains<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);  // warm-up
    cudaEventRecord(a);
    for (int r = 0; r < reps; ++r) k_fma_chains<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(b);
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess || ms <= 0.f)
      rc = HKBE_ERR_CUDA;
  }
  if (rc == HKBE_OK) *tflops = 2.0 * 8.0 * threads * (double)blocks * iters * reps / (ms * 1e-3) / 1e12;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(out);
  return rc;
}

}  // namespace

extern "C" int hkbe_fma_peaks(double* fp64_tflops, double* fp32_tflops) {
  if (!fp64_tflops || !fp32_tflops) return HKBE_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HKBE_ERR_CUDA;
  int rc = time_fma<double>(sms * 8, 1 << 12, fp64_tflops);
  if (rc == HKBE_OK) rc = time_fma<float>(sms * 8, 1 << 14, fp32_tflops);
  return rc;
}

namespace {
__global__ void k_f32_of(int n, const double* x, float* y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = hk::f32_of(x[i]);
}
}  // namespace

extern "C" int hkbe_f32_of(int n, const double* x, float* y) {
  if (n < 0 || (n > 0 && (!x || !y))) return HKBE_ERR_ARG;
  if (n == 0) return HKBE_OK;
  double* dx = nullptr;
  float* dy = nullptr;
  int rc = HKBE_OK;
  if (cudaMalloc(&dx, (size_t)n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dy, (size_t)n * sizeof(float)) != cudaSuccess) {
    rc = HKBE_ERR_NOMEM;
  } else if (cudaMemcpy(dx, x, (size_t)n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    rc = HKBE_ERR_CUDA;
  } else {
    k_f32_of<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256>>>(n, dx, dy);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(y, dy, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = HKBE_ERR_CUDA;
  }
  cudaFree(dx);
  cudaFree(dy);
  return rc;
}
