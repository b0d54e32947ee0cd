// Arithmetic peak of the FP64 and FP32 pipes, measured with the library's own FMA loop
// (sem_measure_fma_peak): the denominators of the element kernels' ALU rooflines.
#include <cuda_runtime.h>

#include <string>

#include "../../include/sem.h"
#include "device.h"

namespace sem {
void count_launch();   // adds one to kernel_launch_count() of this thread
}

namespace {

constexpr int kChains = 8;      // independent FMA chains per thread (hide the pipe latency)
constexpr int kPeakBlock = 256;

// acc <- acc * a + b on kChains chains; a < 1 keeps every chain bounded near b / (1 - a).
// The sum of the chains is stored, so no FMA can be dropped.
template <typename T>
__global__ void __launch_bounds__(kPeakBlock) fma_peak_kernel(int iters, T a, T b, T* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  T acc[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc[k] = (T)(t & 1023) * (T)1e-3 + (T)k;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = fma(acc[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += acc[k];
  out[t] = s;
}

template <typename T>
int measure(int iters, double* tflops, double* ms_out, std::string& err) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = nsm * 8;   // 2048 threads per SM
  T* out = nullptr;
  if (cudaMalloc((void**)&out, sizeof(T) * blocks * kPeakBlock) != cudaSuccess) {
    err = "cudaMalloc failed";
    return SEM_ERR_OOM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  cudaError_t e = cudaSuccess;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first launch warms up
    cudaEventRecord(e0, 0);
    fma_peak_kernel<T><<<blocks, kPeakBlock, 0, 0>>>(iters, (T)0.999999, (T)1e-6, out);
    sem::count_launch();
    cudaEventRecord(e1, 0);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    float ms = 0.f;
    if (e == cudaSuccess && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    return SEM_ERR_CUDA;
  }
  const double flops = 2.0 * kChains * (double)iters * blocks * kPeakBlock;
  *ms_out = best;
  *tflops = flops / (best * 1e-3) / 1e12;
  return SEM_OK;
}

}  // namespace

int sem_measure_fma_peak(int precision, int64_t iters, double* tflops_host, double* ms_host) {
  if (tflops_host == nullptr || ms_host == nullptr || iters <= 0 || iters > (1 << 30) ||
      (precision != SEM_PREC_FP64 && precision != SEM_PREC_FP32))
    return sem::report_error(SEM_ERR_ARG, "bad arguments");
  std::string err;
  const int rc = precision == SEM_PREC_FP64 ? measure<double>((int)iters, tflops_host, ms_host, err)
                                            : measure<float>((int)iters, tflops_host, ms_host, err);
  if (rc != SEM_OK) return sem::report_error(rc, err);
  return SEM_OK;
}
