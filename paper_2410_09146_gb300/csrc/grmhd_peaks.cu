// Arithmetic peaks of the current device: the dense FP64 and FP32 fused multiply-add rates, measured with
// CUDA events. They are the roofline denominators of the ALU-bound kernels (the double-precision update
// and con2prim are bound by the FP64 pipe on GB300, the float flux kernels by the FP32 pipe).
#include <cuda_runtime.h>

#include "../../include/grmhd.h"

namespace {

constexpr int kChains = 8;  // independent dependency chains per thread, enough to fill the pipes

template <class T>
__global__ void k_fma_chains(T* sink, int iters, T s) {
  T a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = T(1) + T(1e-3) * T(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], s, T(1e-9));
  }
  T t = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) t += a[c];
  if (t == T(-1)) *sink = t;  // never true: keeps the chains without a store per thread
}

template <class T>
int time_fma(T* sink, int iters, cudaStream_t s, double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GRMHD_E_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GRMHD_E_CUDA;
  const int blocks = sms * 8, threads = 256;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return GRMHD_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return GRMHD_E_CUDA;
  }
  k_fma_chains<T><<<blocks, threads, 0, s>>>(sink, iters / 8, T(0.999999));  // warm-up
  cudaEventRecord(e0, s);
  k_fma_chains<T><<<blocks, threads, 0, s>>>(sink, iters, T(0.999999));
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || !(ms > 0.f)) return GRMHD_E_CUDA;
  const double flops = 2.0 * kChains * (double)iters * blocks * threads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return GRMHD_OK;
}

}  // namespace

extern "C" int grmhd_fp_peaks(double* sink, void* stream, double* fp64_tflops, double* fp32_tflops) {
  if (!sink || !fp64_tflops || !fp32_tflops) return GRMHD_E_INVALID;
  const cudaStream_t s = (cudaStream_t)stream;
  int r = time_fma<double>(sink, 8192, s, fp64_tflops);
  if (r) return r;
  return time_fma<float>((float*)sink, 131072, s, fp32_tflops);
}
