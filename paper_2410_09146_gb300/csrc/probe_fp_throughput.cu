// Arithmetic-throughput probe: FP64 / FP32 FMA, add, mul, divide and square root on eight
// independent chains per thread, 152 x 8 blocks of 256 threads. Prints operations per second; then the
// DFMA rate when only some lanes of every warp take part (how the FP64 pipe charges a partly active warp).
// The all-FP64 stage is bound by the FP64 pipe on GB300, and its roofline peak is this probe's
// DFMA rate. Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o probe_fp probe_fp_throughput.cu && ./probe_fp
#include <cuda_runtime.h>

#include <cstdio>

#define NCH 8

template <int OP>
__global__ void chains64(double* out, int iters, double s) {
  double a[NCH];
  for (int c = 0; c < NCH; ++c) a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      if (OP == 0) a[c] = fma(a[c], s, 1e-9);
      else if (OP == 1) a[c] = a[c] + s;
      else if (OP == 2) a[c] = a[c] * s;
      else if (OP == 3) a[c] = 1.0 / a[c] + s;
      else if (OP == 4) a[c] = sqrt(a[c]) + s;
    }
  }
  double t = 0;
  for (int c = 0; c < NCH; ++c) t += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = t;  // one slot per thread: grid * block entries
}

template <int OP>
__global__ void chains32(float* out, int iters, float s) {
  float a[NCH];
  for (int c = 0; c < NCH; ++c) a[c] = 1.0f + 1e-3f * (threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      if (OP == 0) a[c] = fmaf(a[c], s, 1e-9f);
      else if (OP == 3) a[c] = 1.0f / a[c] + s;
      else if (OP == 4) a[c] = sqrtf(a[c]) + s;
    }
  }
  float t = 0;
  for (int c = 0; c < NCH; ++c) t += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

// Float -> double and double -> float conversions, independent per chain, fed and consumed by integer
// operations only (a float add on the input side of the first), so that the conversions are the only
// candidate for the FP64 pipe.
__global__ void cvt_f2d(unsigned long long* out, int iters, float s) {
  float f[NCH];
  for (int c = 0; c < NCH; ++c) f[c] = 1.0f + 1e-3f * (threadIdx.x + c);
  unsigned long long acc = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      f[c] += s;
      acc ^= (unsigned long long)__double_as_longlong((double)f[c]);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

__global__ void cvt_d2f(unsigned long long* out, int iters, float s) {
  long long b[NCH];
  for (int c = 0; c < NCH; ++c) b[c] = __double_as_longlong(1.0 + 1e-3 * (threadIdx.x + c) + (double)s);
  unsigned int acc = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      b[c] += 1;
      acc ^= __float_as_uint((float)__longlong_as_double(b[c]));
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// DFMA chains and float -> double conversions interleaved (NCH of each per iteration): the time is the sum
// of the two alone when they share the FP64 pipe, their maximum when they do not.
__global__ void dfma_cvt(unsigned long long* out, int iters, float s) {
  double a[NCH];
  float f[NCH];
  for (int c = 0; c < NCH; ++c) {
    a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    f[c] = 1.0f + 1e-3f * (threadIdx.x + c);
  }
  unsigned long long acc = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      a[c] = fma(a[c], 0.999999, 1e-9);
      f[c] += s;
      acc ^= (unsigned long long)__double_as_longlong((double)f[c]);
    }
  }
  double t = 0;
  for (int c = 0; c < NCH; ++c) t += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc ^ (unsigned long long)__double_as_longlong(t);
}

// DFMA chains in the lanes below `lanes` of every warp only.
__global__ void chains64_lanes(double* out, int iters, double s, int lanes) {
  double a[NCH];
  for (int c = 0; c < NCH; ++c) a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  if ((int)(threadIdx.x & 31) < lanes) {
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int c = 0; c < NCH; ++c) a[c] = fma(a[c], s, 1e-9);
    }
  }
  double t = 0;
  for (int c = 0; c < NCH; ++c) t += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

template <typename K, typename T, typename S>
static void timed(const char* name, K kern, T* buf, int iters, S s, int blocks, int threads, double flop_per_op) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  kern<<<blocks, threads>>>(buf, iters, s);  // warm-up
  cudaDeviceSynchronize();
  cudaEventRecord(e0);
  kern<<<blocks, threads>>>(buf, iters, s);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  const double ops = (double)blocks * threads * iters * NCH;
  printf("%-10s %8.3f ms  %10.3f Gop/s  (%.3f TFLOP/s at %.0f flop/op)\n", name, ms, ops / ms / 1e6,
         ops * flop_per_op / ms / 1e9, flop_per_op);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

int main() {
  const int blocks = 152 * 8, threads = 256;
  double* d64 = nullptr;
  float* d32 = nullptr;
  cudaMalloc(&d64, sizeof(double) * blocks * threads);
  cudaMalloc(&d32, sizeof(float) * blocks * threads);
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, 0);
  printf("%s SMs=%d cc=%d.%d\n", prop.name, prop.multiProcessorCount, prop.major, prop.minor);
  timed("dfma", chains64<0>, d64, 2000, 0.999999, blocks, threads, 2);
  timed("dadd", chains64<1>, d64, 2000, 1e-12, blocks, threads, 1);
  timed("dmul", chains64<2>, d64, 2000, 0.9999999, blocks, threads, 1);
  timed("ddiv+add", chains64<3>, d64, 200, 1e-12, blocks, threads, 1);
  timed("dsqrt+add", chains64<4>, d64, 200, 1e-12, blocks, threads, 1);
  timed("ffma", chains32<0>, d32, 20000, 0.999999f, blocks, threads, 2);
  timed("fdiv+add", chains32<3>, d32, 2000, 1e-7f, blocks, threads, 1);
  timed("fsqrt+add", chains32<4>, d32, 2000, 1e-7f, blocks, threads, 1);
  unsigned long long* du = nullptr;
  cudaMalloc(&du, sizeof(unsigned long long) * blocks * threads);
  timed("cvt f->d", cvt_f2d, du, 2000, 1e-7f, blocks, threads, 1);
  timed("cvt d->f", cvt_d2f, du, 2000, 1e-7f, blocks, threads, 1);
  timed("dfma+cvt", dfma_cvt, du, 2000, 1e-7f, blocks, threads, 1);
  cudaFree(du);
  for (int lanes : {32, 16, 8, 1}) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    chains64_lanes<<<blocks, threads>>>(d64, 2000, 0.999999, lanes);  // warm-up
    cudaEventRecord(e0);
    chains64_lanes<<<blocks, threads>>>(d64, 2000, 0.999999, lanes);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double warp_ops = (double)blocks * threads / 32.0 * 2000 * NCH;
    printf("dfma, %2d active lanes per warp: %8.3f ms  %8.2f G warp-instructions/s  %7.3f TFLOP/s of active lanes\n",
           lanes, ms, warp_ops / ms / 1e6, warp_ops * lanes * 2 / ms / 1e9);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  const cudaError_t e = cudaGetLastError();
  printf("status %s\n", cudaGetErrorString(e));
  cudaFree(d64);
  cudaFree(d32);
  return e == cudaSuccess ? 0 : 1;
}
