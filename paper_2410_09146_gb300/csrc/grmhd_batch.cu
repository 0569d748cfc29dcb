// Launch-size helper, the time-step finalisation and the flat con2prim / prim2con batches (built with FMA).
#include "grmhd_kernels.cuh"
#include "grmhd_launch.h"

namespace grmhd {

int grid_for(long long n, int threads) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  long long b = (n + threads - 1) / threads;
  const long long cap = (long long)sms * 16;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t launch_finalize_dt(const unsigned long long* ms, double* dt, const DevParams& p, cudaStream_t s) {
  k_finalize_dt<<<1, 32, 0, s>>>(ms, dt, p);
  return cudaGetLastError();
}

cudaError_t launch_batch_finalize_dt(const unsigned long long* ms, double* dt, double cfl, cudaStream_t s) {
  k_batch_finalize_dt<<<1, 32, 0, s>>>(ms, dt, cfl);
  return cudaGetLastError();
}

cudaError_t launch_c2p_batch(const double* U, double* P, uint8_t* status, int* iters, long long n, int flags,
                             const DevParams& p, unsigned long long* stats, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_c2p_batch<<<grid_for(n, 128), 128, 0, s>>>(U, P, status, iters, n, flags, p, stats);
  return cudaGetLastError();
}

cudaError_t launch_p2c_batch(const double* P, double* U, long long n, const DevParams& p, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_p2c_batch<<<grid_for(n, 128), 128, 0, s>>>(P, U, n, p);
  return cudaGetLastError();
}

}  // namespace grmhd
