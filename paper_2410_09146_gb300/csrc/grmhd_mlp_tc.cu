// Fused learned-guess con2prim on the fifth-generation tensor cores: one CTA of 128 threads takes a
// tile of 128 flat-space states (thread t owns state t of the tile and row t of every matrix), and
//   1. computes the master-function invariants, the bracket end mu_+ and the features (FP64 / FP32);
//   2. layer 1 (8 -> 64) in FP32 on the CUDA cores, h1 rounded to BF16 into shared memory;
//   3. layers 2 and 3 (64 -> 64) as tcgen05.mma kind::f16 (BF16 operands from shared memory, FP32
//      accumulators in 64 TMEM columns; M = 128 states, N = 64, K = 4 x 16), read back with tcgen05.ld;
//   4. the output layer in FP32 from the TMEM chunks, mu_0 = mu_+ (1 - e^{-y0});
//   5. the safeguarded Newton iteration of the Kastaun master function (Sec. 3.1) from mu_0 (at most 8
//      iterations), falling back to the standard start mu_+/2 with the full budget.
// One elected thread issues the MMAs and waits for their completion on an mbarrier with an iteration
// limit; on a timeout the CTA records it in the statistics, waits once more (bounded) for the MMA in
// flight, frees its TMEM and returns.
#include <cmath>
#include <cstdio>

#include "grmhd_launch.h"
#include "grmhd_mlp.cuh"
#include "grmhd_tc.cuh"

namespace {

using namespace grmhd;
using namespace grmhd::mlp;

constexpr int TC_M = 128;  // states per tile = threads per CTA = MMA M
constexpr int TC_N = HID;  // MMA N (outputs of the layer)
constexpr int TC_K = HID;  // K of layers 2 and 3
constexpr uint32_t TMEM_COLS = 64;
constexpr uint32_t IDESC = tc::idesc_bf16(TC_M, TC_N);
using tc::fence_after_sync;
using tc::fence_async_smem;
using tc::fence_before_sync;
using tc::mbar_wait;
using tc::mma_commit;
using tc::smem_addr;
using tc::smem_desc;
using tc::tmem_ld16;

// Operands in the canonical K-major layout without swizzle (grmhd_tc.cuh).
struct __align__(128) TcSmem {
  __nv_bfloat16 A[TC_M * TC_K];   // activations h1 / h2 (16 KB)
  __nv_bfloat16 B2[TC_N * TC_K];  // W2 (8 KB)
  __nv_bfloat16 B3[TC_N * TC_K];  // W3 (8 KB)
  float W1[HID * NIN];
  float b1[HID], b2[HID], b3[HID];
  float w4[HID];                  // first output row of W4 (only y0 is needed for the guess)
  float norm[NNORM];
  float b4;
  unsigned long long mbar;
  uint32_t tmem_base;
  int ok;
};

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  tc::mma_bf16(tmem_d, adesc, bdesc, IDESC, accumulate);
}

// Eight BF16 values of row r, K group g of the activation operand (one 16-byte store).
__device__ __forceinline__ void store_a8(__nv_bfloat16* A, int r, int g, const float h[8]) {
  __align__(16) __nv_bfloat162 q[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) q[i] = __floats2bfloat162_rn(h[2 * i], h[2 * i + 1]);
  *reinterpret_cast<uint4*>(A + (size_t)g * TC_M * 8 + r * 8) = *reinterpret_cast<const uint4*>(q);
}

// Issue one 64 x 64 layer (K = 4 x 16) from thread 0 and wait for it; returns false (for every thread)
// when the completion was not observed within the limit.
__device__ __forceinline__ bool run_layer(TcSmem& S, const __nv_bfloat16* B, uint32_t& phase) {
  fence_async_smem();  // this thread's generic-proxy stores to A become visible to the tensor cores
  fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0) {
    fence_after_sync();
    const uint32_t a0 = smem_addr(S.A), b0 = smem_addr(B);
#pragma unroll
    for (int s = 0; s < TC_K / 16; ++s) {
      const uint64_t ad = smem_desc(a0 + s * 2 * TC_M * 16, TC_M * 16, 128);
      const uint64_t bd = smem_desc(b0 + s * 2 * TC_N * 16, TC_N * 16, 128);
      mma_bf16(S.tmem_base, ad, bd, s > 0 ? 1u : 0u);
    }
    mma_commit(smem_addr(&S.mbar));
    S.ok = mbar_wait(smem_addr(&S.mbar), phase) ? 1 : 0;
    fence_before_sync();
  }
  __syncthreads();
  fence_after_sync();
  phase ^= 1u;
  return S.ok != 0;
}

__global__ void __launch_bounds__(TC_M) k_c2p_net_tc(const double* __restrict__ U, double* __restrict__ P,
                                                    uint8_t* __restrict__ status, int* __restrict__ iters_out,
                                                    long long n, DevParams p, const __nv_bfloat16* __restrict__ w,
                                                    const float* __restrict__ norm, double* __restrict__ guess,
                                                    unsigned long long* stats) {
  extern __shared__ __align__(128) unsigned char smraw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>(smraw);
  const int t = threadIdx.x, warp = t >> 5;
  // ---- per-CTA set-up: weights into the operand layouts, TMEM, mbarrier
  for (int e = t; e < TC_N * TC_K; e += TC_M) {
    const int r = e / TC_K, k = e % TC_K;  // W[r][k], r = output, k = input
    const int off = (k / 8) * TC_N * 8 + r * 8 + (k % 8);
    S.B2[off] = w[OFF_W2 + e];
    S.B3[off] = w[OFF_W3 + e];
  }
  for (int e = t; e < HID * NIN; e += TC_M) S.W1[e] = __bfloat162float(w[OFF_W1 + e]);
  for (int e = t; e < HID; e += TC_M) {
    S.b1[e] = __bfloat162float(w[OFF_B1 + e]);
    S.b2[e] = __bfloat162float(w[OFF_B2 + e]);
    S.b3[e] = __bfloat162float(w[OFF_B3 + e]);
    S.w4[e] = __bfloat162float(w[OFF_W4 + e]);
  }
  for (int e = t; e < NNORM; e += TC_M) S.norm[e] = norm[e];
  if (t == 0) {
    S.b4 = __bfloat162float(w[OFF_B4]);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&S.mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");  // visible to the async proxy
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&S.tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem_row = S.tmem_base + ((uint32_t)(warp * 32) << 16);  // this warp's 32 TMEM lanes
  uint32_t phase = 0;
  unsigned int it_sum = 0, nconv = 0, nfall = 0;
  bool abandoned = false;
  for (long long base = (long long)blockIdx.x * TC_M; base < n; base += (long long)gridDim.x * TC_M) {
    const long long i = base + t;
    const bool valid = i < n;
    // ---- invariants, mu_+, features, layer 1 (FP32) -> h1 (BF16) into A
    double Uc[NV], ru[3], bu[3];
    C2PIn<double> c;
    bool good = false;
    double mup = 0.0;
    float x[NIN];
#pragma unroll
    for (int k = 0; k < NIN; ++k) x[k] = 0.f;
    if (valid) {
      good = flat_invariants(p, U, n, i, Uc, c, ru, bu);
      if (good) {
        mup = c2p_mu_plus_fast(c);
        raw_features(c, mup, x);
#pragma unroll
        for (int k = 0; k < NIN; ++k) x[k] = (x[k] - S.norm[k]) * S.norm[NIN + k];
      }
    }
#pragma unroll 1
    for (int g = 0; g < HID / 8; ++g) {
      float h[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int j = g * 8 + q;
        float a = S.b1[j];
#pragma unroll
        for (int k = 0; k < NIN; ++k) a = fmaf(S.W1[j * NIN + k], x[k], a);
        h[q] = silu(a);
      }
      store_a8(S.A, t, g, h);
    }
    // ---- layer 2 on the tensor cores -> h2 (BF16) into A
    if (!run_layer(S, S.B2, phase)) {
      abandoned = true;
      break;
    }
#pragma unroll 1
    for (int cb = 0; cb < HID / 16; ++cb) {
      float z[16];
      tmem_ld16(tmem_row + cb * 16, z);
      float h[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) h[q] = silu(z[q] + S.b2[cb * 16 + q]);
      store_a8(S.A, t, 2 * cb, h);
      store_a8(S.A, t, 2 * cb + 1, h + 8);
    }
    // ---- layer 3 on the tensor cores, output layer from the accumulator chunks
    if (!run_layer(S, S.B3, phase)) {
      abandoned = true;
      break;
    }
    float y0 = S.b4;
#pragma unroll 1
    for (int cb = 0; cb < HID / 16; ++cb) {
      float z[16];
      tmem_ld16(tmem_row + cb * 16, z);
#pragma unroll
      for (int q = 0; q < 16; ++q) y0 = fmaf(S.w4[cb * 16 + q], silu(z[q] + S.b3[cb * 16 + q]), y0);
    }
    y0 = y0 * S.norm[2 * NIN + NOUT] + S.norm[2 * NIN];
    if (!valid) continue;
    // ---- Newton from the network's start, fallback to the standard start
    const unsigned lanes = __activemask();  // each of these lanes reaches the __syncwarp below once
    double Pn[NV];
    int st = 0, iters = 0;
    double mu0 = 0.0, mu = 0.0;
    if (good) {
      const float yc = fminf(fmaxf(y0, 0.f), Y0_MAX);  // NaN -> 0 -> mu_0 = 0 -> fallback
      mu = mup - mup * (double)__expf(-yc);
      mu0 = mu;
      bool done = false;
      if (mu > 0.0 && mu < mup) done = c2p_newton<double>(c, mup, mu, p.c2p_tol, GUESS_MAX_ITER, iters, true) == 0;
      if (!done) {
        ++nfall;
        mu = 0.5 * mup;
        st = c2p_newton<double>(c, mup, mu, p.c2p_tol, p.c2p_max_iter, iters, true);
      }
      if (st) ++nconv;
    }
    __syncwarp(lanes);  // iterations of different lengths: run the output once per warp
    if (!good) {
      c2p_bad_output(Uc, Pn);
      st = ST_BAD_INPUT;
    } else {
      c2p_output(c, mu, ru, bu, Uc, Pn);
    }
    Metric<double> m;
    metric_at<double, MINKOWSKI>(p, 0.0, 0.0, 0.0, m);
    st |= apply_floors<MINKOWSKI>(p, m.gam, 1.0, Pn);
#pragma unroll
    for (int q = 0; q < NV; ++q) P[q * n + i] = Pn[q];
    if (status) status[i] = (uint8_t)st;
    if (iters_out) iters_out[i] = iters;
    if (guess) {
      guess[i] = mu0;
      guess[n + i] = mup;
    }
    it_sum += iters;
  }
  // ---- tear-down (uniform: `abandoned` is the same in every thread)
  if (abandoned && t == 0) {
    mbar_wait(smem_addr(&S.mbar), phase ^ 1u);  // the MMA still in flight, bounded
    if (stats) atomicAdd(stats + 6, 1ull);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem_base), "r"(TMEM_COLS) : "memory");
  if (stats) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      it_sum += __shfl_xor_sync(0xffffffffu, it_sum, o);
      nconv += __shfl_xor_sync(0xffffffffu, nconv, o);
      nfall += __shfl_xor_sync(0xffffffffu, nfall, o);
    }
    if ((t & 31) == 0) {
      atomicAdd(stats + 0, (unsigned long long)it_sum);
      if (nconv) atomicAdd(stats + 4, (unsigned long long)nconv);
      if (nfall) atomicAdd(stats + 7, (unsigned long long)nfall);
    }
  }
}

}  // namespace

namespace grmhd {
cudaError_t launch_c2p_net_tc(const void* mlp_ws, const double* U, double* P, uint8_t* status, int* iters,
                              long long n, const DevParams& p, double* guess, unsigned long long* stats,
                              cudaStream_t s) {
  static int attr_dev = -1, ctas = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (attr_dev != dev) {
    e = cudaFuncSetAttribute(k_c2p_net_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcSmem));
    // the launch takes the largest shared-memory carveout (residency below assumes it)
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_c2p_net_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    // resident CTAs per SM from the kernel's registers (per warp, rounded to the 256-register allocation
    // unit), its shared memory (plus the per-block reservation) and the 512 TMEM columns of an SM
    int sms = 0, regs_sm = 0, smem_sm = 0, smem_rsv = 0;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k_c2p_net_tc);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e != cudaSuccess) return e;
    const int warp_regs = ((fa.numRegs * 32 + 255) / 256) * 256;
    int per_sm = regs_sm / (warp_regs * (TC_M / 32));
    const int by_smem = smem_sm / ((int)sizeof(TcSmem) + (int)fa.sharedSizeBytes + smem_rsv);
    if (by_smem < per_sm) per_sm = by_smem;
    if (per_sm > (int)(512 / TMEM_COLS)) per_sm = 512 / TMEM_COLS;
    ctas = sms * (per_sm > 0 ? per_sm : 1);
    attr_dev = dev;
  }
  if (n <= 0) return cudaSuccess;
  const long long tiles = (n + TC_M - 1) / TC_M;
  const int grid = (int)(tiles < ctas ? tiles : ctas);
  const MlpPtrs m = ptrs(mlp_ws);
  k_c2p_net_tc<<<grid, TC_M, sizeof(TcSmem), s>>>(U, P, status, iters, n, p, m.w, m.norm, guess, stats);
  return cudaGetLastError();
}
}  // namespace grmhd
