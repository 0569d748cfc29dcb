// Training kernel of the learned con2prim guess on the fifth-generation tensor cores: fused forward +
// backward over tiles of 128 samples, the network's four 64 x 64 products of a tile and its two 64 x 64
// weight gradients as tcgen05.mma kind::f16 (BF16 operands from shared memory, FP32 accumulators in tensor
// memory), the rest (layer 1, the output layer, the activations and their derivatives, the gradients of the
// first and last layers) in FP32 on the CUDA cores.
//
// One CTA of 128 threads per SM (thread s owns sample s of a tile and row s of every per-sample matrix),
// tensor-memory columns:
//   [0, 64)    z2 = h1 W2^T            (layer 2 before its bias)
//   [64, 128)  z3 = h2 W3^T            (layer 3)
//   [128, 192) delta3 W3               (back through layer 3)
//   [192, 256) delta2 W2               (back through layer 2)
//   [256, 400) [delta3^T; delta2^T] [h2^T; h1^T; 1]^T, accumulated over all tiles of the CTA: rows 0-63,
//              columns 0-63 hold the gradient of W3, rows 64-127, columns 64-127 that of W2, column 128 the
//              bias gradients (the ones row of the second operand).
// The BF16 operands are the forward activations h1, h2 (rounded as in every forward pass of the library)
// and the back-propagated deltas delta3, delta2, rounded to BF16 where they enter a product; delta1 and the
// output-layer quantities stay FP32. The FP64 reference network applies the same roundings
// (oracle/guess_mlp.py, round_delta). One elected thread issues the MMAs and waits for their completion on an
// mbarrier with an iteration limit; on a timeout the CTA stops, records it (*abandon += 1), waits once more
// (bounded) for the MMA in flight and frees its tensor memory.
#include "grmhd_mlp.cuh"
#include "grmhd_tc.cuh"

namespace grmhd {
namespace mlp {
namespace {

using namespace grmhd::tc;

constexpr int TM = TILE;              // samples per tile = threads = MMA M
constexpr int WG_N = 2 * HID + 16;    // N of the weight-gradient product: h2, h1 and the ones row (padded)
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t C_Z2 = 0, C_Z3 = 64, C_D2 = 128, C_D1 = 192, C_WG = 256;
constexpr uint32_t IDESC_64 = idesc_bf16(TM, HID);
constexpr uint32_t IDESC_WG = idesc_bf16(TM, WG_N);
constexpr int LDF = HID + 1;  // padded FP32 rows

struct __align__(128) TrainSmem {
  __nv_bfloat16 A[TM * HID];          // A operand of the per-tile products: h1, h2, delta3, delta2 (16 KB)
  __nv_bfloat16 W2f[HID * HID];       // B of layer 2 forward: W2[j][k] as (n = j, K = k)
  __nv_bfloat16 W3f[HID * HID];       // B of layer 3 forward
  __nv_bfloat16 W3b[HID * HID];       // B of delta3 W3: W3[j][k] as (n = k, K = j)
  __nv_bfloat16 W2b[HID * HID];       // B of delta2 W2
  __nv_bfloat16 Awg[TM * TM];         // [delta3^T; delta2^T], K = the tile's samples (32 KB)
  __nv_bfloat16 Bwg[WG_N * TM];       // [h2^T; h1^T; ones; zeros], K = the tile's samples (36 KB)
  float Z1[TM * LDF];                 // z1, then delta1
  float H3[TM * LDF];                 // h3
  float Xs[TM * NIN];                 // standardised inputs
  float Do[TM * NOUT];                // output deltas
  float W1[HID * NIN], b1[HID], b2[HID], b3[HID], W4[NOUT * HID], b4[NOUT];
  float norm[NNORM];
  float gW1[HID * NIN], gb1[HID], gW4[NOUT * HID], gb4[NOUT];
  unsigned long long mbar;
  uint32_t tmem_base;
  int ok;
};

// Issue `ksteps` K-steps of 16 of D = A B^T (A of RA rows, B of RB rows, both K-major) from thread 0 and
// wait for them; false (for every thread) when the completion was not observed within the limit.
__device__ __forceinline__ bool run_mma(TrainSmem& S, const __nv_bfloat16* A, int RA, const __nv_bfloat16* B, int RB,
                                        int ksteps, uint32_t tmem_d, uint32_t idesc, bool accumulate,
                                        uint32_t& phase) {
  fence_async_smem();  // this thread's generic-proxy stores to the operands become visible to the tensor cores
  fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0) {
    fence_after_sync();
    const uint32_t a0 = smem_addr(A), b0 = smem_addr(B);
    for (int s = 0; s < ksteps; ++s) {
      const uint64_t ad = smem_desc(a0 + s * 2 * RA * 16, RA * 16, 128);
      const uint64_t bd = smem_desc(b0 + s * 2 * RB * 16, RB * 16, 128);
      mma_bf16(tmem_d, ad, bd, idesc, (accumulate || s > 0) ? 1u : 0u);
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

// Row s (a sample) of a K-major operand of R rows: eight values at K group g (one 16-byte store).
__device__ __forceinline__ void store_row8(__nv_bfloat16* A, int R, int s, int g, const float v[8]) {
  __align__(16) __nv_bfloat162 q[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) q[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
  *reinterpret_cast<uint4*>(A + (size_t)g * R * 8 + s * 8) = *reinterpret_cast<const uint4*>(q);
}

// Column s (a sample) of a K-major operand of R rows whose K runs over the samples: rows r0 .. r0 + 15.
__device__ __forceinline__ void store_col16(__nv_bfloat16* A, int R, int s, int r0, const float v[16]) {
#pragma unroll
  for (int i = 0; i < 16; ++i) A[kmajor_off(r0 + i, s, R)] = __float2bfloat16_rn(v[i]);
}

__global__ void __launch_bounds__(TM, 1) k_mlp_train_tc(long long n, const float* __restrict__ X,
                                                        const float* __restrict__ T,
                                                        const __nv_bfloat16* __restrict__ w,
                                                        const float* __restrict__ norm, float* __restrict__ grad,
                                                        float* __restrict__ loss, float* __restrict__ abandon,
                                                        float aux) {
  extern __shared__ __align__(128) unsigned char smraw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smraw);
  const int s = threadIdx.x, warp = s >> 5;
  // ---- per-CTA set-up: weights into the operand layouts and FP32 copies, accumulators, TMEM, mbarrier
  for (int e = s; e < HID * HID; e += TM) {
    const int j = e / HID, k = e % HID;  // W[j][k]: output j, input k
    S.W2f[kmajor_off(j, k, HID)] = w[OFF_W2 + e];
    S.W3f[kmajor_off(j, k, HID)] = w[OFF_W3 + e];
    S.W2b[kmajor_off(k, j, HID)] = w[OFF_W2 + e];
    S.W3b[kmajor_off(k, j, HID)] = w[OFF_W3 + e];
  }
  for (int e = s; e < HID * NIN; e += TM) {
    S.W1[e] = __bfloat162float(w[OFF_W1 + e]);
    S.gW1[e] = 0.f;
  }
  for (int e = s; e < HID; e += TM) {
    S.b1[e] = __bfloat162float(w[OFF_B1 + e]);
    S.b2[e] = __bfloat162float(w[OFF_B2 + e]);
    S.b3[e] = __bfloat162float(w[OFF_B3 + e]);
    S.gb1[e] = 0.f;
  }
  for (int e = s; e < NOUT * HID; e += TM) {
    S.W4[e] = __bfloat162float(w[OFF_W4 + e]);
    S.gW4[e] = 0.f;
  }
  if (s < NOUT) {
    S.b4[s] = __bfloat162float(w[OFF_B4 + s]);
    S.gb4[s] = 0.f;
  }
  for (int e = s; e < NNORM; e += TM) S.norm[e] = norm[e];
  // the ones row (128) and the zero padding (129 .. WG_N - 1) of the weight-gradient operand, fixed
  for (int k = 0; k < TM; ++k)
    for (int r = 2 * HID + (s % 16); r < WG_N; r += 16)
      if (s < 16) S.Bwg[kmajor_off(r, k, WG_N)] = __float2bfloat16_rn(r == 2 * HID ? 1.f : 0.f);
  if (s == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&S.mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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
  const uint32_t trow = S.tmem_base + ((uint32_t)(warp * 32) << 16);  // this warp's 32 TMEM lanes
  const float inv_n = 1.f / (float)n;
  float lsum = 0.f;
  uint32_t phase = 0;
  bool abandoned = false, first = true;
  for (long long base = (long long)blockIdx.x * TM; base < n; base += (long long)gridDim.x * TM) {
    const long long t = base + s;
    const bool valid = t < n;
    float* z1 = S.Z1 + s * LDF;
    // ---- layer 1 (FP32): z1 kept for its derivative, h1 = bf16(silu(z1)) into A and into the gradient operand
    float x[NIN];
#pragma unroll
    for (int k = 0; k < NIN; ++k) {
      x[k] = valid ? (X[t * NIN + k] - S.norm[k]) * S.norm[NIN + k] : 0.f;
      S.Xs[s * NIN + k] = x[k];
    }
#pragma unroll 1
    for (int g = 0; g < HID / 16; ++g) {
      float h[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int j = g * 16 + q;
        float a = S.b1[j];
#pragma unroll
        for (int k = 0; k < NIN; ++k) a = fmaf(S.W1[j * NIN + k], x[k], a);
        z1[j] = a;
        h[q] = valid ? silu(a) : 0.f;  // padding samples contribute nothing to the gradient
      }
      store_row8(S.A, TM, s, 2 * g, h);
      store_row8(S.A, TM, s, 2 * g + 1, h + 8);
      store_col16(S.Bwg, WG_N, s, HID + g * 16, h);  // rows 64..127: h1^T
    }
    // ---- layer 2 on the tensor cores: z2 -> TMEM [0, 64); h2 into A and into the gradient operand
    if (!run_mma(S, S.A, TM, S.W2f, HID, HID / 16, S.tmem_base + C_Z2, IDESC_64, false, phase)) {
      abandoned = true;
      break;
    }
#pragma unroll 1
    for (int cb = 0; cb < HID / 16; ++cb) {
      float z[16], h[16];
      tmem_ld16(trow + C_Z2 + cb * 16, z);
#pragma unroll
      for (int q = 0; q < 16; ++q) h[q] = valid ? silu(z[q] + S.b2[cb * 16 + q]) : 0.f;
      store_row8(S.A, TM, s, 2 * cb, h);
      store_row8(S.A, TM, s, 2 * cb + 1, h + 8);
      store_col16(S.Bwg, WG_N, s, cb * 16, h);  // rows 0..63: h2^T
    }
    // ---- layer 3 on the tensor cores: z3 -> TMEM [64, 128); h3, the output layer and its deltas (FP32)
    if (!run_mma(S, S.A, TM, S.W3f, HID, HID / 16, S.tmem_base + C_Z3, IDESC_64, false, phase)) {
      abandoned = true;
      break;
    }
    float o[NOUT] = {S.b4[0], S.b4[1]};
#pragma unroll 1
    for (int cb = 0; cb < HID / 16; ++cb) {
      float z[16];
      tmem_ld16(trow + C_Z3 + cb * 16, z);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float h3 = silu(z[q] + S.b3[cb * 16 + q]);
        S.H3[s * LDF + cb * 16 + q] = h3;
        o[0] = fmaf(S.W4[cb * 16 + q], h3, o[0]);
        o[1] = fmaf(S.W4[HID + cb * 16 + q], h3, o[1]);
      }
    }
    float d[NOUT];
#pragma unroll
    for (int i = 0; i < NOUT; ++i) {
      const float wgt = i == 0 ? 1.f : aux;
      const float tt = valid ? (T[t * NOUT + i] - S.norm[2 * NIN + i]) / S.norm[2 * NIN + NOUT + i] : 0.f;
      const float e = valid ? o[i] - tt : 0.f;
      lsum += wgt * e * e;
      d[i] = 2.f * wgt * e * inv_n;
      S.Do[s * NOUT + i] = d[i];
    }
    // delta3 = dsilu(z3) (W4^T d), BF16 into A (the next product) and into the gradient operand's rows 0..63
#pragma unroll 1
    for (int cb = 0; cb < HID / 16; ++cb) {
      float z[16], dl[16];
      tmem_ld16(trow + C_Z3 + cb * 16, z);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int k = cb * 16 + q;
        dl[q] = dsilu(z[q] + S.b3[k]) * fmaf(S.W4[k], d[0], S.W4[HID + k] * d[1]);
      }
      store_row8(S.A, TM, s, 2 * cb, dl);
      store_row8(S.A, TM, s, 2 * cb + 1, dl + 8);
      store_col16(S.Awg, TM, s, cb * 16, dl);
    }
    // ---- delta3 W3 on the tensor cores -> TMEM [128, 192); delta2 = dsilu(z2) (delta3 W3)
    if (!run_mma(S, S.A, TM, S.W3b, HID, HID / 16, S.tmem_base + C_D2, IDESC_64, false, phase)) {
      abandoned = true;
      break;
    }
#pragma unroll 1
    for (int cb = 0; cb < HID / 16; ++cb) {
      float z[16], g[16], dl[16];
      tmem_ld16(trow + C_Z2 + cb * 16, z);
      tmem_ld16(trow + C_D2 + cb * 16, g);
#pragma unroll
      for (int q = 0; q < 16; ++q) dl[q] = dsilu(z[q] + S.b2[cb * 16 + q]) * g[q];
      store_row8(S.A, TM, s, 2 * cb, dl);
      store_row8(S.A, TM, s, 2 * cb + 1, dl + 8);
      store_col16(S.Awg, TM, s, HID + cb * 16, dl);  // rows 64..127: delta2^T
    }
    // ---- delta2 W2 on the tensor cores -> TMEM [192, 256); delta1 = dsilu(z1) (delta2 W2), FP32, in place of z1
    if (!run_mma(S, S.A, TM, S.W2b, HID, HID / 16, S.tmem_base + C_D1, IDESC_64, false, phase)) {
      abandoned = true;
      break;
    }
#pragma unroll 1
    for (int cb = 0; cb < HID / 16; ++cb) {
      float g[16];
      tmem_ld16(trow + C_D1 + cb * 16, g);
#pragma unroll
      for (int q = 0; q < 16; ++q) z1[cb * 16 + q] = dsilu(z1[cb * 16 + q]) * g[q];
    }
    // ---- the gradients of W3, b3, W2, b2 on the tensor cores, accumulated over the CTA's tiles
    if (!run_mma(S, S.Awg, TM, S.Bwg, WG_N, TM / 16, S.tmem_base + C_WG, IDESC_WG, !first, phase)) {
      abandoned = true;
      break;
    }
    first = false;
    // ---- the gradients of W1, b1, W4, b4 (FP32): sums over the tile's samples
    {
#pragma unroll
      for (int i = 0; i < HID * NIN / TM; ++i) {
        const int e = s + TM * i, j = e / NIN, k = e % NIN;
        float acc = 0.f;
        for (int r = 0; r < TM; ++r) acc = fmaf(S.Z1[r * LDF + j], S.Xs[r * NIN + k], acc);
        S.gW1[e] += acc;
      }
      if (s < HID) {
        float bs = 0.f;
        for (int r = 0; r < TM; ++r) bs += S.Z1[r * LDF + s];
        S.gb1[s] += bs;
      }
      const int i = s / HID, k = s % HID;  // NOUT * HID == TM entries of gW4
      float acc = 0.f;
      for (int r = 0; r < TM; ++r) acc = fmaf(S.Do[r * NOUT + i], S.H3[r * LDF + k], acc);
      S.gW4[s] += acc;
      if (s < NOUT) {
        float bs = 0.f;
        for (int r = 0; r < TM; ++r) bs += S.Do[r * NOUT + s];
        S.gb4[s] += bs;
      }
    }
    __syncthreads();  // the next tile overwrites Z1, H3, Xs, Do
  }
  // ---- write the gradients: weight gradients of the 64 x 64 layers from TMEM, the rest from shared memory
  if (!abandoned && !first) {
    fence_after_sync();
#pragma unroll 1
    for (int cb = 0; cb < HID / 16; ++cb) {
      float g[16];
      // lanes 0..63 (warps 0, 1): row j of the W3 gradient in columns 0..63; lanes 64..127: row j of W2's in 64..127
      const uint32_t col = C_WG + (warp < 2 ? 0u : (uint32_t)HID) + cb * 16;
      tmem_ld16(trow + col, g);
      const int j = s % HID;
      float* dst = grad + (warp < 2 ? OFF_W3 : OFF_W2) + j * HID + cb * 16;
#pragma unroll
      for (int q = 0; q < 16; ++q) atomicAdd(dst + q, g[q]);
    }
    float g[16];
    tmem_ld16(trow + C_WG + 2 * HID, g);  // column 128: the bias gradients
    atomicAdd(grad + (warp < 2 ? OFF_B3 : OFF_B2) + s % HID, g[0]);
  }
  if (!abandoned) {
    for (int e = s; e < HID * NIN; e += TM) atomicAdd(grad + OFF_W1 + e, S.gW1[e]);
    for (int e = s; e < HID; e += TM) atomicAdd(grad + OFF_B1 + e, S.gb1[e]);
    for (int e = s; e < NOUT * HID; e += TM) atomicAdd(grad + OFF_W4 + e, S.gW4[e]);
    if (s < NOUT) atomicAdd(grad + OFF_B4 + s, S.gb4[s]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((s & 31) == 0) atomicAdd(loss, lsum * inv_n);
  }
  // ---- tear-down (uniform: `abandoned` is the same in every thread)
  if (abandoned && s == 0) {
    mbar_wait(smem_addr(&S.mbar), phase ^ 1u);  // the MMA still in flight, bounded
    atomicAdd(abandon, 1.f);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem_base), "r"(TMEM_COLS) : "memory");
}

}  // namespace

constexpr size_t kTrainTcSmem = sizeof(TrainSmem);
static_assert(kTrainTcSmem <= 227 * 1024, "tensor-core training tile exceeds shared memory");

cudaError_t launch_train_tc(const MlpPtrs& m, long long n, const float* X, const float* T, float aux, float* loss,
                            cudaStream_t s) {
  // loss[1] of the workspace counts CTAs that gave up on a tensor-core wait
  static int attr_dev = -1;
  int dev = 0, sms = 152;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (attr_dev != dev) {
    e = cudaFuncSetAttribute(k_mlp_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainTcSmem);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long tiles = (n + TM - 1) / TM;
  const int grid = (int)(tiles < sms ? tiles : sms);  // one CTA per SM: each allocates all 512 TMEM columns
  k_mlp_train_tc<<<grid, TM, kTrainTcSmem, s>>>(n, X, T, m.w, m.norm, m.grad, loss, m.loss + 1, aux);
  return cudaGetLastError();
}

}  // namespace mlp
}  // namespace grmhd
