// Device code shared by the learned con2prim guess (grmhd_mlp.cu) and its training kernel
// (grmhd_mlp_train.cu): network layout, workspace layout, features and the per-sample forward pass.
// The network is an 8 -> 64 -> 64 -> 64 -> 2 multilayer perceptron with SiLU activations, BF16 weights
// and FP32 arithmetic; its inputs are eight functions of the invariants of the Kastaun master function
// (q = tau/D, r^2 = S^2/D^2, b^2 = B^2/D, (r.b)^2) and of the intermediates at the bracket end mu_+
// (Sec. 3.1), its outputs y0 = -ln(1 - mu/mu_+) and y1 = ln W at the root mu = 1/(h W).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/grmhd.h"
#include "grmhd_device.cuh"

namespace grmhd {
namespace mlp {

constexpr int NIN = 8, HID = 64, NOUT = 2;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + HID * NIN, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID,
              OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID * HID, OFF_W4 = OFF_B3 + HID, OFF_B4 = OFF_W4 + NOUT * HID,
              NPARAM = OFF_B4 + NOUT;
static_assert(NPARAM == GRMHD_MLP_NPARAM, "parameter count");
static_assert(OFF_W2 % 4 == 0 && OFF_W3 % 4 == 0 && OFF_W4 % 4 == 0, "16-byte aligned weight rows");
constexpr int NNORM = 2 * NIN + 2 * NOUT;  // mean_x, invstd_x, mean_y, std_y
static_assert(NNORM == GRMHD_MLP_NNORM, "standardisation length");
constexpr int TILE = 128;                  // samples per training tile (= threads per training block)
constexpr int LD = HID + 1;                // padded activation row: conflict-free per-sample rows
constexpr float Y0_MAX = 30.f;
constexpr float EPS_P_MIN = 1e-30f;
constexpr int GUESS_MAX_ITER = 8;    // Newton iterations from the network's start before the fallback

// Workspace layout: FP32 master weights, Adam moments, gradient, standardisation, loss, BF16 weights.
constexpr size_t WS_MASTER = 0, WS_M = WS_MASTER + NPARAM, WS_V = WS_M + NPARAM, WS_GRAD = WS_V + NPARAM,
                 WS_NORM = WS_GRAD + NPARAM, WS_LOSS = WS_NORM + NNORM, WS_FLOATS = WS_LOSS + 4;
constexpr size_t WS_BF16_OFF = ((WS_FLOATS * 4 + 255) / 256) * 256;
constexpr size_t WS_BYTES = WS_BF16_OFF + ((NPARAM * 2 + 255) / 256) * 256;

struct MlpPtrs {
  float *master, *m, *v, *grad, *norm, *loss;
  __nv_bfloat16* w;
};

inline MlpPtrs ptrs(const void* ws) {
  float* f = (float*)ws;
  MlpPtrs p;
  p.master = f + WS_MASTER;
  p.m = f + WS_M;
  p.v = f + WS_V;
  p.grad = f + WS_GRAD;
  p.norm = f + WS_NORM;
  p.loss = f + WS_LOSS;
  p.w = (__nv_bfloat16*)((char*)ws + WS_BF16_OFF);
  return p;
}

__device__ __forceinline__ float sigm(float z) { return 1.f / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu(float z) { return z * sigm(z); }
// The activations h1, h2 that feed the two 64 x 64 layers are rounded to BF16 in every forward pass
// (they are the tensor-core operands of the fused kernel; training and the FP32-core path round alike).
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float dsilu(float z) {
  const float s = sigm(z);
  return s * (1.f + z * (1.f - s));
}

// Raw features (FP32) from the master-function invariants and the bracket end mu_+: six functions of
// q, r^2, b^2, (r.b)^2 and, from the intermediates at mu_+ (FP64), ln(eps)/10 and ln W. eps(mu_+) is the
// thermal content that fixes how close the root lies to mu_+ (zero exactly in the cold limit).
__device__ __forceinline__ void raw_features(const C2PIn<double>& c, double mup, float x[NIN]) {
  const C2PEval<double> e = c2p_master_value(c, mup);  // eps clamped at 0 as in the solve
  const float q = fmaxf((float)c.q, 0.f), r2 = (float)c.r2, b2 = (float)c.b2, rb2 = (float)c.rb2;
  x[0] = log1pf(q);
  x[1] = 0.5f * log1pf(r2);
  x[2] = 0.5f * log1pf(b2);
  x[3] = 0.25f * log1pf(rb2);
  x[4] = sqrtf(r2) / (1.f + q);
  x[5] = b2 / (1.f + q);
  x[6] = 0.1f * logf(fmaxf((float)e.eps, EPS_P_MIN));
  x[7] = logf((float)e.W);
}

// Invariants of a flat-space conserved state U [8][n] at t (false: bad input).
__device__ __forceinline__ bool flat_invariants(const DevParams& p, const double* __restrict__ U, long long n,
                                                long long t, double Uc[NV], C2PIn<double>& c, double ru[3],
                                                double bu[3]) {
  Metric<double> m;
  metric_at<double, MINKOWSKI>(p, 0.0, 0.0, 0.0, m);
#pragma unroll
  for (int q = 0; q < NV; ++q) Uc[q] = U[q * n + t];
  return c2p_setup<double>(p, m, Uc, c, ru, bu) == 0;
}

__device__ __forceinline__ void load_weights(float* Ws, float* normS, const __nv_bfloat16* __restrict__ w,
                                             const float* __restrict__ norm) {
  for (int e = threadIdx.x; e < NPARAM; e += blockDim.x) Ws[e] = __bfloat162float(w[e]);
  for (int e = threadIdx.x; e < NNORM; e += blockDim.x) normS[e] = norm[e];
  __syncthreads();
}

// One dense layer for one sample, 4 outputs at a time (independent FMA chains), rows of W 16-byte aligned.
template <int K>
__device__ __forceinline__ void dense_regs(const float* __restrict__ W, const float* __restrict__ b, const float in[K],
                                           float out[HID], bool act) {
#pragma unroll
  for (int j = 0; j < HID; j += 4) {
    float a0 = b[j], a1 = b[j + 1], a2 = b[j + 2], a3 = b[j + 3];
#pragma unroll
    for (int k = 0; k < K; k += 4) {
      const float4 w0 = *reinterpret_cast<const float4*>(W + (j + 0) * K + k);
      const float4 w1 = *reinterpret_cast<const float4*>(W + (j + 1) * K + k);
      const float4 w2 = *reinterpret_cast<const float4*>(W + (j + 2) * K + k);
      const float4 w3 = *reinterpret_cast<const float4*>(W + (j + 3) * K + k);
      a0 = fmaf(w0.w, in[k + 3], fmaf(w0.z, in[k + 2], fmaf(w0.y, in[k + 1], fmaf(w0.x, in[k], a0))));
      a1 = fmaf(w1.w, in[k + 3], fmaf(w1.z, in[k + 2], fmaf(w1.y, in[k + 1], fmaf(w1.x, in[k], a1))));
      a2 = fmaf(w2.w, in[k + 3], fmaf(w2.z, in[k + 2], fmaf(w2.y, in[k + 1], fmaf(w2.x, in[k], a2))));
      a3 = fmaf(w3.w, in[k + 3], fmaf(w3.z, in[k + 2], fmaf(w3.y, in[k + 1], fmaf(w3.x, in[k], a3))));
    }
    out[j] = act ? silu(a0) : a0;
    out[j + 1] = act ? silu(a1) : a1;
    out[j + 2] = act ? silu(a2) : a2;
    out[j + 3] = act ? silu(a3) : a3;
  }
}

// One dense layer + SiLU for one sample with its activations in a shared-memory row `act` (padded
// stride LD per thread: conflict-free): inputs are read into registers, then the outputs overwrite the
// row four at a time. The loop over output groups stays rolled so that the code fits the instruction
// cache (a fully unrolled 64 x 64 layer does not).
template <int K, bool ROUND>
__device__ __forceinline__ void dense_row(const float* __restrict__ W, const float* __restrict__ b, float* act) {
  float in[K];
#pragma unroll
  for (int k = 0; k < K; ++k) in[k] = act[k];
#pragma unroll 1
  for (int j = 0; j < HID; j += 4) {
    float a0 = b[j], a1 = b[j + 1], a2 = b[j + 2], a3 = b[j + 3];
#pragma unroll
    for (int k = 0; k < K; k += 4) {
      const float4 w0 = *reinterpret_cast<const float4*>(W + (j + 0) * K + k);
      const float4 w1 = *reinterpret_cast<const float4*>(W + (j + 1) * K + k);
      const float4 w2 = *reinterpret_cast<const float4*>(W + (j + 2) * K + k);
      const float4 w3 = *reinterpret_cast<const float4*>(W + (j + 3) * K + k);
      a0 = fmaf(w0.w, in[k + 3], fmaf(w0.z, in[k + 2], fmaf(w0.y, in[k + 1], fmaf(w0.x, in[k], a0))));
      a1 = fmaf(w1.w, in[k + 3], fmaf(w1.z, in[k + 2], fmaf(w1.y, in[k + 1], fmaf(w1.x, in[k], a1))));
      a2 = fmaf(w2.w, in[k + 3], fmaf(w2.z, in[k + 2], fmaf(w2.y, in[k + 1], fmaf(w2.x, in[k], a2))));
      a3 = fmaf(w3.w, in[k + 3], fmaf(w3.z, in[k + 2], fmaf(w3.y, in[k + 1], fmaf(w3.x, in[k], a3))));
    }
    act[j] = ROUND ? bf16r(silu(a0)) : silu(a0);
    act[j + 1] = ROUND ? bf16r(silu(a1)) : silu(a1);
    act[j + 2] = ROUND ? bf16r(silu(a2)) : silu(a2);
    act[j + 3] = ROUND ? bf16r(silu(a3)) : silu(a3);
  }
}

// Forward pass of one sample (weights in shared memory as float; `act` the sample's activation row of
// LD floats in shared memory); raw features in, raw outputs out.
__device__ __forceinline__ void forward_one(const float* __restrict__ Ws, const float* __restrict__ normS, float* act,
                                            const float xin[NIN], float y[NOUT]) {
#pragma unroll
  for (int k = 0; k < NIN; ++k) act[k] = (xin[k] - normS[k]) * normS[NIN + k];
  dense_row<NIN, true>(Ws + OFF_W1, Ws + OFF_B1, act);   // h1 (BF16)
  dense_row<HID, true>(Ws + OFF_W2, Ws + OFF_B2, act);   // h2 (BF16)
  dense_row<HID, false>(Ws + OFF_W3, Ws + OFF_B3, act);  // h3
  float h[HID];
#pragma unroll
  for (int k = 0; k < HID; ++k) h[k] = act[k];
#pragma unroll
  for (int i = 0; i < NOUT; ++i) {
    float acc = Ws[OFF_B4 + i];
#pragma unroll
    for (int k = 0; k < HID; ++k) acc = fmaf(Ws[OFF_W4 + i * HID + k], h[k], acc);
    y[i] = acc * normS[2 * NIN + NOUT + i] + normS[2 * NIN + i];
  }
}

// forward kernels: weights, standardisation, one activation row of LD floats per thread (128 threads)
constexpr int FWD_ACT_OFF = NPARAM + 2 + NNORM;
constexpr size_t kForwardSmem = (FWD_ACT_OFF + 128 * LD) * sizeof(float);
constexpr size_t kTrainSmem = (2 * (NPARAM + 2) + NNORM + TILE * NIN + 4 * TILE * LD + TILE * NOUT) * sizeof(float);
static_assert(kTrainSmem <= 227 * 1024, "training tile exceeds shared memory");

// Forward + backward of one batch into the workspace gradient; loss added to *loss (device).
// The same gradient with the 64 x 64 products and weight gradients on the tensor cores (grmhd_mlp_train_tc.cu);
// the back-propagated deltas are rounded to BF16 where they enter a product. m.loss[1] counts abandoned CTAs.
cudaError_t launch_train_tc(const MlpPtrs& m, long long n, const float* X, const float* T, float aux, float* loss,
                            cudaStream_t s);
cudaError_t launch_train(const MlpPtrs& m, long long n, const float* X, const float* T, float aux, float* loss,
                         cudaStream_t s);

}  // namespace mlp
}  // namespace grmhd
