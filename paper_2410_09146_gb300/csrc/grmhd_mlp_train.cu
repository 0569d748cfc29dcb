// Training kernel of the learned con2prim guess: fused forward + backward over tiles of 128 samples.
#include "grmhd_mlp.cuh"

namespace grmhd {
namespace mlp {
namespace {

// Fused forward + backward over tiles of TILE samples (thread s owns sample s of a tile). The forward
// pass rounds h1 and h2 to BF16 like inference; the backward pass treats the rounding as the identity. Accumulates
// into grad the gradient of L = (1/n) sum_s [(o0 - t0)^2 + aux (o1 - t1)^2] (standardised outputs and
// targets) with respect to the weights as used in the forward pass (the BF16 copy), and L into loss[0].
// T holds raw targets [n][2].
__global__ void __launch_bounds__(TILE, 1) k_mlp_train(long long n, const float* __restrict__ X,
                                                       const float* __restrict__ T, const __nv_bfloat16* __restrict__ w,
                                                       const float* __restrict__ norm, float* __restrict__ grad,
                                                       float* __restrict__ loss, float aux) {
  extern __shared__ __align__(16) float sm[];
  float* Ws = sm;                 // NPARAM
  float* Gs = Ws + NPARAM + 2;    // NPARAM, entry e owned by thread e % TILE
  float* normS = Gs + NPARAM + 2; // NNORM
  float* Xs = normS + NNORM;      // TILE x NIN standardised inputs
  float* A1 = Xs + TILE * NIN;    // z1, later delta1
  float* A2 = A1 + TILE * LD;     // z2, later delta2
  float* A3 = A2 + TILE * LD;     // z3, later delta3
  float* Hb = A3 + TILE * LD;     // activations h1 / h2 / h3 as needed
  float* Do = Hb + TILE * LD;     // TILE x NOUT output deltas
  load_weights(Ws, normS, w, norm);
  const int s = threadIdx.x;
  for (int e = s; e < NPARAM; e += TILE) Gs[e] = 0.f;
  const float inv_n = 1.f / (float)n;
  float lsum = 0.f;
  const int kc = s % HID, jr = s / HID;  // gradient-ownership pattern of the 64x64 layers
  for (long long base = (long long)blockIdx.x * TILE; base < n; base += (long long)gridDim.x * TILE) {
    const long long t = base + s;
    const bool valid = t < n;
    float* xs = Xs + s * NIN;
    float* a1 = A1 + s * LD;
    float* a2 = A2 + s * LD;
    float* a3 = A3 + s * LD;
    float* hb = Hb + s * LD;
    // ---- forward
#pragma unroll
    for (int k = 0; k < NIN; ++k) xs[k] = valid ? (X[t * NIN + k] - normS[k]) * normS[NIN + k] : 0.f;
    {
      float x[NIN], z[HID];
#pragma unroll
      for (int k = 0; k < NIN; ++k) x[k] = xs[k];
      dense_regs<NIN>(Ws + OFF_W1, Ws + OFF_B1, x, z, false);
#pragma unroll
      for (int j = 0; j < HID; ++j) {
        a1[j] = z[j];
        hb[j] = bf16r(silu(z[j]));  // h1
      }
    }
    {
      float h[HID], z[HID];
#pragma unroll
      for (int k = 0; k < HID; ++k) h[k] = hb[k];
      dense_regs<HID>(Ws + OFF_W2, Ws + OFF_B2, h, z, false);
#pragma unroll
      for (int j = 0; j < HID; ++j) {
        a2[j] = z[j];
        h[j] = bf16r(silu(z[j]));  // h2
      }
      dense_regs<HID>(Ws + OFF_W3, Ws + OFF_B3, h, z, false);
#pragma unroll
      for (int j = 0; j < HID; ++j) {
        a3[j] = z[j];
        h[j] = silu(z[j]);
        hb[j] = h[j];  // h3
      }
      float d[NOUT];
#pragma unroll
      for (int i = 0; i < NOUT; ++i) {
        float acc = Ws[OFF_B4 + i];
#pragma unroll
        for (int k = 0; k < HID; ++k) acc = fmaf(Ws[OFF_W4 + i * HID + k], h[k], acc);
        const float wgt = i == 0 ? 1.f : aux;
        const float tt = valid ? (T[t * NOUT + i] - normS[2 * NIN + i]) / normS[2 * NIN + NOUT + i] : 0.f;
        const float e = valid ? acc - tt : 0.f;
        lsum += wgt * e * e;
        d[i] = 2.f * wgt * e * inv_n;
        Do[s * NOUT + i] = d[i];
      }
      // delta3 = dsilu(z3) * W4^T d (own row)
#pragma unroll
      for (int k = 0; k < HID; ++k)
        a3[k] = dsilu(a3[k]) * fmaf(Ws[OFF_W4 + k], d[0], Ws[OFF_W4 + HID + k] * d[1]);
    }
    __syncthreads();
    // ---- gW4[i][k] = sum_r Do[r][i] h3[r][k] (thread s owns entry s), gb4
    {
      const int i = s / HID, k = s % HID;
      float acc = 0.f;
      for (int r = 0; r < TILE; ++r) acc = fmaf(Do[r * NOUT + i], Hb[r * LD + k], acc);
      Gs[OFF_W4 + s] += acc;
      if (s < NOUT) {
        float bs = 0.f;
        for (int r = 0; r < TILE; ++r) bs += Do[r * NOUT + s];
        Gs[OFF_B4 + s] += bs;
      }
    }
    __syncthreads();
    for (int k = 0; k < HID; ++k) hb[k] = bf16r(silu(a2[k]));  // h2
    __syncthreads();
    // ---- gW3[j][k] = sum_r delta3[r][j] h2[r][k]: thread owns column kc, rows jr + 2i; gb3
    {
      float acc[HID / 2];
#pragma unroll
      for (int i = 0; i < HID / 2; ++i) acc[i] = 0.f;
      float bs = 0.f;
      for (int r = 0; r < TILE; ++r) {
        const float h = Hb[r * LD + kc];
        const float* dr = A3 + r * LD;
#pragma unroll
        for (int i = 0; i < HID / 2; ++i) acc[i] = fmaf(dr[jr + 2 * i], h, acc[i]);
        if (s < HID) bs += dr[s];
      }
#pragma unroll
      for (int i = 0; i < HID / 2; ++i) Gs[OFF_W3 + (jr + 2 * i) * HID + kc] += acc[i];
      if (s < HID) Gs[OFF_B3 + s] += bs;
    }
    // delta2 = dsilu(z2) * W3^T delta3 (own row, in place of z2)
#pragma unroll 4
    for (int k = 0; k < HID; ++k) {
      float acc = 0.f;
#pragma unroll 16
      for (int j = 0; j < HID; ++j) acc = fmaf(Ws[OFF_W3 + j * HID + k], a3[j], acc);
      a2[k] = acc * dsilu(a2[k]);
    }
    __syncthreads();
    for (int k = 0; k < HID; ++k) hb[k] = bf16r(silu(a1[k]));  // h1
    __syncthreads();
    // ---- gW2[j][k] = sum_r delta2[r][j] h1[r][k]; gb2
    {
      float acc[HID / 2];
#pragma unroll
      for (int i = 0; i < HID / 2; ++i) acc[i] = 0.f;
      float bs = 0.f;
      for (int r = 0; r < TILE; ++r) {
        const float h = Hb[r * LD + kc];
        const float* dr = A2 + r * LD;
#pragma unroll
        for (int i = 0; i < HID / 2; ++i) acc[i] = fmaf(dr[jr + 2 * i], h, acc[i]);
        if (s < HID) bs += dr[s];
      }
#pragma unroll
      for (int i = 0; i < HID / 2; ++i) Gs[OFF_W2 + (jr + 2 * i) * HID + kc] += acc[i];
      if (s < HID) Gs[OFF_B2 + s] += bs;
    }
    // delta1 = dsilu(z1) * W2^T delta2 (own row, in place of z1)
#pragma unroll 4
    for (int k = 0; k < HID; ++k) {
      float acc = 0.f;
#pragma unroll 16
      for (int j = 0; j < HID; ++j) acc = fmaf(Ws[OFF_W2 + j * HID + k], a2[j], acc);
      a1[k] = acc * dsilu(a1[k]);
    }
    __syncthreads();
    // ---- gW1[j][k] = sum_r delta1[r][j] x[r][k] (thread owns e = s + TILE i), gb1
    {
#pragma unroll
      for (int i = 0; i < HID * NIN / TILE; ++i) {
        const int e = s + TILE * i, j = e / NIN, k = e % NIN;
        float acc = 0.f;
        for (int r = 0; r < TILE; ++r) acc = fmaf(A1[r * LD + j], Xs[r * NIN + k], acc);
        Gs[OFF_W1 + e] += acc;
      }
      if (s < HID) {
        float bs = 0.f;
        for (int r = 0; r < TILE; ++r) bs += A1[r * LD + s];
        Gs[OFF_B1 + s] += bs;
      }
    }
    __syncthreads();
  }
  for (int e = s; e < NPARAM; e += TILE) atomicAdd(grad + e, Gs[e]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if ((s & 31) == 0) atomicAdd(loss, lsum * inv_n);
}

}  // namespace

cudaError_t launch_train(const MlpPtrs& m, long long n, const float* X, const float* T, float aux, float* loss,
                         cudaStream_t s) {
  static int attr_dev = -1;
  int dev = 0, sms = 152;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (attr_dev != dev) {
    e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long tiles = (n + TILE - 1) / TILE;
  const int grid = (int)(tiles < sms ? tiles : sms);
  k_mlp_train<<<grid, TILE, kTrainSmem, s>>>(n, X, T, m.w, m.norm, m.grad, loss, aux);
  return cudaGetLastError();
}

}  // namespace mlp
}  // namespace grmhd
