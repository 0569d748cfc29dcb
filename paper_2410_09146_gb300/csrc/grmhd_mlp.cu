// Learned initial guess for con2prim: evaluation of the network, Adam, weight I/O, and the guided
// con2prim batch (the training kernel is in grmhd_mlp_train.cu).
//
// The guided con2prim starts the safeguarded Newton iteration of the Kastaun master function
// (Sec. 3.1) at mu_0 = mu_+ (1 - e^{-y0}) instead of the standard mu_+/2; the iteration keeps the full
// bracket (0, mu_+], and when it has not converged after a few iterations the solve restarts from the
// standard start, so a poor guess costs iterations, never the root.
#include <cmath>
#include <cstdio>

#include "grmhd_launch.h"
#include "grmhd_mlp.cuh"

namespace grmhd {
char* create_error_buffer();
}

namespace {

using namespace grmhd;
using namespace grmhd::mlp;

// Network outputs for raw features X [n][8] -> Y [n][2].
__global__ void __launch_bounds__(128) k_mlp_forward(long long n, const float* __restrict__ X, float* __restrict__ Y,
                                                     const __nv_bfloat16* __restrict__ w,
                                                     const float* __restrict__ norm) {
  extern __shared__ __align__(16) float sm[];
  float* Ws = sm;
  float* normS = sm + NPARAM + 2;
  load_weights(Ws, normS, w, norm);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    float x[NIN], y[NOUT];
#pragma unroll
    for (int k = 0; k < NIN; ++k) x[k] = X[t * NIN + k];
    forward_one(Ws, normS, sm + FWD_ACT_OFF + threadIdx.x * LD, x, y);
    Y[t * NOUT] = y[0];
    Y[t * NOUT + 1] = y[1];
  }
}

// The network's start for flat-space conserved states U [8][n]: guess[t] = mu_0 = mu_+ (1 - e^{-y0})
// and guess[n + t] = mu_+ (both double). Bad states get mu_0 = mu_+ = 0 (the solve flags them).
__global__ void __launch_bounds__(128) k_mlp_guess(long long n, const double* __restrict__ U,
                                                   double* __restrict__ guess, DevParams p,
                                                   const __nv_bfloat16* __restrict__ w,
                                                   const float* __restrict__ norm) {
  extern __shared__ __align__(16) float sm[];
  float* Ws = sm;
  float* normS = sm + NPARAM + 2;
  load_weights(Ws, normS, w, norm);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double Uc[NV], ru[3], bu[3];
    C2PIn<double> c;
    double mu0 = 0.0, mup = 0.0;
    if (flat_invariants(p, U, n, t, Uc, c, ru, bu)) {
      mup = c2p_mu_plus_fast(c);
      float x[NIN], y[NOUT];
      raw_features(c, mup, x);
      forward_one(Ws, normS, sm + FWD_ACT_OFF + threadIdx.x * LD, x, y);
      const float y0 = fminf(fmaxf(y[0], 0.f), Y0_MAX);  // NaN -> 0 -> mu_0 = 0 -> fallback
      mu0 = mup - mup * (double)__expf(-y0);
    }
    guess[t] = mu0;
    guess[n + t] = mup;
  }
}

// Adam on the FP32 master weights; refreshes the BF16 copy and clears the gradient. The learning rate
// and the bias corrections c1 = 1 - b1^step, c2 = 1 - b2^step come from the host.
__global__ void k_mlp_adam(float* master, float* m, float* v, float* grad, __nv_bfloat16* w, float lr, float b1,
                           float b2, float eps, float c1, float c2) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NPARAM) return;
  const float g = grad[e];
  const float mm = b1 * m[e] + (1.f - b1) * g;
  const float vv = b2 * v[e] + (1.f - b2) * g * g;
  m[e] = mm;
  v[e] = vv;
  const float nw = master[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  master[e] = nw;
  w[e] = __float2bfloat16_rn(nw);
  grad[e] = 0.f;
}

__global__ void k_mlp_refresh(const float* master, __nv_bfloat16* w) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < NPARAM) w[e] = __float2bfloat16_rn(master[e]);
}

// Flat-space con2prim batch with the standard start mu_+/2 (guess == NULL) or the network's start
// (guess [2][n] = (mu_0, mu_+) from k_mlp_guess): at most GUESS_MAX_ITER Newton iterations from mu_0,
// then, if they did not converge (or mu_0 is not inside (0, mu_+)), the standard start with the full
// iteration budget. Optionally records the features X [n][8] and the targets T [n][2] of the solved
// states (y0 = -ln(1 - mu/mu_+) clipped to [0, 30], y1 = ln W at the root): training pairs.
// stats: [0] iterations (all attempts), [4] not converged, [7] fallbacks to the standard start.
__global__ void __launch_bounds__(128) k_c2p_guided(const double* __restrict__ U, double* __restrict__ P,
                                                    uint8_t* __restrict__ status, int* __restrict__ iters_out,
                                                    long long n, DevParams p, const double* __restrict__ guess,
                                                    float* __restrict__ X, float* __restrict__ T,
                                                    unsigned long long* stats) {
  unsigned int it_sum = 0, nconv = 0, nfall = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const unsigned lanes = __activemask();  // each of these lanes reaches the __syncwarp below once
    double Uc[NV], ru[3], bu[3], Pn[NV];
    C2PIn<double> c;
    int st = 0, iters = 0;
    const bool good = flat_invariants(p, U, n, t, Uc, c, ru, bu);
    double mup = 0.0, mu = 0.0;
    if (good) {
      bool done = false;
      if (guess) {
        mu = guess[t];
        mup = guess[n + t];
        if (mu > 0.0 && mu < mup) {
          done = c2p_newton<double>(c, mup, mu, p.c2p_tol, GUESS_MAX_ITER, iters, true) == 0;
        }
        if (!done) ++nfall;
      } else {
        mup = c2p_mu_plus_fast(c);
      }
      if (!done) {
        mu = 0.5 * mup;
        st = c2p_newton<double>(c, mup, mu, p.c2p_tol, p.c2p_max_iter, iters, true);
      }
      if (st) ++nconv;
    }
    __syncwarp(lanes);  // iterations of different lengths: run the output once per warp
    if (!good) {
      c2p_bad_output(Uc, Pn);
      st = ST_BAD_INPUT;
      if (X)
        for (int k = 0; k < NIN; ++k) X[t * NIN + k] = 0.f;
      if (T) T[t * NOUT] = T[t * NOUT + 1] = 0.f;
    } else {
      c2p_output(c, mu, ru, bu, Uc, Pn);
      if (X) {
        float x[NIN];
        raw_features(c, mup, x);
#pragma unroll
        for (int k = 0; k < NIN; ++k) X[t * NIN + k] = x[k];
      }
      if (T) {
        const double ratio = fmin(mu / mup, 1.0);
        const double y0 = ratio >= 1.0 ? (double)Y0_MAX : fmin(-log1p(-ratio), (double)Y0_MAX);
        const C2PEval<double> e = c2p_master_value(c, mu);
        T[t * NOUT] = (float)fmax(y0, 0.0);
        T[t * NOUT + 1] = (float)log(e.W);
      }
    }
    Metric<double> m;
    metric_at<double, MINKOWSKI>(p, 0.0, 0.0, 0.0, m);
    st |= apply_floors<MINKOWSKI>(p, m.gam, 1.0, Pn);
#pragma unroll
    for (int q = 0; q < NV; ++q) P[q * n + t] = Pn[q];
    if (status) status[t] = (uint8_t)st;
    if (iters_out) iters_out[t] = iters;
    it_sum += iters;
  }
  if (stats) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      it_sum += __shfl_xor_sync(0xffffffffu, it_sum, o);
      nconv += __shfl_xor_sync(0xffffffffu, nconv, o);
      nfall += __shfl_xor_sync(0xffffffffu, nfall, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(stats + 0, (unsigned long long)it_sum);
      if (nconv) atomicAdd(stats + 4, (unsigned long long)nconv);
      if (nfall) atomicAdd(stats + 7, (unsigned long long)nfall);
    }
  }
}

int fail(int code, const char* msg) {
  snprintf(create_error_buffer(), 256, "%s", msg);
  return code;
}

#define MCK(expr, what)                                                \
  do {                                                                 \
    cudaError_t e_ = (expr);                                           \
    if (e_ != cudaSuccess) {                                           \
      char m_[200];                                                    \
      snprintf(m_, sizeof m_, "%s: %s", what, cudaGetErrorString(e_)); \
      return fail(GRMHD_E_CUDA, m_);                                   \
    }                                                                  \
  } while (0)

cudaError_t smem_attributes() {
  static int attr_dev = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || attr_dev == dev) return e;
  e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kForwardSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_mlp_guess, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kForwardSmem);
  if (e == cudaSuccess) attr_dev = dev;
  return e;
}

void launch_adam(const MlpPtrs& m, double lr, int step, cudaStream_t s) {
  const double b1 = 0.9, b2 = 0.999;
  k_mlp_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(m.master, m.m, m.v, m.grad, m.w, (float)lr, (float)b1, (float)b2,
                                                  1e-8f, (float)(1.0 - pow(b1, step)), (float)(1.0 - pow(b2, step)));
}

bool aligned(const void* ws) { return ((uintptr_t)ws) % 256 == 0; }

}  // namespace

namespace grmhd {
cudaError_t launch_c2p_guided(const double* U, double* P, uint8_t* status, int* iters, long long n,
                              const DevParams& p, const double* guess, float* X, float* T, unsigned long long* stats,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_c2p_guided<<<grid_for(n, 128), 128, 0, s>>>(U, P, status, iters, n, p, guess, X, T, stats);
  return cudaGetLastError();
}

cudaError_t launch_mlp_guess(const void* ws, const double* U, double* guess, long long n, const DevParams& p,
                             cudaStream_t s) {
  cudaError_t e = smem_attributes();
  if (e != cudaSuccess || n <= 0) return e;
  const MlpPtrs m = ptrs(ws);
  k_mlp_guess<<<grid_for(n, 128), 128, kForwardSmem, s>>>(n, U, guess, p, m.w, m.norm);
  return cudaGetLastError();
}
}  // namespace grmhd

extern "C" {

size_t grmhd_mlp_workspace_bytes(void) { return WS_BYTES; }

int grmhd_mlp_set_weights(void* ws, const float* theta, const float* norm, void* stream) {
  if (!ws || !theta || !norm) return fail(GRMHD_E_INVALID, "grmhd_mlp_set_weights: NULL pointer");
  if (!aligned(ws)) return fail(GRMHD_E_WORKSPACE, "grmhd_mlp_set_weights: workspace not 256-byte aligned");
  const cudaStream_t s = (cudaStream_t)stream;
  const MlpPtrs m = ptrs(ws);
  MCK(cudaMemsetAsync(ws, 0, WS_BYTES, s), "clearing the network workspace");
  MCK(cudaMemcpyAsync(m.master, theta, NPARAM * sizeof(float), cudaMemcpyHostToDevice, s), "copying weights");
  MCK(cudaMemcpyAsync(m.norm, norm, NNORM * sizeof(float), cudaMemcpyHostToDevice, s), "copying the standardisation");
  k_mlp_refresh<<<(NPARAM + 255) / 256, 256, 0, s>>>(m.master, m.w);
  MCK(cudaGetLastError(), "converting weights to BF16");
  MCK(cudaStreamSynchronize(s), "synchronising");
  return GRMHD_OK;
}

int grmhd_mlp_get_weights(const void* ws, float* theta, float* theta_bf16, void* stream) {
  if (!ws || !theta) return fail(GRMHD_E_INVALID, "grmhd_mlp_get_weights: NULL pointer");
  const cudaStream_t s = (cudaStream_t)stream;
  const MlpPtrs m = ptrs(ws);
  MCK(cudaMemcpyAsync(theta, m.master, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, s), "copying weights");
  if (theta_bf16) {
    __nv_bfloat16 tmp[NPARAM];
    MCK(cudaMemcpyAsync(tmp, m.w, NPARAM * sizeof(__nv_bfloat16), cudaMemcpyDeviceToHost, s), "copying BF16 weights");
    MCK(cudaStreamSynchronize(s), "synchronising");
    for (int e = 0; e < NPARAM; ++e) theta_bf16[e] = __bfloat162float(tmp[e]);
  }
  MCK(cudaStreamSynchronize(s), "synchronising");
  return GRMHD_OK;
}

int grmhd_mlp_forward(const void* ws, long long n, const float* X, float* Y, void* stream) {
  if (!ws || n < 0 || (n > 0 && (!X || !Y))) return fail(GRMHD_E_INVALID, "grmhd_mlp_forward: bad arguments");
  if (!aligned(ws)) return fail(GRMHD_E_WORKSPACE, "grmhd_mlp_forward: workspace not 256-byte aligned");
  MCK(smem_attributes(), "shared-memory limit");
  if (n == 0) return GRMHD_OK;
  const MlpPtrs m = ptrs(ws);
  k_mlp_forward<<<grid_for(n, 128), 128, kForwardSmem, (cudaStream_t)stream>>>(n, X, Y, m.w, m.norm);
  MCK(cudaGetLastError(), "forward");
  return GRMHD_OK;
}

namespace {
using TrainFn = cudaError_t (*)(const MlpPtrs&, long long, const float*, const float*, float, float*, cudaStream_t);

int mlp_grad(TrainFn fn, void* ws, long long n, const float* X, const float* T, double aux, float* grad, float* loss,
             void* stream) {
  if (!ws || n <= 0 || !X || !T) return fail(GRMHD_E_INVALID, "grmhd_mlp_grad: bad arguments");
  if (!aligned(ws)) return fail(GRMHD_E_WORKSPACE, "grmhd_mlp_grad: workspace not 256-byte aligned");
  const cudaStream_t s = (cudaStream_t)stream;
  const MlpPtrs m = ptrs(ws);
  MCK(cudaMemsetAsync(m.grad, 0, NPARAM * sizeof(float), s), "clearing the gradient");
  MCK(cudaMemsetAsync(m.loss, 0, sizeof(float), s), "clearing the loss");  // loss[1]: timed-out waits, kept
  MCK(fn(m, n, X, T, (float)aux, m.loss, s), "forward + backward");
  float hl[2] = {0.f, 0.f};
  MCK(cudaMemcpyAsync(hl, m.loss, 2 * sizeof(float), cudaMemcpyDeviceToHost, s), "copying");
  if (grad) MCK(cudaMemcpyAsync(grad, m.grad, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, s), "copying");
  MCK(cudaStreamSynchronize(s), "synchronising");
  if (hl[1] != 0.f) {
    MCK(cudaMemset(m.loss + 1, 0, sizeof(float)), "clearing the wait counter");
    return fail(GRMHD_E_CUDA, "grmhd_mlp_grad: a tensor-core wait timed out (this or an earlier tensor-core "
                              "gradient is incomplete)");
  }
  if (loss) *loss = hl[0];
  return GRMHD_OK;
}
}  // namespace

int grmhd_mlp_grad(void* ws, long long n, const float* X, const float* T, double aux, float* grad, float* loss,
                   void* stream) {
  return mlp_grad(launch_train, ws, n, X, T, aux, grad, loss, stream);
}

int grmhd_mlp_grad_tc(void* ws, long long n, const float* X, const float* T, double aux, float* grad, float* loss,
                      void* stream) {
  return mlp_grad(launch_train_tc, ws, n, X, T, aux, grad, loss, stream);
}

int grmhd_mlp_adam(void* ws, double lr, int step, void* stream) {
  if (!ws || step < 1 || !(lr >= 0.0)) return fail(GRMHD_E_INVALID, "grmhd_mlp_adam: bad arguments");
  if (!aligned(ws)) return fail(GRMHD_E_WORKSPACE, "grmhd_mlp_adam: workspace not 256-byte aligned");
  launch_adam(ptrs(ws), lr, step, (cudaStream_t)stream);
  MCK(cudaGetLastError(), "Adam");
  return GRMHD_OK;
}

namespace {
int mlp_train(TrainFn fn, void* ws, long long n, const float* X, const float* T, long long batch, int steps, double lr,
              double lr_end, double aux, int first_step, float* loss_dev, void* stream) {
  if (!ws || n <= 0 || !X || !T || batch <= 0 || steps < 0 || first_step < 1 || !(lr > 0.0) || !(lr_end >= 0.0))
    return fail(GRMHD_E_INVALID, "grmhd_mlp_train: bad arguments");
  if (!aligned(ws)) return fail(GRMHD_E_WORKSPACE, "grmhd_mlp_train: workspace not 256-byte aligned");
  const cudaStream_t s = (cudaStream_t)stream;
  const MlpPtrs m = ptrs(ws);
  if (batch > n) batch = n;
  MCK(cudaMemsetAsync(m.grad, 0, NPARAM * sizeof(float), s), "clearing the gradient");
  MCK(cudaMemsetAsync(m.loss, 0, sizeof(float), s), "clearing the loss");  // loss[1]: timed-out waits, kept
  if (loss_dev && steps > 0)
    MCK(cudaMemsetAsync(loss_dev, 0, (size_t)steps * sizeof(float), s), "clearing the loss history");
  long long off = 0;
  for (int k = 0; k < steps; ++k) {
    if (off + batch > n) off = 0;  // contiguous minibatches of i.i.d. samples, wrapping at the end
    MCK(fn(m, batch, X + off * NIN, T + off * NOUT, (float)aux, loss_dev ? loss_dev + k : m.loss, s),
        "forward + backward");
    off += batch;
    // cosine decay from lr to lr_end over the call
    const double rate = lr_end + 0.5 * (lr - lr_end) * (1.0 + cos(M_PI * (double)k / (double)(steps > 1 ? steps : 1)));
    launch_adam(m, rate, first_step + k, s);
    MCK(cudaGetLastError(), "Adam");
  }
  return GRMHD_OK;
}
}  // namespace

int grmhd_mlp_train(void* ws, long long n, const float* X, const float* T, long long batch, int steps, double lr,
                    double lr_end, double aux, int first_step, float* loss_dev, void* stream) {
  return mlp_train(launch_train, ws, n, X, T, batch, steps, lr, lr_end, aux, first_step, loss_dev, stream);
}

int grmhd_mlp_train_tc(void* ws, long long n, const float* X, const float* T, long long batch, int steps, double lr,
                       double lr_end, double aux, int first_step, float* loss_dev, void* stream) {
  return mlp_train(launch_train_tc, ws, n, X, T, batch, steps, lr, lr_end, aux, first_step, loss_dev, stream);
}

}  // extern "C"
