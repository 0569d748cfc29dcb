// Passive scalar (Sec. 2.1: (X rho u^mu)_{;mu} = S, the electron fraction Y_e being the paper's use; S = 0
// without radiation). Conserved sqrt(gamma) D X (three double slots paired with the U slots), primitive X
// (ghosted, in the storage type of P). The face flux of sqrt(gamma) D X is the stage's face mass flux
// (component 0 of F^d, after the Riemann solver) times X reconstructed, with the stage's reconstruction,
// on the upwind side of that flux; the update takes the stage's RK weights, and X = DX / (sqrt(gamma) D)
// with the stage's final densitized D (a density floor dilutes X; D X stays conserved). The fluid kernels
// are untouched: the scalar runs in two light kernels after the stage's cell passes.
#pragma once

#include <algorithm>

#include "grmhd_kernels.cuh"
#include "grmhd_launch.h"

namespace grmhd {

// Face fluxes of sqrt(gamma) D X through the d-faces of the interior, in runs of kRun consecutive faces
// along d: face f (0 <= f <= n_d) is the lower d-face of cell f and sits between cells f - 1 and f. A
// thread slides a 6-cell window along its run and reconstructs each cell once (both faces): the face's
// left value is the previous cell's upper face, its right value this cell's lower face.
// Grid: x over (run, transverse a) in 32-bit indices, y over transverse b; for d = y, z the x direction of
// the mesh is the fastest index (coalesced loads), for d = x the run index is.
constexpr int kRun = 16;

// One run: the unit (u, v) of the x index and c2 of the grid (see k_scalar_flux).
template <class R, class T, int RECON>
__device__ __forceinline__ void scalar_flux_run(const T* __restrict__ X, const R* __restrict__ F, R* __restrict__ FX,
                                                const DevParams& p, int d, int u, int v, int c2) {
  const int n[3] = {p.nx, p.ny, p.nz};
  const long long st = d == 0 ? 1 : (d == 1 ? (long long)p.gx : (long long)p.gx * p.gy);
  const R eps = par<R>(p.weno_eps, p.fweno_eps);
  int c[3], r;
  if (d == 0) { r = u; c[1] = v; c[2] = c2; c[0] = 0; }
  else if (d == 1) { c[0] = u; r = v; c[2] = c2; c[1] = 0; }
  else { c[0] = u; r = v; c[1] = c2; c[2] = 0; }
  const int f0 = r * kRun;
  const int f1 = min(f0 + kRun, n[d] + 1);
  c[d] = f0;
  long long g = gidx(p, c[0], c[1], c[2]);  // lower face of cell f0
  R w[6];
#pragma unroll
  for (int q = 0; q < 5; ++q) w[q] = R(X[g + (q - 3) * st]);  // cells f0-3 .. f0+1
  R qm, qp;
  recon_cell<R, RECON>(w[0], w[1], w[2], w[3], w[4], eps, qm, qp);  // cell f0 - 1
  R XL = qp;
  for (int f = f0; f < f1; ++f, g += st) {
    w[5] = R(X[g + 2 * st]);  // cell f + 2
    recon_cell<R, RECON>(w[1], w[2], w[3], w[4], w[5], eps, qm, qp);  // cell f
    const R mdot = F[g];  // component 0 (mass) of the face flux
    FX[g] = mdot * (mdot >= R(0) ? XL : qm);
    XL = qp;
#pragma unroll
    for (int q = 0; q < 5; ++q) w[q] = w[q + 1];
  }
}

// (fast, slow) extents of the x index of the run grid: d = 0: (runs, ny), with z on the grid's y; d = 1:
// (nx, runs), z on y; d = 2: (nx, runs), y on y.
__device__ __forceinline__ void scalar_run_extents(const DevParams& p, int d, int& a_fast, int& a_slow, int& nc2) {
  const int n[3] = {p.nx, p.ny, p.nz};
  const int nrun = (n[d] + 1 + kRun - 1) / kRun;
  a_fast = d == 0 ? nrun : n[0];
  a_slow = d == 0 ? n[1] : nrun;
  nc2 = d == 2 ? n[1] : n[2];
}

template <class R, class T, int RECON>
__global__ void __launch_bounds__(256) k_scalar_flux(const T* __restrict__ X, const R* __restrict__ F,
                                                     R* __restrict__ FX, DevParams p, int d) {
  int a_fast, a_slow, nc2;
  scalar_run_extents(p, d, a_fast, a_slow, nc2);
  const int total = a_fast * a_slow;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x)
    scalar_flux_run<R, T, RECON>(X, F, FX, p, d, t % a_fast, t / a_fast, (int)blockIdx.y);
}

// Batched: grid y over the blocks, x over all runs of the block (grid-stride).
template <class R, class T, int RECON>
__global__ void __launch_bounds__(256) k_batch_scalar_flux(const BlockDesc* __restrict__ blocks, int d) {
  const BlockDesc& B = blocks[blockIdx.y];
  int a_fast, a_slow, nc2;
  scalar_run_extents(B.p, d, a_fast, a_slow, nc2);
  const int plane = a_fast * a_slow, total = plane * nc2;
  const T* X = (const T*)B.X;
  const R* F = (const R*)B.F[d];
  R* FX = (R*)B.FX + (long long)d * B.p.gsize;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int w = t % plane;
    scalar_flux_run<R, T, RECON>(X, F, FX, B.p, d, w % a_fast, w / a_fast, t / plane);
  }
}

// DXnew = g0 DX0 + g1 DXcur + beta dt (-div FX) in double; X = DXnew / D (Unew component 0) on the interior,
// in the storage type of X. Grid: x over the cells of an xy-plane, y over z.
template <class R, class T>
__device__ __forceinline__ void scalar_update_cell(T* __restrict__ X, const R* __restrict__ FX,
                                                   const double* __restrict__ DX0, const double* __restrict__ DXcur,
                                                   double* __restrict__ DXnew, const double* __restrict__ Unew,
                                                   const DevParams& p, const StageArgs& a, double bdt, int i, int j,
                                                   int k) {
  const long long G = p.gsize, sy = p.gx, sz = (long long)p.gx * p.gy;
  const long long t = i + (long long)p.nx * (j + (long long)p.ny * k);
  const long long g = gidx(p, i, j, k);
  const R* Fx = FX;
  const R* Fy = FX + G;
  const R* Fz = FX + 2 * G;
  const R div = (Fx[g + 1] - Fx[g]) * par<R>(p.idx[0], p.fidx[0]) + (Fy[g + sy] - Fy[g]) * par<R>(p.idx[1], p.fidx[1]) +
                (Fz[g + sz] - Fz[g]) * par<R>(p.idx[2], p.fidx[2]);
  double u = a.g1 * DXcur[t];
  if (a.g0 != 0.0) u += a.g0 * DX0[t];
  const double dxn = u + bdt * (double)(-div);
  DXnew[t] = dxn;
  if constexpr (sizeof(T) == sizeof(float)) {
    // mixed form: X is stored in float, so divide in float (a double divide is ~10 FP64 issue slots)
    X[g] = (float)dxn / (float)Unew[t];
  } else {
    X[g] = (T)(dxn / Unew[t]);
  }
}

template <class R, class T>
__global__ void __launch_bounds__(256) k_scalar_update(T* __restrict__ X, const R* __restrict__ FX,
                                                       const double* __restrict__ DX0, const double* __restrict__ DXcur,
                                                       double* __restrict__ DXnew, const double* __restrict__ Unew,
                                                       DevParams p, StageArgs a) {
  const double dt = a.use_dev_dt ? *a.dt_dev : a.dt;
  const int plane = p.nx * p.ny;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < plane; q += gridDim.x * blockDim.x)
    scalar_update_cell<R, T>(X, FX, DX0, DXcur, DXnew, Unew, p, a, a.beta * dt, q % p.nx, q / p.nx, (int)blockIdx.y);
}

// Batched: grid y over the blocks, x over the block's cells (grid-stride).
template <class R, class T>
__global__ void __launch_bounds__(256) k_batch_scalar_update(const BlockDesc* __restrict__ blocks, BatchArgs ba) {
  const BlockDesc& B = blocks[blockIdx.y];
  const double dt = ba.use_dev_dt ? *ba.dt_dev : ba.dt;
  StageArgs a{};
  a.g0 = ba.g0;
  a.g1 = ba.g1;
  const int plane = B.p.nx * B.p.ny, total = plane * B.p.nz;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int q = t % plane;
    scalar_update_cell<R, T>((T*)B.X, (const R*)B.FX, B.DX[ba.s0], B.DX[ba.sc], B.DX[ba.dst], B.U[ba.dst], B.p, a,
                             ba.beta * dt, q % B.p.nx, q / B.p.nx, t / plane);
  }
}

// Load X (double, ghosted) into the storage type and form DX = D X on the interior from the densitized D.
template <class T>
__global__ void k_scalar_load(const double* __restrict__ Xd, T* __restrict__ X, const double* __restrict__ U,
                              double* __restrict__ DX, DevParams p) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < p.gsize; t += (long long)gridDim.x * blockDim.x) {
    X[t] = (T)Xd[t];
    const int i = (int)(t % p.gx) - p.ng, j = (int)((t / p.gx) % p.gy) - p.ng, k = (int)(t / ((long long)p.gx * p.gy)) - p.ng;
    if (i >= 0 && i < p.nx && j >= 0 && j < p.ny && k >= 0 && k < p.nz) {
      const long long c = i + (long long)p.nx * (j + (long long)p.ny * k);
      DX[c] = U[c] * (double)(T)Xd[t];
    }
  }
}

template <class T>
__global__ void k_scalar_store(const T* __restrict__ X, double* __restrict__ Xd, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    Xd[t] = (double)X[t];
}

template <class R, class T>
struct ScalarLaunch {
  static cudaError_t flux(const DevParams& p, const void* X, const void* F, void* FX, int d, cudaStream_t s) {
    const int n[3] = {p.nx, p.ny, p.nz};
    const long long nrun = (n[d] + 1 + kRun - 1) / kRun;
    const long long per = d == 0 ? nrun * n[1] : (long long)n[0] * nrun;  // x indices per grid row
    const dim3 grid((unsigned)((per + 255) / 256), (unsigned)(d == 2 ? n[1] : n[2]));
    const T* x = (const T*)X;
    const R* f = (const R*)F;
    R* fx = (R*)FX + (long long)d * p.gsize;
    switch (p.recon) {
      case RECON_CONSTANT: k_scalar_flux<R, T, RECON_CONSTANT><<<grid, 256, 0, s>>>(x, f, fx, p, d); break;
      case RECON_PLM_MINMOD: k_scalar_flux<R, T, RECON_PLM_MINMOD><<<grid, 256, 0, s>>>(x, f, fx, p, d); break;
      case RECON_PLM_MC: k_scalar_flux<R, T, RECON_PLM_MC><<<grid, 256, 0, s>>>(x, f, fx, p, d); break;
      case RECON_WENO5Z: k_scalar_flux<R, T, RECON_WENO5Z><<<grid, 256, 0, s>>>(x, f, fx, p, d); break;
      case RECON_MP5: k_scalar_flux<R, T, RECON_MP5><<<grid, 256, 0, s>>>(x, f, fx, p, d); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  static cudaError_t update(const DevParams& p, void* X, const void* FX, const double* DX0, const double* DXcur,
                            double* DXnew, const double* Unew, const StageArgs& a, cudaStream_t s) {
    const dim3 grid((unsigned)(((long long)p.nx * p.ny + 255) / 256), (unsigned)p.nz);
    k_scalar_update<R, T><<<grid, 256, 0, s>>>((T*)X, (const R*)FX, DX0, DXcur, DXnew, Unew, p, a);
    return cudaGetLastError();
  }
  static cudaError_t load(const DevParams& p, const double* Xd, void* X, const double* U, double* DX, cudaStream_t s) {
    k_scalar_load<T><<<grid_for(p.gsize, 256), 256, 0, s>>>(Xd, (T*)X, U, DX, p);
    return cudaGetLastError();
  }
  static cudaError_t store(const DevParams& p, const void* X, double* Xd, cudaStream_t s) {
    k_scalar_store<T><<<grid_for(p.gsize, 256), 256, 0, s>>>((const T*)X, Xd, p.gsize);
    return cudaGetLastError();
  }
  // batched forms: grid y over the blocks (at most 65535), x sized for the largest block
  static cudaError_t batch_flux(const BlockDesc* b, int nblocks, long long max_units, int recon, int d, cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    const dim3 grid((unsigned)std::min<long long>((max_units + 255) / 256, 4096), (unsigned)nblocks);
    switch (recon) {
      case RECON_CONSTANT: k_batch_scalar_flux<R, T, RECON_CONSTANT><<<grid, 256, 0, s>>>(b, d); break;
      case RECON_PLM_MINMOD: k_batch_scalar_flux<R, T, RECON_PLM_MINMOD><<<grid, 256, 0, s>>>(b, d); break;
      case RECON_PLM_MC: k_batch_scalar_flux<R, T, RECON_PLM_MC><<<grid, 256, 0, s>>>(b, d); break;
      case RECON_WENO5Z: k_batch_scalar_flux<R, T, RECON_WENO5Z><<<grid, 256, 0, s>>>(b, d); break;
      case RECON_MP5: k_batch_scalar_flux<R, T, RECON_MP5><<<grid, 256, 0, s>>>(b, d); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  static cudaError_t batch_update(const BlockDesc* b, int nblocks, long long max_cells, const BatchArgs& a,
                                  cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    const dim3 grid((unsigned)std::min<long long>((max_cells + 255) / 256, 4096), (unsigned)nblocks);
    k_batch_scalar_update<R, T><<<grid, 256, 0, s>>>(b, a);
    return cudaGetLastError();
  }
  static cudaError_t ghost(const DevParams& p, void* X, cudaStream_t s) {
    k_ghost_periodic<T, 1><<<grid_for(p.gsize, 256), 256, 0, s>>>((T*)X, p);
    return cudaGetLastError();
  }
};

}  // namespace grmhd
