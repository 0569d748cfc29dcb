// Passive scalar (Sec. 2.1: (X rho u^mu)_{;mu} = S, the electron fraction Y_e being the paper's use; S = 0
// without radiation). Conserved sqrt(gamma) D X (three double slots paired with the U slots), primitive X
// (ghosted, in the storage type of P). The face flux of sqrt(gamma) D X is the stage's face mass flux
// (component 0 of F^d, after the Riemann solver) times X reconstructed, with the stage's reconstruction,
// on the upwind side of that flux; the update takes the stage's RK weights, and X = DX / (sqrt(gamma) D)
// with the stage's final densitized D (a density floor dilutes X; D X stays conserved). The fluid kernels
// are untouched: the scalar runs in two light kernels after the stage's cell passes.
#pragma once

#include "grmhd_kernels.cuh"
#include "grmhd_launch.h"

namespace grmhd {

// Face flux of sqrt(gamma) D X through the d-faces of the interior: face (i, j, k), i along d in [0, n_d],
// is the lower d-face of ghosted cell (i, j, k) and sits between cells c - e_d and c.
template <class R, class T, int RECON>
__global__ void __launch_bounds__(256) k_scalar_flux(const T* __restrict__ X, const R* __restrict__ F,
                                                     R* __restrict__ FX, DevParams p, int d) {
  const int n[3] = {p.nx, p.ny, p.nz};
  int m[3] = {n[0], n[1], n[2]};
  m[d] = n[d] + 1;
  const long long nf = (long long)m[0] * m[1] * m[2];
  const long long st = d == 0 ? 1 : (d == 1 ? (long long)p.gx : (long long)p.gx * p.gy);
  const R eps = R(p.weno_eps);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nf; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % m[0]), j = (int)((t / m[0]) % m[1]), k = (int)(t / ((long long)m[0] * m[1]));
    const long long g = gidx(p, i, j, k);
    R f[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) f[q] = R(X[g + (q - 3) * st]);  // cells c-3 .. c+2 along d
    R qm, qp, XL, XR;
    recon_cell<R, RECON>(f[0], f[1], f[2], f[3], f[4], eps, qm, qp);  // the cell below the face
    XL = qp;
    recon_cell<R, RECON>(f[1], f[2], f[3], f[4], f[5], eps, qm, qp);  // the cell above it
    XR = qm;
    const R mdot = F[g];  // component 0 (mass) of the face flux
    FX[g] = mdot * (mdot >= R(0) ? XL : XR);
  }
}

// DXnew = g0 DX0 + g1 DXcur + beta dt (-div FX); X = DXnew / D (Unew component 0) on the interior.
template <class R, class T>
__global__ void __launch_bounds__(256) k_scalar_update(T* __restrict__ X, const R* __restrict__ FX,
                                                       const double* __restrict__ DX0, const double* __restrict__ DXcur,
                                                       double* __restrict__ DXnew, const double* __restrict__ Unew,
                                                       DevParams p, StageArgs a) {
  const double dt = a.use_dev_dt ? *a.dt_dev : a.dt;
  const double bdt = a.beta * dt;
  const long long G = p.gsize, sy = p.gx, sz = (long long)p.gx * p.gy;
  const R* Fx = FX;
  const R* Fy = FX + G;
  const R* Fz = FX + 2 * G;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < p.isize; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % p.nx), j = (int)((t / p.nx) % p.ny), k = (int)(t / ((long long)p.nx * p.ny));
    const long long g = gidx(p, i, j, k);
    const R div = (Fx[g + 1] - Fx[g]) * R(p.idx[0]) + (Fy[g + sy] - Fy[g]) * R(p.idx[1]) +
                  (Fz[g + sz] - Fz[g]) * R(p.idx[2]);
    double u = a.g1 * DXcur[t];
    if (a.g0 != 0.0) u += a.g0 * DX0[t];
    const double dxn = u + bdt * (double)(-div);
    DXnew[t] = dxn;
    X[g] = (T)(dxn / Unew[t]);
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
    long long nf = (long long)p.nx * p.ny * p.nz / (d == 0 ? p.nx : (d == 1 ? p.ny : p.nz)) *
                   ((d == 0 ? p.nx : (d == 1 ? p.ny : p.nz)) + 1);
    const int grid = grid_for(nf, 256);
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
    k_scalar_update<R, T><<<grid_for(p.isize, 256), 256, 0, s>>>((T*)X, (const R*)FX, DX0, DXcur, DXnew, Unew, p, a);
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
  static cudaError_t ghost(const DevParams& p, void* X, cudaStream_t s) {
    k_ghost_periodic<T, 1><<<grid_for(p.gsize, 256), 256, 0, s>>>((T*)X, p);
    return cudaGetLastError();
  }
};

}  // namespace grmhd
