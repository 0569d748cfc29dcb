// Face-centred constrained transport: the field lives on the faces (the paper names face-centred CT as
// planned work without a scheme; this is the upwind "contact" CT of Gardiner & Stone 2005, J. Comput.
// Phys. 205, 509). Layouts (x fastest, entry (i,j,k) of component d is the lower d-face of ghosted cell
// (i,j,k)):
//   Bf   [3][gz][gy][gx] double  densitized normal field sqrt(gamma) B^d of every face
//   Ecc  [3][gz][gy][gx] R       cell-centred EMFs Omega_c = sqrt(gamma) (B^a v~^b - B^b v~^a), (c, a, b)
//                                cyclic, on cells [-1, n] of every direction
//   E    [3][gz][gy][gx] R       edge EMFs, stored as in flux-CT (component c at the lower corner of cell
//                                (i,j,k) in the two directions transverse to c)
// With that sign, Omega_c = F^b_{B^a} = -F^a_{B^b} for the face fluxes F of the densitized field.
#pragma once

#include "grmhd_kernels.cuh"
#include "grmhd_launch.h"

namespace grmhd {

// Cell-centred EMFs of cell t of the box [-1, nx] x [-1, ny] x [-1, nz], in the flux type R with the
// metric evaluated at the cell centre in R.
template <class R, class T, int METRIC>
__global__ void __launch_bounds__(128) k_emf_cc(const T* __restrict__ P, R* __restrict__ Ecc, DevParams p) {
  const int ex = p.nx + 2, ey = p.ny + 2;
  const long long n = (long long)ex * ey * (p.nz + 2);
  const long long G = p.gsize;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % ex) - 1, j = (int)((t / ex) % ey) - 1, k = (int)(t / ((long long)ex * ey)) - 1;
    const long long g = gidx(p, i, j, k);
    Metric<R> m;
    metric_at<R, METRIC>(p, par<R>(p.x0[0], p.fx0[0]) + (R(i) + R(0.5)) * par<R>(p.dx[0], p.fdx[0]), par<R>(p.x0[1], p.fx0[1]) + (R(j) + R(0.5)) * par<R>(p.dx[1], p.fdx[1]),
                         par<R>(p.x0[2], p.fx0[2]) + (R(k) + R(0.5)) * par<R>(p.dx[2], p.fdx[2]), m);
    R ut[3], B[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      ut[q] = R(P[(1 + q) * G + g]);
      B[q] = R(P[(5 + q) * G + g]);
    }
    R utl[3];
    lower3(m.gam, ut, utl);
    const R W = sqrt(R(1) + ut[0] * utl[0] + ut[1] * utl[1] + ut[2] * utl[2]);
    R vt[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) vt[q] = m.alpha * (ut[q] / W) - m.beta[q];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int a = (c + 1) % 3, b = (c + 2) % 3;
      Ecc[c * G + g] = m.sqrtgam * (B[a] * vt[b] - B[b] * vt[a]);
    }
  }
}

// Edge EMF of component c = the direction not in {a, b} at ghosted index g (its lower corner in a and b),
// with sa, sb the index strides of directions a and b. Four face EMFs around the edge (a-faces below
// and above the edge along b give -F^a_{B^b}, b-faces left and right along a give F^b_{B^a}), plus on
// each of the four half-faces the difference between face and cell-centred EMF in the cell its face's
// mass flux comes from (the mean of both cells when that flux is zero).
template <class R>
__device__ __forceinline__ R emf_upwind_edge(const R* __restrict__ Fa, const R* __restrict__ Fb,
                                             const R* __restrict__ Ec, long long G, long long g, long long sa,
                                             long long sb, int a, int b) {
  const R oa_lo = -Fa[(5 + b) * G + g - sb], oa_hi = -Fa[(5 + b) * G + g];   // a-faces (fa, fb - 1), (fa, fb)
  const R ob_lo = Fb[(5 + a) * G + g - sa], ob_hi = Fb[(5 + a) * G + g];     // b-faces (fa - 1, fb), (fa, fb)
  const R c_mm = Ec[g - sa - sb], c_pm = Ec[g - sb], c_mp = Ec[g - sa], c_pp = Ec[g];  // cells (ia, ib)
  const R da_lo = Fa[g - sb], da_hi = Fa[g];  // mass fluxes through the a-faces
  const R db_lo = Fb[g - sa], db_hi = Fb[g];  // and through the b-faces
  auto pick = [](R m, R lo_cell, R hi_cell) {
    return m > R(0) ? lo_cell : (m < R(0) ? hi_cell : R(0.5) * (lo_cell + hi_cell));
  };
  const R xb_lo = pick(da_lo, ob_lo - c_mm, ob_hi - c_pm);
  const R xb_hi = pick(da_hi, c_mp - ob_lo, c_pp - ob_hi);
  const R xa_lo = pick(db_lo, oa_lo - c_mm, oa_hi - c_mp);
  const R xa_hi = pick(db_hi, c_pm - oa_lo, c_pp - oa_hi);
  return R(0.25) * (oa_lo + oa_hi + ob_lo + ob_hi) + R(0.25) * (xb_lo - xb_hi) + R(0.25) * (xa_lo - xa_hi);
}

// Upwind edge EMFs for edge box index t in [0, nx] x [0, ny] x [0, nz] (the edges flux-CT covers), formed in
// the flux type and stored in double: k_face_update differences them in double, and a conversion here, once
// per edge in a kernel that leaves the FP64 pipe idle, saves four in that FP64-bound kernel (each edge
// bounds four faces); the values are the same bits.
template <class R>
__global__ void __launch_bounds__(128) k_emf_upwind(const R* __restrict__ Fx, const R* __restrict__ Fy,
                                                    const R* __restrict__ Fz, const R* __restrict__ Ecc,
                                                    double* __restrict__ E, DevParams p) {
  const int ex = p.nx + 1, ey = p.ny + 1;
  const long long n = (long long)ex * ey * (p.nz + 1);
  const long long G = p.gsize, sx = 1, sy = p.gx, sz = (long long)p.gx * p.gy;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % ex), j = (int)((t / ex) % ey), k = (int)(t / ((long long)ex * ey));
    const long long g = gidx(p, i, j, k);
    if (i < p.nx) E[g] = (double)emf_upwind_edge<R>(Fy, Fz, Ecc, G, g, sy, sz, 1, 2);               // x: a = y, b = z
    if (j < p.ny) E[G + g] = (double)emf_upwind_edge<R>(Fz, Fx, Ecc + G, G, g, sz, sx, 2, 0);     // y: a = z, b = x
    if (k < p.nz) E[2 * G + g] = (double)emf_upwind_edge<R>(Fx, Fy, Ecc + 2 * G, G, g, sx, sy, 0, 1);  // z: a = x, b = y
  }
}

// Faces of box index t in [0, nx] x [0, ny] x [0, nz] advanced by the discrete Stokes theorem:
//   Bfnew = g0 Bf0 + g1 Bfcur + beta dt curl(E), curl differenced in double (so that the face divergence
//   changes by double roundoff only, whatever the EMF type):
//   x: -dE_z/dy + dE_y/dz,  y: dE_z/dx - dE_x/dz,  z: -dE_y/dx + dE_x/dy.
template <class R>  // the form's flux type (one instance per form; the EMFs are double in both)
__global__ void __launch_bounds__(256) k_face_update(const double* __restrict__ Bf0, const double* __restrict__ Bfc,
                                                     double* __restrict__ Bfn, const double* __restrict__ E,
                                                     StageArgs a, DevParams p) {
  const int ex = p.nx + 1, ey = p.ny + 1;
  const long long n = (long long)ex * ey * (p.nz + 1);
  const long long G = p.gsize, sy = p.gx, sz = (long long)p.gx * p.gy;
  const double dt = a.use_dev_dt ? *a.dt_dev : a.dt;
  const double bdt = a.beta * dt;
  const double cx = bdt * p.idx[0], cy = bdt * p.idx[1], cz = bdt * p.idx[2];  // beta dt / dx_d
  const bool with0 = a.g0 != 0.0;  // uniform: first stages have no step-start term
  const double* Ex = E;
  const double* Ey = E + G;
  const double* Ez = E + 2 * G;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % ex), j = (int)((t / ex) % ey), k = (int)(t / ((long long)ex * ey));
    const long long g = gidx(p, i, j, k);
    const double ez = Ez[g], ey_ = Ey[g], ex_ = Ex[g];
    if (j < p.ny && k < p.nz) {
      double b = a.g1 * Bfc[g] + ((Ey[g + sz] - ey_) * cz - (Ez[g + sy] - ez) * cy);
      if (with0) b += a.g0 * Bf0[g];
      Bfn[g] = b;
    }
    if (i < p.nx && k < p.nz) {
      double b = a.g1 * Bfc[G + g] + ((Ez[g + 1] - ez) * cx - (Ex[g + sz] - ex_) * cz);
      if (with0) b += a.g0 * Bf0[G + g];
      Bfn[G + g] = b;
    }
    if (i < p.nx && j < p.ny) {
      double b = a.g1 * Bfc[2 * G + g] + ((Ex[g + sy] - ex_) * cy - (Ey[g + 1] - ey_) * cx);
      if (with0) b += a.g0 * Bf0[2 * G + g];
      Bfn[2 * G + g] = b;
    }
  }
}

// Cell field from the faces for every ghosted cell whose two d-faces are stored (all but the last ghost
// layer along d): B^d = (Bf_d(lower) + Bf_d(upper)) / (2 sqrt(gamma)) at the cell centre.
template <class T, int METRIC>
__global__ void k_face_to_cells(const double* __restrict__ Bf, T* __restrict__ P, DevParams p) {
  const long long G = p.gsize;
  const long long st[3] = {1, p.gx, (long long)p.gx * p.gy};
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < G; t += (long long)gridDim.x * blockDim.x) {
    const int gi = (int)(t % p.gx), gj = (int)((t / p.gx) % p.gy), gk = (int)(t / ((long long)p.gx * p.gy));
    Metric<double> m;
    metric_at<double, METRIC>(p, p.x0[0] + (gi - p.ng + 0.5) * p.dx[0], p.x0[1] + (gj - p.ng + 0.5) * p.dx[1],
                              p.x0[2] + (gk - p.ng + 0.5) * p.dx[2], m);
    const int c[3] = {gi, gj, gk}, gn[3] = {p.gx, p.gy, p.gz};
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (c[d] + 1 < gn[d]) P[(5 + d) * G + t] = (T)(0.5 * (Bf[d * G + t] + Bf[d * G + t + st[d]]) / m.sqrtgam);
  }
}

// Launchers of one arithmetic form (R: flux / EMF type, T: storage type of P).
template <class R, class T>
struct FaceCtLaunch {
  static cudaError_t emf(const DevParams& p, const void* P, const void* Fx, const void* Fy, const void* Fz, void* Ecc,
                         void* E, cudaStream_t s) {
    const long long ncell = (long long)(p.nx + 2) * (p.ny + 2) * (p.nz + 2);
    if (p.metric == KERR_SCHILD)
      k_emf_cc<R, T, KERR_SCHILD><<<grid_for(ncell, 128), 128, 0, s>>>((const T*)P, (R*)Ecc, p);
    else
      k_emf_cc<R, T, MINKOWSKI><<<grid_for(ncell, 128), 128, 0, s>>>((const T*)P, (R*)Ecc, p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long nedge = (long long)(p.nx + 1) * (p.ny + 1) * (p.nz + 1);
    k_emf_upwind<R><<<grid_for(nedge, 128), 128, 0, s>>>((const R*)Fx, (const R*)Fy, (const R*)Fz, (const R*)Ecc,
                                                         (double*)E, p);
    return cudaGetLastError();
  }
  static cudaError_t faces(const DevParams& p, const double* Bf0, const double* Bfc, double* Bfn, const void* E,
                           const StageArgs& a, cudaStream_t s) {
    const long long n = (long long)(p.nx + 1) * (p.ny + 1) * (p.nz + 1);
    k_face_update<R><<<grid_for(n, 256), 256, 0, s>>>(Bf0, Bfc, Bfn, (const double*)E, a, p);
    return cudaGetLastError();
  }
  static cudaError_t to_cells(const DevParams& p, const double* Bf, void* P, cudaStream_t s) {
    if (p.metric == KERR_SCHILD)
      k_face_to_cells<T, KERR_SCHILD><<<grid_for(p.gsize, 128), 128, 0, s>>>(Bf, (T*)P, p);
    else
      k_face_to_cells<T, MINKOWSKI><<<grid_for(p.gsize, 128), 128, 0, s>>>(Bf, (T*)P, p);
    return cudaGetLastError();
  }
  static cudaError_t ghost_faces(const DevParams& p, double* Bf, cudaStream_t s) {
    k_ghost_periodic<double, 3><<<grid_for(p.gsize, 256), 256, 0, s>>>(Bf, p);
    return cudaGetLastError();
  }
};

}  // namespace grmhd
