// Two-level block meshes: the ghost exchange between levels and the refluxing of coarse cells at
// coarse-fine faces (the multi-block / AMR fill of the meshblock method).
//
// Ghosts are exchanged as primitives in two passes at the start of every stage. Pass 1: a ghost whose
// point lies in a leaf of its own level copies that leaf's cell; a coarse ghost over a fine leaf takes the
// mean of the 8 fine cells it covers (restriction). Pass 2: a fine ghost over a coarse leaf is the coarse
// cell's value plus, per direction, the minmod-limited slope times the offset (+-1/4 of the coarse width)
// of the fine centre (prolongation); its slope stencil may read coarse ghosts, which pass 1 filled.
// After the stage's update (and its floor and deferred passes) every coarse cell with a face on a fine
// leaf replaces that face's flux by the mean of the 4 fine face fluxes covering it (Berger-Colella
// refluxing; for B the flux-CT face fluxes formed from the edge EMFs), and takes con2prim, floors and the
// re-derived hydro state again.
#pragma once

#include "grmhd_kernels.cuh"

namespace grmhd {

__device__ __forceinline__ int mesh_leaf(const MeshDesc& M, int fx, int fy, int fz, const int n[3]) {
  return M.leaf[fx / n[0] + 2 * M.nb[0] * (fy / n[1] + 2 * M.nb[1] * (fz / n[2]))];
}

// One pass of the exchange. Grid: (x: ghost cells of a block, y: blocks; pass 2: the level-1 blocks only).
// The restriction and prolongation arithmetic is in the storage type of the primitives (float in the mixed
// form, where conversions to double would share the FP64 pipe; double in the all-FP64 form).
template <class T>
__global__ void __launch_bounds__(256) k_mesh_exchange(const BlockDesc* __restrict__ blocks, MeshDesc M, int pass) {
  const int b = pass == 2 ? M.fine[blockIdx.y] : (int)blockIdx.y;
  const BlockDesc& D = blocks[b];
  const DevParams& p = D.p;  // every block of a mesh has the same cell counts
  const long long G = p.gsize;
  const int n[3] = {p.nx, p.ny, p.nz};
  const int lev = D.level;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M.nghost; e += gridDim.x * blockDim.x) {
    const unsigned pk = M.ghost[e];
    const int c[3] = {(int)(pk & 1023u) - p.ng, (int)((pk >> 10) & 1023u) - p.ng, (int)(pk >> 20) - p.ng};
    int gl[3];
    bool outside = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int N = M.nb[d] * n[d] << lev;
      int gd = D.pos[d] * n[d] + c[d];
      if (gd < 0 || gd >= N) {
        outside = true;
        gd = gd < 0 ? gd + N : gd - N;  // ghosts are at most ng < n cells outside, so one wrap suffices
      }
      gl[d] = gd;
    }
    if (outside && !M.periodic) continue;
    const int src = lev ? mesh_leaf(M, gl[0], gl[1], gl[2], n) : mesh_leaf(M, 2 * gl[0], 2 * gl[1], 2 * gl[2], n);
    const BlockDesc& S = blocks[src];
    const long long g = gidx(p, c[0], c[1], c[2]);
    const T* __restrict__ Ps = (const T*)S.P;
    T* __restrict__ Pd = (T*)D.P;
    // the passive scalar, when the batch carries one, is exchanged like one more primitive
    const T* __restrict__ Xs = (const T*)S.X;
    T* __restrict__ Xd = (T*)D.X;
    if (pass == 1 && S.level == lev) {
      const long long gs = gidx(S.p, gl[0] - S.pos[0] * n[0], gl[1] - S.pos[1] * n[1], gl[2] - S.pos[2] * n[2]);
#pragma unroll
      for (int q = 0; q < NV; ++q) Pd[q * G + g] = Ps[q * G + gs];
      if (Xs) Xd[g] = Xs[gs];
    } else if (pass == 1 && lev == 0 && S.level == 1) {
      // restriction: the 8 fine interior cells under this coarse ghost (n even: all in leaf S)
      const long long g0 = gidx(S.p, 2 * gl[0] - S.pos[0] * n[0], 2 * gl[1] - S.pos[1] * n[1], 2 * gl[2] - S.pos[2] * n[2]);
      const long long sy = S.p.gx, sz = (long long)S.p.gx * S.p.gy;
#pragma unroll
      for (int q = 0; q <= NV; ++q) {
        if (q == NV && !Xs) break;
        const T* a = q < NV ? Ps + q * G + g0 : Xs + g0;
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc += a[(k & 1) + ((k >> 1) & 1) * sy + (k >> 2) * sz];
        if (q < NV) Pd[q * G + g] = acc / T(8); else Xd[g] = acc / T(8);
      }
    } else if (pass == 2 && S.level == 0) {
      // prolongation from the coarse cell containing this fine ghost (an interior cell of S)
      const long long gc = gidx(S.p, (gl[0] >> 1) - S.pos[0] * n[0], (gl[1] >> 1) - S.pos[1] * n[1],
                                (gl[2] >> 1) - S.pos[2] * n[2]);
      const long long st[3] = {1, S.p.gx, (long long)S.p.gx * S.p.gy};
      T off[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) off[d] = (gl[d] & 1) ? T(0.25) : T(-0.25);
#pragma unroll
      for (int q = 0; q <= NV; ++q) {
        if (q == NV && !Xs) break;
        const T* a = q < NV ? Ps + q * G + gc : Xs + gc;
        const T pc = a[0];
        T v = pc;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const T up = a[st[d]] - pc, dn = pc - a[-st[d]];
          // minmod: the smaller slope in magnitude when both have the same sign, else 0
          const T m = up * dn > T(0) ? (up > T(0) ? (up < dn ? up : dn) : (up > dn ? up : dn)) : T(0);
          v = v + off[d] * m;
        }
        if (q < NV) Pd[q * G + g] = v; else Xd[g] = v;
      }
    }
  }
}

// Fluxes an update uses through the lower d-face of ghosted cell g: the hydro face fluxes and the flux-CT
// fluxes of B (the same expressions as the update's).
template <class R>
__device__ __forceinline__ void face_flux_used(const DevParams& p, const R* __restrict__ F, const R* __restrict__ E,
                                               int d, long long g, double out[NV]) {
  const long long G = p.gsize, sy = p.gx, sz = (long long)p.gx * p.gy;
#pragma unroll
  for (int q = 0; q < 5; ++q) out[q] = (double)F[q * G + g];
  const R* Ex = E;
  const R* Ey = E + G;
  const R* Ez = E + 2 * G;
  const R h = R(0.5);
  if (d == 0) {
    out[5] = 0.0;
    out[6] = (double)(-h * (Ez[g] + Ez[g + sy]));
    out[7] = (double)(h * (Ey[g] + Ey[g + sz]));
  } else if (d == 1) {
    out[5] = (double)(h * (Ez[g] + Ez[g + 1]));
    out[6] = 0.0;
    out[7] = (double)(-h * (Ex[g] + Ex[g + sz]));
  } else {
    out[5] = (double)(-h * (Ey[g] + Ey[g + 1]));
    out[6] = (double)(h * (Ex[g] + Ex[g + sy]));
    out[7] = 0.0;
  }
}

template <int METRIC, class R, class T>
__global__ void __launch_bounds__(64) k_mesh_reflux(const BlockDesc* __restrict__ blocks,
                                                     const RefluxCell* __restrict__ cells, int ncells, BatchArgs a) {
  const double dt = a.use_dev_dt ? *a.dt_dev : a.dt;
  const double bdt = a.beta * dt;
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < ncells; w += gridDim.x * blockDim.x) {
    const RefluxCell rc = cells[w];
    const BlockDesc& B = blocks[rc.block];
    const DevParams& p = B.p;
    const long long t = rc.cell, n = p.isize, G = p.gsize;
    const int nn[3] = {p.nx, p.ny, p.nz};
    const int ci[3] = {(int)(t % p.nx), (int)((t / p.nx) % p.ny), (int)(t / ((long long)p.nx * p.ny))};
    const long long g = gidx(p, ci[0], ci[1], ci[2]);
    const long long st[3] = {1, p.gx, (long long)p.gx * p.gy};
    double dU[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) dU[q] = 0.0;
    for (int d = 0; d < 3; ++d) {
      const int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
      for (int s = 0; s < 2; ++s) {
        const int fb = rc.fine[2 * d + s];
        if (fb < 0) continue;
        const BlockDesc& S = blocks[fb];
        double Fc[NV], Ff[NV], f4[NV];
        face_flux_used<R>(p, (const R*)B.F[d], (const R*)B.E, d, g + (s ? st[d] : 0), Fc);
#pragma unroll
        for (int q = 0; q < NV; ++q) Ff[q] = 0.0;
        int ff[3];
        ff[d] = s ? 0 : nn[d];  // the fine block's lower boundary face when it lies above, else its upper
        for (int c2 = 0; c2 < 2; ++c2)
          for (int c1 = 0; c1 < 2; ++c1) {
            ff[a1] = 2 * (B.pos[a1] * nn[a1] + ci[a1]) - S.pos[a1] * nn[a1] + c1;
            ff[a2] = 2 * (B.pos[a2] * nn[a2] + ci[a2]) - S.pos[a2] * nn[a2] + c2;
            face_flux_used<R>(S.p, (const R*)S.F[d], (const R*)S.E, d, gidx(S.p, ff[0], ff[1], ff[2]), f4);
#pragma unroll
            for (int q = 0; q < NV; ++q) Ff[q] += f4[q];
          }
        const double sg = s ? 1.0 : -1.0;
#pragma unroll
        for (int q = 0; q < NV; ++q) dU[q] += sg * (Fc[q] - Ff[q] / 4.0) / p.dx[d];
      }
    }
    double Un[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) Un[q] = B.U[a.dst][q * n + t] + bdt * dU[q];
    // con2prim (the double solver in both forms: these are few cells), floors, re-derived hydro state
    Metric<double> m;
    double isg, fr;
    cell_metric<METRIC>(p, t, p.x0[0] + (ci[0] + 0.5) * p.dx[0], p.x0[1] + (ci[1] + 0.5) * p.dx[1],
                        p.x0[2] + (ci[2] + 0.5) * p.dx[2], m, isg, fr);
    T* P = (T*)B.P;
    double Pc[NV], Uc[NV], Pn[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      Pc[q] = (double)P[q * G + g];
      Uc[q] = Un[q] * isg;
    }
    const double mu0 = mu_of_prims<double>(Pc, m.gam, p.gamma_eos);
    int iters;
    int stt = con2prim<double>(p, m, Uc, mu0, Pn, iters);
    stt |= apply_floors_fr(p, m.gam, fr, Pn);
    if (stt) {
      double U5[5];
      prim_to_cons5<double>(Pn, m, p.gamma_eos, U5);
#pragma unroll
      for (int q = 0; q < 5; ++q) Un[q] = U5[q];
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      B.U[a.dst][q * n + t] = Un[q];
      P[q * G + g] = (T)Pn[q];
    }
    B.status[t] = (uint8_t)stt;
  }
}

// Refluxing of the passive scalar after its update: every coarse cell at a coarse-fine face corrects its
// sqrt(gamma) D X by the difference between its face flux and the mean of the 4 fine ones (the same faces
// as the fluid's refluxing), then X = DX / D with its refluxed D.
template <class R, class T>
__global__ void __launch_bounds__(64) k_mesh_reflux_scalar(const BlockDesc* __restrict__ blocks,
                                                            const RefluxCell* __restrict__ cells, int ncells,
                                                            BatchArgs a) {
  const double dt = a.use_dev_dt ? *a.dt_dev : a.dt;
  const double bdt = a.beta * dt;
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < ncells; w += gridDim.x * blockDim.x) {
    const RefluxCell rc = cells[w];
    const BlockDesc& B = blocks[rc.block];
    const DevParams& p = B.p;
    const long long t = rc.cell;
    const int nn[3] = {p.nx, p.ny, p.nz};
    const int ci[3] = {(int)(t % p.nx), (int)((t / p.nx) % p.ny), (int)(t / ((long long)p.nx * p.ny))};
    const long long g = gidx(p, ci[0], ci[1], ci[2]);
    const long long st[3] = {1, p.gx, (long long)p.gx * p.gy};
    double dX = 0.0;
    for (int d = 0; d < 3; ++d) {
      const int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
      for (int s = 0; s < 2; ++s) {
        const int fb = rc.fine[2 * d + s];
        if (fb < 0) continue;
        const BlockDesc& S = blocks[fb];
        const double Fc = (double)((const R*)B.FX)[(long long)d * p.gsize + g + (s ? st[d] : 0)];
        double Ff = 0.0;
        int ff[3];
        ff[d] = s ? 0 : nn[d];
        for (int c2 = 0; c2 < 2; ++c2)
          for (int c1 = 0; c1 < 2; ++c1) {
            ff[a1] = 2 * (B.pos[a1] * nn[a1] + ci[a1]) - S.pos[a1] * nn[a1] + c1;
            ff[a2] = 2 * (B.pos[a2] * nn[a2] + ci[a2]) - S.pos[a2] * nn[a2] + c2;
            Ff += (double)((const R*)S.FX)[(long long)d * S.p.gsize + gidx(S.p, ff[0], ff[1], ff[2])];
          }
        dX += (s ? 1.0 : -1.0) * (Fc - Ff / 4.0) / p.dx[d];
      }
    }
    double* DX = B.DX[a.dst];
    const double dxn = DX[t] + bdt * dX;
    DX[t] = dxn;
    ((T*)B.X)[g] = (T)(dxn / B.U[a.dst][t]);
  }
}

}  // namespace grmhd
