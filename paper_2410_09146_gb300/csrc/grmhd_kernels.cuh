// Kernels of one GRMHD Runge-Kutta stage (a0 ghost fill, a1 metric, a2 reconstruction,
// a3 Riemann flux, a4 constrained transport, a5 divergence + sources + RK combination,
// a6 con2prim + floors, a7 time step). Layouts, all with x fastest:
//   P   [8][gz][gy][gx]  primitives incl. ghosts (type T: double, or float in the mixed form)
//   U   [8][nz][ny][nx]  densitized conserved state (double)
//   F_d [8][gz][gy][gx]  face fluxes of direction d; entry (i,j,k) is the lower d-face of cell (i,j,k)
//   E   [3][gz][gy][gx]  edge EMFs; component c at (i,j,k) is the c-directed edge at the lower
//                        corner of cell (i,j,k) in the two directions transverse to c
#pragma once

#include "grmhd_device.cuh"

namespace grmhd {

__device__ __forceinline__ long long gidx(const DevParams& p, int i, int j, int k) {
  return ((long long)(k + p.ng) * p.gy + (j + p.ng)) * p.gx + (i + p.ng);
}

__device__ __forceinline__ long long iidx(const DevParams& p, int i, int j, int k) {
  return ((long long)k * p.ny + j) * p.nx + i;
}

// a0: periodic ghost fill (every ghost cell copies its wrapped interior cell); NVAR arrays gsize apart
// (the 8 primitives, or the 3 face-field components, whose canonical faces wrap the same way).
template <class T, int NVAR = NV>
__global__ void k_ghost_periodic(T* __restrict__ P, DevParams p) {
  const long long n = p.gsize;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int gi = (int)(t % p.gx);
    const int gj = (int)((t / p.gx) % p.gy);
    const int gk = (int)(t / ((long long)p.gx * p.gy));
    const int i = gi - p.ng, j = gj - p.ng, k = gk - p.ng;
    if (i >= 0 && i < p.nx && j >= 0 && j < p.ny && k >= 0 && k < p.nz) continue;
    const int si = ((i % p.nx) + p.nx) % p.nx, sj = ((j % p.ny) + p.ny) % p.ny, sk = ((k % p.nz) + p.nz) % p.nz;
    const long long src = gidx(p, si, sj, sk);
#pragma unroll
    for (int q = 0; q < NVAR; ++q) STC(P, q * n + t, NVAR * n, LDC(P, q * n + src, NVAR * n));
  }
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// a1 + a3 for the face between cells (i, j, k) - e_d and (i, j, k) of direction d, given the two
// reconstructed sides PL, PR: evaluate the metric at the face centre, floor the two sides (Sec. 3.2: rho >=
// rho_flr, rho eps >= rho eps_flr at the face; continuous in the data, unlike a switch to other values),
// their (U, F, lambda), and the Riemann flux Fh; returns max |lambda|. With a face-centred field (p.bface)
// both sides take the face's normal field B^d = Bf_d / sqrt(gamma).
template <class R, int METRIC>
__device__ __forceinline__ R face_flux(const DevParams& p, int d, int i, int j, int k, R PL[NV], R PR[NV],
                                       R Fh[NV]) {
  // face centre, in the flux arithmetic type
  R xf[3] = {par<R>(p.x0[0], p.fx0[0]) + (R(i) + R(0.5)) * par<R>(p.dx[0], p.fdx[0]), par<R>(p.x0[1], p.fx0[1]) + (R(j) + R(0.5)) * par<R>(p.dx[1], p.fdx[1]),
             par<R>(p.x0[2], p.fx0[2]) + (R(k) + R(0.5)) * par<R>(p.dx[2], p.fdx[2])};
  const int cd = d == 0 ? i : (d == 1 ? j : k);
  const R xd = sel3(d, par<R>(p.x0[0], p.fx0[0]), par<R>(p.x0[1], p.fx0[1]), par<R>(p.x0[2], p.fx0[2])) +
               R(cd) * sel3(d, par<R>(p.dx[0], p.fdx[0]), par<R>(p.dx[1], p.fdx[1]), par<R>(p.dx[2], p.fdx[2]));
  if (d == 0) xf[0] = xd; else if (d == 1) xf[1] = xd; else xf[2] = xd;
  if (METRIC == KERR_SCHILD_SPHERICAL && d == 1 && fabs(sin(p.x0[1] + j * p.dx[1])) < 1e-12) {
    // a theta face on the polar axis has zero area (sqrt(-g) = 0 there, where the metric is singular): no flux.
    // Decided in double from the double parameters: a float theta of pi (3.1415927) has sin ~ -9e-8.
#pragma unroll
    for (int q = 0; q < NV; ++q) Fh[q] = R(0);
    return R(0);
  }
  Metric<R> m;
  R rks = R(1);
  metric_at<R, METRIC>(p, xf[0], xf[1], xf[2], m, &rks);
  const R fr = METRIC != MINKOWSKI ? (p.floor_r2 ? rcp(rks * rks) : R(pow((double)rks, -p.floor_r_exp)))
                                     : R(1);
  const R rho_flr = par<R>(p.rho_floor0, p.frho_floor0) * fr, eps_flr = par<R>(p.eps_floor0, p.feps_floor0) * fr;
  if (!(PL[0] >= rho_flr)) PL[0] = rho_flr;
  if (!(PR[0] >= rho_flr)) PR[0] = rho_flr;
  if (!(PL[4] >= PL[0] * eps_flr)) PL[4] = PL[0] * eps_flr;
  if (!(PR[4] >= PR[0] * eps_flr)) PR[4] = PR[0] * eps_flr;
  if (p.bface != nullptr) {
    const R bn = fdiv(R(LDC(p.bface, d * p.gsize + gidx(p, i, j, k), 3 * p.gsize)), m.sqrtgam);
    if (d == 0) { PL[5] = bn; PR[5] = bn; }
    else if (d == 1) { PL[6] = bn; PR[6] = bn; }
    else { PL[7] = bn; PR[7] = bn; }
  }
  const R smg = METRIC == KERR_SCHILD_SPHERICAL ? m.alpha * m.sqrtgam : R(1);  // sqrt(-g) at the face
  if constexpr (sizeof(R) == 4) {
    // both sides at once in paired float arithmetic
    float2 P2[NV], U2[NV], F2[NV], lm, lp;
#pragma unroll
    for (int q = 0; q < NV; ++q) P2[q] = make_float2(PL[q], PR[q]);
    prim_to_face_x2(P2, m, d, p.fgamma, U2, F2, lm, lp);
    if constexpr (METRIC == KERR_SCHILD_SPHERICAL) {
#pragma unroll
      for (int q = 0; q < NV; ++q) F2[q] = mul2(F2[q], x2(smg));  // densitized flux sqrt(-g) F^d
    }
    return riemann_flux_x2(p.riemann, U2, F2, lm, lp, Fh);
  } else {
    FaceSide<R> L, Rs;
    prim_to_face<R>(PL, m, d, p.gamma_eos, L, smg);
    prim_to_face<R>(PR, m, d, p.gamma_eos, Rs, smg);
    return riemann_flux<R>(p.riemann, L, Rs, Fh);
  }
}

// a2 for face t of direction d: reconstruct the two cells beside the face, then face_flux. Writes F and
// returns max |lambda| of the face when it is an interior face (0 otherwise).
template <class R, class T, int METRIC, int RECON>
__device__ __forceinline__ R flux_face(const DevParams& p, const T* __restrict__ P, R* __restrict__ F, int d,
                                       long long t) {
  int ex, ey;
  face_box(p, d, ex, ey);
  const long long stride = d == 0 ? 1 : (d == 1 ? (long long)p.gx : (long long)p.gx * p.gy);
  const int i = (int)(t % ex) + (d == 0 ? 0 : -1);
  const int j = (int)((t / ex) % ey) + (d == 1 ? 0 : -1);
  const int k = (int)(t / ((long long)ex * ey)) + (d == 2 ? 0 : -1);
  const long long g = gidx(p, i, j, k);
  R PL[NV], PR[NV];
  const R eps = par<R>(p.weno_eps, p.fweno_eps);
  // Spherical coordinates: the phi components of W v and B (variables 3 and 7) grow like 1/sin(theta)
  // towards the axis, and sin(theta) times them is regular there (continuing through it with the sign of
  // sin(theta)), so that product is reconstructed and divided by sin(theta) at the face. The stencil cell
  // at offset o along d has theta index j + o for d = 1, j otherwise.
  const bool sph = METRIC == KERR_SCHILD_SPHERICAL;
  R sfc = R(1), sw[6] = {R(1), R(1), R(1), R(1), R(1), R(1)};
  if (sph) {
    const R th0 = par<R>(p.x0[1], p.fx0[1]), dth = par<R>(p.dx[1], p.fdx[1]);
    sfc = sin(d == 1 ? th0 + R(j) * dth : th0 + (R(j) + R(0.5)) * dth);
#pragma unroll
    for (int o = 0; o < 6; ++o) sw[o] = sin(th0 + (R(j + (d == 1 ? o - 3 : 0)) + R(0.5)) * dth);
  }
  // no weighting on an axis face (it carries no flux; decided in double, as in face_flux)
  const bool reg_ok = sph && !(d == 1 && fabs(sin(p.x0[1] + j * p.dx[1])) < 1e-12);
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    const long long c0 = q * p.gsize + g, PN = NV * p.gsize;
    const bool reg = reg_ok && (q == 3 || q == 7);
    const R fm3 = cell_centric(RECON) ? R(LDC(P, c0 - 3 * stride, PN)) * (reg ? sw[0] : R(1)) : R(0);
    const R fm2 = RECON != RECON_CONSTANT ? R(LDC(P, c0 - 2 * stride, PN)) * (reg ? sw[1] : R(1)) : R(0);
    const R fm1 = R(LDC(P, c0 - stride, PN)) * (reg ? sw[2] : R(1));
    const R f0 = R(LDC(P, c0, PN)) * (reg ? sw[3] : R(1));
    const R fp1 = RECON != RECON_CONSTANT ? R(LDC(P, c0 + stride, PN)) * (reg ? sw[4] : R(1)) : R(0);
    const R fp2 = cell_centric(RECON) ? R(LDC(P, c0 + 2 * stride, PN)) * (reg ? sw[5] : R(1)) : R(0);
    R qm, qp;
    recon_cell<R, RECON>(fm3, fm2, fm1, f0, fp1, eps, qm, qp);  // cell c - e_d
    PL[q] = reg ? qp / sfc : qp;
    recon_cell<R, RECON>(fm2, fm1, f0, fp1, fp2, eps, qm, qp);  // cell c
    PR[q] = reg ? qm / sfc : qm;
  }
  R Fh[NV];
  const R cm = face_flux<R, METRIC>(p, d, i, j, k, PL, PR, Fh);
#pragma unroll
  for (int q = 0; q < NV; ++q) STC(F, q * p.gsize + g, NV * p.gsize, Fh[q]);
  const bool interior = (d == 0 || (i >= 0 && i < p.nx)) && (d == 1 || (j >= 0 && j < p.ny)) &&
                        (d == 2 || (k >= 0 && k < p.nz));
  return interior ? cm : R(0);
}

// Block-wide max of v (non-negative) folded into *dst with one atomic per block.
template <class R>
__device__ __forceinline__ void block_max_to(R v, unsigned long long* dst) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __shared__ R red[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : R(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) atomic_max_pos(dst, (double)v);
  }
}

// One thread per face of direction d; for interior faces max |lambda| is reduced into ms[d].
template <class R, class T, int METRIC, int RECON>
__global__ void __launch_bounds__(128) k_flux(const T* __restrict__ P, R* __restrict__ F,
                                              unsigned long long* __restrict__ ms, DevParams p, int d,
                                              int track_speed) {
  int ex, ey;
  const long long nface = face_box(p, d, ex, ey);
  R cm_local = R(0);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nface;
       t += (long long)gridDim.x * blockDim.x) {
    const R cm = flux_face<R, T, METRIC, RECON>(p, P, F, d, t);
    if (cm > cm_local) cm_local = cm;
  }
  if (track_speed) block_max_to<R>(cm_local, ms + d);
}

// Stencil rows ahead of the cell being reconstructed that the float y / z flux runs prefetch into L1: each
// cell adds one row (its f + 2 neighbour) to the rows the cell before loaded, and that row is the one whose
// load waits on L2.
constexpr int kFluxPrefetch = 1;

template <class T>
__device__ __forceinline__ void prefetch_l1(const T* a) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(a));
}

// Minus / plus face values of every variable of the cell at ghosted index g, its five-cell stencil along the
// sweep at stride sd (every stencil cell inside the ghosted block): the float WENO5-Z-AOAH form reconstructs
// the variables in pairs (recon_weno5z_x2), the others one at a time (recon_cell).
template <class R, class T, int RECON>
__device__ __forceinline__ void recon_cell_all(const DevParams& p, const T* __restrict__ P, long long g,
                                               long long sd, R eps, R qm[NV], R qp[NV]) {
  const long long PN = NV * p.gsize;
  if constexpr (sizeof(R) == 4 && RECON == RECON_WENO5Z) {
#pragma unroll
    for (int q = 0; q < NV; q += 2) {
      float2 f[5];
#pragma unroll
      for (int s = 0; s < 5; ++s) {
        const long long c = q * p.gsize + g + (s - 2) * sd;
        f[s] = make_float2(float(LDC(P, c, PN)), float(LDC(P, c + p.gsize, PN)));
      }
      float2 m, pl;
      recon_weno5z_x2(f[0], f[1], f[2], f[3], f[4], eps, m, pl);
      qm[q] = m.x;
      qm[q + 1] = m.y;
      qp[q] = pl.x;
      qp[q + 1] = pl.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      R f[5];
#pragma unroll
      for (int s = 0; s < 5; ++s) f[s] = R(LDC(P, q * p.gsize + g + (s - 2) * sd, PN));
      recon_cell<R, RECON>(f[0], f[1], f[2], f[3], f[4], eps, qm[q], qp[q]);
    }
  }
}

// Cell-centric fluxes of direction d = 1, 2 for WENO5-Z-AOAH, unit t of flux_units: one transverse
// position and a run of flux_run_length faces along d. Each cell is reconstructed once (both of its faces),
// and face f pairs the plus side of cell f - 1 with the minus side of cell f (face_flux, as in the
// face-centric flux_face). The five-cell stencil is loaded afresh for each cell: four of its rows were
// loaded by the warp for the cell before (its lanes hold consecutive x positions) and come from L1, and
// not holding a 40-value window across face_flux cuts the spills at 64 registers (y / z sweeps 1.75 ->
// 1.45 ms at 256^3). Returns max |lambda| over the run's interior faces.
template <class R, class T, int METRIC, int RECON>
__device__ __forceinline__ R flux_run(const DevParams& p, const T* __restrict__ P, R* __restrict__ F, int d,
                                      long long t) {
  // transverse coordinates: a fastest (x for d = 1, 2; y for d = 0), b the other
  const int nd = d == 0 ? p.nx : (d == 1 ? p.ny : p.nz);
  const int na = d == 0 ? p.ny : p.nx;
  const int nb = d == 2 ? p.ny : p.nz;
  const long long sd = d == 0 ? 1 : (d == 1 ? (long long)p.gx : (long long)p.gx * p.gy);
  const R eps = par<R>(p.weno_eps, p.fweno_eps);
  const int a = (int)(t % (na + 2)) - 1;
  const long long rest = t / (na + 2);
  const int b = (int)(rest % (nb + 2)) - 1;
  const int run = flux_run_length(p, nd);
  const int f0 = (int)(rest / (nb + 2)) * run;
  const int f1 = min(f0 + run, nd + 1);
  // start at the cell before the run: its plus side is the left state of the run's first face
  int i = d == 0 ? f0 - 1 : a;
  int j = d == 1 ? f0 - 1 : (d == 0 ? a : b);
  int k = d == 2 ? f0 - 1 : b;
  const bool inner_t = a >= 0 && a < na && b >= 0 && b < nb;  // interior transverse position
  long long g = gidx(p, i, j, k);
  // Every cell, the one before the run included, is reconstructed at the one call site below, so a cell's
  // face values do not depend on where runs start (float FMA contraction could otherwise round two inlined
  // copies differently): the float form gives the same bits for any run layout, hence for any run length
  // and block size.
  R PL[NV];
  R cm_run = R(0);
  for (int f = f0 - 1; f < f1; ++f) {
    if constexpr (sizeof(R) == 4 && kFluxPrefetch > 0) {
      // the row that cell f + kFluxPrefetch adds to its stencil, into L1 ahead of its use (when it is a cell
      // of the ghosted block)
      if (f + 2 + kFluxPrefetch < nd + p.ng) {
#pragma unroll
        for (int q = 0; q < NV; ++q) prefetch_l1(P + q * p.gsize + g + (2 + kFluxPrefetch) * sd);
      }
    }
    // stencil of cell f: cells f - 2 .. f + 2
    R PR[NV], QP[NV];
    recon_cell_all<R, T, RECON>(p, P, g, sd, eps, PR, QP);
    if (f >= f0) {  // face f: the plus side of cell f - 1 and the minus side of cell f
      R Fh[NV];
      const R cm = face_flux<R, METRIC>(p, d, i, j, k, PL, PR, Fh);
#pragma unroll
      for (int q = 0; q < NV; ++q) STC(F, q * p.gsize + g, NV * p.gsize, Fh[q]);
      if (inner_t && cm > cm_run) cm_run = cm;
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) PL[q] = QP[q];
    g += sd;
    if (d == 0) ++i; else if (d == 1) ++j; else ++k;
  }
  return cm_run;
}

// Cell-centric x fluxes for WENO5-Z-AOAH, unit t of flux_units(p, 0): lane l of warp w reconstructs cell
// s = 31 w - 1 + l of the sequence of x rows (cells -1..nx of each row, end to end) and, when l >= 1 and
// the cell is not the first of its row, evaluates the face between it and the previous cell with that
// cell's plus side from lane l - 1. Units come in whole, aligned warps (every lane of the warp takes part in
// the shuffles). Returns max |lambda| of the lane's face when interior, 0 otherwise.
template <class R, class T, int METRIC, int RECON>
__device__ __forceinline__ R flux_lane(const DevParams& p, const T* __restrict__ P, R* __restrict__ F,
                                       long long t) {
  const int lane = (int)(t & 31);
  const long long seq = (t >> 5) * FLUX_WARP_FACES - 1 + lane;
  const long long ncell = (long long)(p.ny + 2) * (p.nz + 2) * (p.nx + 2);
  const bool live = seq >= 0 && seq < ncell;
  const long long row = live ? seq / (p.nx + 2) : 0;
  const int c = live ? (int)(seq % (p.nx + 2)) - 1 : 0;
  const int j = (int)(row % (p.ny + 2)) - 1, k = (int)(row / (p.ny + 2)) - 1;
  const R eps = par<R>(p.weno_eps, p.fweno_eps);
  const long long g = gidx(p, c, j, k);
  R qm[NV], qp[NV];
  // a lane past either end of the sequence (!live) reconstructs cell (0, -1, -1), inside the ghosted block; its
  // values reach no face
  recon_cell_all<R, T, RECON>(p, P, g, 1, eps, qm, qp);
  R PL[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) PL[q] = __shfl_up_sync(0xffffffffu, qp[q], 1);
  if (lane == 0 || !live || c < 0) return R(0);
  R Fh[NV];
  const R cm = face_flux<R, METRIC>(p, 0, c, j, k, PL, qm, Fh);
#pragma unroll
  for (int q = 0; q < NV; ++q) STC(F, q * p.gsize + g, NV * p.gsize, Fh[q]);
  return (j >= 0 && j < p.ny && k >= 0 && k < p.nz) ? cm : R(0);
}

// Resident CTAs per SM the float cell-centric flux kernels are compiled for: 6 x 128 threads at 80
// registers, the best of the occupancy / spill trade-off measured at 256^3 with the paired float arithmetic
// (x / y / z 0.98 / 0.95 / 0.95 ms; 7 CTAs at 72 registers 1.00 / 0.96 / 0.96, 8 at 64 1.02 / 0.98 / 0.98);
// the double form is bound by FP64 issue and keeps its registers.
template <class R>
constexpr int kFluxMinBlocks = sizeof(R) == 4 ? 6 : 1;

template <class R, class T, int METRIC, int RECON>
__global__ void __launch_bounds__(128, kFluxMinBlocks<R>) k_flux_cc(const T* __restrict__ P, R* __restrict__ F,
                                                 unsigned long long* __restrict__ ms, DevParams p, int d,
                                                 int track_speed) {
  const long long total = flux_units(p, d);
  R cm_local = R(0);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const R cm = d == 0 ? flux_lane<R, T, METRIC, RECON>(p, P, F, t) : flux_run<R, T, METRIC, RECON>(p, P, F, d, t);
    if (cm > cm_local) cm_local = cm;
  }
  if (track_speed) block_max_to<R>(cm_local, ms + d);
}

// Geometric sources in spherical Kerr-Schild coordinates (x^1, x^2, x^3) = (ln r, theta, phi), not
// densitized (Sec. 2.1 eq. (source vector), without the radiation four-force). The metric is stationary and
// axisymmetric, so only d_1 and d_2 of g_{mu nu} are nonzero, and for a symmetric T the momentum source
// T^{mu nu}(d_mu g_{nu j} - Gamma^d_{nu mu} g_{d j}) reduces to S_j = 1/2 T^{mu nu} d_j g_{mu nu} (S_3 = 0).
// The energy source alpha (T^{mu 0} d_mu ln alpha - T^{mu nu} Gamma^0_{mu nu}) uses
// T^{mu nu} Gamma^0_{mu nu} = g^{0 d} (T^{mu nu} d_mu g_{d nu} - 1/2 T^{mu nu} d_d g_{mu nu}), where
// g^{00} = -(1+q), g^{01} = q/r and g^{02} = g^{03} = 0. The 4-metric in (t, r, theta, phi): g_tt = -(1-q),
// g_tr = q, g_tphi = -a sin^2 q, g_rr = 1+q, g_rphi = -a sin^2 (1+q), g_thth = Sigma, g_phph =
// sin^2 (Sigma + a^2 sin^2 (1+q)); a component with k r indices carries r^k, and d_1 = r d/dr.
template <class R>
__device__ __forceinline__ void sks_sources(const DevParams& p, R x, R y, const R P[NV], const Metric<R>& m,
                                            R S[5]) {
  const R a = par<R>(p.a, p.fa), M = par<R>(p.M, p.fM);
  const R r = exp(x), sn = sin(y), cs = cos(y), s2 = sn * sn, sc = sn * cs;
  const R Sig = r * r + a * a * cs * cs;
  const R q = R(2) * M * r / Sig;
  const R dSr = R(2) * r, dSt = -R(2) * a * a * sc;         // d Sigma / dr, d Sigma / dtheta
  const R dqr = R(2) * M * (Sig - r * dSr) / (Sig * Sig);    // dq / dr
  const R dqt = -R(2) * M * r * dSt / (Sig * Sig);           // dq / dtheta
  const R Ep = Sig + a * a * s2 * (R(1) + q);
  // g, d_r g, d_theta g in (t, r, theta, phi), upper triangle: 00 01 03 11 13 22 33
  const R gs[7] = {-(R(1) - q), q, -a * s2 * q, R(1) + q, -a * s2 * (R(1) + q), Sig, s2 * Ep};
  const R gr[7] = {dqr, dqr, -a * s2 * dqr, dqr, -a * s2 * dqr, dSr, s2 * (dSr + a * a * s2 * dqr)};
  const R gt[7] = {dqt, dqt, -a * (R(2) * sc * q + s2 * dqt), dqt, -a * (R(2) * sc * (R(1) + q) + s2 * dqt), dSt,
                   R(2) * sc * Ep + s2 * (dSt + a * a * (R(2) * sc * (R(1) + q) + s2 * dqt))};
  const int mi[7] = {0, 0, 0, 1, 1, 2, 3}, ni[7] = {0, 1, 3, 1, 3, 2, 3};
  // in (t, x^1, theta, phi): d_1 (r^k g) = k r^k g + r^k r d_r g, d_2 (r^k g) = r^k d_theta g
  R d1[4][4], d2[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) d1[u][v] = d2[u][v] = R(0);
#pragma unroll
  for (int c = 0; c < 7; ++c) {
    const int k = (mi[c] == 1) + (ni[c] == 1);
    const R fac = k == 0 ? R(1) : (k == 1 ? r : r * r);
    const R v1 = R(k) * fac * gs[c] + fac * r * gr[c], v2 = fac * gt[c];
    d1[mi[c]][ni[c]] = d1[ni[c]][mi[c]] = v1;
    d2[mi[c]][ni[c]] = d2[ni[c]][mi[c]] = v2;
  }
  // fluid four-vectors and T^{mu nu}, from the 3+1 metric
  const R ut[3] = {P[1], P[2], P[3]};
  const R B[3] = {P[5], P[6], P[7]};
  R utl[3], Bl[3];
  lower3(m.gam, ut, utl);
  lower3(m.gam, B, Bl);
  const R W = sqrt(R(1) + ut[0] * utl[0] + ut[1] * utl[1] + ut[2] * utl[2]);
  const R iW = R(1) / W, ia = R(1) / m.alpha;
  R vt[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) vt[i] = m.alpha * ut[i] * iW - m.beta[i];
  const R Bv = (B[0] * utl[0] + B[1] * utl[1] + B[2] * utl[2]) * iW;
  const R B2 = B[0] * Bl[0] + B[1] * Bl[1] + B[2] * Bl[2];
  const R ab0 = W * Bv;
  const R b2 = (B2 + ab0 * ab0) * iW * iW;
  R uc[4], bc[4];
  uc[0] = W * ia;
  bc[0] = ab0 * ia;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    uc[1 + i] = W * ia * vt[i];
    bc[1 + i] = B[i] * iW + bc[0] * vt[i];
  }
  const R pg = (par<R>(p.gamma_eos, p.fgamma) - R(1)) * P[4];
  const R w = P[0] + P[4] + pg + b2;
  const R pt = pg + R(0.5) * b2;
  const R ia2 = ia * ia;
  R gu[4][4];
  gu[0][0] = -ia2;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    gu[0][1 + i] = gu[1 + i][0] = m.beta[i] * ia2;
#pragma unroll
    for (int j = 0; j < 3; ++j) gu[1 + i][1 + j] = m.gamu[sym3(i, j)] - m.beta[i] * m.beta[j] * ia2;
  }
  R T[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) T[u][v] = w * uc[u] * uc[v] + pt * gu[u][v] - bc[u] * bc[v];
  R td1 = R(0), td2 = R(0);  // T^{mu nu} d_1 g_{mu nu}, T^{mu nu} d_2 g_{mu nu}
  R h0 = R(0), h1 = R(0);    // T^{mu nu} d_mu g_{0 nu}, T^{mu nu} d_mu g_{1 nu} (mu = 1, 2)
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      td1 += T[u][v] * d1[u][v];
      td2 += T[u][v] * d2[u][v];
    }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    h0 += T[1][v] * d1[0][v] + T[2][v] * d2[0][v];
    h1 += T[1][v] * d1[1][v] + T[2][v] * d2[1][v];
  }
  S[0] = R(0);
  S[1] = R(0.5) * td1;
  S[2] = R(0.5) * td2;
  S[3] = R(0);
  const R g00 = -(R(1) + q), g01 = q / r;
  const R TG = g00 * h0 + g01 * (h1 - R(0.5) * td1);   // T^{mu nu} Gamma^0_{mu nu}
  // d_mu ln alpha = -1/2 d_mu q / (1 + q): d_1 with d_1 q = r dq/dr, d_2 with dq/dtheta
  const R dla1 = -R(0.5) * r * dqr / (R(1) + q), dla2 = -R(0.5) * dqt / (R(1) + q);
  S[4] = m.alpha * (T[1][0] * dla1 + T[2][0] * dla2 - TG);
}

// Spherical coordinates: the edges along r on the polar axis (theta faces 0 and ny) are one line for every
// phi, where E_r is single-valued: each takes the mean over phi of the values k_emf computed there (summed
// in phi order). One thread per (radial cell, pole).
template <class R>
__global__ void k_emf_axis(R* __restrict__ E, DevParams p) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * p.nx) return;
  const int i = t % p.nx, fj = t < p.nx ? 0 : p.ny;
  if (!(fabs(sin(p.x0[1] + fj * p.dx[1])) < 1e-12)) return;
  const long long G = p.gsize;
  R m = R(0);
  for (int fk = 0; fk < p.nz; ++fk) m += LDC(E, gidx(p, i, fj, fk), 3 * G);
  m /= R(p.nz);
  for (int fk = 0; fk <= p.nz; ++fk) STC(E, gidx(p, i, fj, fk), 3 * G, m);
}

// a0 for a spherical block covering theta in [0, pi] and phi in [0, 2 pi) (nz even): phi is periodic, and a
// ghost beyond a pole is the cell mirrored across it and turned by pi in phi, where the coordinate map
// continues through the pole with d/dtheta reversed: the theta components of W v and B (variables 2 and 6)
// change sign, the rest is copied. Radial ghosts keep their loaded values.
template <class T>
__global__ void k_ghost_spherical(T* __restrict__ P, DevParams p) {
  const long long n = p.gsize;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % p.gx) - p.ng;
    const int j = (int)((t / p.gx) % p.gy) - p.ng;
    const int k = (int)(t / ((long long)p.gx * p.gy)) - p.ng;
    if (i < 0 || i >= p.nx) continue;
    const bool jin = j >= 0 && j < p.ny, kin = k >= 0 && k < p.nz;
    if (jin && kin) continue;
    int sj = j, sk = ((k % p.nz) + p.nz) % p.nz;
    bool flip = false;
    if (!jin) {
      sj = j < 0 ? -j - 1 : 2 * p.ny - j - 1;
      sk = (sk + p.nz / 2) % p.nz;
      flip = true;
    }
    const long long src = gidx(p, i, sj, sk);
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const T v = LDC(P, q * n + src, NV * n);
      STC(P, q * n + t, NV * n, (flip && (q == 2 || q == 6)) ? -v : v);
    }
  }
}

// a7: dt = cfl / max_d(max|lambda_d| / dx_d)
static __global__ void k_finalize_dt(const unsigned long long* ms, double* dt, DevParams p) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double m = 0.0;
    for (int d = 0; d < 3; ++d) m = fmax(m, __longlong_as_double((long long)ms[d]) / p.dx[d]);
    *dt = p.cfl / m;
  }
}

// a4: Toth flux-CT edge EMFs, Omega_k = 1/4 (sum of the 4 F^j_{B^i} - sum of the 4 F^i_{B^j})
// around the edge for (i, j, k) cyclic, for edge box index t in [0, nx] x [0, ny] x [0, nz].
template <class R>
__device__ __forceinline__ void emf_edge(const DevParams& p, const R* __restrict__ Fx, const R* __restrict__ Fy,
                                         const R* __restrict__ Fz, R* __restrict__ E, long long t) {
  const int ex = p.nx + 1, ey = p.ny + 1;
  const long long G = p.gsize;
  const long long sy = p.gx, sz = (long long)p.gx * p.gy;
  const int i = (int)(t % ex), j = (int)((t / ex) % ey), k = (int)(t / ((long long)ex * ey));
  const long long g = gidx(p, i, j, k);
  // spherical coordinates: an edge along phi on the polar axis has zero length, hence a zero EMF (Omega_phi,
  // the covariant phi component of E, carries a factor sin(theta))
  const bool axis_z = p.metric == KERR_SCHILD_SPHERICAL && fabs(sin(p.x0[1] + j * p.dx[1])) < 1e-12;
  if (k < p.nz)  // Omega_z(fi = i, fj = j, k)
    STC(E, 2 * G + g, 3 * G, axis_z ? R(0) : R(0.25) * (LDC(Fy, 5 * G + g - 1, 8 * G) + LDC(Fy, 5 * G + g, 8 * G) -
                                                     LDC(Fx, 6 * G + g - sy, 8 * G) - LDC(Fx, 6 * G + g, 8 * G)));
  if (i < p.nx)  // Omega_x(i, fj = j, fk = k)
    STC(E, 0 * G + g, 3 * G, R(0.25) * (LDC(Fz, 6 * G + g - sy, 8 * G) + LDC(Fz, 6 * G + g, 8 * G) -
                                       LDC(Fy, 7 * G + g - sz, 8 * G) - LDC(Fy, 7 * G + g, 8 * G)));
  if (j < p.ny)  // Omega_y(fi = i, j, fk = k)
    STC(E, 1 * G + g, 3 * G, R(0.25) * (LDC(Fx, 7 * G + g - sz, 8 * G) + LDC(Fx, 7 * G + g, 8 * G) -
                                       LDC(Fz, 5 * G + g - 1, 8 * G) - LDC(Fz, 5 * G + g, 8 * G)));
}

template <class R>
__global__ void k_emf(const R* __restrict__ Fx, const R* __restrict__ Fy, const R* __restrict__ Fz,
                      R* __restrict__ E, DevParams p) {
  const long long n = (long long)(p.nx + 1) * (p.ny + 1) * (p.nz + 1);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    emf_edge<R>(p, Fx, Fy, Fz, E, t);
}

// Geometric source terms at a cell centre (Sec. 2.1 source vector, without the radiation
// four-force), returned densitized (sqrt(-g) = 1): S[0] = 0, S[1..3] = S_j, S[4] = S_tau.
// For Kerr-Schild, g = eta + f l l makes S_j = 1/2 T^{mu nu} d_j g_{mu nu}
//   = 1/2 [d_j f (l.T.l) + 2 f (d_j l).T.l],
// and S_tau = alpha (T^{k0} d_k ln alpha - T^{mu nu} Gamma^0_{mu nu}) with
//   T^{mu nu} Gamma^0_{mu nu} = g^{0 lambda} (Q_lambda - S_lambda), Q_lambda = T^{k nu} d_k g_{lambda nu}.
template <class R>
__device__ __forceinline__ void ks_sources(const DevParams& p, R x, R y, R z, const R P[NV], const Metric<R>& m,
                                           R S[5]) {
  const R a = par<R>(p.a, p.fa), M = par<R>(p.M, p.fM);
  R r, r2, f, l[3];
  ks_core<R>(x, y, z, a, M, r, r2, f, l);
  const R xs[3] = {x, y, z};
  const R R2 = x * x + y * y + z * z;
  const R sq = R(2) * r2 - (R2 - a * a);
  const R Sig = r2 * r2 + a * a * z * z;
  const R ira = rcp(r2 + a * a);
  const R ir = rcp(r);
  R dr[3], df[3], dl[3][3];  // dl[k][i] = d_k l_i
#pragma unroll
  for (int kk = 0; kk < 3; ++kk) {
    dr[kk] = (xs[kk] * r2 + (kk == 2 ? a * a * z : R(0))) * ir / sq;
    const R dSig = R(4) * r * r2 * dr[kk] + (kk == 2 ? R(2) * a * a * z : R(0));
    df[kk] = f * (R(3) * dr[kk] * ir - dSig / Sig);
    dl[kk][0] = ((dr[kk] * x + (kk == 0 ? r : R(0)) + (kk == 1 ? a : R(0))) - R(2) * r * dr[kk] * l[0]) * ira;
    dl[kk][1] = ((dr[kk] * y + (kk == 1 ? r : R(0)) - (kk == 0 ? a : R(0))) - R(2) * r * dr[kk] * l[1]) * ira;
    dl[kk][2] = ((kk == 2 ? R(1) : R(0)) - l[2] * dr[kk]) * ir;
  }
  // fluid four-vectors
  const R ut[3] = {P[1], P[2], P[3]};
  const R B[3] = {P[5], P[6], P[7]};
  R utl[3], Bl[3];
  lower3(m.gam, ut, utl);
  lower3(m.gam, B, Bl);
  const R W = sqrt(R(1) + ut[0] * utl[0] + ut[1] * utl[1] + ut[2] * utl[2]);
  const R iW = rcp(W), ia = rcp(m.alpha);
  R vt[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) vt[i] = m.alpha * ut[i] * iW - m.beta[i];
  const R Bv = (B[0] * utl[0] + B[1] * utl[1] + B[2] * utl[2]) * iW;
  const R B2 = B[0] * Bl[0] + B[1] * Bl[1] + B[2] * Bl[2];
  const R ab0 = W * Bv;
  const R b2 = (B2 + ab0 * ab0) * iW * iW;
  R uc[4], bc[4];
  uc[0] = W * ia;
  bc[0] = ab0 * ia;
  const R b0 = bc[0];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    uc[1 + i] = W * ia * vt[i];
    bc[1 + i] = B[i] * iW + b0 * vt[i];
  }
  const R pg = (par<R>(p.gamma_eos, p.fgamma) - R(1)) * P[4];
  const R w = P[0] + P[4] + pg + b2;
  const R pt = pg + R(0.5) * b2;
  // g^{mu nu}
  const R ia2 = ia * ia;
  R gu[4][4];
  gu[0][0] = -ia2;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    gu[0][1 + i] = gu[1 + i][0] = m.beta[i] * ia2;
#pragma unroll
    for (int j = 0; j < 3; ++j) gu[1 + i][1 + j] = m.gamu[sym3(i, j)] - m.beta[i] * m.beta[j] * ia2;
  }
  R T[4][4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu)
#pragma unroll
    for (int nu = 0; nu < 4; ++nu) T[mu][nu] = w * uc[mu] * uc[nu] + pt * gu[mu][nu] - bc[mu] * bc[nu];
  const R L4[4] = {R(1), l[0], l[1], l[2]};
  R tv[4];  // t^mu = T^{mu nu} l_nu
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) tv[mu] = T[mu][0] + T[mu][1] * l[0] + T[mu][2] * l[1] + T[mu][3] * l[2];
  const R ltl = tv[0] + l[0] * tv[1] + l[1] * tv[2] + l[2] * tv[3];
  R Sj[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const R dlt = dl[j][0] * tv[1] + dl[j][1] * tv[2] + dl[j][2] * tv[3];
    Sj[j] = R(0.5) * df[j] * ltl + f * dlt;
  }
  R A = R(0), C = R(0), Bq[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int kk = 0; kk < 3; ++kk) {
    A += df[kk] * tv[1 + kk];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      C += T[1 + kk][1 + i] * dl[kk][i];
      Bq[i] += dl[kk][i] * tv[1 + kk];
    }
  }
  const R AfC = A + f * C;
  // g^{00} = -(1+f), g^{0i} = f l_i; Q_0 = A + f C, Q_j = l_j (A + f C) + f B_j
  R tg = -(R(1) + f) * AfC;
#pragma unroll
  for (int j = 0; j < 3; ++j) tg += f * l[j] * (l[j] * AfC + f * Bq[j] - Sj[j]);
  const R dla = -R(0.5) * (T[1][0] * df[0] + T[2][0] * df[1] + T[3][0] * df[2]) / (R(1) + f);
  S[0] = R(0);
  S[1] = Sj[0];
  S[2] = Sj[1];
  S[3] = Sj[2];
  S[4] = m.alpha * (dla - tg);
  (void)L4;
}

// Double-precision metric at the centre of interior cell t, 1/sqrt(gamma) and the floor radius factor:
// from the block's geometry cache when it has one (Kerr-Schild), else evaluated in place.
template <int METRIC>
__device__ __forceinline__ void cell_metric(const DevParams& p, long long t, double xc, double yc, double zc,
                                            Metric<double>& m, double& isg, double& fr) {
  if (METRIC == KERR_SCHILD && p.geo != nullptr) {
#ifdef GRMHD_BOUNDS_CHECK
    if (t < 0 || t >= p.isize) {  // every cache entry is a multiple of isize away: one check covers them
      bounds_fault(p, __LINE__, t);
      t = 0;
    }
#endif
    geo_load(p.geo, p.isize, t, m, isg, fr);
  } else {
    double r;
    metric_at<double, METRIC>(p, xc, yc, zc, m, &r);
    isg = 1.0 / m.sqrtgam;
    fr = METRIC != MINKOWSKI ? floor_factor(p, r) : 1.0;
  }
}

// Fill the geometry cache of a block (once, at context creation).
template <int METRIC>
__global__ void k_geometry(DevParams p, double* __restrict__ geo) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < p.isize; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % p.nx), j = (int)((t / p.nx) % p.ny), k = (int)(t / ((long long)p.nx * p.ny));
    Metric<double> m;
    double r;
    const double x = p.x0[0] + (i + 0.5) * p.dx[0], y = p.x0[1] + (j + 0.5) * p.dx[1], z = p.x0[2] + (k + 0.5) * p.dx[2];
    metric_at<double, METRIC>(p, x, y, z, m, &r);
    KSGeo kg{0.0, 0.0, {0.0, 0.0, 0.0}};
    if (METRIC == KERR_SCHILD) {
      double rr, r2;
      ks_core<double>(x, y, z, p.a, p.M, rr, r2, kg.f, kg.l);
      kg.kappa = kg.f / (1.0 + kg.f);
    }
    geo_store(geo, p.isize, t, m, 1.0 / m.sqrtgam, METRIC == KERR_SCHILD ? floor_factor(p, r) : 1.0, kg);
  }
}

// Per-thread con2prim statistics, folded into StageArgs::stats once per warp.
struct CellStats {
  unsigned int it_sum = 0, c_rho = 0, c_eps = 0, c_w = 0, c_nc = 0, c_bad = 0, it_max = 0;
  __device__ __forceinline__ void add(int st, int iters) {
    it_sum += iters;
    it_max = iters > (int)it_max ? iters : it_max;
    c_rho += (st & ST_RHO_FLOOR) != 0;
    c_eps += (st & ST_EPS_FLOOR) != 0;
    c_w += (st & ST_W_CAP) != 0;
    c_nc += (st & ST_NOT_CONVERGED) != 0;
    c_bad += (st & ST_BAD_INPUT) != 0;
  }
  __device__ __forceinline__ void flush(unsigned long long* stats) {
    if (!stats) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      it_sum += __shfl_xor_sync(0xffffffffu, it_sum, o);
      c_rho += __shfl_xor_sync(0xffffffffu, c_rho, o);
      c_eps += __shfl_xor_sync(0xffffffffu, c_eps, o);
      c_w += __shfl_xor_sync(0xffffffffu, c_w, o);
      c_nc += __shfl_xor_sync(0xffffffffu, c_nc, o);
      c_bad += __shfl_xor_sync(0xffffffffu, c_bad, o);
      it_max = max(it_max, __shfl_xor_sync(0xffffffffu, it_max, o));
    }
    if ((threadIdx.x & 31) == 0) {
      if (it_sum) atomicAdd(stats + 0, (unsigned long long)it_sum);
      if (c_rho) atomicAdd(stats + 1, (unsigned long long)c_rho);
      if (c_eps) atomicAdd(stats + 2, (unsigned long long)c_eps);
      if (c_w) atomicAdd(stats + 3, (unsigned long long)c_w);
      if (c_nc) atomicAdd(stats + 4, (unsigned long long)c_nc);
      if (c_bad) atomicAdd(stats + 5, (unsigned long long)c_bad);
      atomicMax(stats + 6, (unsigned long long)it_max);
    }
  }
};

// The part of a geometry-cache entry the mixed form's con2prim needs in double: the Kerr-Schild factors of
// the 3-metric and 1/sqrt(gamma).
__device__ __forceinline__ void geo_load_c2p(const double* __restrict__ geo, long long n, long long t, KSGeo& k,
                                             double& isg) {
  k.f = geo[19 * n + t];
  k.kappa = geo[20 * n + t];
#pragma unroll
  for (int i = 0; i < 3; ++i) k.l[i] = geo[(21 + i) * n + t];
  isg = geo[17 * n + t];
}

// Mixed form of a5 + a6 for interior cell t, after the float flux divergence L (CT fluxes for B): float
// sources, the RK combination in double, con2prim_mixed_f, floors in float on the float primitives and, for
// a floored cell, its hydro state re-derived from them in float. A cell whose double step from the float
// root is not small is queued for deferred_cell.
template <int METRIC>
__device__ __forceinline__ void update_cell_mixed(const DevParams& p, float* __restrict__ P, const StageArgs& a,
                                                  float L[NV], double dt, long long t, long long g, int i, int j,
                                                  int k, float xr, float yr, float zr,
                                                  const float Pr[NV], long long wl_tag, CellStats& cs) {
  const long long n = p.isize, G = p.gsize, sy = p.gx, sz = (long long)p.gx * p.gy;
  Metric<float> mr;
  float rf = 1.f;
  metric_at<float, METRIC>(p, xr, yr, zr, mr, &rf);
  if (METRIC == KERR_SCHILD) {
    float Sr[5];
    ks_sources<float>(p, xr, yr, zr, Pr, mr, Sr);
#pragma unroll
    for (int q = 1; q < 5; ++q) L[q] += Sr[q];
  } else if (METRIC == KERR_SCHILD_SPHERICAL) {
    float Sr[5];
    sks_sources<float>(p, xr, yr, Pr, mr, Sr);
    const float smg = mr.alpha * mr.sqrtgam;  // sqrt(-g) S
#pragma unroll
    for (int q = 1; q < 5; ++q) L[q] += smg * Sr[q];
  }
  // the RK combination in double; a first stage of SSP-RK2 (g0 = 0, g1 = 1) skips the zero and unit terms
  const double bdt = a.beta * dt;
  double Un[NV];
  if (a.g0 == 0.0 && a.g1 == 1.0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) Un[q] = LDC(a.Ucur, q * n + t, NV * n) + bdt * (double)L[q];
  } else {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double u = a.g1 * LDC(a.Ucur, q * n + t, NV * n);
      if (a.g0 != 0.0) u += a.g0 * LDC(a.U0, q * n + t, NV * n);
      Un[q] = u + bdt * (double)L[q];
    }
  }
  if (a.bface_new != nullptr) {
    // face-centred CT: the cell's densitized field is the mean of its two advanced faces of each direction
    const double* bn = a.bface_new;
    Un[5] = 0.5 * (LDC(bn, g, 3 * G) + LDC(bn, g + 1, 3 * G));
    Un[6] = 0.5 * (LDC(bn, G + g, 3 * G) + LDC(bn, G + g + sy, 3 * G));
    Un[7] = 0.5 * (LDC(bn, 2 * G + g, 3 * G) + LDC(bn, 2 * G + g + sz, 3 * G));
  }
  // the 3-metric of the double solve: the Kerr-Schild factors (Cartesian metrics), or the matrices
  using Geo = typename std::conditional<METRIC == KERR_SCHILD_SPHERICAL, Metric<double>, KSGeo>::type;
  Geo gm{};
  double isg = 1.0;
  if constexpr (METRIC == KERR_SCHILD_SPHERICAL) {
    metric_at<double, METRIC>(p, p.x0[0] + (i + 0.5) * p.dx[0], p.x0[1] + (j + 0.5) * p.dx[1],
                              p.x0[2] + (k + 0.5) * p.dx[2], gm);
    isg = 1.0 / gm.sqrtgam;
  } else if (METRIC == KERR_SCHILD && p.geo != nullptr) {
#ifdef GRMHD_BOUNDS_CHECK
    if (t < 0 || t >= n) {
      bounds_fault(p, __LINE__, t);
      t = 0;
    }
#endif
    geo_load_c2p(p.geo, n, t, gm, isg);
  } else if (METRIC == KERR_SCHILD) {
    double r, r2;
    ks_core<double>(p.x0[0] + (i + 0.5) * p.dx[0], p.x0[1] + (j + 0.5) * p.dx[1], p.x0[2] + (k + 0.5) * p.dx[2],
                    p.a, p.M, r, r2, gm.f, gm.l);
    gm.kappa = gm.f / (1.0 + gm.f);
    isg = 1.0 / sqrt(1.0 + gm.f);
  }
  // warm start mu = 1/(h W) of the current primitives, in float (it only seeds the float phase)
  const float mu0 = mu_of_prims<float>(Pr, mr.gam, p.fgamma);
  float Pn[NV];
  int iters;
  double mu_r;
  int st = con2prim_mixed_f(p, gm, isg, Un, mu0, a.worklist != nullptr, Pn, iters, mu_r);
  if (st == C2P_DEFERRED) {
    // finished by deferred_cell: keep P (the warm start), store the new conserved state
#pragma unroll
    for (int q = 0; q < NV; ++q) STC(a.Unew, q * n + t, NV * n, Un[q]);
    const unsigned int slot = atomicAdd(a.wl_count, 1u);
    STC(a.worklist, slot, n, (int)(wl_tag + t));
    STC(a.wl_mu, slot, n, mu_r);
    cs.it_sum += iters;
    return;
  }
  const float fr = METRIC != MINKOWSKI ? (p.floor_r2 ? 1.f / (rf * rf) : powf(rf, -(float)p.floor_r_exp))
                                         : 1.f;
  st |= apply_floors_f(p, mr.gam, fr, Pn);
  if (st) {
    // the hydro state re-derived from the floored float primitives, in float like the floors themselves
    // (the FP32 pipe is idle in this FP64-bound kernel, so the lanes of a warp that take this branch cost
    // next to nothing; the forms without cancellation keep it to the rounding of the primitives)
    float U5[5];
    prim_to_cons5<float>(Pn, mr, p.fgamma, U5);
#pragma unroll
    for (int q = 0; q < 5; ++q) Un[q] = (double)U5[q];
  }
#pragma unroll
  for (int q = 0; q < NV; ++q) STC(a.Unew, q * n + t, NV * n, Un[q]);
#pragma unroll
  for (int q = 0; q < NV; ++q) STC(P, q * G + g, NV * G, Pn[q]);
  STC(a.status, t, n, (uint8_t)st);
  cs.add(st, iters);
}

// a5 + a6 for interior cell t: divergence of the face fluxes (CT fluxes for B), sources, RK
// combination Unew = g0 U0 + g1 Ucur + beta dt L, con2prim warm-started from the current primitives,
// floors, and the re-derived hydro state when a floor fired. In the mixed form a cell whose float
// con2prim phase does not settle is queued (wl_tag identifies its block) and finished by
// deferred_cell. dt is the stage's time step.
template <int METRIC, class R, class T>
__device__ __forceinline__ void update_cell(const DevParams& p, T* __restrict__ P, const R* __restrict__ Fx,
                                            const R* __restrict__ Fy, const R* __restrict__ Fz,
                                            const R* __restrict__ E, const StageArgs& a, double dt, long long t,
                                            long long wl_tag, CellStats& cs) {
  const long long n = p.isize;
  const long long G = p.gsize, sy = p.gx, sz = (long long)p.gx * p.gy;
  const int i = (int)(t % p.nx), j = (int)((t / p.nx) % p.ny), k = (int)(t / ((long long)p.nx * p.ny));
  const long long g = gidx(p, i, j, k);
  const double xc = p.x0[0] + (i + 0.5) * p.dx[0];
  const double yc = p.x0[1] + (j + 0.5) * p.dx[1];
  const double zc = p.x0[2] + (k + 0.5) * p.dx[2];
  // the cell centre in the source / warm-start precision, formed in that precision (no conversion from double)
  const R xr = par<R>(p.x0[0], p.fx0[0]) + (R(i) + R(0.5)) * par<R>(p.dx[0], p.fdx[0]);
  const R yr = par<R>(p.x0[1], p.fx0[1]) + (R(j) + R(0.5)) * par<R>(p.dx[1], p.fdx[1]);
  const R zr = par<R>(p.x0[2], p.fx0[2]) + (R(k) + R(0.5)) * par<R>(p.dx[2], p.fdx[2]);
  T Pt[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) Pt[q] = LDC(P, q * G + g, NV * G);
  R L[NV];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const R div = (LDC(Fx, q * G + g + 1, NV * G) - LDC(Fx, q * G + g, NV * G)) * par<R>(p.idx[0], p.fidx[0]) + (LDC(Fy, q * G + g + sy, NV * G) - LDC(Fy, q * G + g, NV * G)) * par<R>(p.idx[1], p.fidx[1]) +
                  (LDC(Fz, q * G + g + sz, NV * G) - LDC(Fz, q * G + g, NV * G)) * par<R>(p.idx[2], p.fidx[2]);
    L[q] = -div;
  }
  if (a.bface_new == nullptr) {
    const R* Ex = E;
    const R* Ey = E + G;
    const R* Ez = E + 2 * G;
    const R h = R(0.5);
    // CT fluxes of B (normal components vanish)
    const R FyBx_p = h * (LDC(Ez, g + sy, G) + LDC(Ez, g + sy + 1, G)), FyBx_m = h * (LDC(Ez, g, G) + LDC(Ez, g + 1, G));
    const R FzBx_p = -h * (LDC(Ey, g + sz, G) + LDC(Ey, g + sz + 1, G)), FzBx_m = -h * (LDC(Ey, g, G) + LDC(Ey, g + 1, G));
    const R FxBy_p = -h * (LDC(Ez, g + 1, G) + LDC(Ez, g + 1 + sy, G)), FxBy_m = -h * (LDC(Ez, g, G) + LDC(Ez, g + sy, G));
    const R FzBy_p = h * (LDC(Ex, g + sz, G) + LDC(Ex, g + sz + sy, G)), FzBy_m = h * (LDC(Ex, g, G) + LDC(Ex, g + sy, G));
    const R FxBz_p = h * (LDC(Ey, g + 1, G) + LDC(Ey, g + 1 + sz, G)), FxBz_m = h * (LDC(Ey, g, G) + LDC(Ey, g + sz, G));
    const R FyBz_p = -h * (LDC(Ex, g + sy, G) + LDC(Ex, g + sy + sz, G)), FyBz_m = -h * (LDC(Ex, g, G) + LDC(Ex, g + sz, G));
    L[5] = -((FyBx_p - FyBx_m) * par<R>(p.idx[1], p.fidx[1]) + (FzBx_p - FzBx_m) * par<R>(p.idx[2], p.fidx[2]));
    L[6] = -((FxBy_p - FxBy_m) * par<R>(p.idx[0], p.fidx[0]) + (FzBy_p - FzBy_m) * par<R>(p.idx[2], p.fidx[2]));
    L[7] = -((FxBz_p - FxBz_m) * par<R>(p.idx[0], p.fidx[0]) + (FyBz_p - FyBz_m) * par<R>(p.idx[1], p.fidx[1]));
  } else {
    L[5] = L[6] = L[7] = R(0);  // the field comes from the advanced faces below
  }
  if constexpr (sizeof(T) == 4) {
    update_cell_mixed<METRIC>(p, P, a, L, dt, t, g, i, j, k, xr, yr, zr, Pt, wl_tag, cs);
  } else {
    const double bdt = a.beta * dt;
    Metric<double> m;
    double isg, fr;
    cell_metric<METRIC>(p, t, xc, yc, zc, m, isg, fr);
    // metric in the source / warm-start precision: the double one itself in the FP64 form
    Metric<R> mr;
    if constexpr (sizeof(R) == sizeof(double)) {
      mr = m;
    } else {
      metric_at<R, METRIC>(p, xr, yr, zr, mr);
    }
    R Pr[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) Pr[q] = R(Pt[q]);
    if (METRIC == KERR_SCHILD) {
      R Sr[5];
      ks_sources<R>(p, xr, yr, zr, Pr, mr, Sr);
#pragma unroll
      for (int q = 1; q < 5; ++q) L[q] += Sr[q];
    } else if (METRIC == KERR_SCHILD_SPHERICAL) {
      R Sr[5];
      sks_sources<R>(p, xr, yr, Pr, mr, Sr);
      const R smg = mr.alpha * mr.sqrtgam;  // sqrt(-g) S
#pragma unroll
      for (int q = 1; q < 5; ++q) L[q] += smg * Sr[q];
    }
    double Un[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double u = a.g1 * LDC(a.Ucur, q * n + t, NV * n);
      if (a.g0 != 0.0) u += a.g0 * LDC(a.U0, q * n + t, NV * n);
      Un[q] = u + bdt * (double)L[q];
    }
    if (a.bface_new != nullptr) {
      // face-centred CT: the cell's densitized field is the mean of its two advanced faces of each direction
      const double* bn = a.bface_new;
      Un[5] = 0.5 * (LDC(bn, g, 3 * G) + LDC(bn, g + 1, 3 * G));
      Un[6] = 0.5 * (LDC(bn, G + g, 3 * G) + LDC(bn, G + g + sy, 3 * G));
      Un[7] = 0.5 * (LDC(bn, 2 * G + g, 3 * G) + LDC(bn, 2 * G + g + sz, 3 * G));
    }
    // a6: con2prim on the undensitized state, warm-started from the current primitives
    double Uc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) Uc[q] = Un[q] * isg;
    const double mu0 = (double)mu_of_prims<R>(Pr, mr.gam, par<R>(p.gamma_eos, p.fgamma));
    double Pn[NV];
    int iters;
    int st = con2prim<double>(p, m, Uc, mu0, Pn, iters);
    st |= apply_floors_fr(p, m.gam, fr, Pn);
    if (st) {
      if (a.floorlist) {
        // the hydro state of this cell is re-derived from the floored P by floor_cell, in a pass whose warps
        // hold only such cells (a few percent of cells, but present in most warps of this pass)
        STC(a.floorlist, atomicAdd(a.fl_count, 1u), n, (int)(wl_tag + t));
      } else {
        double U5[5];
        prim_to_cons5<double>(Pn, m, p.gamma_eos, U5);
#pragma unroll
        for (int q = 0; q < 5; ++q) Un[q] = U5[q];
      }
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) STC(a.Unew, q * n + t, NV * n, Un[q]);
#pragma unroll
    for (int q = 0; q < NV; ++q) STC(P, q * G + g, NV * G, (T)Pn[q]);
    STC(a.status, t, n, (uint8_t)st);
    cs.add(st, iters);
  }
}

// Resident CTAs per SM the update kernel is compiled for: the mixed form's (double solve, ~170 registers
// unbounded) is latency-bound at two CTAs per SM; held to four (123 registers, no spills) it runs 5.38 ms per
// 256^3 stage, against 6.35 at five (96 registers, spilling); the FP64 form keeps its registers.
template <class T>
constexpr int kUpdateMinBlocks = sizeof(T) == 4 ? 4 : 1;

template <int METRIC, class R, class T>
__global__ void __launch_bounds__(128, kUpdateMinBlocks<T>) k_update(T* __restrict__ P, const R* __restrict__ Fx,
                                                const R* __restrict__ Fy, const R* __restrict__ Fz,
                                                const R* __restrict__ E, StageArgs a, DevParams p) {
  const double dt = a.use_dev_dt ? *a.dt_dev : a.dt;
  CellStats cs;
  const long long t1 = a.t_end > 0 ? a.t_end : p.isize;
  for (long long t = a.t_begin + blockIdx.x * (long long)blockDim.x + threadIdx.x; t < t1;
       t += (long long)gridDim.x * blockDim.x)
    update_cell<METRIC, R, T>(p, P, Fx, Fy, Fz, E, a, dt, t, 0, cs);
  cs.flush(a.stats);
}

// Mixed form, passes over the cells whose float con2prim phase in k_update did not settle (Unew holds their
// conserved state). Pass 1 (full = false, cell t with tag wl_tag + t from the worklist): one double Newton
// step resumed from that phase's double iterate mu_r; a cell whose step does not settle is queued on the
// solve list (or solved in place without one). Pass 2 (full = true, from the solve list): the full double
// con2prim, warm-started from the current primitives. Nine in ten worklist cells settle in pass 1, and the
// full iteration, ten times as long, runs only in warps of cells that need it.
template <int METRIC, class T>
__device__ __forceinline__ void deferred_cell(const DevParams& p, T* __restrict__ P, const StageArgs& a, long long t,
                                              double mu_r, bool full, long long wl_tag, CellStats& cs) {
  const long long n = p.isize, G = p.gsize;
  const int i = (int)(t % p.nx), j = (int)((t / p.nx) % p.ny), k = (int)(t / ((long long)p.nx * p.ny));
  const long long g = gidx(p, i, j, k);
  Metric<double> m;
  double isg, fr;
  cell_metric<METRIC>(p, t, p.x0[0] + (i + 0.5) * p.dx[0], p.x0[1] + (j + 0.5) * p.dx[1],
                      p.x0[2] + (k + 0.5) * p.dx[2], m, isg, fr);
  double Uc[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) Uc[q] = LDC(a.Unew, q * n + t, NV * n) * isg;
  double Pn[NV];
  int iters = 0, st = 0;
  if (full || !con2prim_resume_step<double>(p, m, Uc, mu_r, Pn, iters)) {
    if (!full && a.solvelist != nullptr) {
      STC(a.solvelist, atomicAdd(a.sl_count, 1u), n, (int)(wl_tag + t));
      cs.it_sum += iters;
      return;
    }
    double Pc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) Pc[q] = (double)LDC(P, q * G + g, NV * G);
    const double mu0 = mu_of_prims<double>(Pc, m.gam, p.gamma_eos);
    int it2 = 0;
    st = con2prim<double>(p, m, Uc, mu0, Pn, it2, true);
    iters += it2;
  }
  st |= apply_floors_fr(p, m.gam, fr, Pn);
  if (st) {
    double U5[5];
    prim_to_cons5<double>(Pn, m, p.gamma_eos, U5);
#pragma unroll
    for (int q = 0; q < 5; ++q) STC(a.Unew, q * n + t, NV * n, U5[q]);
  }
#pragma unroll
  for (int q = 0; q < NV; ++q) STC(P, q * G + g, NV * G, (T)Pn[q]);
  STC(a.status, t, n, (uint8_t)st);
  cs.add(st, iters);
}

// Hydro part of the conserved state of a cell whose floors (or status) fired in update_cell,
// re-derived from the primitives it stored.
template <int METRIC, class T>
__device__ __forceinline__ void floor_cell(const DevParams& p, const T* __restrict__ P, const StageArgs& a, long long t) {
  const long long n = p.isize, G = p.gsize;
  const int i = (int)(t % p.nx), j = (int)((t / p.nx) % p.ny), k = (int)(t / ((long long)p.nx * p.ny));
  const long long g = gidx(p, i, j, k);
  Metric<double> m;
  double isg, fr;
  cell_metric<METRIC>(p, t, p.x0[0] + (i + 0.5) * p.dx[0], p.x0[1] + (j + 0.5) * p.dx[1],
                      p.x0[2] + (k + 0.5) * p.dx[2], m, isg, fr);
  double Pn[NV], U5[5];
#pragma unroll
  for (int q = 0; q < NV; ++q) Pn[q] = (double)LDC(P, q * G + g, NV * G);
  prim_to_cons5<double>(Pn, m, p.gamma_eos, U5);
#pragma unroll
  for (int q = 0; q < 5; ++q) STC(a.Unew, q * n + t, NV * n, U5[q]);
}

template <int METRIC, class T>
__global__ void __launch_bounds__(128) k_update_floors(const T* __restrict__ P, StageArgs a, DevParams p) {
  const unsigned int cnt = *a.fl_count;
  for (unsigned int w = blockIdx.x * blockDim.x + threadIdx.x; w < cnt; w += gridDim.x * blockDim.x)
    floor_cell<METRIC, T>(p, P, a, LDC(a.floorlist, w, p.isize));
}

template <int METRIC, class T>
__global__ void __launch_bounds__(128) k_update_deferred(T* __restrict__ P, StageArgs a, DevParams p, int full) {
  const unsigned int cnt = full ? *a.sl_count : *a.wl_count;
  CellStats cs;
  for (unsigned int w = blockIdx.x * blockDim.x + threadIdx.x; w < cnt; w += gridDim.x * blockDim.x) {
    if (full)
      deferred_cell<METRIC, T>(p, P, a, LDC(a.solvelist, w, p.isize), 0.0, true, 0, cs);
    else
      deferred_cell<METRIC, T>(p, P, a, LDC(a.worklist, w, p.isize), LDC(a.wl_mu, w, p.isize), false, 0, cs);
  }
  cs.flush(a.stats);
  // deferred cells of the stage (summed over the slabs of an update run in z slabs)
  if (!full && a.stats && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.stats + 7, (unsigned long long)cnt);
}

// ------------------------------------------------------------------ batched (many meshblocks)
// Persistent kernels: each CTA takes work items from a device counter until the list is empty,
// so one launch covers every block of the batch for one phase.
__device__ __forceinline__ int next_item(unsigned int* counter) {
  __shared__ int s_item;
  __syncthreads();
  if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
  __syncthreads();
  return s_item;
}

__device__ __forceinline__ StageArgs block_stage_args(const BlockDesc& b, const BatchArgs& a) {
  StageArgs s{};
  s.U0 = b.U[a.s0];
  s.Ucur = b.U[a.sc];
  s.Unew = b.U[a.dst];
  s.status = b.status;
  s.dt_dev = a.dt_dev;
  s.stats = a.stats;
  s.g0 = a.g0;
  s.g1 = a.g1;
  s.beta = a.beta;
  s.dt = a.dt;
  s.use_dev_dt = a.use_dev_dt;
  s.worklist = a.worklist;
  s.wl_count = a.wl_count;
  s.wl_mu = a.wl_mu;
  s.floorlist = a.floorlist;
  s.fl_count = a.fl_count;
  s.solvelist = a.solvelist;
  s.sl_count = a.sl_count;
  return s;
}

// Same-level ghost exchange of a lattice batch: every ghost cell of every block takes the primitives of
// the cell with the same global index in the block that owns it. Outside the lattice the global index
// wraps when periodic; otherwise the ghost keeps its value (fixed outer boundary). Sources are interior
// cells and destinations ghost cells, so the copies never overlap.
template <class T>
__global__ void k_batch_exchange(const BlockDesc* __restrict__ blocks, int nblocks, Lattice L) {
  const DevParams& p0 = blocks[0].p;  // every block of a lattice has the same sizes
  const long long G = p0.gsize;
  const int n[3] = {p0.nx, p0.ny, p0.nz};
  const long long total = (long long)nblocks * G;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / G);
    const long long g = t - (long long)b * G;
    const int c[3] = {(int)(g % p0.gx) - p0.ng, (int)((g / p0.gx) % p0.gy) - p0.ng,
                      (int)(g / ((long long)p0.gx * p0.gy)) - p0.ng};
    if (c[0] >= 0 && c[0] < n[0] && c[1] >= 0 && c[1] < n[1] && c[2] >= 0 && c[2] < n[2]) continue;
    const int bc[3] = {b % L.nb[0], (b / L.nb[0]) % L.nb[1], b / (L.nb[0] * L.nb[1])};
    int src[3], sb[3];
    bool outside = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const long long N = (long long)L.nb[d] * n[d];
      long long gd = (long long)bc[d] * n[d] + c[d];
      if (gd < 0 || gd >= N) {
        outside = true;
        gd = ((gd % N) + N) % N;
      }
      sb[d] = (int)(gd / n[d]);
      src[d] = (int)(gd - (long long)sb[d] * n[d]);
    }
    if (outside && !L.periodic) continue;
    const BlockDesc& S = blocks[sb[0] + L.nb[0] * (sb[1] + L.nb[1] * sb[2])];
    const T* __restrict__ Ps = (const T*)S.P;
    T* __restrict__ Pd = (T*)blocks[b].P;
    const long long gs = gidx(S.p, src[0], src[1], src[2]);
#pragma unroll
    for (int q = 0; q < NV; ++q) Pd[q * G + g] = Ps[q * G + gs];
    if (S.X) ((T*)blocks[b].X)[g] = ((const T*)S.X)[gs];  // the passive scalar, when the batch has one
  }
}

// Fluxes of every direction of every block; ms[0] collects max |lambda| / dx over the batch.
template <class R, class T, int METRIC, int RECON>
__global__ void __launch_bounds__(128, kFluxMinBlocks<R>) k_batch_flux(const BlockDesc* __restrict__ blocks,
                                                    const WorkItem* __restrict__ items, int nitems,
                                                    unsigned int* counter, unsigned long long* ms, int track_speed) {
  R cm_local = R(0);
  for (;;) {
    const int it = next_item(counter);
    if (it >= nitems) break;
    const WorkItem w = items[it];
    const BlockDesc& b = blocks[w.block];
    const R idx = R(b.p.idx[w.phase]);
    for (int k = threadIdx.x; k < w.count; k += blockDim.x) {
      // units of flux_units: runs of faces for the five-point reconstructions (cell-centric), single faces otherwise
      const R cm = (!cell_centric(RECON)
                        ? flux_face<R, T, METRIC, RECON>(b.p, (const T*)b.P, (R*)b.F[w.phase], w.phase, w.start + k)
                        : (w.phase == 0 ? flux_lane<R, T, METRIC, RECON>(b.p, (const T*)b.P, (R*)b.F[0], w.start + k)
                                        : flux_run<R, T, METRIC, RECON>(b.p, (const T*)b.P, (R*)b.F[w.phase], w.phase,
                                                                        w.start + k))) *
                   idx;
      if (cm > cm_local) cm_local = cm;
    }
  }
  if (track_speed) block_max_to<R>(cm_local, ms);
}

template <class R>
__global__ void __launch_bounds__(128) k_batch_emf(const BlockDesc* __restrict__ blocks,
                                                   const WorkItem* __restrict__ items, int nitems,
                                                   unsigned int* counter) {
  for (;;) {
    const int it = next_item(counter);
    if (it >= nitems) break;
    const WorkItem w = items[it];
    const BlockDesc& b = blocks[w.block];
    for (int k = threadIdx.x; k < w.count; k += blockDim.x)
      emf_edge<R>(b.p, (const R*)b.F[0], (const R*)b.F[1], (const R*)b.F[2], (R*)b.E, w.start + k);
  }
}

// The block descriptor and the stage arguments of the CTA's current item sit in shared memory: read from
// global memory into registers they had held ~40 of them across the cell loop (the single-block k_update reads
// its arguments from the constant bank), 187 registers in all; staged, the mixed form fits the same 4 CTAs per
// SM as k_update (640-block batch: 11.17 ms per stage against 11.60 at 2 CTAs per SM; 3 CTAs: 11.89).
template <int METRIC, class R, class T>
__global__ void __launch_bounds__(128, kUpdateMinBlocks<T>) k_batch_update(const BlockDesc* __restrict__ blocks,
                                                      const WorkItem* __restrict__ items, int nitems,
                                                      unsigned int* counter, BatchArgs a) {
  const double dt = a.use_dev_dt ? *a.dt_dev : a.dt;
  CellStats cs;
  __shared__ BlockDesc s_b;
  __shared__ StageArgs s_sa;
  for (;;) {
    const int it = next_item(counter);  // barrier before and after: the previous item is finished
    if (it >= nitems) break;
    const WorkItem w = items[it];
    if (threadIdx.x == 0) {
      s_b = blocks[w.block];
      s_sa = block_stage_args(s_b, a);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < w.count; k += blockDim.x)
      update_cell<METRIC, R, T>(s_b.p, (T*)s_b.P, (const R*)s_b.F[0], (const R*)s_b.F[1], (const R*)s_b.F[2],
                                (const R*)s_b.E, s_sa, dt, w.start + k, s_b.cell_offset, cs);
  }
  cs.flush(a.stats);
}

// Deferred con2prim cells of the batch (deferred_cell's two passes): list entries are batch-wide cell indices.
template <int METRIC, class T>
__global__ void __launch_bounds__(128) k_batch_deferred(const BlockDesc* __restrict__ blocks, int nblocks,
                                                        BatchArgs a, int full) {
  const unsigned int cnt = full ? *a.sl_count : *a.wl_count;
  CellStats cs;
  for (unsigned int w = blockIdx.x * blockDim.x + threadIdx.x; w < cnt; w += gridDim.x * blockDim.x) {
    const long long gcell = full ? a.solvelist[w] : a.worklist[w];
    int lo = 0, hi = nblocks - 1;  // last block whose cell_offset <= gcell
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (blocks[mid].cell_offset <= gcell) lo = mid; else hi = mid - 1;
    }
    const BlockDesc& b = blocks[lo];
    const StageArgs sa = block_stage_args(b, a);
    deferred_cell<METRIC, T>(b.p, (T*)b.P, sa, gcell - b.cell_offset, full ? 0.0 : a.wl_mu[w], full != 0,
                             b.cell_offset, cs);
  }
  cs.flush(a.stats);
  // deferred cells of the stage
  if (!full && a.stats && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.stats + 7, (unsigned long long)cnt);
}

template <int METRIC, class T>
__global__ void __launch_bounds__(128) k_batch_floors(const BlockDesc* __restrict__ blocks, int nblocks, BatchArgs a) {
  const unsigned int cnt = *a.fl_count;
  for (unsigned int w = blockIdx.x * blockDim.x + threadIdx.x; w < cnt; w += gridDim.x * blockDim.x) {
    const long long gcell = a.floorlist[w];
    int lo = 0, hi = nblocks - 1;  // last block whose cell_offset <= gcell
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (blocks[mid].cell_offset <= gcell) lo = mid; else hi = mid - 1;
    }
    const BlockDesc& b = blocks[lo];
    const StageArgs sa = block_stage_args(b, a);
    floor_cell<METRIC, T>(b.p, (const T*)b.P, sa, gcell - b.cell_offset);
  }
}

// dt = cfl / (max over the batch of |lambda| / dx)
static __global__ void k_batch_finalize_dt(const unsigned long long* ms, double* dt, double cfl) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *dt = cfl / __longlong_as_double((long long)ms[0]);
}

// Densitized conserved state of interior cells t0 <= t < t1 from the primitives (set-up and checkpoint restore).
template <int METRIC, class T>
__global__ void k_prim2con(const T* __restrict__ P, double* __restrict__ U, DevParams p, long long t0, long long t1) {
  const long long n = p.isize, G = p.gsize;
  for (long long t = t0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; t < t1; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % p.nx), j = (int)((t / p.nx) % p.ny), k = (int)(t / ((long long)p.nx * p.ny));
    const long long g = gidx(p, i, j, k);
    double Pc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) Pc[q] = (double)P[q * G + g];
    Metric<double> m;
    double isg, fr;  // the metric from the block's geometry cache when it has one (same values as in place)
    cell_metric<METRIC>(p, t, p.x0[0] + (i + 0.5) * p.dx[0], p.x0[1] + (j + 0.5) * p.dx[1],
                        p.x0[2] + (k + 0.5) * p.dx[2], m, isg, fr);
    double U5[5];
    prim_to_cons5<double>(Pc, m, p.gamma_eos, U5);
#pragma unroll
    for (int q = 0; q < 5; ++q) U[q * n + t] = U5[q];
#pragma unroll
    for (int q = 5; q < NV; ++q) U[q * n + t] = m.sqrtgam * Pc[q];
  }
}

// Flat-space prim->cons over a batch: P, U are [8][n] (structure of arrays).
static __global__ void k_p2c_batch(const double* __restrict__ P, double* __restrict__ U, long long n, DevParams p) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    Metric<double> m;
    metric_at<double, MINKOWSKI>(p, 0.0, 0.0, 0.0, m);
    double Pc[NV], U5[5];
#pragma unroll
    for (int q = 0; q < NV; ++q) Pc[q] = P[q * n + t];
    prim_to_cons5<double>(Pc, m, p.gamma_eos, U5);
#pragma unroll
    for (int q = 0; q < 5; ++q) U[q * n + t] = U5[q];
#pragma unroll
    for (int q = 5; q < NV; ++q) U[q * n + t] = Pc[q];
  }
}

// Flat-space con2prim over a batch: U, P are [8][n] (structure of arrays).
// flags bit 0: use P as the warm start.
static __global__ void k_c2p_batch(const double* __restrict__ U, double* __restrict__ P, uint8_t* __restrict__ status,
                            int* __restrict__ iters_out, long long n, int flags, DevParams p,
                            unsigned long long* stats) {
  unsigned int it_sum = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    Metric<double> m;
    metric_at<double, MINKOWSKI>(p, 0.0, 0.0, 0.0, m);
    double Uc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) Uc[q] = U[q * n + t];
    double mu0 = -1.0;
    if (flags & 1) {
      double Pg[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) Pg[q] = P[q * n + t];
      mu0 = mu_of_prims<double>(Pg, m.gam, p.gamma_eos);
    }
    double Pn[NV];
    int iters;
    int st = con2prim<double>(p, m, Uc, mu0, Pn, iters, true);
    st |= apply_floors<MINKOWSKI>(p, m.gam, 1.0, Pn);
#pragma unroll
    for (int q = 0; q < NV; ++q) P[q * n + t] = Pn[q];
    if (status) status[t] = (uint8_t)st;
    if (iters_out) iters_out[t] = iters;
    it_sum += iters;
  }
  if (stats) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) it_sum += __shfl_xor_sync(0xffffffffu, it_sum, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(stats, (unsigned long long)it_sum);
  }
}

template <class Tin, class Tout>
__global__ void k_convert(const Tin* __restrict__ a, Tout* __restrict__ b, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    b[t] = (Tout)a[t];
}

}  // namespace grmhd
