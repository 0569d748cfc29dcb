// Device-side building blocks of the GRMHD Runge-Kutta stage (sm_103a).
//
// Method: Barker et al., "Phoebus" (arXiv:2410.09146) -- Valencia GRMHD, Sec. 2.1;
// analytic metric, Sec. 2.3; second-order FV with LLF/HLL, PLM/WENO5-Z-AOAH, Toth flux-CT
// and Kastaun con2prim, Sec. 3.1; floors, Sec. 3.2; WENO5-Z-AOAH, App. B.
//
// Everything here is templated on the arithmetic type R (double for the all-FP64 form,
// float for the reconstruction / flux / EMF / source part of the mixed form).
#pragma once

#include <type_traits>
#include <cuda_runtime.h>
#include <stdint.h>

namespace grmhd {

// metrics: flat, Cartesian Kerr-Schild, Kerr-Schild in spherical coordinates (x^1, x^2, x^3) = (ln r, theta, phi)
enum { MINKOWSKI = 0, KERR_SCHILD = 1, KERR_SCHILD_SPHERICAL = 2 };
// boundaries: periodic, fixed ghosts, spherical (polar ghosts mirrored across the axis, phi periodic)
enum { BC_PERIODIC = 0, BC_FIXED = 1, BC_SPHERICAL = 2 };
enum { RECON_CONSTANT = 0, RECON_PLM_MINMOD = 1, RECON_PLM_MC = 2, RECON_WENO5Z = 3, RECON_MP5 = 4 };

// Five-point reconstructions (WENO5-Z-AOAH, MP5) run on the cell-centric flux path.
__host__ __device__ constexpr bool cell_centric(int recon) { return recon == RECON_WENO5Z || recon == RECON_MP5; }
enum { RIEMANN_LLF = 0, RIEMANN_HLL = 1 };
enum { ST_RHO_FLOOR = 1, ST_EPS_FLOOR = 2, ST_W_CAP = 4, ST_NOT_CONVERGED = 8, ST_BAD_INPUT = 16 };
enum { NV = 8 };

// Kernel-side copy of the run parameters (passed by value).
struct DevParams {
  int nx, ny, nz, ng;
  int gx, gy, gz;            // ghosted extents
  long long gsize;           // gx*gy*gz: stride between variables of P, F, E
  long long isize;           // nx*ny*nz: stride between variables of U
  double x0[3], dx[3], idx[3];
  double a, M;               // spin parameter a = spin*M, mass M
  double gamma_eos;
  int metric, recon, riemann, bc;
  double rho_floor0, eps_floor0, floor_r_exp, w_max;
  double w_max2, v0sq_cap;   // w_max^2 and 1 - 1/w_max^2 (velocity bound of the con2prim solve)
  double c2p_tol;
  int c2p_max_iter;
  double cfl, weno_eps;
  // Geometry cache: NGEO doubles per interior cell (structure of arrays, isize apart) holding the
  // static Kerr-Schild metric at the cell centre, filled once per block; NULL: computed in place.
  const double* geo;
  // Face-centred CT: the stage's face field sqrt(gamma) B^d, [3][gsize] double (entry (i,j,k) of
  // component d on the lower d-face of cell (i,j,k)); the flux kernels take the normal field from it.
  // NULL: cell-centred field (flux-CT).
  const double* bface;
  double shift[3];  // Minkowski: constant shift beta^i (flat space in coordinates moving at -beta)
  // Float copies of the parameters the float kernels read (set with the double ones): a double -> float
  // conversion costs an FP64 issue slot on this part, so the float code reads these instead.
  float fx0[3], fdx[3], fidx[3], fa, fM, fgamma, fweno_eps, frho_floor0, feps_floor0, fw_max2, fshift[3];
  float fv0sq_cap;
  int floor_r2;  // floor_r_exp == 2 (the radius factor is 1/r^2)
  int flux_run;  // faces per run of the cell-centric y / z flux units (0: FLUX_RUN)
  // Bounds-check build (GRMHD_BOUNDS_CHECK): the word where the first out-of-range access of a stage kernel
  // is recorded (see bounds_fault); unused otherwise.
  unsigned long long* fault;
};

// Checked global-memory access of the stage kernels. In the bounds-check build (-DGRMHD_BOUNDS_CHECK) every
// load / store through ldc / stc compares its index with the extent of the array; the first index outside
// [0, n) is recorded in *p.fault as (source line << 48) | (sign << 47) | |index|, plus one (0 = none), and the
// access is skipped (a load returns 0). Nothing traps, so a faulty index leaves the context usable. In the
// normal build both are the plain access.
__device__ __forceinline__ void bounds_fault(const DevParams& p, int line, long long i) {
  if (p.fault == nullptr) return;
  const unsigned long long mag = (unsigned long long)(i < 0 ? -i : i) & ((1ull << 47) - 1);
  const unsigned long long w = (((unsigned long long)line & 0xffffull) << 48) | ((i < 0 ? 1ull : 0ull) << 47) | mag;
  atomicCAS(p.fault, 0ull, w + 1);
}

template <class X>
__device__ __forceinline__ X ldc(const DevParams& p, const X* __restrict__ a, long long i, long long n, int line) {
#ifdef GRMHD_BOUNDS_CHECK
  if (i < 0 || i >= n) {
    bounds_fault(p, line, i);
    return X(0);
  }
#endif
  (void)p; (void)n; (void)line;
  return a[i];
}

template <class X>
__device__ __forceinline__ void stc(const DevParams& p, X* __restrict__ a, long long i, long long n, X v, int line) {
#ifdef GRMHD_BOUNDS_CHECK
  if (i < 0 || i >= n) {
    bounds_fault(p, line, i);
    return;
  }
#endif
  (void)p; (void)n; (void)line;
  a[i] = v;
}

#define LDC(arr, i, n) ldc(p, (arr), (long long)(i), (long long)(n), __LINE__)
#define STC(arr, i, n, v) stc(p, (arr), (long long)(i), (long long)(n), (v), __LINE__)

// A parameter in the arithmetic type R: the double field in double code, its float copy in float code.
template <class R>
__host__ __device__ __forceinline__ R par(double d, float f) {
  if constexpr (sizeof(R) == 4) {
    return f;
  } else {
    return (R)d;
  }
}

// Arguments of the update kernel (a5 + a6).
struct StageArgs {
  const double* U0;
  const double* Ucur;
  double* Unew;
  uint8_t* status;
  const double* dt_dev;          // used when use_dev_dt != 0
  unsigned long long* stats;     // [0] iterations, [1] rho floor, [2] eps floor, [3] W cap, [4] not converged,
                                 // [5] bad input, [6] max iterations
  double g0, g1, beta, dt;
  int use_dev_dt;
  int* worklist;                 // mixed form: cells whose float con2prim phase did not settle
  unsigned int* wl_count;        // number of entries in worklist
  double* wl_mu;                 // per worklist entry: the double iterate to resume from (0: none)
  int* floorlist;                // cells whose floors / status re-derive U in a compacted pass (NULL: inline)
  unsigned int* fl_count;        // number of entries in floorlist
  const double* bface_new;       // face-centred CT: the advanced faces [3][gsize]; NULL: flux-CT
  int* solvelist;                // mixed form: worklist cells whose resumed double step did not settle, for
  unsigned int* sl_count;        // the full double iteration in a last pass (NULL: inline); its count
  long long t_begin, t_end;      // single-block update: interior cells [t_begin, t_end) (t_end = 0: all)
};


// Face box of direction d: face index along d in [0, n_d], transverse cell indices in [-1, n_t]
// (the transverse halo feeds the CT edge averages).
__host__ __device__ __forceinline__ long long face_box(const DevParams& p, int d, int& ex, int& ey) {
  ex = p.nx + (d == 0 ? 1 : 2);
  ey = p.ny + (d == 1 ? 1 : 2);
  const int ez = p.nz + (d == 2 ? 1 : 2);
  return (long long)ex * ey * ez;
}

// One meshblock of a batch: its geometry and where its arrays live in the workspace.
struct BlockDesc {
  DevParams p;
  void* P;                // primitives [8][gz][gy][gx] (storage type of the form)
  void* F[3];             // face fluxes per direction
  void* E;                // edge EMFs
  double* U[3];           // conserved-state slots
  uint8_t* status;
  long long cell_offset;  // index of the block's first interior cell in the batch
  int level;              // two-level mesh: 0 (root block) or 1 (child of a refined root block)
  int pos[3];             // two-level mesh: position in its level's block lattice
  void* X;                // passive scalar X [gsize] (storage type of P), NULL without one
  double* DX[3];          // passive scalar: sqrt(gamma) D X slots [isize], paired with U
  void* FX;               // passive scalar: face fluxes [3][gsize] (flux type)
};

// A contiguous range of flux units (faces, or runs of faces: flux_units) / edges / cells of one block
// (phase 0..2: fluxes of direction d, 3: EMFs, 4: cell update).
struct WorkItem {
  int block;
  int phase;
  long long start;
  int count;
  int pad;
};

// A batch whose blocks, all of the same size, tile an nb[0] x nb[1] x nb[2] lattice: block b sits at
// lattice position (b % nb[0], (b / nb[0]) % nb[1], b / (nb[0] nb[1])). periodic: the lattice wraps.
struct Lattice {
  int nb[3];
  int periodic;
};

// A batch whose blocks, all of the same size, are the leaves of a two-level mesh over an nb[0] x nb[1] x
// nb[2] grid of root blocks (BlockDesc::level / pos). leaf: the block covering each fine-block-sized unit
// of the mesh, [2 nb[2]][2 nb[1]][2 nb[0]] (a root block covers 2 x 2 x 2 units). periodic: the mesh wraps.
struct MeshDesc {
  int nb[3];
  int periodic;
  const int* leaf;
  // the ghost cells of a block (all blocks have the same extents): ghosted indices packed as
  // i | j << 10 | k << 20, nghost of them
  const unsigned* ghost;
  int nghost;
  // the level-1 blocks (the only ones pass 2 writes to)
  const int* fine;
  int nfine;
};

// A coarse cell with at least one face on a fine leaf: fine[2 d + s] is the fine block across its lower
// (s = 0) or upper (s = 1) face of direction d, or -1.
struct RefluxCell {
  int block;
  int cell;
  int fine[6];
};

// Coefficients and bookkeeping shared by every block of a batched stage.
struct BatchArgs {
  double g0, g1, beta, dt;
  int use_dev_dt, s0, sc, dst;
  const double* dt_dev;
  unsigned long long* stats;
  int* worklist;
  unsigned int* wl_count;
  double* wl_mu;
  int* floorlist;
  unsigned int* fl_count;
  int* solvelist;
  unsigned int* sl_count;
};

// ------------------------------------------------------------------ metric (Sec. 2.3)
// gam / gamu hold the symmetric 3x3 in the order xx, xy, xz, yy, yz, zz.
template <class R>
struct Metric {
  R alpha, beta[3], gam[6], gamu[6], sqrtgam;
};

__host__ __device__ constexpr int sym3(int i, int j) {
  return i <= j ? (i == 0 ? j : (i == 1 ? 2 + j : 5)) : (j == 0 ? i : (j == 1 ? 2 + i : 5));
}

// Geometry cache entries: alpha, beta^i (3), gamma_ij (6), gamma^ij (6), sqrt(gamma), 1/sqrt(gamma), the
// floor radius factor r^-floor_r_exp, then the Kerr-Schild factors f, kappa = f/(1+f) and l_i (5), from which
// gamma_ij = delta_ij + f l_i l_j and gamma^ij = delta^ij - kappa l^i l^j: the mixed form's con2prim reads
// these and 1/sqrt(gamma) (6 doubles) instead of the two matrices (13).
constexpr int NGEO = 24;

// The spatial metric as the mixed form's con2prim takes it: gamma_ij = delta_ij + f l_i l_j,
// gamma^ij = delta^ij - kappa l^i l^j (Kerr-Schild, kappa = f/(1+f); flat space: f = kappa = 0).
struct KSGeo {
  double f, kappa, l[3];
};

__device__ __forceinline__ void geo_store(double* __restrict__ geo, long long n, long long t, const Metric<double>& m,
                                          double isg, double fr, const KSGeo& k) {
  geo[t] = m.alpha;
#pragma unroll
  for (int i = 0; i < 3; ++i) geo[(1 + i) * n + t] = m.beta[i];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    geo[(4 + i) * n + t] = m.gam[i];
    geo[(10 + i) * n + t] = m.gamu[i];
  }
  geo[16 * n + t] = m.sqrtgam;
  geo[17 * n + t] = isg;
  geo[18 * n + t] = fr;
  geo[19 * n + t] = k.f;
  geo[20 * n + t] = k.kappa;
#pragma unroll
  for (int i = 0; i < 3; ++i) geo[(21 + i) * n + t] = k.l[i];
}

__device__ __forceinline__ void geo_load(const double* __restrict__ geo, long long n, long long t, Metric<double>& m,
                                         double& isg, double& fr) {
  m.alpha = geo[t];
#pragma unroll
  for (int i = 0; i < 3; ++i) m.beta[i] = geo[(1 + i) * n + t];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    m.gam[i] = geo[(4 + i) * n + t];
    m.gamu[i] = geo[(10 + i) * n + t];
  }
  m.sqrtgam = geo[16 * n + t];
  isg = geo[17 * n + t];
  fr = geo[18 * n + t];
}

template <class R>
__device__ __forceinline__ R fdiv(R x, R y) { return x / y; }

// Quotients of the float flux path: the approximate quotient (reciprocal approximation times x, within
// 2 ulp for 2^-126 <= |y| <= 2^126) instead of the correctly rounded one, whose divide sequence takes ~4x
// the instructions (~85 quotients per face); the double form keeps the IEEE quotient.
template <>
__device__ __forceinline__ float fdiv<float>(float x, float y) { return __fdividef(x, y); }

template <class R>
__device__ __forceinline__ R rcp(R x) { return fdiv(R(1), x); }

// x finite, and x > 0 for finite x, from the bit pattern: integer instructions, where a double compare
// would take a slot of the FP64 pipe that binds the mixed form's update.
__device__ __forceinline__ bool dfinite(double x) { return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000; }
__device__ __forceinline__ bool dpositive(double x) { return __double_as_longlong(x) > 0; }

// Kerr-Schild core: r, f = 2 M r^3/(r^4 + a^2 z^2), spatial l_i (l_0 = 1).
template <class R>
__device__ __forceinline__ void ks_core(R x, R y, R z, R a, R M, R& r, R& r2, R& f, R l[3]) {
  const R R2 = x * x + y * y + z * z;
  const R A = R2 - a * a;
  const R sq = sqrt(A * A + R(4) * a * a * z * z);
  r2 = R(0.5) * (A + sq);
  r = sqrt(r2);
  f = fdiv(R(2) * M * r * r2, r2 * r2 + a * a * z * z);
  const R ira = rcp(r2 + a * a);
  l[0] = (r * x + a * y) * ira;
  l[1] = (r * y - a * x) * ira;
  l[2] = fdiv(z, r);
}

// 3+1 quantities in closed form: alpha = (1+f)^-1/2, beta^i = f l^i/(1+f),
// gamma_ij = delta_ij + f l_i l_j, gamma^ij = delta^ij - f l^i l^j/(1+f), sqrt(gamma) = (1+f)^1/2,
// sqrt(-g) = alpha sqrt(gamma) = 1.
template <class R, int METRIC>
__device__ __forceinline__ void metric_at(const DevParams& p, R x, R y, R z, Metric<R>& m, R* rks = nullptr) {
  if (METRIC == MINKOWSKI) {
    m.alpha = R(1);
    m.sqrtgam = R(1);
#pragma unroll
    for (int i = 0; i < 3; ++i) m.beta[i] = par<R>(p.shift[i], p.fshift[i]);
#pragma unroll
    for (int t = 0; t < 6; ++t) m.gam[t] = m.gamu[t] = (t == 0 || t == 3 || t == 5) ? R(1) : R(0);
    if (rks) *rks = R(1);
  } else if (METRIC == KERR_SCHILD_SPHERICAL) {
    // (x, y, z) = (ln r, theta, phi). In (r, theta, phi), with Sigma = r^2 + a^2 cos^2, q = 2 M r / Sigma:
    // alpha = (1+q)^-1/2, beta^r = q/(1+q) (beta^theta = beta^phi = 0), gamma_rr = 1+q, gamma_rphi =
    // -a sin^2 (1+q), gamma_thth = Sigma, gamma_phph = sin^2 (Sigma + a^2 sin^2 (1+q)); the inverse of the
    // (r, phi) block has determinant (1+q) sin^2 Sigma, so gamma^rr = 1/(1+q) + a^2 sin^2/Sigma, gamma^rphi =
    // a/Sigma, gamma^phph = 1/(Sigma sin^2), gamma^thth = 1/Sigma; sqrt(gamma) = Sigma |sin| (1+q)^1/2. Each r
    // index then carries a factor r (dr = r dx^1), an upper one 1/r.
    const R a = par<R>(p.a, p.fa), M = par<R>(p.M, p.fM);
    const R r = exp(x), sn = sin(y), cs = cos(y), s2 = sn * sn;
    const R Sig = r * r + a * a * cs * cs;
    const R iS = rcp(Sig);
    const R q = R(2) * M * r * iS;
    const R ip = rcp(R(1) + q);
    const R ir = rcp(r);
    m.alpha = sqrt(ip);
    m.beta[0] = q * ip * ir;
    m.beta[1] = m.beta[2] = R(0);
    m.gam[0] = r * r * (R(1) + q);
    m.gam[1] = R(0);
    m.gam[2] = -r * a * s2 * (R(1) + q);
    m.gam[3] = Sig;
    m.gam[4] = R(0);
    m.gam[5] = s2 * (Sig + a * a * s2 * (R(1) + q));
    m.gamu[0] = (ip + a * a * s2 * iS) * ir * ir;
    m.gamu[1] = R(0);
    m.gamu[2] = a * iS * ir;
    m.gamu[3] = iS;
    m.gamu[4] = R(0);
    m.gamu[5] = iS * rcp(s2);
    m.sqrtgam = r * Sig * fabs(sn) * sqrt(R(1) + q);
    if (rks) *rks = r;
  } else {
    R r, r2, f, l[3];
    ks_core<R>(x, y, z, par<R>(p.a, p.fa), par<R>(p.M, p.fM), r, r2, f, l);
    if (rks) *rks = r;
    const R sg = sqrt(R(1) + f);
    const R ip = rcp(R(1) + f);
    m.sqrtgam = sg;
    m.alpha = rcp(sg);
#pragma unroll
    for (int i = 0; i < 3; ++i) m.beta[i] = f * ip * l[i];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        const R ll = l[i] * l[j];
        m.gam[sym3(i, j)] = (i == j ? R(1) : R(0)) + f * ll;
        m.gamu[sym3(i, j)] = (i == j ? R(1) : R(0)) - f * ip * ll;
      }
  }
}

// Component d of a 3-vector by selects (d is a run-time direction: indexing an array with it would put the
// array in local memory).
template <class R>
__host__ __device__ __forceinline__ R sel3(int d, R a0, R a1, R a2) {
  return d == 0 ? a0 : (d == 1 ? a1 : a2);
}

template <class R>
__device__ __forceinline__ void lower3(const R g[6], const R v[3], R out[3]) {
  out[0] = g[0] * v[0] + g[1] * v[1] + g[2] * v[2];
  out[1] = g[1] * v[0] + g[3] * v[1] + g[4] * v[2];
  out[2] = g[2] * v[0] + g[4] * v[1] + g[5] * v[2];
}

// ------------------------------------------------------------------ fluid (Sec. 2.1)
// Densitized conserved vector sqrt(gamma) U, flux sqrt(-g) F^d and the two characteristic
// speeds of one face side, from the primitive vector P = (rho, W v^i, rho eps, B^i).
template <class R>
struct FaceSide {
  R U[NV], F[NV], lm, lp;
};

// smg: sqrt(-g) at the face (1 in the Cartesian metrics, where the flux needs no factor). The double form;
// float faces are formed two sides at a time by prim_to_face_x2.
template <class R>
__device__ __forceinline__ void prim_to_face(const R P[NV], const Metric<R>& m, int d, R gamma_eos,
                                             FaceSide<R>& s, R smg = R(1)) {
  static_assert(sizeof(R) == 8, "float face states are formed by prim_to_face_x2");
  const R rho = P[0], u = P[4];
  const R ut[3] = {P[1], P[2], P[3]};
  const R B[3] = {P[5], P[6], P[7]};
  R utl[3], Bl[3];
  lower3(m.gam, ut, utl);
  lower3(m.gam, B, Bl);
  const R usq = ut[0] * utl[0] + ut[1] * utl[1] + ut[2] * utl[2];
  const R W = sqrt(R(1) + usq);
  const R iW = rcp(W);
  const R ia = rcp(m.alpha);
  R v[3], vl[3], vt[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    v[i] = ut[i] * iW;
    vl[i] = utl[i] * iW;
    vt[i] = m.alpha * v[i] - m.beta[i];
  }
  const R B2 = B[0] * Bl[0] + B[1] * Bl[1] + B[2] * Bl[2];
  const R Bv = B[0] * vl[0] + B[1] * vl[1] + B[2] * vl[2];
  const R ab0 = W * Bv;                       // alpha b^0
  const R b2 = (B2 + ab0 * ab0) * iW * iW;    // b^2
  R bl[3];                                    // b_j = B_j / W + alpha b^0 v_j
#pragma unroll
  for (int i = 0; i < 3; ++i) bl[i] = Bl[i] * iW + ab0 * vl[i];
  const R pgas = (gamma_eos - R(1)) * u;
  const R rhoh = rho + u + pgas;
  const R pstar = pgas + R(0.5) * b2;
  const R D = rho * W;
  R Uc[NV];
  Uc[0] = D;
  const R wW2 = (rhoh + b2) * W * W;
#pragma unroll
  for (int j = 0; j < 3; ++j) Uc[1 + j] = wW2 * vl[j] - ab0 * bl[j];
  Uc[4] = wW2 - pstar - ab0 * ab0 - D;
#pragma unroll
  for (int k = 0; k < 3; ++k) Uc[5 + k] = B[k];
  const R vtd = sel3(d, vt[0], vt[1], vt[2]) * ia;
  const R Bd = sel3(d, B[0], B[1], B[2]);
  const R vd = sel3(d, v[0], v[1], v[2]);
  s.F[0] = D * vtd;
#pragma unroll
  for (int j = 0; j < 3; ++j) s.F[1 + j] = Uc[1 + j] * vtd + (j == d ? pstar : R(0)) - bl[j] * Bd * iW;
  s.F[4] = Uc[4] * vtd + pstar * vd - ab0 * Bd * iW;
#pragma unroll
  for (int k = 0; k < 3; ++k) s.F[5 + k] = B[k] * vtd - Bd * vt[k] * ia;
#pragma unroll
  for (int q = 0; q < NV; ++q) s.U[q] = m.sqrtgam * Uc[q];
#pragma unroll
  for (int q = 0; q < NV; ++q) s.F[q] *= smg;  // densitized flux sqrt(-g) F^d (a no-op in Cartesian metrics)
  // Valencia characteristic speeds with the approximate fast speed c^2 = vA^2 + cs^2 (1 - vA^2).
  const R cs2 = fdiv(gamma_eos * pgas, rhoh);
  const R va2 = fdiv(b2, rhoh + b2);
  const R c2 = va2 + cs2 * (R(1) - va2);
  // 1 - v^2 = 1/W^2, 1 - c^2 = (1 - vA^2)(1 - cs^2) with 1 - vA^2 = rho h/(rho h + b^2), and
  // 1 - v^2 c^2 = (1 - c^2) + c^2/W^2, instead of differences whose rounding grows like W^2
  const R one_v2 = rcp(W * W);
  const R one_c2 = fdiv(rhoh, rhoh + b2) * (R(1) - cs2);
  const R one_v2c2 = one_c2 + c2 * one_v2;
  R disc = one_v2 * (sel3(d, m.gamu[0], m.gamu[3], m.gamu[5]) * one_v2c2 - vd * vd * one_c2);
  disc = disc > R(0) ? disc : R(0);
  const R pre = fdiv(m.alpha, one_v2c2);
  const R sq = sqrt(c2 * disc);
  const R base = vd * one_c2;
  const R bd = sel3(d, m.beta[0], m.beta[1], m.beta[2]);
  s.lp = pre * (base + sq) - bd;
  s.lm = pre * (base - sq) - bd;
}

// Paired FP32 arithmetic: one f32x2 instruction applies the operation to both halves, each rounded as the
// scalar instruction rounds it, in one issue slot.
__device__ __forceinline__ float2 x2(float c) { return make_float2(c, c); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, x2(-1.f), a); }  // a - b, exact product
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(rcp(a.x), rcp(a.y)); }
__device__ __forceinline__ float2 sqrt2(float2 a) { return make_float2(sqrtf(a.x), sqrtf(a.y)); }
__device__ __forceinline__ float2 dot2(const float2 a[3], const float2 b[3]) {
  return fma2(a[2], b[2], fma2(a[1], b[1], mul2(a[0], b[0])));
}

// prim_to_face of both sides of a face at once, in float: the left state in the x halves of P and the right
// state in the y halves; every add, multiply and fma is issued once for the two sides (f32x2), the square
// roots and reciprocals per side. Outputs the densitized U and F^d of each side (F not yet times sqrt(-g))
// and their characteristic speeds.
// S_j and tau are taken in forms without cancellation. The printed forms
// S_j = (rho h + b^2) W^2 v_j - alpha b^0 b_j and tau = (rho h + b^2) W^2 - p* - (alpha b^0)^2 - D subtract
// terms of size W^2 (B.v)^2 (and rho W from rho h W^2), so their float rounding grows like W^2 in magnetised,
// relativistic cells. With b^2 W^2 = B^2 + (alpha b^0)^2 they are equal to
//   S_j = (rho h W^2 + B^2) v_j - (B.v) B_j,
//   tau = rho W u^2/(W + 1) + rho eps W^2 + p u^2 + B^2 - (B^2 + (alpha b^0)^2)/(2 W^2)   (u^2 = W^2 - 1),
// whose terms are all of the size of the result. The speeds use 1 - v^2 = 1/W^2 and
// 1 - c^2 = (1 - vA^2)(1 - cs^2) (prim_to_face).
__device__ __forceinline__ void prim_to_face_x2(const float2 P[NV], const Metric<float>& m, int d, float gamma_eos,
                                                float2 U[NV], float2 F[NV], float2& lm, float2& lp) {
  const float2 rho = P[0], u = P[4];
  const float2 ut[3] = {P[1], P[2], P[3]};
  const float2 B[3] = {P[5], P[6], P[7]};
  const float2 g0 = x2(m.gam[0]), g1 = x2(m.gam[1]), g2 = x2(m.gam[2]), g3 = x2(m.gam[3]), g4 = x2(m.gam[4]),
               g5 = x2(m.gam[5]);
  float2 utl[3], Bl[3];
  utl[0] = fma2(g2, ut[2], fma2(g1, ut[1], mul2(g0, ut[0])));
  utl[1] = fma2(g4, ut[2], fma2(g3, ut[1], mul2(g1, ut[0])));
  utl[2] = fma2(g5, ut[2], fma2(g4, ut[1], mul2(g2, ut[0])));
  Bl[0] = fma2(g2, B[2], fma2(g1, B[1], mul2(g0, B[0])));
  Bl[1] = fma2(g4, B[2], fma2(g3, B[1], mul2(g1, B[0])));
  Bl[2] = fma2(g5, B[2], fma2(g4, B[1], mul2(g2, B[0])));
  const float2 one = x2(1.f), neg = x2(-1.f);
  const float2 usq = dot2(ut, utl);
  const float2 W = sqrt2(add2(one, usq));
  const float2 iW = rcp2(W);
  const float ia = rcp(m.alpha);
  const float2 al = x2(m.alpha);
  float2 v[3], vl[3], vt[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    v[i] = mul2(ut[i], iW);
    vl[i] = mul2(utl[i], iW);
    vt[i] = fma2(al, v[i], x2(-m.beta[i]));
  }
  const float2 B2 = dot2(B, Bl);
  const float2 Bv = dot2(B, vl);
  const float2 ab0 = mul2(W, Bv);                              // alpha b^0
  const float2 W2 = mul2(W, W);
  const float2 b2 = mul2(mul2(fma2(ab0, ab0, B2), iW), iW);    // b^2
  const float2 pgas = mul2(x2(gamma_eos - 1.f), u);
  const float2 rhoh = add2(add2(rho, u), pgas);
  const float2 pstar = fma2(x2(0.5f), b2, pgas);
  const float2 D = mul2(rho, W);
  float2 Uc[NV];
  Uc[0] = D;
  const float2 wB = fma2(rhoh, W2, B2);                        // rho h W^2 + B^2
  const float2 nBv = mul2(Bv, neg);
#pragma unroll
  for (int j = 0; j < 3; ++j) Uc[1 + j] = fma2(wB, vl[j], mul2(nBv, Bl[j]));
  Uc[4] = add2(mul2(mul2(D, usq), rcp2(add2(W, one))), fma2(u, W2, fma2(pgas, usq, fma2(x2(-0.5f), b2, B2))));
#pragma unroll
  for (int k = 0; k < 3; ++k) Uc[5 + k] = B[k];
  const float2 vtd = mul2(sel3(d, vt[0], vt[1], vt[2]), x2(ia));
  const float2 Bd = sel3(d, B[0], B[1], B[2]);
  const float2 vd = sel3(d, v[0], v[1], v[2]);
  const float2 nBdiW = mul2(mul2(Bd, iW), neg);                // -B^d / W
  F[0] = mul2(D, vtd);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    // b_j = B_j / W + alpha b^0 v_j
    const float2 bl = fma2(ab0, vl[j], mul2(Bl[j], iW));
    F[1 + j] = fma2(Uc[1 + j], vtd, fma2(bl, nBdiW, j == d ? pstar : x2(0.f)));
  }
  F[4] = fma2(Uc[4], vtd, fma2(pstar, vd, mul2(ab0, nBdiW)));
  const float2 nBdia = mul2(Bd, x2(-ia));
#pragma unroll
  for (int k = 0; k < 3; ++k) F[5 + k] = fma2(B[k], vtd, mul2(nBdia, vt[k]));
  const float2 sg = x2(m.sqrtgam);
#pragma unroll
  for (int q = 0; q < NV; ++q) U[q] = mul2(sg, Uc[q]);
  // Valencia characteristic speeds with the approximate fast speed c^2 = vA^2 + cs^2 (1 - vA^2)
  const float2 irb = rcp2(add2(rhoh, b2));                     // 1 / (rho h + b^2)
  const float2 cs2 = mul2(mul2(x2(gamma_eos), pgas), rcp2(rhoh));
  const float2 va2 = mul2(b2, irb);
  const float2 c2 = fma2(cs2, sub2(one, va2), va2);
  const float2 one_v2 = rcp2(W2);
  const float2 one_c2 = mul2(mul2(rhoh, irb), sub2(one, cs2));
  const float2 one_v2c2 = fma2(c2, one_v2, one_c2);
  float2 disc = mul2(one_v2, fma2(x2(sel3(d, m.gamu[0], m.gamu[3], m.gamu[5])), one_v2c2,
                                  mul2(mul2(vd, vd), mul2(one_c2, neg))));
  disc = make_float2(disc.x > 0.f ? disc.x : 0.f, disc.y > 0.f ? disc.y : 0.f);
  const float2 pre = mul2(al, rcp2(one_v2c2));
  const float2 sq = sqrt2(mul2(c2, disc));
  const float2 base = mul2(vd, one_c2);
  const float2 nbd = x2(-sel3(d, m.beta[0], m.beta[1], m.beta[2]));
  lp = fma2(pre, add2(base, sq), nbd);
  lm = fma2(pre, sub2(base, sq), nbd);
}

// Hydro part of the densitized conserved vector only (used after floors).
template <class R>
__device__ __forceinline__ void prim_to_cons5(const R P[NV], const Metric<R>& m, R gamma_eos, R U5[5]) {
  const R ut[3] = {P[1], P[2], P[3]};
  const R B[3] = {P[5], P[6], P[7]};
  R utl[3], Bl[3];
  lower3(m.gam, ut, utl);
  lower3(m.gam, B, Bl);
  const R usq = ut[0] * utl[0] + ut[1] * utl[1] + ut[2] * utl[2];
  const R W = sqrt(R(1) + usq);
  const R iW = rcp(W);
  R vl[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) vl[i] = utl[i] * iW;
  const R B2 = B[0] * Bl[0] + B[1] * Bl[1] + B[2] * Bl[2];
  const R Bv = B[0] * vl[0] + B[1] * vl[1] + B[2] * vl[2];
  const R ab0 = W * Bv;
  const R b2 = (B2 + ab0 * ab0) * iW * iW;
  const R pgas = (gamma_eos - R(1)) * P[4];
  const R D = P[0] * W;
  U5[0] = m.sqrtgam * D;
  if constexpr (sizeof(R) == 4) {
    // float: the forms without cancellation of prim_to_face
    const R rhohW2 = (P[0] + P[4] + pgas) * W * W;
#pragma unroll
    for (int j = 0; j < 3; ++j) U5[1 + j] = m.sqrtgam * ((rhohW2 + B2) * vl[j] - Bv * Bl[j]);
    U5[4] = m.sqrtgam * (fdiv(D * usq, W + R(1)) + P[4] * W * W + pgas * usq + (B2 - R(0.5) * b2));
  } else {
    const R w = P[0] + P[4] + pgas + b2;
    const R wW2 = w * W * W;
#pragma unroll
    for (int j = 0; j < 3; ++j) U5[1 + j] = m.sqrtgam * (wW2 * vl[j] - ab0 * (Bl[j] * iW + ab0 * vl[j]));
    U5[4] = m.sqrtgam * (wW2 - (pgas + R(0.5) * b2) - ab0 * ab0 - D);
  }
}

// ------------------------------------------------------------------ reconstruction (Sec. 3.1, App. B)
template <class R>
__device__ __forceinline__ R mc_slope(R dm, R dp) {
  if (!(dm * dp > R(0))) return R(0);
  const R c = R(0.5) * (dm + dp);
  const R m = fmin(fmin(R(2) * fabs(dm), R(2) * fabs(dp)), fabs(c));
  return dm > R(0) ? m : -m;
}

template <class R>
__device__ __forceinline__ R minmod_slope(R dm, R dp) {
  if (!(dm * dp > R(0))) return R(0);
  const R m = fmin(fabs(dm), fabs(dp));
  return dm > R(0) ? m : -m;
}

// WENO5-Z values at both faces of the cell with centre value f2 (stencil f0..f4), and their nonlinear
// weights. Candidates are the third-order cell-average forms, linear weights (1/10, 6/10, 3/10),
// tau_Z = |beta_2 - beta_0|, exponent p = 2. The plus face comes from (f0..f4), the minus face from the
// mirrored stencil (f4..f0). The mirrored stencil has the same smoothness indicators in reverse order (beta_0 <-> beta_2)
// and the same tau, so they and the ratios tau/(beta + eps) are computed once; only the candidate values
// and the linear weights (gamma is not symmetric) differ between the two sides.
template <class R>
__device__ __forceinline__ void weno5z_both(R f0, R f1, R f2, R f3, R f4, R eps, R& qp, R& qm, R wp[3], R wm[3],
                                            R z[3]) {
  const R P0 = (R(2) * f0 - R(7) * f1 + R(11) * f2) * R(1.0 / 6.0);
  const R P1 = (-f1 + R(5) * f2 + R(2) * f3) * R(1.0 / 6.0);
  const R P2 = (R(2) * f2 + R(5) * f3 - f4) * R(1.0 / 6.0);
  const R M0 = (R(2) * f4 - R(7) * f3 + R(11) * f2) * R(1.0 / 6.0);  // mirrored candidates
  const R M1 = (-f3 + R(5) * f2 + R(2) * f1) * R(1.0 / 6.0);
  const R M2 = (R(2) * f2 + R(5) * f1 - f0) * R(1.0 / 6.0);
  const R t0 = f0 - R(2) * f1 + f2, s0 = f0 - R(4) * f1 + R(3) * f2;
  const R t1 = f1 - R(2) * f2 + f3, s1 = f1 - f3;
  const R t2 = f2 - R(2) * f3 + f4, s2 = R(3) * f2 - R(4) * f3 + f4;
  const R b0 = R(13.0 / 12.0) * t0 * t0 + R(0.25) * s0 * s0;
  const R b1 = R(13.0 / 12.0) * t1 * t1 + R(0.25) * s1 * s1;
  const R b2 = R(13.0 / 12.0) * t2 * t2 + R(0.25) * s2 * s2;
  const R tau = fabs(b2 - b0);
  R q0 = fdiv(tau, b0 + eps), q1 = fdiv(tau, b1 + eps), q2 = fdiv(tau, b2 + eps);
  if (sizeof(R) == 4) {  // keep q^2 inside the float range; a clamped q still dominates its weight
    q0 = fmin(q0, R(1e15));
    q1 = fmin(q1, R(1e15));
    q2 = fmin(q2, R(1e15));
  }
  const R z0 = R(1) + q0 * q0, z1 = R(1) + q1 * q1, z2 = R(1) + q2 * q2;
  z[0] = z0;
  z[1] = z1;
  z[2] = z2;
  const R a0 = R(0.1) * z0, a1 = R(0.6) * z1, a2 = R(0.3) * z2;      // plus side
  const R c0 = R(0.1) * z2, c1 = R(0.6) * z1, c2 = R(0.3) * z0;      // minus side (stencils mirrored)
  const R is = rcp(a0 + a1 + a2), im = rcp(c0 + c1 + c2);
  wp[0] = a0 * is;
  wp[1] = a1 * is;
  wp[2] = a2 * is;
  wm[0] = c0 * im;
  wm[1] = c1 * im;
  wm[2] = c2 * im;
  qp = wp[0] * P0 + wp[1] * P1 + wp[2] * P2;
  qm = wm[0] * M0 + wm[1] * M1 + wm[2] * M2;
}

template <class R>
__device__ __forceinline__ R weno_sigma_side(const R w[3]) {
  return R(3) * w[0] * w[1] * w[2] / (R(0.3) * w[0] * w[1] + R(0.6) * w[0] * w[2] + R(0.1) * w[1] * w[2]);
}

// MP5 (Sec. 3.1; the monotonicity-preserving scheme of Suresh & Huynh 1997): value at the upper face of the
// centre cell of (f0..f4). The fifth-order interpolant is kept when it lies between f2 and the
// monotonicity-preserving bound f2 + minmod(f3 - f2, 4 (f2 - f1)); otherwise it is moved to the nearest
// end of the accuracy-preserving interval built from the upper, median and large-curvature limits with
// the limited second differences d^M4. Acceptance test (v - f2)(v - v_MP) <= 0, alpha = 4.
template <class R>
__device__ __forceinline__ R sgn1(R a) {
  return a > R(0) ? R(1) : (a < R(0) ? R(-1) : R(0));
}

template <class R>
__device__ __forceinline__ R minmod2(R a, R b) {
  return R(0.5) * (sgn1(a) + sgn1(b)) * fmin(fabs(a), fabs(b));
}

template <class R>
__device__ __forceinline__ R minmod4(R w, R x, R y, R z) {
  const R sw = sgn1(w);
  const R s = R(0.125) * (sw + sgn1(x)) * fabs((sw + sgn1(y)) * (sw + sgn1(z)));
  return s * fmin(fmin(fabs(w), fabs(x)), fmin(fabs(y), fabs(z)));
}

template <class R>
__device__ __forceinline__ R mp5_face(R f0, R f1, R f2, R f3, R f4) {
  const R alpha = R(4);
  const R v = fdiv(R(2) * f0 - R(13) * f1 + R(47) * f2 + R(27) * f3 - R(3) * f4, R(60));
  const R vmp = f2 + minmod2(f3 - f2, alpha * (f2 - f1));
  if ((v - f2) * (v - vmp) <= R(0)) return v;
  const R dm = f0 - R(2) * f1 + f2, d0 = f1 - R(2) * f2 + f3, dp = f2 - R(2) * f3 + f4;
  const R dhp = minmod4(R(4) * d0 - dp, R(4) * dp - d0, d0, dp);
  const R dhm = minmod4(R(4) * d0 - dm, R(4) * dm - d0, d0, dm);
  const R vul = f2 + alpha * (f2 - f1);
  const R vav = R(0.5) * (f2 + f3);
  const R vmd = vav - R(0.5) * dhp;
  const R vlc = f2 + R(0.5) * (f2 - f1) + R(4) / R(3) * dhm;
  const R vmin = fmax(fmin(fmin(f2, f3), vmd), fmin(fmin(f2, vul), vlc));
  const R vmax = fmin(fmax(fmax(f2, f3), vmd), fmax(fmax(f2, vul), vlc));
  return v + minmod2(vmin - v, vmax - v);
}

// Face values of the centre cell c = f[2]: qm at its lower face, qp at its upper face.
template <class R, int RECON>
__device__ __forceinline__ void recon_cell(R f0, R f1, R f2, R f3, R f4, R eps, R& qm, R& qp) {
  if (RECON == RECON_CONSTANT) {
    qm = qp = f2;
  } else if (RECON == RECON_MP5) {  // the lower face from the mirrored stencil
    qp = mp5_face<R>(f0, f1, f2, f3, f4);
    qm = mp5_face<R>(f4, f3, f2, f1, f0);
  } else if (RECON == RECON_PLM_MINMOD || RECON == RECON_PLM_MC) {
    const R s = RECON == RECON_PLM_MC ? mc_slope(f2 - f1, f3 - f2) : minmod_slope(f2 - f1, f3 - f2);
    qm = f2 - R(0.5) * s;
    qp = f2 + R(0.5) * s;
  } else {
    R wp[3], wm[3], z[3], P5p, P5m;
    weno5z_both<R>(f0, f1, f2, f3, f4, eps, P5p, P5m, wp, wm, z);
    R sigma;
    if constexpr (sizeof(R) == 4) {
      // The same sigma from the unnormalised weights: with w_k = gamma_k z_k / S (S = sum gamma_k z_k) the
      // reciprocal of a side's sigma is (S / 3) (1/z_0 + 1/z_1 + 1/z_2), the same sum on both sides (the
      // mirrored side permutes z and gamma together), so the harmonic mean of the two sides is
      // 6 / ((S_+ + S_-) H) = 15 / ((z_0 + 3 z_1 + z_2) H), H = 1/z_0 + 1/z_1 + 1/z_2: one quotient and three
      // reciprocals instead of three quotients of products (which can also underflow in float). z_k is
      // in [1, 1e30] (q clamped), so neither factor leaves the float range.
      const R H = rcp(z[0]) + rcp(z[1]) + rcp(z[2]);
      sigma = fdiv(R(15), (z[0] + R(3) * z[1] + z[2]) * H);
    } else {
      const R sp = weno_sigma_side(wp), sm = weno_sigma_side(wm);
      sigma = sp + sm > R(0) ? R(2) * sp * sm / (sp + sm) : R(0);
    }
    sigma = sigma > R(1) ? R(1) : sigma;
    const R s = mc_slope(f2 - f1, f3 - f2);
    qp = sigma * P5p + (R(1) - sigma) * (f2 + R(0.5) * s);
    qm = sigma * P5m + (R(1) - sigma) * (f2 - R(0.5) * s);
  }
}

// The MC slope of recon_cell from the paired differences dm, dp, their product and their mean c.
__device__ __forceinline__ float mc_pick(float dm, float dp, float pr, float c) {
  if (!(pr > 0.f)) return 0.f;
  const float m = fminf(fminf(fabsf(dm + dm), fabsf(dp + dp)), fabsf(c));
  return dm > 0.f ? m : -m;
}

// WENO5-Z-AOAH face values (recon_cell<float, RECON_WENO5Z>) of two variables at once, one in each half of
// the float2 operands: the candidates, smoothness indicators, Z weights, the blend factor sigma and the
// blend with the MC-limited linear values, every FP32 add, multiply and fma issued once for both
// variables; the reciprocals and the limiter's compares stay per variable. The candidates are formed as
// fmas with the coefficients divided by 6 and the weights applied before the sum, so the values agree with
// recon_cell's float form to rounding (a few ulps), not bit for bit; the float cell-centric fluxes use this
// form for every cell, so a cell's face values still do not depend on the run layout.
__device__ __forceinline__ void recon_weno5z_x2(float2 f0, float2 f1, float2 f2, float2 f3, float2 f4, float eps,
                                                float2& qm, float2& qp) {
  const float2 t3 = x2(1.f / 3.f), s6 = x2(-1.f / 6.f), f56 = x2(5.f / 6.f), e6 = x2(11.f / 6.f),
               m76 = x2(-7.f / 6.f);
  const float2 a11 = mul2(f2, e6), a5 = mul2(f2, f56), a3 = mul2(f2, t3);
  const float2 P0 = fma2(f0, t3, fma2(f1, m76, a11));  // plus face: (2 f0 - 7 f1 + 11 f2) / 6
  const float2 P1 = fma2(f1, s6, fma2(f3, t3, a5));    // (-f1 + 5 f2 + 2 f3) / 6
  const float2 P2 = fma2(f4, s6, fma2(f3, f56, a3));   // (2 f2 + 5 f3 - f4) / 6
  const float2 M0 = fma2(f4, t3, fma2(f3, m76, a11));  // minus face: the mirrored stencil
  const float2 M1 = fma2(f3, s6, fma2(f1, t3, a5));
  const float2 M2 = fma2(f0, s6, fma2(f1, f56, a3));
  const float2 m2 = x2(-2.f), m4 = x2(-4.f), c3 = x2(3.f);
  const float2 t0 = fma2(f1, m2, add2(f0, f2)), s0 = fma2(f1, m4, fma2(f2, c3, f0));
  const float2 t1 = fma2(f2, m2, add2(f1, f3)), s1 = sub2(f1, f3);
  const float2 t2 = fma2(f3, m2, add2(f2, f4)), s2 = fma2(f3, m4, fma2(f2, c3, f4));
  const float2 k13 = x2(13.f / 12.f), k4 = x2(0.25f);
  const float2 b0 = fma2(mul2(t0, k13), t0, mul2(mul2(s0, s0), k4));
  const float2 b1 = fma2(mul2(t1, k13), t1, mul2(mul2(s1, s1), k4));
  const float2 b2 = fma2(mul2(t2, k13), t2, mul2(mul2(s2, s2), k4));
  const float2 db = sub2(b2, b0);
  const float2 tau = make_float2(fabsf(db.x), fabsf(db.y));
  const float2 e2 = x2(eps);
  float2 q0 = mul2(tau, rcp2(add2(b0, e2))), q1 = mul2(tau, rcp2(add2(b1, e2))), q2 = mul2(tau, rcp2(add2(b2, e2)));
  // q^2 kept inside the float range, as in recon_cell
  q0 = make_float2(fminf(q0.x, 1e15f), fminf(q0.y, 1e15f));
  q1 = make_float2(fminf(q1.x, 1e15f), fminf(q1.y, 1e15f));
  q2 = make_float2(fminf(q2.x, 1e15f), fminf(q2.y, 1e15f));
  const float2 one = x2(1.f);
  const float2 z0 = fma2(q0, q0, one), z1 = fma2(q1, q1, one), z2 = fma2(q2, q2, one);
  const float2 a0 = mul2(z0, x2(0.1f)), a1 = mul2(z1, x2(0.6f)), a2 = mul2(z2, x2(0.3f));  // plus side
  const float2 c0 = mul2(z2, x2(0.1f)), c2 = mul2(z0, x2(0.3f));                           // minus side
  const float2 is = rcp2(add2(add2(a0, a1), a2)), im = rcp2(add2(add2(c0, a1), c2));
  const float2 P5p = fma2(mul2(a2, is), P2, fma2(mul2(a1, is), P1, mul2(mul2(a0, is), P0)));
  const float2 P5m = fma2(mul2(c2, im), M2, fma2(mul2(a1, im), M1, mul2(mul2(c0, im), M0)));
  // sigma = 15 / ((z0 + 3 z1 + z2) (1/z0 + 1/z1 + 1/z2)), at most 1
  const float2 H = add2(add2(rcp2(z0), rcp2(z1)), rcp2(z2));
  const float2 den = mul2(fma2(z1, c3, add2(z0, z2)), H);
  float2 sg = mul2(x2(15.f), rcp2(den));
  sg = make_float2(fminf(sg.x, 1.f), fminf(sg.y, 1.f));
  const float2 dm = sub2(f2, f1), dp = sub2(f3, f2);
  const float2 h = x2(0.5f), nh = x2(-0.5f);
  const float2 pr = mul2(dm, dp), cs = mul2(h, add2(dm, dp));
  const float2 s = make_float2(mc_pick(dm.x, dp.x, pr.x, cs.x), mc_pick(dm.y, dp.y, pr.y, cs.y));
  const float2 om = sub2(one, sg);
  qp = fma2(sg, P5p, mul2(om, fma2(s, h, f2)));
  qm = fma2(sg, P5m, mul2(om, fma2(s, nh, f2)));
}

// ------------------------------------------------------------------ Riemann solvers (Sec. 3.1)
template <class R>
__device__ __forceinline__ R riemann_flux(int riemann, const FaceSide<R>& L, const FaceSide<R>& Rs, R Fh[NV]) {
  const R cmax = fmax(fmax(fabs(L.lm), fabs(L.lp)), fmax(fabs(Rs.lm), fabs(Rs.lp)));
  if (riemann == RIEMANN_LLF) {
#pragma unroll
    for (int q = 0; q < NV; ++q) Fh[q] = R(0.5) * (L.F[q] + Rs.F[q]) - R(0.5) * cmax * (Rs.U[q] - L.U[q]);
  } else {
    const R cl = fmin(R(0), fmin(L.lm, Rs.lm));
    const R cr = fmax(R(0), fmax(L.lp, Rs.lp));
    const R den = cr - cl;
    if (den == R(0)) {
#pragma unroll
      for (int q = 0; q < NV; ++q) Fh[q] = R(0.5) * (L.F[q] + Rs.F[q]);
    } else {
      const R id = rcp(den);
#pragma unroll
      for (int q = 0; q < NV; ++q) Fh[q] = (cr * L.F[q] - cl * Rs.F[q] + cr * cl * (Rs.U[q] - L.U[q])) * id;
    }
  }
  return cmax;
}

// riemann_flux for the paired float sides of prim_to_face_x2 (left in the x halves, right in the y halves).
__device__ __forceinline__ float riemann_flux_x2(int riemann, const float2 U[NV], const float2 F[NV], float2 lm,
                                                 float2 lp, float Fh[NV]) {
  const float cmax = fmaxf(fmaxf(fabsf(lm.x), fabsf(lp.x)), fmaxf(fabsf(lm.y), fabsf(lp.y)));
  if (riemann == RIEMANN_LLF) {
#pragma unroll
    for (int q = 0; q < NV; ++q) Fh[q] = 0.5f * (F[q].x + F[q].y) - 0.5f * cmax * (U[q].y - U[q].x);
  } else {
    const float cl = fminf(0.f, fminf(lm.x, lm.y));
    const float cr = fmaxf(0.f, fmaxf(lp.x, lp.y));
    const float den = cr - cl;
    if (den == 0.f) {
#pragma unroll
      for (int q = 0; q < NV; ++q) Fh[q] = 0.5f * (F[q].x + F[q].y);
    } else {
      const float id = rcp(den);
#pragma unroll
      for (int q = 0; q < NV; ++q) Fh[q] = (cr * F[q].x - cl * F[q].y + cr * cl * (U[q].y - U[q].x)) * id;
    }
  }
  return cmax;
}

// ------------------------------------------------------------------ con2prim (Sec. 3.1)
// Kastaun, Kalinani & Ciolfi (2021): with q = tau/D, r_i = S_i/D, b^i = B^i/sqrt(D), the unknown
// mu = 1/(h W) is the root of f(mu) = mu - 1/(nu(mu) + mu rbar^2(mu)) in [0, mu_+], mu_+ the root
// of mu^2 (1 + rbar^2(mu)) = 1 (h0 = 1 for the ideal gas). Solved by a bracketed Newton iteration
// whose derivative comes from forward-mode dual numbers, warm-started from the previous primitives.
// The all-FP64 form iterates in double; the mixed form iterates in float and finishes with one
// double Newton step (quadratic convergence turns the float root into a double one), falling back
// to the double iteration when the float phase does not settle.
template <class T>
struct Dual {
  T v, d;
};
template <class T>
__device__ __forceinline__ Dual<T> operator+(Dual<T> a, Dual<T> b) { return {a.v + b.v, a.d + b.d}; }
template <class T>
__device__ __forceinline__ Dual<T> operator-(Dual<T> a, Dual<T> b) { return {a.v - b.v, a.d - b.d}; }
template <class T>
__device__ __forceinline__ Dual<T> operator*(Dual<T> a, Dual<T> b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <class T>
__device__ __forceinline__ Dual<T> operator*(T a, Dual<T> b) { return {a * b.v, a * b.d}; }
template <class T>
__device__ __forceinline__ Dual<T> operator+(T a, Dual<T> b) { return {a + b.v, b.d}; }
template <class T>
__device__ __forceinline__ Dual<T> operator-(T a, Dual<T> b) { return {a - b.v, -b.d}; }
template <class T>
__device__ __forceinline__ Dual<T> drcp(Dual<T> a) {
  const T r = T(1) / a.v;
  return {r, -a.d * r * r};
}
template <class T>
__device__ __forceinline__ Dual<T> dsqrt(Dual<T> a) {
  const T s = sqrt(a.v);
  return {s, a.d * T(0.5) / s};
}

// Work units of the flux phase of direction d: faces (face-centric reconstructions), or, for
// WENO5-Z-AOAH and MP5, (transverse position, run of ~p.flux_run faces along d) pairs (cell-centric: each
// cell reconstructed once per direction, plus the cell before each run). The transverse positions span
// [-1, n] in both directions. Runs of 32 faces by default: at 256^3 the y / z sweeps took 1.95 ms against
// 2.08 with runs of 16 and 2.23 with runs of 8. A single-block context picks shorter runs (down to
// FLUX_RUN_MIN) when its columns are too few to fill the GPU with runs of 32 (flux_run_for): at 64^3 the
// y / z sweeps take 0.039 ms with runs of 4, 0.047 with 8; at 96^3 and 128^3 runs of 4 to 8 tie.
constexpr int FLUX_RUN = 32;
constexpr int FLUX_RUN_MIN = 4;

// Run length for a block of nx x ny x nz cells alone on a GPU of nsm SMs: long enough to amortise the extra
// cell of each run, short enough that the y / z units give every SM two waves of 8 CTAs of 128 threads.
__host__ __forceinline__ int flux_run_for(int nx, int ny, int nz, int nsm) {
  const long long target = (long long)nsm * 8 * 128 * 2;
  const long long cols = (long long)(nx + 2) * ((ny < nz ? ny : nz) + 2);
  const int nd = ny > nz ? ny : nz;
  long long run = (long long)(nd + 1) * cols / (target > 0 ? target : 1);
  run = run < FLUX_RUN_MIN ? FLUX_RUN_MIN : (run > FLUX_RUN ? FLUX_RUN : run);
  return (int)run;
}

// Runs per column of nd + 1 faces (nd + 1 >= FLUX_RUN: runs of FLUX_RUN to 2 FLUX_RUN - 1 faces) and their
// common length (the last run takes the remainder).
__host__ __device__ __forceinline__ int flux_runs(const DevParams& p, int nd) {
  const int r = (nd + 1) / (p.flux_run > 0 ? p.flux_run : FLUX_RUN);
  return r > 0 ? r : 1;
}
__host__ __device__ __forceinline__ int flux_run_length(const DevParams& p, int nd) {
  const int r = flux_runs(p, nd);
  return (nd + 1 + r - 1) / r;
}

// Direction x (d = 0) is cell-centric per warp instead: the x rows of cells -1..nx are laid end to end,
// and warp w takes the 32 consecutive cells 31 w - 1 .. 31 w + 30 of that sequence (x-coalesced loads and
// stores). A lane whose cell is not the first of its row evaluates the face below its cell with the plus
// side of the previous cell passed by a lane shuffle; lane 0 only supplies that side (its face belongs to
// the previous warp). The units are whole warps.
constexpr int FLUX_WARP_FACES = 31;

__host__ __device__ __forceinline__ long long flux_units(const DevParams& p, int d) {
  if (cell_centric(p.recon) && d == 0) {
    const long long cells = (long long)(p.ny + 2) * (p.nz + 2) * (p.nx + 2);
    return (cells + FLUX_WARP_FACES - 1) / FLUX_WARP_FACES * 32;
  }
  if (cell_centric(p.recon)) {
    const int nd = d == 0 ? p.nx : (d == 1 ? p.ny : p.nz);
    const int na = d == 0 ? p.ny : p.nx, nb = d == 2 ? p.ny : p.nz;
    return (long long)(na + 2) * (nb + 2) * flux_runs(p, nd);
  }
  int ex, ey;
  return face_box(p, d, ex, ey);
}

template <class T>
struct C2PIn {
  T D, q, r2, b2, rb, rb2, gm1, v0sq;
};

template <class T>
__device__ __forceinline__ T c2p_rbar2(const C2PIn<T>& c, T mu, T& x) {
  x = T(1) / (T(1) + mu * c.b2);
  return x * x * c.r2 + mu * x * (T(1) + x) * c.rb2;
}

// Master function value and derivative at mu; also the intermediate W, rho, eps and x.
template <class T>
struct C2PEval {
  T f, df, x, W, rho, eps;
  T dx, dW, drho, deps;  // derivatives of x, W, rho, eps with respect to mu (0 from c2p_master_value)
};

template <class T>
__device__ __forceinline__ C2PEval<T> c2p_master(const C2PIn<T>& c, T mu_v) {
  typedef Dual<T> D;
  const D mu = {mu_v, T(1)};
  const D x = drcp(T(1) + c.b2 * mu);
  const D rb = c.r2 * (x * x) + c.rb2 * (mu * x * (T(1) + x));
  const D qbar = (c.q - T(0.5) * c.b2) - (T(0.5) * (c.b2 * c.r2 - c.rb2)) * (mu * mu * x * x);
  D vh2 = mu * mu * rb;
  if (vh2.v > c.v0sq) vh2 = {c.v0sq, T(0)};
  const D iW = dsqrt(T(1) - vh2);  // 1/W
  const D W = drcp(iW);
  const D rho = c.D * iW;
  D eps = W * (qbar - mu * rb) + vh2 * W * W * drcp(T(1) + W);
  if (eps.v < T(0)) eps = {T(0), T(0)};
  // a = P/(rho (1 + eps)) = (Gamma - 1) eps/(1 + eps) for the ideal gas
  const D onepe = T(1) + eps;
  const D a = c.gm1 * eps * drcp(onepe);
  const D nuA = (T(1) + a) * onepe * iW;
  const D nuB = (T(1) + a) * (T(1) + qbar - mu * rb);
  const D nu = nuA.v >= nuB.v ? nuA : nuB;
  const D f = mu - drcp(nu + mu * rb);
  C2PEval<T> e;
  e.f = f.v;
  e.df = f.d;
  e.x = x.v;
  e.W = W.v;
  e.rho = rho.v;
  e.eps = eps.v;
  e.dx = x.d;
  e.dW = W.d;
  e.drho = rho.d;
  e.deps = eps.d;
  return e;
}

// Master-function intermediates without the derivative (final evaluation at the root).
template <class T>
__device__ __forceinline__ C2PEval<T> c2p_master_value(const C2PIn<T>& c, T mu) {
  const T x = T(1) / (T(1) + c.b2 * mu);
  const T rb = c.r2 * (x * x) + c.rb2 * (mu * x * (T(1) + x));
  const T qbar = (c.q - T(0.5) * c.b2) - (T(0.5) * (c.b2 * c.r2 - c.rb2)) * (mu * mu * x * x);
  T vh2 = mu * mu * rb;
  if (vh2 > c.v0sq) vh2 = c.v0sq;
  const T iW = sqrt(T(1) - vh2);
  const T W = T(1) / iW;
  T eps = W * (qbar - mu * rb) + vh2 * W * W / (T(1) + W);
  if (eps < T(0)) eps = T(0);
  C2PEval<T> e;
  e.f = T(0);
  e.df = T(0);
  e.x = x;
  e.W = W;
  e.rho = c.D / W;
  e.eps = eps;
  e.dx = e.dW = e.drho = e.deps = T(0);
  return e;
}

// Upper end of the bracket: root of g(mu) = mu^2 (1 + rbar^2(mu)) - 1 on (0, 1], Newton safeguarded
// by bisection, from `mu` (<= 0: the b = 0 root), to relative step `rtol`.
template <class T>
__device__ __forceinline__ T c2p_mu_plus(const C2PIn<T>& c, T mu, T rtol, int maxit) {
  T x;
  const T g1 = (T(1) + c2p_rbar2(c, T(1), x)) - T(1);
  if (!(g1 > T(0))) return T(1);
  T lo = T(0), hi = T(1);
  if (!(mu > lo && mu < hi)) mu = T(1) / sqrt(T(1) + c.r2);
  if (!(mu > lo && mu < hi)) mu = T(0.5);
  for (int it = 0; it < maxit; ++it) {
    const T xx = T(1) / (T(1) + mu * c.b2);
    const T dx = -c.b2 * xx * xx;
    const T rb = xx * xx * c.r2 + mu * xx * (T(1) + xx) * c.rb2;
    const T drb = T(2) * xx * dx * c.r2 + c.rb2 * (xx * (T(1) + xx) + mu * dx * (T(1) + T(2) * xx));
    const T g = mu * mu * (T(1) + rb) - T(1);
    const T dg = T(2) * mu * (T(1) + rb) + mu * mu * drb;
    if (g == T(0)) return mu;  // exact root
    if (g < T(0)) lo = mu; else hi = mu;
    T nmu = mu - g / dg;
    if (!(nmu >= lo && nmu <= hi)) nmu = T(0.5) * (lo + hi);
    const bool done = fabs(nmu - mu) <= rtol * nmu;
    mu = nmu;
    if (done || hi - lo <= rtol * hi) break;
  }
  return mu;
}

// mu_+ of a double-precision set-up, iterated in float to a relative step of 1e-7 and then polished
// in double to 1e-15 (the same root as c2p_mu_plus<double> to rounding, in about half the double
// iterations). Used by the flat con2prim batches.
__device__ __forceinline__ double c2p_mu_plus_fast(const C2PIn<double>& c) {
  C2PIn<float> cf;
  cf.D = (float)c.D; cf.q = (float)c.q; cf.r2 = (float)c.r2; cf.b2 = (float)c.b2; cf.rb = (float)c.rb;
  cf.rb2 = (float)c.rb2; cf.gm1 = (float)c.gm1; cf.v0sq = (float)c.v0sq;
  const float muf = c2p_mu_plus<float>(cf, -1.f, 1e-7f, 40);
  return c2p_mu_plus<double>(c, (double)muf, 1e-15, 12);
}

// Bracketed Newton iteration on [0, mup] from mu (double or float). Returns 0 when converged (the
// root, or mu_+ when f(mu_+) <= 0: the cold limit eps = 0), ST_NOT_CONVERGED otherwise.
template <class T>
__device__ __forceinline__ int c2p_newton(const C2PIn<T>& c, T mup, T& mu, T tol, int maxit, int& iters,
                                          bool extra_step) {
  T lo = T(0), hi = mup;
  if (!(mu > lo && mu < hi)) mu = T(0.5) * mup;
  for (int it = 0; it < maxit; ++it) {
    const C2PEval<T> e = c2p_master(c, mu);
    ++iters;
    if (e.f == T(0) || (e.f < T(0) && mu == mup)) return 0;
    if (e.f < T(0)) lo = mu; else hi = mu;
    T nmu = mu - e.f / e.df;
    if (!(nmu >= lo && nmu <= hi) || !(e.df > T(0)))
      nmu = (nmu > hi && hi == mup && e.df > T(0)) ? mup : T(0.5) * (lo + hi);  // try the unevaluated end first
    const bool conv = fabs(nmu - mu) <= tol * nmu;
    mu = nmu;
    if (conv) {
      if (extra_step) {  // one more Newton step past the tolerance
        const C2PEval<T> e2 = c2p_master(c, mu);
        ++iters;
        nmu = mu - e2.f / e2.df;
        if (nmu >= lo && nmu <= hi && e2.df > T(0)) mu = nmu;
      }
      return 0;
    }
    if (hi - lo <= T(1e-16) * hi) return 0;
  }
  return ST_NOT_CONVERGED;
}

// Undensitized (D, S_j, tau, B^k) -> inputs of the master function. Returns ST_BAD_INPUT for
// non-finite values or D <= 0.
template <class R>
__device__ __forceinline__ int c2p_setup(const DevParams& p, const Metric<R>& m, const double Uc[NV], C2PIn<double>& c,
                                         double ru[3], double bu[3]) {
  bool finite = true;
#pragma unroll
  for (int q = 0; q < NV; ++q) finite = finite && isfinite(Uc[q]);
  if (!finite || !(Uc[0] > 0.0)) return ST_BAD_INPUT;
  double gam[6], gamu[6];
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    gam[t] = (double)m.gam[t];
    gamu[t] = (double)m.gamu[t];
  }
  c.D = Uc[0];
  const double isD = rsqrt(c.D);  // 1/sqrt(D), and 1/D as its square
  const double iD = isD * isD;
  c.q = Uc[4] * iD;
  const double rl[3] = {Uc[1] * iD, Uc[2] * iD, Uc[3] * iD};
  lower3(gamu, rl, ru);
  bu[0] = Uc[5] * isD;
  bu[1] = Uc[6] * isD;
  bu[2] = Uc[7] * isD;
  double bl[3];
  lower3(gam, bu, bl);
  c.r2 = rl[0] * ru[0] + rl[1] * ru[1] + rl[2] * ru[2];
  c.b2 = bu[0] * bl[0] + bu[1] * bl[1] + bu[2] * bl[2];
  c.rb = rl[0] * bu[0] + rl[1] * bu[1] + rl[2] * bu[2];
  c.rb2 = c.rb * c.rb;
  c.gm1 = p.gamma_eos - 1.0;
  // velocity bound of the solve: physical bound r^2/(1 + r^2) and the Lorentz-factor ceiling
  c.v0sq = fmin(c.r2 / (1.0 + c.r2), p.v0sq_cap);
  return 0;
}

// Primitives at the root mu.
__device__ __forceinline__ void c2p_output_eval(const C2PIn<double>& c, const C2PEval<double>& e, double mu,
                                                const double ru[3], const double bu[3], const double Uc[NV],
                                                double Pout[NV]) {
  const double W = e.W;
  Pout[0] = e.rho;
  const double mx = mu * e.x;
#pragma unroll
  for (int i = 0; i < 3; ++i) Pout[1 + i] = W * mx * (ru[i] + mu * c.rb * bu[i]);
  Pout[4] = e.rho * e.eps;
#pragma unroll
  for (int k = 0; k < 3; ++k) Pout[5 + k] = Uc[5 + k];
}

__device__ __forceinline__ void c2p_output(const C2PIn<double>& c, double mu, const double ru[3], const double bu[3],
                                           const double Uc[NV], double Pout[NV]) {
  c2p_output_eval(c, c2p_master_value(c, mu), mu, ru, bu, Uc, Pout);
}

__device__ __forceinline__ void c2p_bad_output(const double Uc[NV], double Pout[NV]) {
#pragma unroll
  for (int q = 0; q < 5; ++q) Pout[q] = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) Pout[5 + k] = isfinite(Uc[5 + k]) ? Uc[5 + k] : 0.0;
}

// All-FP64 con2prim: double Newton to |d mu| <= c2p_tol mu plus one more step. Returns the status
// bits of the solve (0, ST_NOT_CONVERGED or ST_BAD_INPUT); floors are separate. fast_mup: the bracket
// end from c2p_mu_plus_fast (flat batches) instead of the all-double iteration (the FP64 stage).
template <class R>
__device__ __forceinline__ int con2prim(const DevParams& p, const Metric<R>& m, const double Uc[NV],
                                        double mu_guess, double Pout[NV], int& iters, bool fast_mup = false) {
  const unsigned lanes = __activemask();  // each of these lanes reaches the __syncwarp below once
  iters = 0;
  C2PIn<double> c;
  double ru[3], bu[3];
  const bool bad = c2p_setup<R>(p, m, Uc, c, ru, bu) != 0;
  double mu = mu_guess;
  int st = ST_BAD_INPUT;
  if (!bad) {
    const double mup = fast_mup ? c2p_mu_plus_fast(c) : c2p_mu_plus<double>(c, -1.0, 1e-15, 60);
    st = c2p_newton<double>(c, mup, mu, p.c2p_tol, p.c2p_max_iter, iters, true);
  }
  __syncwarp(lanes);  // reconverge after iterations of different lengths: the output runs once per warp
  if (bad) {
    c2p_bad_output(Uc, Pout);
    return ST_BAD_INPUT;
  }
  c2p_output(c, mu, ru, bu, Uc, Pout);
  return st;
}

// One double Newton step of the master function from mue, accepted when it is smaller than 3e-6 mue
// (its error is then of order step^2) and stays below the float bracket end (with margin): on success
// returns true with the root mu and the intermediates there, to first order in the step.
__device__ __forceinline__ bool c2p_accept_step(const C2PIn<double>& c, const C2PEval<double>& e, double mue,
                                                float mupf, double& mu, C2PEval<double>& ev) {
  const double step = -e.f / e.df;
  const double nmu = mue + step;
  mu = nmu;
  if (!(e.df > 0.0 && nmu > 0.0 && fabs(step) <= 3e-6 * nmu && nmu <= (double)mupf * (1.0 + 1e-5))) return false;
  ev = e;
  ev.x += e.dx * step;
  ev.W += e.dW * step;
  ev.rho += e.drho * step;
  ev.eps = fmax(e.eps + e.deps * step, 0.0);
  return true;
}

// The resumed step of a deferred cell: from the double iterate mu_r of the first pass (when it has one), one
// more evaluation and the same acceptance as the first pass. False: the cell needs the full double con2prim.
template <class R>
__device__ __forceinline__ bool con2prim_resume_step(const DevParams& p, const Metric<R>& m, const double Uc[NV],
                                                     double mu_r, double Pout[NV], int& iters) {
  iters = 0;
  if (!(mu_r > 0.0)) return false;
  C2PIn<double> c;
  double ru[3], bu[3];
  if (c2p_setup<R>(p, m, Uc, c, ru, bu) != 0) return false;
  C2PIn<float> cf;
  cf.D = (float)c.D; cf.q = (float)c.q; cf.r2 = (float)c.r2; cf.b2 = (float)c.b2; cf.rb = (float)c.rb;
  cf.rb2 = (float)c.rb2; cf.gm1 = (float)c.gm1; cf.v0sq = (float)c.v0sq;
  const float mupf = c2p_mu_plus<float>(cf, -1.f, 1e-7f, 40);
  const C2PEval<double> e = c2p_master(c, mu_r);
  iters = 1;
  double mu;
  C2PEval<double> ev;
  if (!c2p_accept_step(c, e, mu_r, mupf, mu, ev)) return false;
  c2p_output_eval(c, ev, mu, ru, bu, Uc, Pout);
  return true;
}

// Returned by con2prim_mixed_f(defer = true): the cell needs the double iteration of deferred_cell.
enum { C2P_DEFERRED = 256 };

// Mixed form of the stage's con2prim (a6), from the densitized conserved state, with the primitives returned
// in float, the storage type of the mixed form. Only what the solve's conditioning needs is double: the
// master function's invariants q, r^2, b^2, (r.b)^2 and the velocity bound (from the double state and the
// cell's double metric), mu_+ when the float root sits on it (one double Newton step), the master function at
// the float root and the specific internal energy there. Everything the float primitives are formed from
// to float accuracy anyway (x, the Newton step, the output velocities, density and field) is float.
// Two identities (exact in real arithmetic, with W = 1/sqrt(1 - v^2) and W (1 + qbar - mu rbar^2) = 1 + eps)
// remove the master function's divisions besides x:
//   eps = W (qbar - mu rbar^2) + v^2 W^2/(1 + W) = W (1 + qbar - mu rbar^2) - 1,
//   nu = max((1 + a)(1 + eps)/W, (1 + a)(1 + qbar - mu rbar^2)) = (1 + Gamma eps)/W  (eps clamped at 0),
// and the root is taken on K f = mu K - 1 (K = nu + mu rbar^2 > 0, the same root), whose Newton step at the
// root equals f's. Returns the status bits of the solve (floors are applied by the caller) or C2P_DEFERRED
// when the double step from the float root is not small (defer == true; mu_r then holds the double iterate
// the double pass resumes from); without defer such a cell takes the full double iteration here.
// The two contractions of the solve's invariants with the 3-metric: r^i = gamma^ij r_j and b^2 = gamma_ij b^i b^j,
// from the Cartesian Kerr-Schild factors (r_i - kappa (l.r) l^i, b.b + f (l.b)^2) or from the matrices.
__device__ __forceinline__ double c2p_contract(const KSGeo& gm, const double rl[3], const double bu[3], double ru[3]) {
  const double klr = gm.kappa * (gm.l[0] * rl[0] + gm.l[1] * rl[1] + gm.l[2] * rl[2]);
#pragma unroll
  for (int i = 0; i < 3; ++i) ru[i] = rl[i] - klr * gm.l[i];
  const double lb = gm.l[0] * bu[0] + gm.l[1] * bu[1] + gm.l[2] * bu[2];
  return bu[0] * bu[0] + bu[1] * bu[1] + bu[2] * bu[2] + gm.f * lb * lb;
}
__device__ __forceinline__ double c2p_contract(const Metric<double>& m, const double rl[3], const double bu[3],
                                               double ru[3]) {
  double bl[3];
  lower3(m.gamu, rl, ru);
  lower3(m.gam, bu, bl);
  return bu[0] * bl[0] + bu[1] * bl[1] + bu[2] * bl[2];
}

template <class Geo>
__device__ __forceinline__ int con2prim_mixed_f(const DevParams& p, const Geo& gm, double isg,
                                                const double Un[NV], float mu_guess, bool defer, float Pf[NV],
                                                int& iters, double& mu_r) {
  // Lanes entering together; each of them reaches the __syncwarp below exactly once (no return before it).
  const unsigned lanes = __activemask();
  iters = 0;
  mu_r = 0.0;
  bool finite = true;
#pragma unroll
  for (int q = 0; q < NV; ++q) finite = finite && dfinite(Un[q]);
  const bool bad = !finite || !dpositive(Un[0]);
  C2PIn<double> c;
  C2PIn<float> cf;
  float ruf[3], buf[3];
  float mupf = 1.f, muf = 0.f;
  int itf = 0, stf = ST_NOT_CONVERGED;
  if (!bad) {
    // q = tau/D and r_i = S_i/D are ratios of densitized values; b^i = B^i/sqrt(D) takes sqrt(gamma) once
    const double D = Un[0] * isg;
    const double isD = rsqrt(D);
    const double s = isg * isD * isD;
    const double rl[3] = {Un[1] * s, Un[2] * s, Un[3] * s};
    const double tb = isg * isD;
    const double bu[3] = {Un[5] * tb, Un[6] * tb, Un[7] * tb};
    double ru[3];
    c.b2 = c2p_contract(gm, rl, bu, ru);
    c.D = D;
    c.q = Un[4] * s;
    c.r2 = rl[0] * ru[0] + rl[1] * ru[1] + rl[2] * ru[2];
    c.rb = rl[0] * bu[0] + rl[1] * bu[1] + rl[2] * bu[2];
    c.rb2 = c.rb * c.rb;
    c.gm1 = p.gamma_eos - 1.0;
    c.v0sq = 0.0;  // formed below where the double part needs it (it costs a double quotient)
    cf.D = (float)c.D; cf.q = (float)c.q; cf.r2 = (float)c.r2; cf.b2 = (float)c.b2; cf.rb = (float)c.rb;
    cf.rb2 = cf.rb * cf.rb; cf.gm1 = p.fgamma - 1.f;
    cf.v0sq = fminf(__fdividef(cf.r2, 1.f + cf.r2), p.fv0sq_cap);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      ruf[i] = (float)ru[i];
      buf[i] = (float)bu[i];
    }
    mupf = c2p_mu_plus<float>(cf, -1.f, 1e-7f, 40);
    muf = mu_guess;
    stf = c2p_newton<float>(cf, mupf, muf, 2e-6f, 24, itf, false);
  }
  // The float iterations end at different counts in different lanes: reconverge, so that the double part
  // below runs once for the warp rather than once per group of lanes (FP64 issue is per warp instruction).
  __syncwarp(lanes);
  if (bad) {
#pragma unroll
    for (int q = 0; q < 5; ++q) Pf[q] = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) Pf[5 + k] = isfinite(Un[5 + k]) ? (float)(Un[5 + k] * isg) : 0.f;
    return ST_BAD_INPUT;
  }
  iters = itf;
  bool done = false;
  double mu = (double)muf, eps = 0.0;
  float Wf = 1.f, xf = 1.f;  // the intermediates at the accepted root
  if (stf == 0 && isfinite(muf) && muf > 0.f) {
    const bool cold = muf >= mupf;
    double mue = mu;
    if (__any_sync(__activemask(), cold)) {  // the same instructions for every lane of the warp
      // mu_+ in double: one Newton step on mu^2 (1 + rbar^2(mu)) - 1 from the float root (relative error
      // ~1e-7 -> ~1e-14), the derivative in float (it only scales that step)
      double m1 = (double)mupf;
      if (mupf < 1.f) {
        const double xx = 1.0 / (1.0 + m1 * c.b2);
        const double rb = xx * xx * c.r2 + m1 * xx * (1.0 + xx) * c.rb2;
        const double gp = m1 * m1 * (1.0 + rb) - 1.0;
        const float xr = 1.f / (1.f + mupf * cf.b2);
        const float dxr = -cf.b2 * xr * xr;
        const float rbr = xr * xr * cf.r2 + mupf * xr * (1.f + xr) * cf.rb2;
        const float drb = 2.f * xr * dxr * cf.r2 + cf.rb2 * (xr * (1.f + xr) + mupf * dxr * (1.f + 2.f * xr));
        const float dg = 2.f * mupf * (1.f + rbr) + mupf * mupf * drb;
        m1 -= (double)__fdividef((float)gp, dg);
      }
      if (cold) mue = m1;
    }
    // the master function times K at mue, in double
    const double x = 1.0 / (1.0 + c.b2 * mue);
    const double rb = c.r2 * (x * x) + c.rb2 * (mue * x * (1.0 + x));
    const double qbar = (c.q - 0.5 * c.b2) - (0.5 * (c.b2 * c.r2 - c.rb2)) * (mue * mue * x * x);
    double vh2 = mue * mue * rb;
    // vh2 > v0sq = min(r^2/(1 + r^2), v0sq_cap), without the quotient unless the bound binds
    if (vh2 * (1.0 + c.r2) > c.r2 || vh2 > p.v0sq_cap) vh2 = fmin(c.r2 / (1.0 + c.r2), p.v0sq_cap);
    const double W = rsqrt(1.0 - vh2);
    const double iW = (1.0 - vh2) * W;
    const double e0 = fmax(W * (1.0 + qbar - mue * rb) - 1.0, 0.0);
    const double K = (1.0 + p.gamma_eos * e0) * iW + mue * rb;
    const double gK = mue * K - 1.0;
    // the derivatives, in float at the same point
    const C2PEval<float> ed = c2p_master<float>(cf, (float)mue);
    ++iters;
    if (cold && !(gK > 0.0)) {  // root on mu_+: the cold limit
      mu = mue;
      eps = e0;
      Wf = (float)W;
      xf = ed.x;
      done = true;
    } else {
      const float step = -__fdividef((float)gK, (float)K * ed.df);
      const double nmu = mue + (double)step;
      mu = nmu;
      const float nmuf = (float)nmu;
      done = ed.df > 0.f && nmuf > 0.f && fabsf(step) <= 3e-6f * nmuf && nmuf <= mupf * (1.f + 1e-5f);
      if (done) {
        // the intermediates at the root to first order in the step (the neglected term is O(step^2))
        eps = fmax(e0 + (double)(ed.deps * step), 0.0);
        Wf = (float)W + ed.dW * step;
        xf = ed.x + ed.dx * step;
      } else if (defer && dfinite(nmu) && nmuf > 0.f && nmuf < mupf * (1.f + 1e-3f)) {
        mu_r = nmu;  // the double pass resumes from this iterate
      }
    }
  }
  if (!done && defer) return C2P_DEFERRED;
  int st = 0;
  if (!done) {  // float phase did not settle: double iteration on the full bracket, from the float root
    c.v0sq = fmin(c.r2 / (1.0 + c.r2), p.v0sq_cap);
    const double mup = c2p_mu_plus_fast(c);
    if (!(stf == 0 && isfinite(mu) && mu > 0.0)) mu = (double)mu_guess;
    int it64 = 0;
    st = c2p_newton<double>(c, mup, mu, p.c2p_tol, p.c2p_max_iter, it64, true);
    iters += it64;
    const C2PEval<double> ev = c2p_master_value(c, mu);
    eps = ev.eps;
    Wf = (float)ev.W;
    xf = (float)ev.x;
  }
  // primitives in float: rho = D/W, W v^i = W mu x (r^i + mu (r.b) b^i), rho eps, B^i = b^i sqrt(D)
  const float muF = (float)mu;
  const float mx = Wf * muF * xf;
  const float mrb = muF * cf.rb;
  Pf[0] = cf.D / Wf;
#pragma unroll
  for (int i = 0; i < 3; ++i) Pf[1 + i] = mx * (ruf[i] + mrb * buf[i]);
  Pf[4] = Pf[0] * (float)eps;
  const float sD = sqrtf(cf.D);
#pragma unroll
  for (int k = 0; k < 3; ++k) Pf[5 + k] = buf[k] * sD;
  return st;
}

// The floors of apply_floors_fr on float primitives (the mixed form's storage type), with the float metric
// and radius factor.
__device__ __forceinline__ int apply_floors_f(const DevParams& p, const float gam[6], float fr, float P[NV]) {
  const float rho_flr = p.frho_floor0 * fr;
  const float eps_flr = p.feps_floor0 * fr;
  int st = 0;
  if (!(P[0] >= rho_flr)) {
    P[0] = rho_flr;
    st |= ST_RHO_FLOOR;
  }
  if (!(P[4] >= P[0] * eps_flr)) {
    P[4] = P[0] * eps_flr;
    st |= ST_EPS_FLOOR;
  }
  const float ut[3] = {P[1], P[2], P[3]};
  float utl[3];
  lower3(gam, ut, utl);
  const float usq = ut[0] * utl[0] + ut[1] * utl[1] + ut[2] * utl[2];
  const float wm2 = p.fw_max2;
  if (1.f + usq > wm2) {  // W = sqrt(1 + u^2) > w_max
    const float s = sqrtf((wm2 - 1.f) / usq);
    P[1] *= s;
    P[2] *= s;
    P[3] *= s;
    st |= ST_W_CAP;
  }
  return st;
}

// Floors (Sec. 3.2): rho >= rho0 r^-n, rho eps >= rho eps0 r^-n (r the Kerr-Schild radius; 1 in
// Minkowski), and the Lorentz-factor ceiling W <= w_max.
// Floors with the radius factor fr = r^-floor_r_exp already evaluated (1 in Minkowski).
__device__ __forceinline__ int apply_floors_fr(const DevParams& p, const double gam[6], double fr, double P[NV]) {
  const double rho_flr = p.rho_floor0 * fr;
  const double eps_flr = p.eps_floor0 * fr;
  int st = 0;
  if (!(P[0] >= rho_flr)) {
    P[0] = rho_flr;
    st |= ST_RHO_FLOOR;
  }
  if (!(P[4] >= P[0] * eps_flr)) {
    P[4] = P[0] * eps_flr;
    st |= ST_EPS_FLOOR;
  }
  const double ut[3] = {P[1], P[2], P[3]};
  double utl[3];
  lower3(gam, ut, utl);
  const double usq = ut[0] * utl[0] + ut[1] * utl[1] + ut[2] * utl[2];
  if (1.0 + usq > p.w_max2) {  // W = sqrt(1 + u^2) > w_max
    const double s = sqrt((p.w_max2 - 1.0) / usq);
    P[1] *= s;
    P[2] *= s;
    P[3] *= s;
    st |= ST_W_CAP;
  }
  return st;
}

// Radius factor of the floors at Kerr-Schild radius r.
__device__ __forceinline__ double floor_factor(const DevParams& p, double r) {
  return p.floor_r_exp == 2.0 ? 1.0 / (r * r) : pow(r, -p.floor_r_exp);
}

template <int METRIC>
__device__ __forceinline__ int apply_floors(const DevParams& p, const double gam[6], double r, double P[NV]) {
  return apply_floors_fr(p, gam, METRIC != MINKOWSKI ? floor_factor(p, r) : 1.0, P);
}

// mu = 1/(h W) of a primitive state, the con2prim warm start (in the arithmetic type R).
template <class R>
__device__ __forceinline__ R mu_of_prims(const R P[NV], const R gam[6], R gamma_eos) {
  const R ut[3] = {P[1], P[2], P[3]};
  R utl[3];
  lower3(gam, ut, utl);
  const R W = sqrt(R(1) + ut[0] * utl[0] + ut[1] * utl[1] + ut[2] * utl[2]);
  const R h = R(1) + gamma_eos * P[4] / P[0];  // 1 + eps + p/rho = 1 + Gamma u/rho
  return R(1) / (h * W);
}

}  // namespace grmhd
