// All-FP64 form of the stage kernels (every step in double precision). Built without FMA
// contraction (-fmad=false) so that every double operation rounds as the FP64 reference does.
#include "grmhd_kernels.cuh"
#include "grmhd_face_ct.cuh"
#include "grmhd_launch.h"
#include "grmhd_batch_launch.cuh"
#include "grmhd_scalar.cuh"

namespace grmhd {

namespace {

using R = double;
using T = double;

template <int METRIC>
cudaError_t flux_m(const DevParams& p, const T* P, R* F, unsigned long long* ms, int d, int track, cudaStream_t s) {
  const long long n = (long long)(p.nx + (d == 0 ? 1 : 2)) * (p.ny + (d == 1 ? 1 : 2)) * (p.nz + (d == 2 ? 1 : 2));
  const int g = grid_for(n, 128);
  if (METRIC == KERR_SCHILD_SPHERICAL) {  // face-centric for every reconstruction (its sin(theta) weighting)
    switch (p.recon) {
      case RECON_CONSTANT: k_flux<R, T, METRIC, RECON_CONSTANT><<<g, 128, 0, s>>>(P, F, ms, p, d, track); break;
      case RECON_PLM_MINMOD: k_flux<R, T, METRIC, RECON_PLM_MINMOD><<<g, 128, 0, s>>>(P, F, ms, p, d, track); break;
      case RECON_PLM_MC: k_flux<R, T, METRIC, RECON_PLM_MC><<<g, 128, 0, s>>>(P, F, ms, p, d, track); break;
      case RECON_WENO5Z: k_flux<R, T, METRIC, RECON_WENO5Z><<<g, 128, 0, s>>>(P, F, ms, p, d, track); break;
      case RECON_MP5: k_flux<R, T, METRIC, RECON_MP5><<<g, 128, 0, s>>>(P, F, ms, p, d, track); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  switch (p.recon) {
    case RECON_CONSTANT: k_flux<R, T, METRIC, RECON_CONSTANT><<<g, 128, 0, s>>>(P, F, ms, p, d, track); break;
    case RECON_PLM_MINMOD: k_flux<R, T, METRIC, RECON_PLM_MINMOD><<<g, 128, 0, s>>>(P, F, ms, p, d, track); break;
    case RECON_PLM_MC: k_flux<R, T, METRIC, RECON_PLM_MC><<<g, 128, 0, s>>>(P, F, ms, p, d, track); break;
    case RECON_WENO5Z:  // cell-centric: each cell reconstructed once per direction
      k_flux_cc<R, T, METRIC, RECON_WENO5Z><<<grid_for(flux_units(p, d), 128), 128, 0, s>>>(P, F, ms, p, d, track);
      break;
    case RECON_MP5:
      k_flux_cc<R, T, METRIC, RECON_MP5><<<grid_for(flux_units(p, d), 128), 128, 0, s>>>(P, F, ms, p, d, track);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t ghost(const DevParams& p, void* P, cudaStream_t s) {
  if (p.bc == BC_SPHERICAL)
    k_ghost_spherical<T><<<grid_for(p.gsize, 256), 256, 0, s>>>((T*)P, p);
  else
    k_ghost_periodic<T><<<grid_for(p.gsize, 256), 256, 0, s>>>((T*)P, p);
  return cudaGetLastError();
}

cudaError_t flux(const DevParams& p, const void* P, void* F, unsigned long long* ms, int d, int track, cudaStream_t s) {
  if (p.metric == KERR_SCHILD_SPHERICAL) return flux_m<KERR_SCHILD_SPHERICAL>(p, (const T*)P, (R*)F, ms, d, track, s);
  return p.metric == KERR_SCHILD ? flux_m<KERR_SCHILD>(p, (const T*)P, (R*)F, ms, d, track, s)
                                 : flux_m<MINKOWSKI>(p, (const T*)P, (R*)F, ms, d, track, s);
}

cudaError_t emf(const DevParams& p, const void* Fx, const void* Fy, const void* Fz, void* E, cudaStream_t s) {
  const long long n = (long long)(p.nx + 1) * (p.ny + 1) * (p.nz + 1);
  k_emf<R><<<grid_for(n, 256), 256, 0, s>>>((const R*)Fx, (const R*)Fy, (const R*)Fz, (R*)E, p);
  if (p.metric == KERR_SCHILD_SPHERICAL) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_emf_axis<R><<<(2 * p.nx + 127) / 128, 128, 0, s>>>((R*)E, p);
  }
  return cudaGetLastError();
}

cudaError_t update(const DevParams& p, void* P, const void* Fx, const void* Fy, const void* Fz, const void* E,
                   const StageArgs& a, cudaStream_t s) {
  const int g = grid_for((a.t_end > 0 ? a.t_end : p.isize) - a.t_begin, 128);
  if (p.metric == KERR_SCHILD)
    k_update<KERR_SCHILD, R, T><<<g, 128, 0, s>>>((T*)P, (const R*)Fx, (const R*)Fy, (const R*)Fz, (const R*)E, a, p);
  else if (p.metric == KERR_SCHILD_SPHERICAL)
    k_update<KERR_SCHILD_SPHERICAL, R, T><<<g, 128, 0, s>>>((T*)P, (const R*)Fx, (const R*)Fy, (const R*)Fz,
                                                            (const R*)E, a, p);
  else
    k_update<MINKOWSKI, R, T><<<g, 128, 0, s>>>((T*)P, (const R*)Fx, (const R*)Fy, (const R*)Fz, (const R*)E, a, p);
  return cudaGetLastError();
}

// Pass over the cells queued by k_update (count known on the device only): re-derivation of the hydro
// state of floored cells. (This form has no deferred con2prim cells.)
cudaError_t cell_passes(const DevParams& p, void* P, const StageArgs& a, cudaStream_t s) {
  if (a.floorlist == nullptr) return cudaSuccess;
  const int g2 = grid_for(p.isize / 8 + 1, 128);
  if (p.metric == KERR_SCHILD)
    k_update_floors<KERR_SCHILD, T><<<g2, 128, 0, s>>>((const T*)P, a, p);
  else if (p.metric == KERR_SCHILD_SPHERICAL)
    k_update_floors<KERR_SCHILD_SPHERICAL, T><<<g2, 128, 0, s>>>((const T*)P, a, p);
  else
    k_update_floors<MINKOWSKI, T><<<g2, 128, 0, s>>>((const T*)P, a, p);
  return cudaGetLastError();
}

cudaError_t prim2con(const DevParams& p, const void* P, double* U, long long t0, long long t1, cudaStream_t s) {
  if (t1 <= t0) return cudaSuccess;
  const int g = grid_for(t1 - t0, 128);
  if (p.metric == KERR_SCHILD)
    k_prim2con<KERR_SCHILD, T><<<g, 128, 0, s>>>((const T*)P, U, p, t0, t1);
  else if (p.metric == KERR_SCHILD_SPHERICAL)
    k_prim2con<KERR_SCHILD_SPHERICAL, T><<<g, 128, 0, s>>>((const T*)P, U, p, t0, t1);
  else
    k_prim2con<MINKOWSKI, T><<<g, 128, 0, s>>>((const T*)P, U, p, t0, t1);
  return cudaGetLastError();
}

cudaError_t load_prims(const DevParams& p, const double* src, void* P, cudaStream_t s) {
  return cudaMemcpyAsync(P, src, sizeof(double) * NV * p.gsize, cudaMemcpyDeviceToDevice, s);
}

cudaError_t store_prims(const DevParams& p, const void* P, double* dst, cudaStream_t s) {
  return cudaMemcpyAsync(dst, P, sizeof(double) * NV * p.gsize, cudaMemcpyDeviceToDevice, s);
}

cudaError_t geometry(const DevParams& p, double* geo, cudaStream_t s) {
  if (p.metric != KERR_SCHILD || p.isize == 0) return cudaSuccess;
  k_geometry<KERR_SCHILD><<<grid_for(p.isize, 128), 128, 0, s>>>(p, geo);
  return cudaGetLastError();
}

using FC = FaceCtLaunch<R, T>;
using BL = BatchLaunch<double, double>;
using SL = ScalarLaunch<double, double>;
const FormLaunchers kFp64 = {ghost, flux, emf, update, cell_passes, prim2con, load_prims, store_prims, BL::flux, BL::emf, BL::update,
                                BL::deferred, BL::ctas_per_sm, 8, 8, geometry, BL::floors,
                                FC::emf, FC::faces, FC::to_cells, FC::ghost_faces,
                                BL::flux_ctas_per_sm, BL::exchange, BL::mesh_exchange,
                                BL::mesh_reflux, SL::flux, SL::update, SL::load, SL::store, SL::ghost,
                                SL::batch_flux, SL::batch_update, BL::mesh_reflux_scalar};

}  // namespace

const FormLaunchers& fp64_launchers() { return kFp64; }

}  // namespace grmhd
