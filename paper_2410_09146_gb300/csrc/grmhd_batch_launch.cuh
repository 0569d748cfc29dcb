// Launchers of the batched persistent kernels for one arithmetic form (R: flux type, T: P storage).
#pragma once

#include "grmhd_kernels.cuh"
#include "grmhd_mesh.cuh"
#include "grmhd_launch.h"

namespace grmhd {

template <class R, class T>
struct BatchLaunch {
  template <int METRIC>
  static cudaError_t flux_m(const BlockDesc* b, const WorkItem* it, int n, unsigned int* ctr, unsigned long long* ms,
                            int track, int recon, int grid, cudaStream_t s) {
    switch (recon) {
      case RECON_CONSTANT: k_batch_flux<R, T, METRIC, RECON_CONSTANT><<<grid, 128, 0, s>>>(b, it, n, ctr, ms, track); break;
      case RECON_PLM_MINMOD: k_batch_flux<R, T, METRIC, RECON_PLM_MINMOD><<<grid, 128, 0, s>>>(b, it, n, ctr, ms, track); break;
      case RECON_PLM_MC: k_batch_flux<R, T, METRIC, RECON_PLM_MC><<<grid, 128, 0, s>>>(b, it, n, ctr, ms, track); break;
      case RECON_WENO5Z: k_batch_flux<R, T, METRIC, RECON_WENO5Z><<<grid, 128, 0, s>>>(b, it, n, ctr, ms, track); break;
      case RECON_MP5: k_batch_flux<R, T, METRIC, RECON_MP5><<<grid, 128, 0, s>>>(b, it, n, ctr, ms, track); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  static cudaError_t flux(const BlockDesc* b, const WorkItem* it, int n, unsigned int* ctr, unsigned long long* ms,
                          int track, int metric, int recon, int grid, cudaStream_t s) {
    return metric == KERR_SCHILD ? flux_m<KERR_SCHILD>(b, it, n, ctr, ms, track, recon, grid, s)
                                 : flux_m<MINKOWSKI>(b, it, n, ctr, ms, track, recon, grid, s);
  }
  static cudaError_t emf(const BlockDesc* b, const WorkItem* it, int n, unsigned int* ctr, int grid, cudaStream_t s) {
    k_batch_emf<R><<<grid, 128, 0, s>>>(b, it, n, ctr);
    return cudaGetLastError();
  }
  static cudaError_t update(const BlockDesc* b, const WorkItem* it, int n, unsigned int* ctr, const BatchArgs& a,
                            int metric, int grid, cudaStream_t s) {
    if (metric == KERR_SCHILD)
      k_batch_update<KERR_SCHILD, R, T><<<grid, 128, 0, s>>>(b, it, n, ctr, a);
    else
      k_batch_update<MINKOWSKI, R, T><<<grid, 128, 0, s>>>(b, it, n, ctr, a);
    return cudaGetLastError();
  }
  // the two passes of deferred_cell (the second over the cells the first queued, when there is a solve list)
  static cudaError_t deferred(const BlockDesc* b, int nblocks, const BatchArgs& a, int metric, int grid,
                              cudaStream_t s) {
    for (int full = 0; full < (a.solvelist ? 2 : 1); ++full) {
      if (metric == KERR_SCHILD)
        k_batch_deferred<KERR_SCHILD, T><<<grid, 128, 0, s>>>(b, nblocks, a, full);
      else
        k_batch_deferred<MINKOWSKI, T><<<grid, 128, 0, s>>>(b, nblocks, a, full);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  static cudaError_t floors(const BlockDesc* b, int nblocks, const BatchArgs& a, int metric, int grid,
                            cudaStream_t s) {
    if (sizeof(T) == 4) return cudaSuccess;  // the mixed form re-derives floored cells inside its update
    if (metric == KERR_SCHILD)
      k_batch_floors<KERR_SCHILD, T><<<grid, 128, 0, s>>>(b, nblocks, a);
    else
      k_batch_floors<MINKOWSKI, T><<<grid, 128, 0, s>>>(b, nblocks, a);
    return cudaGetLastError();
  }
  // CTAs per SM of the persistent kernels (occupancy of the update kernel, the heaviest)
  template <int METRIC>
  static int flux_ctas_m(int recon) {
    int n = 0;
    switch (recon) {
      case RECON_CONSTANT: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_flux<R, T, METRIC, RECON_CONSTANT>, 128, 0); break;
      case RECON_PLM_MINMOD: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_flux<R, T, METRIC, RECON_PLM_MINMOD>, 128, 0); break;
      case RECON_PLM_MC: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_flux<R, T, METRIC, RECON_PLM_MC>, 128, 0); break;
      case RECON_WENO5Z: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_flux<R, T, METRIC, RECON_WENO5Z>, 128, 0); break;
      case RECON_MP5: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_flux<R, T, METRIC, RECON_MP5>, 128, 0); break;
      default: break;
    }
    return n > 0 ? n : 1;
  }
  // resident CTAs per SM of the batched flux kernel (its persistent grid is sized from this, the other
  // phases' grid from the update kernel's)
  static int flux_ctas_per_sm(int metric, int recon) {
    return metric == KERR_SCHILD ? flux_ctas_m<KERR_SCHILD>(recon) : flux_ctas_m<MINKOWSKI>(recon);
  }
  static cudaError_t exchange(const BlockDesc* b, int nblocks, long long ghosted_cells, const Lattice& L, cudaStream_t s) {
    k_batch_exchange<T><<<grid_for(ghosted_cells, 256), 256, 0, s>>>(b, nblocks, L);
    return cudaGetLastError();
  }
  static cudaError_t mesh_exchange(const BlockDesc* b, int nblocks, const MeshDesc& M, int pass, cudaStream_t s) {
    const int ny = pass == 2 ? M.nfine : nblocks;
    if (ny <= 0 || M.nghost <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((M.nghost + 255) / 256), (unsigned)ny);
    k_mesh_exchange<T><<<grid, 256, 0, s>>>(b, M, pass);
    return cudaGetLastError();
  }
  static cudaError_t mesh_reflux(const BlockDesc* b, const RefluxCell* cells, int ncells, const BatchArgs& a,
                                 int metric, cudaStream_t s) {
    if (ncells <= 0) return cudaSuccess;
    // 64-thread CTAs: the reflux cells are few (a face layer), so spread them over as many SMs as possible
    const int grid = (ncells + 63) / 64;
    if (metric == KERR_SCHILD)
      k_mesh_reflux<KERR_SCHILD, R, T><<<grid, 64, 0, s>>>(b, cells, ncells, a);
    else
      k_mesh_reflux<MINKOWSKI, R, T><<<grid, 64, 0, s>>>(b, cells, ncells, a);
    return cudaGetLastError();
  }
  static cudaError_t mesh_reflux_scalar(const BlockDesc* b, const RefluxCell* cells, int ncells, const BatchArgs& a,
                                        cudaStream_t s) {
    if (ncells <= 0) return cudaSuccess;
    k_mesh_reflux_scalar<R, T><<<(ncells + 63) / 64, 64, 0, s>>>(b, cells, ncells, a);
    return cudaGetLastError();
  }
  static int ctas_per_sm(int metric) {
    int n = 0;
    if (metric == KERR_SCHILD)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_update<KERR_SCHILD, R, T>, 128, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_update<MINKOWSKI, R, T>, 128, 0);
    return n > 0 ? n : 1;
  }
};

}  // namespace grmhd
