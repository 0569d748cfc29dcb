// Internal launcher interface between the C-ABI layer and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "grmhd_device.cuh"

namespace grmhd {

// Launchers for one arithmetic form. R is the flux/EMF type, T the storage type of P:
// form 0 = all double, form 1 = mixed (float fluxes and P).
struct FormLaunchers {
  cudaError_t (*ghost)(const DevParams& p, void* P, cudaStream_t s);
  cudaError_t (*flux)(const DevParams& p, const void* P, void* F, unsigned long long* ms, int d, int track,
                      cudaStream_t s);
  cudaError_t (*emf)(const DevParams& p, const void* Fx, const void* Fy, const void* Fz, void* E, cudaStream_t s);
  cudaError_t (*update)(const DevParams& p, void* P, const void* Fx, const void* Fy, const void* Fz, const void* E,
                        const StageArgs& a, cudaStream_t s);
  // the passes over the cells queued by update (floored cells; deferred con2prim in the mixed form)
  cudaError_t (*cell_passes)(const DevParams& p, void* P, const StageArgs& a, cudaStream_t s);
  // prim->cons of interior cells t0 <= t < t1
  cudaError_t (*prim2con)(const DevParams& p, const void* P, double* U, long long t0, long long t1, cudaStream_t s);
  cudaError_t (*load_prims)(const DevParams& p, const double* src, void* P, cudaStream_t s);   // double -> storage
  cudaError_t (*store_prims)(const DevParams& p, const void* P, double* dst, cudaStream_t s);  // storage -> double
  // batched persistent kernels (many meshblocks, one launch per phase)
  cudaError_t (*batch_flux)(const BlockDesc* b, const WorkItem* it, int n, unsigned int* ctr, unsigned long long* ms,
                            int track, int metric, int recon, int grid, cudaStream_t s);
  cudaError_t (*batch_emf)(const BlockDesc* b, const WorkItem* it, int n, unsigned int* ctr, int grid, cudaStream_t s);
  cudaError_t (*batch_update)(const BlockDesc* b, const WorkItem* it, int n, unsigned int* ctr, const BatchArgs& a,
                              int metric, int grid, cudaStream_t s);
  cudaError_t (*batch_deferred)(const BlockDesc* b, int nblocks, const BatchArgs& a, int metric, int grid,
                                cudaStream_t s);
  int (*batch_ctas_per_sm)(int metric);
  int p_bytes;  // bytes per stored primitive
  int r_bytes;  // bytes per flux / EMF value
  // fill the geometry cache (NGEO x isize doubles) of a Kerr-Schild block
  cudaError_t (*geometry)(const DevParams& p, double* geo, cudaStream_t s);
  // batched re-derivation of the hydro state of floored cells
  cudaError_t (*batch_floors)(const BlockDesc* b, int nblocks, const BatchArgs& a, int metric, int grid,
                              cudaStream_t s);
  // face-centred CT (grmhd_face_ct.cuh): cell-centred and upwind edge EMFs, the Stokes update of the
  // faces, the cell field from the faces, the periodic fill of the face arrays
  cudaError_t (*emf_face)(const DevParams& p, const void* P, const void* Fx, const void* Fy, const void* Fz,
                          void* Ecc, void* E, cudaStream_t s);
  cudaError_t (*face_update)(const DevParams& p, const double* Bf0, const double* Bfc, double* Bfn, const void* E,
                             const StageArgs& a, cudaStream_t s);
  cudaError_t (*face_to_cells)(const DevParams& p, const double* Bf, void* P, cudaStream_t s);
  cudaError_t (*ghost_faces)(const DevParams& p, double* Bf, cudaStream_t s);
  // resident CTAs per SM of the batched flux kernel (metric, recon)
  int (*batch_flux_ctas_per_sm)(int metric, int recon);
  // same-level ghost exchange of a lattice batch (ghosted_cells = nblocks x the block's gsize)
  cudaError_t (*batch_exchange)(const BlockDesc* b, int nblocks, long long ghosted_cells, const Lattice& L,
                                cudaStream_t s);
  // two-level mesh (grmhd_mesh.cuh): one pass (1 or 2) of the ghost exchange, and the refluxing of the
  // coarse cells at coarse-fine faces after the update
  cudaError_t (*mesh_exchange)(const BlockDesc* b, int nblocks, const MeshDesc& M, int pass, cudaStream_t s);
  cudaError_t (*mesh_reflux)(const BlockDesc* b, const RefluxCell* cells, int ncells, const BatchArgs& a, int metric,
                             cudaStream_t s);
  // passive scalar (grmhd_scalar.cuh): face fluxes of direction d (FX holds the 3 directions), the update,
  // loading X (and D X from the current state), widening X to double, the periodic ghost fill of X
  cudaError_t (*scalar_flux)(const DevParams& p, const void* X, const void* F, void* FX, int d, cudaStream_t s);
  cudaError_t (*scalar_update)(const DevParams& p, void* X, const void* FX, const double* DX0, const double* DXcur,
                               double* DXnew, const double* Unew, const StageArgs& a, cudaStream_t s);
  cudaError_t (*scalar_load)(const DevParams& p, const double* Xd, void* X, const double* U, double* DX, cudaStream_t s);
  cudaError_t (*scalar_store)(const DevParams& p, const void* X, double* Xd, cudaStream_t s);
  cudaError_t (*scalar_ghost)(const DevParams& p, void* X, cudaStream_t s);
  // passive scalar of a batch: face fluxes of direction d of every block, the update of every block
  cudaError_t (*batch_scalar_flux)(const BlockDesc* b, int nblocks, long long max_units, int recon, int d,
                                   cudaStream_t s);
  cudaError_t (*batch_scalar_update)(const BlockDesc* b, int nblocks, long long max_cells, const BatchArgs& a,
                                     cudaStream_t s);
  // refluxing of the passive scalar on a two-level mesh, after its update
  cudaError_t (*mesh_reflux_scalar)(const BlockDesc* b, const RefluxCell* cells, int ncells, const BatchArgs& a,
                                    cudaStream_t s);
};

const FormLaunchers& fp64_launchers();
const FormLaunchers& mixed_launchers();

cudaError_t launch_finalize_dt(const unsigned long long* ms, double* dt, const DevParams& p, cudaStream_t s);
cudaError_t launch_batch_finalize_dt(const unsigned long long* ms, double* dt, double cfl, cudaStream_t s);
cudaError_t launch_c2p_batch(const double* U, double* P, uint8_t* status, int* iters, long long n, int flags,
                             const DevParams& p, unsigned long long* stats, cudaStream_t s);
cudaError_t launch_p2c_batch(const double* P, double* U, long long n, const DevParams& p, cudaStream_t s);

// Learned-guess con2prim (grmhd_mlp.cu): the network's start (mu_0, mu_+) [2][n] for flat-space
// states, and the batch solve from it (guess != NULL, with fallback) or from mu_+/2, optionally
// recording training pairs (X, T).
cudaError_t launch_mlp_guess(const void* mlp_ws, const double* U, double* guess, long long n, const DevParams& p,
                             cudaStream_t s);
cudaError_t launch_c2p_guided(const double* U, double* P, uint8_t* status, int* iters, long long n,
                              const DevParams& p, const double* guess, float* X, float* T, unsigned long long* stats,
                              cudaStream_t s);

// Fused learned-guess con2prim with the hidden layers on the tensor cores (grmhd_mlp_tc.cu); guess
// (optional) receives (mu_0, mu_+) [2][n]; stats [6] counts tiles abandoned on an MMA wait timeout.
cudaError_t launch_c2p_net_tc(const void* mlp_ws, const double* U, double* P, uint8_t* status, int* iters,
                              long long n, const DevParams& p, double* guess, unsigned long long* stats,
                              cudaStream_t s);

int grid_for(long long n, int threads);

}  // namespace grmhd
