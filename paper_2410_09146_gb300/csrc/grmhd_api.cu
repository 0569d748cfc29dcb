// C-ABI entry points of libgrmhd.so (declared and documented in include/grmhd.h).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "../../include/grmhd.h"
#include "grmhd_device.cuh"
#include "grmhd_launch.h"
#include "grmhd_mesh_host.h"

using namespace grmhd;

constexpr int kLoadChunks = 8;  // slabs of a chunked host load (grmhd_set_prims_f32)

struct grmhd_ctx {
  grmhd_params prm;
  DevParams dp;
  const FormLaunchers* L;
  cudaStream_t stream;
  char* ws;
  size_t ws_bytes;
  void* P;
  double* Uslot[3];
  void* F[3];
  void* E;
  uint8_t* status;
  int* worklist;             // mixed form: deferred con2prim cells (NULL in the FP64 form)
  double* wl_mu;             // mixed form: the double iterate each deferred cell resumes from
  int* floorlist;            // FP64 form: floored cells (hydro state re-derived in a pass); mixed form:
                             // deferred cells that need the full double con2prim
  unsigned long long* scal;  // [0..2] max speed bits, [3] dt (double), [8..15] stats, [16] worklist count,
                             // [17] floor-list count, [20..23] batch work counters
  double* Bslot[3];          // face-centred CT: face field slots [3][gsize], paired with Uslot
  void* X;                   // passive scalar: X [gsize] (storage type of P)
  double* DXslot[3];         // passive scalar: sqrt(gamma) D X [isize], paired with Uslot
  void* FX;                  // passive scalar: face fluxes [3][gsize] (flux type)
  bool has_scalar;           // passive scalar: grmhd_set_scalar called since grmhd_set_prims
  std::vector<char> block_scalar;  // batches: grmhd_batch_set_scalar called for block b since its set_prims
  long long max_runs, max_cells;   // batches with a scalar: grid sizing (largest block's gsize and isize)
  void* Ecc;                 // face-centred CT: cell-centred EMFs [3][gsize] (flux type)
  bool has_faces;            // face-centred CT: grmhd_set_face_b called since grmhd_set_prims
  int s0, sc;                // slot of U0 and of the current state
  bool has_state;
  // host loads of the float primitives: chunks copied on `stream`, their prim->cons on `load_stream` (created
  // on the first such load), so the two overlap; load_ev[k] marks chunk k's copies, load_ev[kLoadChunks] the end
  cudaStream_t load_stream;
  cudaEvent_t load_ev[kLoadChunks + 1];
  // host reads overlapped with a stage (grmhd_stage_host_f32): out_ev[k] marks slab k's update on `stream`, whose
  // rows are then copied on load_stream; out_ev[kLoadChunks] the end of the copies
  cudaEvent_t out_ev[kLoadChunks + 1];
  bool out_ev_made;
  int load_last;             // load_ev index of the last host load's last copies
  bool timing;               // record CUDA events around each kernel group
  cudaEvent_t ev[8];         // ghost | flux x | flux y | flux z | emf | update | cell passes | end
  double t_ms[7];            // accumulated ms per kernel group since the last read
  int t_stages;              // stages accumulated
  bool t_pending;            // events of the last stage not yet read
  // batch of meshblocks (nblocks == 0: a single-block context)
  int nblocks;
  std::vector<BlockDesc> hblocks;
  BlockDesc* dblocks;
  WorkItem* ditems;
  long long max_items;
  int n_items[3];            // flux | EMF | update items at the current tile
  int tile;
  int grid_persist;
  int grid_flux;             // persistent grid of the batched flux phase
  bool lattice_on;           // the blocks tile a lattice: ghosts exchanged at the start of every stage
  Lattice lattice;
  bool mesh_on;              // the blocks are the leaves of a two-level mesh: exchange and refluxing
  MeshDesc mesh;
  int* dleaf;                // leaf map of the mesh (workspace, capacity leaf_cap)
  unsigned* dghost;          // ghost cells of a mesh block (workspace, capacity ghost_cap)
  int* dfine;                // level-1 blocks of the mesh (workspace, nblocks entries)
  long long ghost_cap;
  RefluxCell* dreflux;       // coarse cells at coarse-fine faces (workspace, capacity reflux_cap)
  long long leaf_cap, reflux_cap;
  int n_reflux;
  long long total_cells;
  long long total_ghosted;   // nblocks x gsize of block 0 (meaningful for lattices, whose blocks are equal)
  bool use_graph;
  int n_tuned;               // the last autotune's timing table: work-item size and ms per stage
  int tuned_tile[8];
  double tuned_ms[8];
  cudaStream_t cap_stream;
  std::map<std::vector<double>, cudaGraphExec_t> graphs;
  char err[256];
};

namespace grmhd {

// Parameter checks and the kernel-side copy of the parameters, shared by every entry point that takes a
// grmhd_params (contexts, batches and the allocation-free stage).
bool valid_params(const grmhd_params* p, char* msg, size_t n) {
  if (!p) { snprintf(msg, n, "params is NULL"); return false; }
  const bool batch_only = p->nx == 0 && p->ny == 0 && p->nz == 0;
  if (!batch_only) {
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) { snprintf(msg, n, "nx, ny, nz must be >= 1"); return false; }
    const int need = p->recon >= GRMHD_RECON_WENO5Z_AOAH ? 3 : (p->recon == GRMHD_RECON_CONSTANT ? 1 : 2);
    if (p->ng < need) { snprintf(msg, n, "ng = %d too small for the reconstruction (needs %d)", p->ng, need); return false; }
    if (p->ng > 16) { snprintf(msg, n, "ng = %d too large", p->ng); return false; }
    for (int d = 0; d < 3; ++d)
      if (!(p->dx[d] > 0.0)) { snprintf(msg, n, "dx[%d] must be > 0", d); return false; }
    const double cells = (double)(p->nx + 2 * p->ng) * (p->ny + 2 * p->ng) * (p->nz + 2 * p->ng);
    if (cells > 4.0e9) { snprintf(msg, n, "block too large"); return false; }
  }
  if (p->metric != GRMHD_MINKOWSKI && p->metric != GRMHD_KERR_SCHILD && p->metric != GRMHD_KERR_SCHILD_SPHERICAL) {
    snprintf(msg, n, "unknown metric");
    return false;
  }
  if (p->recon < 0 || p->recon > 4) { snprintf(msg, n, "unknown reconstruction"); return false; }
  if (p->riemann != GRMHD_RIEMANN_LLF && p->riemann != GRMHD_RIEMANN_HLL) { snprintf(msg, n, "unknown Riemann solver"); return false; }
  if (p->precision != GRMHD_FP64 && p->precision != GRMHD_MIXED) { snprintf(msg, n, "unknown precision"); return false; }
  if (p->bc != GRMHD_BC_PERIODIC && p->bc != GRMHD_BC_FIXED && p->bc != GRMHD_BC_SPHERICAL) {
    snprintf(msg, n, "unknown boundary condition");
    return false;
  }
  if (!(p->gamma_eos > 1.0)) { snprintf(msg, n, "gamma_eos must be > 1"); return false; }
  if (!(p->c2p_tol > 0.0) || p->c2p_max_iter < 1) { snprintf(msg, n, "bad con2prim tolerance / iteration cap"); return false; }
  if (!(p->w_max > 1.0)) { snprintf(msg, n, "w_max must be > 1"); return false; }
  if (p->metric == GRMHD_KERR_SCHILD && !(p->mass > 0.0)) { snprintf(msg, n, "mass must be > 0"); return false; }
  if (p->ct != GRMHD_CT_FLUX && p->ct != GRMHD_CT_FACE) { snprintf(msg, n, "unknown constrained-transport mode"); return false; }
  if (p->scalar != 0 && p->scalar != 1) { snprintf(msg, n, "scalar must be 0 or 1"); return false; }
  if (p->scalar && p->ng < 3) { snprintf(msg, n, "a passive scalar needs ng >= 3"); return false; }
  if (p->scalar && p->ct != GRMHD_CT_FLUX) { snprintf(msg, n, "the passive scalar runs with flux-CT (GRMHD_CT_FLUX)"); return false; }
  if (p->metric == GRMHD_MINKOWSKI && !(p->shift[0] * p->shift[0] + p->shift[1] * p->shift[1] + p->shift[2] * p->shift[2] < 1.0)) {
    snprintf(msg, n, "the shift must have |beta| < 1");
    return false;
  }
  if (p->metric == GRMHD_KERR_SCHILD_SPHERICAL) {
    const char* why = !(p->mass >= 0.0)            ? "mass must be >= 0"
                      : !(std::fabs(p->spin) < 1.0) ? "|spin| must be < 1"
                      : p->ct != GRMHD_CT_FLUX      ? "spherical Kerr-Schild runs with flux-CT (GRMHD_CT_FLUX)"
                      : p->scalar                   ? "spherical Kerr-Schild runs without a passive scalar"
                      : p->bc == GRMHD_BC_PERIODIC  ? "spherical Kerr-Schild takes fixed or spherical ghosts"
                                                    : nullptr;
    if (why) { snprintf(msg, n, "%s", why); return false; }
  }
  if (p->bc == GRMHD_BC_SPHERICAL) {
    const double pi = 3.14159265358979323846;
    const char* why =
        p->metric != GRMHD_KERR_SCHILD_SPHERICAL ? "spherical ghosts need the spherical Kerr-Schild metric"
        : !(std::fabs(p->x0[1]) < 1e-12 && std::fabs(p->x0[1] + p->ny * p->dx[1] - pi) < 1e-9)
            ? "spherical ghosts need a block over theta in [0, pi]"
        : !(std::fabs(p->nz * p->dx[2] - 2.0 * pi) < 1e-9) || p->nz % 2 ? "spherical ghosts need phi over [0, 2 pi) with nz even"
        : p->ng > p->ny ? "spherical ghosts need ng <= ny"
                        : nullptr;
    if (why) { snprintf(msg, n, "%s", why); return false; }
  }
  return true;
}

DevParams dev_params(const grmhd_params* p) {
  DevParams d{};
  d.nx = p->nx; d.ny = p->ny; d.nz = p->nz; d.ng = p->ng;
  d.gx = p->nx + 2 * p->ng; d.gy = p->ny + 2 * p->ng; d.gz = p->nz + 2 * p->ng;
  d.gsize = (long long)d.gx * d.gy * d.gz;
  d.isize = (long long)p->nx * p->ny * p->nz;
  for (int i = 0; i < 3; ++i) {
    d.x0[i] = p->x0[i];
    d.dx[i] = p->dx[i];
    d.idx[i] = p->dx[i] > 0 ? 1.0 / p->dx[i] : 0.0;
  }
  d.a = p->spin * p->mass;
  d.M = p->mass;
  d.gamma_eos = p->gamma_eos;
  d.metric = p->metric; d.recon = p->recon; d.riemann = p->riemann; d.bc = p->bc;
  d.rho_floor0 = p->rho_floor0; d.eps_floor0 = p->eps_floor0; d.floor_r_exp = p->floor_r_exp; d.w_max = p->w_max;
  d.w_max2 = p->w_max * p->w_max;
  d.v0sq_cap = 1.0 - 1.0 / (p->w_max * p->w_max);
  d.c2p_tol = p->c2p_tol; d.c2p_max_iter = p->c2p_max_iter;
  d.cfl = p->cfl; d.weno_eps = p->weno_eps;
  for (int i = 0; i < 3; ++i) d.shift[i] = p->metric == GRMHD_MINKOWSKI ? p->shift[i] : 0.0;
  for (int i = 0; i < 3; ++i) {
    d.fx0[i] = (float)d.x0[i];
    d.fdx[i] = (float)d.dx[i];
    d.fidx[i] = (float)d.idx[i];
    d.fshift[i] = (float)d.shift[i];
  }
  d.fa = (float)d.a;
  d.fM = (float)d.M;
  d.fgamma = (float)d.gamma_eos;
  d.fweno_eps = (float)d.weno_eps;
  d.frho_floor0 = (float)d.rho_floor0;
  d.feps_floor0 = (float)d.eps_floor0;
  d.fw_max2 = (float)d.w_max2;
  d.fv0sq_cap = (float)d.v0sq_cap;
  d.floor_r2 = d.floor_r_exp == 2.0 ? 1 : 0;
  return d;
}

}  // namespace grmhd

namespace {

thread_local char g_create_err[256] = "";

constexpr size_t kAlign = 256;
constexpr int kFaultSlot = 32;  // scal[32]: the bounds-check build's fault word
size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct Layout {
  size_t P, U[3], F[3], E, status, worklist, wl_mu, floorlist, geo, B[3], Ecc, X, DX[3], FX, scal, total;
};

Layout layout_of(const grmhd_params* p) {
  Layout l{};
  const size_t G = (size_t)(p->nx + 2 * p->ng) * (p->ny + 2 * p->ng) * (p->nz + 2 * p->ng);
  const size_t I = (size_t)p->nx * p->ny * p->nz;
  const bool batch_only = I == 0;
  const size_t pb = p->precision == GRMHD_MIXED ? 4 : 8;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  l.scal = take(64 * sizeof(unsigned long long));
  if (!batch_only) {
    l.P = take(8 * G * pb);
    for (int s = 0; s < 3; ++s) l.U[s] = take(8 * I * sizeof(double));
    for (int d = 0; d < 3; ++d) l.F[d] = take(8 * G * pb);
    l.E = take(3 * G * (p->ct == GRMHD_CT_FACE ? sizeof(double) : pb));  // face-centred CT: upwind EMFs in double
    l.status = take(I);
    if (p->precision == GRMHD_MIXED) {
      l.worklist = take(I * sizeof(int));
      l.wl_mu = take(I * sizeof(double));
    }
    l.floorlist = take(I * sizeof(int));
    if (p->metric == GRMHD_KERR_SCHILD) l.geo = take(NGEO * I * sizeof(double));
    if (p->ct == GRMHD_CT_FACE) {
      for (int k = 0; k < 3; ++k) l.B[k] = take(3 * G * sizeof(double));
      l.Ecc = take(3 * G * pb);
    }
    if (p->scalar) {
      l.X = take(G * pb);
      for (int k = 0; k < 3; ++k) l.DX[k] = take(I * sizeof(double));
      l.FX = take(3 * G * pb);
    }
  }
  l.total = off;
  return l;
}

int fail(grmhd_ctx* c, int code, const char* what, cudaError_t e = cudaSuccess) {
  if (e != cudaSuccess)
    snprintf(c->err, sizeof(c->err), "%s: %s", what, cudaGetErrorString(e));
  else
    snprintf(c->err, sizeof(c->err), "%s", what);
  return code;
}

#define CK(expr, what)                                   \
  do {                                                   \
    cudaError_t e_ = (expr);                             \
    if (e_ != cudaSuccess) return fail(c, GRMHD_E_CUDA, what, e_); \
  } while (0)

bool batch_only(const grmhd_ctx* c) { return c->dp.isize == 0; }

// Fold the events of the last timed stage into the per-kernel totals (synchronises on its last event).
cudaError_t collect_timing(grmhd_ctx* c) {
  if (!c->t_pending) return cudaSuccess;
  cudaError_t e = cudaEventSynchronize(c->ev[7]);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < 7; ++k) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]);
    if (e != cudaSuccess) return e;
    c->t_ms[k] += ms;
  }
  c->t_stages += 1;
  c->t_pending = false;
  return cudaSuccess;
}

constexpr int kMinTile = 128;

// Units per work item of a phase: `tile` faces / edges / cells; for the run units of the cell-centric
// five-point fluxes (~flux_run faces each) tile / flux_run of them, at least 128 so that a CTA is filled.
// The x units of those fluxes are lanes of whole warps: their items hold a multiple of 32 of them.
int phase_tile(const DevParams& p, int tile, int phase) {
  if ((phase == 1 || phase == 2) && cell_centric(p.recon)) {
    const int t = tile / (p.flux_run > 0 ? p.flux_run : FLUX_RUN);
    return t < 128 ? 128 : t;
  }
  if (phase == 0 && cell_centric(p.recon)) return (tile + 31) / 32 * 32;
  return tile;
}

long long block_items(const DevParams& p, int tile, int phase) {
  long long n;
  tile = phase_tile(p, tile, phase);
  if (phase < 3) {
    n = flux_units(p, phase);
  } else if (phase == 3) {
    n = (long long)(p.nx + 1) * (p.ny + 1) * (p.nz + 1);
  } else {
    n = p.isize;
  }
  return (n + tile - 1) / tile;
}

std::vector<WorkItem> build_items(const std::vector<BlockDesc>& blocks, int tile, int counts[3]) {
  std::vector<WorkItem> v[3];
  for (int b = 0; b < (int)blocks.size(); ++b) {
    const DevParams& p = blocks[b].p;
    for (int phase = 0; phase < 5; ++phase) {
      long long n;
      if (phase < 3) {
        n = flux_units(p, phase);
      } else if (phase == 3) {
        n = (long long)(p.nx + 1) * (p.ny + 1) * (p.nz + 1);
      } else {
        n = p.isize;
      }
      const int list = phase < 3 ? 0 : phase - 2;
      const int pt = phase_tile(p, tile, phase);
      for (long long s = 0; s < n; s += pt) {
        WorkItem w;
        w.block = b;
        w.phase = phase;
        w.start = s;
        w.count = (int)std::min<long long>(pt, n - s);
        w.pad = 0;
        v[list].push_back(w);
      }
    }
  }
  std::vector<WorkItem> all;
  for (int l = 0; l < 3; ++l) {
    counts[l] = (int)v[l].size();
    all.insert(all.end(), v[l].begin(), v[l].end());
  }
  return all;
}

struct BatchLayout {
  size_t scal, blocks, items, worklist, wl_mu, floorlist, leaf, reflux, ghost, fine, total;
  long long leaf_cap, reflux_cap, ghost_cap;
  std::vector<size_t> P, U, F, E, status, geo;  // per block; U and F hold 3 consecutive regions
  std::vector<size_t> X, DX, FX;                // passive scalar per block (DX: 3 consecutive regions)
};

bool valid_block(const grmhd_block& b, int ng, char* msg, size_t n) {
  if (b.nx < 1 || b.ny < 1 || b.nz < 1) { snprintf(msg, n, "block sizes must be >= 1"); return false; }
  if (!(b.dx[0] > 0 && b.dx[1] > 0 && b.dx[2] > 0)) { snprintf(msg, n, "block cell widths must be > 0"); return false; }
  const double cells = (double)(b.nx + 2 * ng) * (b.ny + 2 * ng) * (b.nz + 2 * ng);
  if (cells > 2.0e9) { snprintf(msg, n, "block too large"); return false; }
  return true;
}

DevParams block_params(const grmhd_params* p, const grmhd_block& b) {
  grmhd_params q = *p;
  q.nx = b.nx; q.ny = b.ny; q.nz = b.nz;
  for (int i = 0; i < 3; ++i) { q.x0[i] = b.x0[i]; q.dx[i] = b.dx[i]; }
  return dev_params(&q);
}

BatchLayout batch_layout(const grmhd_params* p, int nblocks, const grmhd_block* blocks) {
  BatchLayout l;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  const size_t pb = p->precision == GRMHD_MIXED ? 4 : 8;
  l.scal = take(64 * sizeof(unsigned long long));
  l.blocks = take(sizeof(BlockDesc) * (size_t)nblocks);
  long long items = 0, cells = 0;
  std::vector<BlockDesc> tmp(nblocks);
  for (int b = 0; b < nblocks; ++b) {
    const DevParams d = block_params(p, blocks[b]);
    for (int phase = 0; phase < 5; ++phase) items += block_items(d, kMinTile, phase);
    cells += d.isize;
  }
  l.items = take(sizeof(WorkItem) * (size_t)items);
  for (int b = 0; b < nblocks; ++b) {
    const DevParams d = block_params(p, blocks[b]);
    const size_t G = (size_t)d.gsize, I = (size_t)d.isize;
    l.P.push_back(take(8 * G * pb));
    for (int s = 0; s < 3; ++s) l.U.push_back(take(8 * I * sizeof(double)));
    for (int k = 0; k < 3; ++k) l.F.push_back(take(8 * G * pb));
    l.E.push_back(take(3 * G * pb));
    l.status.push_back(take(I));
    l.geo.push_back(p->metric == GRMHD_KERR_SCHILD ? take(NGEO * I * sizeof(double)) : 0);
    if (p->scalar) {
      l.X.push_back(take(G * pb));
      for (int k = 0; k < 3; ++k) l.DX.push_back(take(I * sizeof(double)));
      l.FX.push_back(take(3 * G * pb));
    }
  }
  l.worklist = p->precision == GRMHD_MIXED ? take((size_t)cells * sizeof(int)) : 0;
  l.wl_mu = p->precision == GRMHD_MIXED ? take((size_t)cells * sizeof(double)) : 0;
  l.floorlist = take((size_t)cells * sizeof(int));
  // two-level meshes: a leaf map of at most 8 units per block, and at most every face cell of every block
  // at a coarse-fine face
  l.leaf_cap = 8LL * nblocks;
  l.reflux_cap = 0;
  for (int b = 0; b < nblocks; ++b)
    l.reflux_cap += 2LL * ((long long)blocks[b].nx * blocks[b].ny + (long long)blocks[b].ny * blocks[b].nz +
                           (long long)blocks[b].nx * blocks[b].nz);
  l.ghost_cap = 0;
  for (int b = 0; b < nblocks; ++b) {
    const DevParams d = block_params(p, blocks[b]);
    if (d.gsize - d.isize > l.ghost_cap) l.ghost_cap = d.gsize - d.isize;
  }
  l.leaf = take((size_t)l.leaf_cap * sizeof(int));
  l.reflux = take((size_t)l.reflux_cap * sizeof(RefluxCell));
  l.ghost = take((size_t)l.ghost_cap * sizeof(unsigned));
  l.fine = take((size_t)nblocks * sizeof(int));
  l.total = off;
  return l;
}

}  // namespace

namespace grmhd {
char* create_error_buffer() { return g_create_err; }
}  // namespace grmhd

extern "C" {

size_t grmhd_workspace_bytes(const grmhd_params* p) {
  char msg[256];
  if (!valid_params(p, msg, sizeof msg)) return 0;
  return layout_of(p).total;
}

int grmhd_create(const grmhd_params* p, void* workspace, size_t bytes, void* stream, grmhd_ctx** out) {
  if (!out) {
    snprintf(g_create_err, sizeof g_create_err, "out is NULL");
    return GRMHD_E_INVALID;
  }
  *out = nullptr;
  if (!valid_params(p, g_create_err, sizeof g_create_err)) return GRMHD_E_INVALID;
  const Layout l = layout_of(p);
  if (bytes < l.total || (l.total > 0 && workspace == nullptr)) {
    snprintf(g_create_err, sizeof g_create_err, "workspace of %zu bytes is smaller than the %zu bytes needed", bytes, l.total);
    return GRMHD_E_WORKSPACE;
  }
  if (((uintptr_t)workspace) % kAlign != 0) {
    snprintf(g_create_err, sizeof g_create_err, "workspace must be 256-byte aligned");
    return GRMHD_E_WORKSPACE;
  }
  grmhd_ctx* c = new (std::nothrow) grmhd_ctx();
  if (!c) {
    snprintf(g_create_err, sizeof g_create_err, "host allocation failed");
    return GRMHD_E_INVALID;
  }
  c->prm = *p;
  c->dp = dev_params(p);
  {  // runs of the y / z flux units sized to fill this GPU with this one block (batches keep FLUX_RUN)
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
      c->dp.flux_run = flux_run_for(p->nx, p->ny, p->nz, nsm);
  }
  c->L = p->precision == GRMHD_MIXED ? &mixed_launchers() : &fp64_launchers();
  c->stream = (cudaStream_t)stream;
  c->ws = (char*)workspace;
  c->ws_bytes = bytes;
  c->scal = (unsigned long long*)(c->ws + l.scal);
  c->dp.fault = c->scal + kFaultSlot;
  if (!batch_only(c)) {
    c->P = c->ws + l.P;
    for (int s = 0; s < 3; ++s) c->Uslot[s] = (double*)(c->ws + l.U[s]);
    for (int d = 0; d < 3; ++d) c->F[d] = c->ws + l.F[d];
    c->E = c->ws + l.E;
    c->status = (uint8_t*)(c->ws + l.status);
    c->worklist = p->precision == GRMHD_MIXED ? (int*)(c->ws + l.worklist) : nullptr;
    c->wl_mu = p->precision == GRMHD_MIXED ? (double*)(c->ws + l.wl_mu) : nullptr;
    c->floorlist = (int*)(c->ws + l.floorlist);
    if (p->metric == GRMHD_KERR_SCHILD) c->dp.geo = (const double*)(c->ws + l.geo);
    if (p->ct == GRMHD_CT_FACE) {
      for (int k = 0; k < 3; ++k) c->Bslot[k] = (double*)(c->ws + l.B[k]);
      c->Ecc = c->ws + l.Ecc;
    }
    if (p->scalar) {
      c->X = c->ws + l.X;
      for (int k = 0; k < 3; ++k) c->DXslot[k] = (double*)(c->ws + l.DX[k]);
      c->FX = c->ws + l.FX;
    }
  }
  c->has_faces = false;
  c->has_scalar = false;
  c->s0 = c->sc = 0;
  c->has_state = false;
  cudaError_t e = cudaMemsetAsync(c->ws, 0, l.total, c->stream);
  if (e == cudaSuccess && c->dp.geo) e = c->L->geometry(c->dp, (double*)c->dp.geo, c->stream);
  if (e != cudaSuccess) {
    snprintf(g_create_err, sizeof g_create_err, "initialising the workspace failed: %s", cudaGetErrorString(e));
    delete c;
    return GRMHD_E_CUDA;
  }
  *out = c;
  return GRMHD_OK;
}

int grmhd_set_prims(grmhd_ctx* c, const double* P, int where) {
  if (!c || !P) return c ? fail(c, GRMHD_E_INVALID, "P is NULL") : GRMHD_E_INVALID;
  if (c->nblocks > 0) return fail(c, GRMHD_E_INVALID, "batch context: use grmhd_batch_set_prims");
  if (batch_only(c)) return fail(c, GRMHD_E_INVALID, "context has no grid");
  const size_t bytes = sizeof(double) * NV * (size_t)c->dp.gsize;
  const double* src = P;
  if (where == GRMHD_HOST) {
    // Stage through the flux region: it spans at least 8 G doubles in both forms (one double flux
    // buffer, or three contiguous float flux buffers).
    void* tmp = c->F[0];
    CK(cudaMemcpyAsync(tmp, P, bytes, cudaMemcpyHostToDevice, c->stream), "copying P to the device");
    CK(cudaStreamSynchronize(c->stream), "synchronising");  // a host P is read before the call returns
    src = (const double*)tmp;
  } else if (where != GRMHD_DEVICE) {
    return fail(c, GRMHD_E_INVALID, "where must be GRMHD_HOST or GRMHD_DEVICE");
  }
  CK(c->L->load_prims(c->dp, src, c->P, c->stream), "loading primitives");
  c->s0 = c->sc = 0;
  CK(c->L->prim2con(c->dp, c->P, c->Uslot[0], 0, c->dp.isize, c->stream), "prim->cons");
  c->has_state = true;
  c->has_faces = false;
  c->has_scalar = false;
  return GRMHD_OK;
}

int grmhd_set_face_b(grmhd_ctx* c, const double* Bf, int where) {
  if (!c || !Bf) return c ? fail(c, GRMHD_E_INVALID, "Bf is NULL") : GRMHD_E_INVALID;
  if (c->nblocks > 0 || batch_only(c)) return fail(c, GRMHD_E_INVALID, "context has no single-block grid");
  if (c->prm.ct != GRMHD_CT_FACE) return fail(c, GRMHD_E_INVALID, "not a face-centred CT context (params.ct)");
  if (!c->has_state) return fail(c, GRMHD_E_INVALID, "grmhd_set_prims has not been called");
  if (where != GRMHD_HOST && where != GRMHD_DEVICE) return fail(c, GRMHD_E_INVALID, "bad where");
  const size_t bytes = sizeof(double) * 3 * (size_t)c->dp.gsize;
  double* cur = c->Bslot[c->sc];
  CK(cudaMemcpyAsync(cur, Bf, bytes, where == GRMHD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                     c->stream),
     "copying the face field");
  if (c->prm.bc == GRMHD_BC_PERIODIC) CK(c->L->ghost_faces(c->dp, cur, c->stream), "face ghost fill");
  // every slot starts from these faces: fixed ghost faces are never written by a stage
  for (int k = 0; k < 3; ++k)
    if (c->Bslot[k] != cur) CK(cudaMemcpyAsync(c->Bslot[k], cur, bytes, cudaMemcpyDeviceToDevice, c->stream), "copying faces");
  CK(c->L->face_to_cells(c->dp, cur, c->P, c->stream), "cell field from the faces");
  CK(c->L->prim2con(c->dp, c->P, c->Uslot[c->sc], 0, c->dp.isize, c->stream), "prim->cons");
  if (where == GRMHD_HOST) CK(cudaStreamSynchronize(c->stream), "synchronising");
  c->has_faces = true;
  return GRMHD_OK;
}

// The loading stream and its events, made on first use.
static cudaError_t ensure_load_stream(grmhd_ctx* c) {
  if (c->load_stream) return cudaSuccess;
  cudaError_t e = cudaStreamCreateWithFlags(&c->load_stream, cudaStreamNonBlocking);
  for (cudaEvent_t& ev : c->load_ev)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  return e;
}

// grmhd_set_prims_f32; join = false (host loads inside grmhd_stage_host_f32): the context's stream does not wait
// for the prim->cons and the call does not wait for the copies; the stage that follows joins the prim->cons
// before its update (load_ev[kLoadChunks]) and the caller waits for the copies (load_ev[last chunk]).
static int set_prims_f32(grmhd_ctx* c, const float* P, int where, bool join);

int grmhd_set_prims_f32(grmhd_ctx* c, const float* P, int where) { return set_prims_f32(c, P, where, true); }

static int set_prims_f32(grmhd_ctx* c, const float* P, int where, bool join) {
  if (!c || !P) return c ? fail(c, GRMHD_E_INVALID, "P is NULL") : GRMHD_E_INVALID;
  if (c->nblocks > 0 || batch_only(c)) return fail(c, GRMHD_E_INVALID, "context has no single-block grid");
  if (c->L->p_bytes != 4) return fail(c, GRMHD_E_INVALID, "single-precision primitives need a GRMHD_MIXED context");
  if (where != GRMHD_HOST && where != GRMHD_DEVICE) return fail(c, GRMHD_E_INVALID, "where must be GRMHD_HOST or GRMHD_DEVICE");
  const size_t bytes = sizeof(float) * NV * (size_t)c->dp.gsize;
  c->s0 = c->sc = 0;
  if (where == GRMHD_DEVICE) {
    CK(cudaMemcpyAsync(c->P, P, bytes, cudaMemcpyDeviceToDevice, c->stream), "copying P");
    CK(c->L->prim2con(c->dp, c->P, c->Uslot[0], 0, c->dp.isize, c->stream), "prim->cons");
  } else {
    // In kLoadChunks slabs of ghosted z rows: a slab's rows of the 8 variables are copied on the context's
    // stream, and the prim->cons of the interior cells in those rows runs on the loading stream once they
    // have landed, beside the next slab's copies (a 256^3 load: 0.6 GB at ~210 GB/s, 2.8 ms, against 2.9 ms
    // of double-precision prim->cons). The call returns once the host P has been read; the context's stream
    // waits for the last prim->cons.
    CK(ensure_load_stream(c), "creating the loading stream");
    const long long row = (long long)c->dp.gx * c->dp.gy, G = c->dp.gsize, plane = (long long)c->dp.nx * c->dp.ny;
    const int gz = c->dp.gz, ng = c->dp.ng, nz = c->dp.nz;
    const int nch = gz < kLoadChunks ? gz : kLoadChunks;
    int r0 = 0;
    for (int ch = 0; ch < nch; ++ch) {
      const int r1 = (int)((long long)gz * (ch + 1) / nch);
      for (int q = 0; q < NV; ++q)
        CK(cudaMemcpyAsync((float*)c->P + q * G + r0 * row, P + q * G + r0 * row, sizeof(float) * (r1 - r0) * row,
                           cudaMemcpyHostToDevice, c->stream),
           "copying P");
      CK(cudaEventRecord(c->load_ev[ch], c->stream), "recording a load event");
      CK(cudaStreamWaitEvent(c->load_stream, c->load_ev[ch], 0), "ordering the loading stream");
      const int k0 = r0 - ng > 0 ? r0 - ng : 0, k1 = r1 - ng < nz ? r1 - ng : nz;  // interior z of these rows
      if (k1 > k0) CK(c->L->prim2con(c->dp, c->P, c->Uslot[0], k0 * plane, k1 * plane, c->load_stream), "prim->cons");
      r0 = r1;
    }
    CK(cudaEventRecord(c->load_ev[kLoadChunks], c->load_stream), "recording a load event");
    c->load_last = nch - 1;
    if (join) {
      CK(cudaStreamWaitEvent(c->stream, c->load_ev[kLoadChunks], 0), "ordering the context's stream");
      CK(cudaEventSynchronize(c->load_ev[nch - 1]), "synchronising");  // the host P has been read
    }
  }
  c->has_state = true;
  c->has_faces = false;
  c->has_scalar = false;
  return GRMHD_OK;
}

int grmhd_set_scalar(grmhd_ctx* c, const double* X, int where) {
  if (!c || !X) return c ? fail(c, GRMHD_E_INVALID, "X is NULL") : GRMHD_E_INVALID;
  if (c->nblocks > 0 || batch_only(c)) return fail(c, GRMHD_E_INVALID, "context has no single-block grid");
  if (!c->prm.scalar) return fail(c, GRMHD_E_INVALID, "the context was created without a passive scalar");
  if (!c->has_state) return fail(c, GRMHD_E_INVALID, "grmhd_set_prims has not been called");
  const double* src = X;
  if (where == GRMHD_HOST) {
    // stage through the flux region (at least 8 G doubles)
    CK(cudaMemcpyAsync(c->F[0], X, sizeof(double) * (size_t)c->dp.gsize, cudaMemcpyHostToDevice, c->stream),
       "copying X to the device");
    src = (const double*)c->F[0];
  } else if (where != GRMHD_DEVICE) {
    return fail(c, GRMHD_E_INVALID, "where must be GRMHD_HOST or GRMHD_DEVICE");
  }
  CK(c->L->scalar_load(c->dp, src, c->X, c->Uslot[c->sc], c->DXslot[c->sc], c->stream), "loading X");
  if (where == GRMHD_HOST) CK(cudaStreamSynchronize(c->stream), "synchronising");
  c->has_scalar = true;
  return GRMHD_OK;
}

int grmhd_set_cons(grmhd_ctx* c, const double* U, int where) {
  if (!c || !U) return c ? fail(c, GRMHD_E_INVALID, "U is NULL") : GRMHD_E_INVALID;
  if (c->nblocks > 0) return fail(c, GRMHD_E_INVALID, "not available for batch contexts");
  if (batch_only(c)) return fail(c, GRMHD_E_INVALID, "context has no grid");
  if (where != GRMHD_HOST && where != GRMHD_DEVICE) return fail(c, GRMHD_E_INVALID, "bad where");
  const size_t bytes = sizeof(double) * NV * (size_t)c->dp.isize;
  CK(cudaMemcpyAsync(c->Uslot[c->sc], U, bytes, where == GRMHD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                     c->stream),
     "copying U");
  if (where == GRMHD_HOST) CK(cudaStreamSynchronize(c->stream), "synchronising");
  c->has_state = true;
  c->has_scalar = false;
  return GRMHD_OK;
}

static int batch_stage(grmhd_ctx* c, double g0, double g1, double beta, double dt);
int grmhd_p2c(grmhd_ctx* c, long long n, const double* P, double* U) {
  if (!c) return GRMHD_E_INVALID;
  if (n < 0 || (n > 0 && (!U || !P))) return fail(c, GRMHD_E_INVALID, "bad batch arguments");
  CK(launch_p2c_batch(P, U, n, c->dp, c->stream), "prim2con batch");
  return GRMHD_OK;
}

int grmhd_c2p_guess(grmhd_ctx* c, const void* mlp_ws, long long n, const double* U, double* P, uint8_t* status,
                    int* iters, double* guess, float* X, float* T, int flags) {
  if (!c) return GRMHD_E_INVALID;
  if (n < 0 || (n > 0 && (!U || !P))) return fail(c, GRMHD_E_INVALID, "bad batch arguments");
  if (flags & ~GRMHD_GUESS_FP32) return fail(c, GRMHD_E_INVALID, "unknown flags");
  const bool fp32 = (flags & GRMHD_GUESS_FP32) != 0;
  if (mlp_ws && fp32 && !guess) return fail(c, GRMHD_E_INVALID, "the FP32-core guess needs a guess buffer");
  if (mlp_ws && !fp32 && (X || T))
    return fail(c, GRMHD_E_INVALID, "training pairs are recorded by the standard or the FP32-core path only");
  if (mlp_ws && ((uintptr_t)mlp_ws) % 256 != 0) return fail(c, GRMHD_E_WORKSPACE, "network workspace not 256-byte aligned");
  unsigned long long* stats = c->scal + 8;
  CK(cudaMemsetAsync(stats, 0, 8 * sizeof(unsigned long long), c->stream), "clearing stats");
  if (mlp_ws && !fp32) {
    CK(launch_c2p_net_tc(mlp_ws, U, P, status, iters, n, c->dp, guess, stats, c->stream), "tensor-core guided con2prim");
    return GRMHD_OK;
  }
  if (mlp_ws) CK(launch_mlp_guess(mlp_ws, U, guess, n, c->dp, c->stream), "network guess");
  CK(launch_c2p_guided(U, P, status, iters, n, c->dp, mlp_ws ? guess : nullptr, X, T, stats, c->stream),
     "guided con2prim batch");
  return GRMHD_OK;
}

static int grmhd_get_scalars(grmhd_ctx* c, int what, void* dst, int where);

// One stage of a context (grmhd_stage); host_out != NULL (float primitives, single-block contexts): the stage's
// primitives are also copied to host_out, overlapped with the update (grmhd_stage_host_f32); join_load: a host
// load without join precedes (its prim->cons, on the loading stream, may run beside the ghost fill and fluxes,
// which read only P; the update waits for it).
static int stage_impl(grmhd_ctx* c, double g0, double g1, double beta, double dt, float* host_out,
                      bool join_load = false) {
  if (!c) return GRMHD_E_INVALID;
  if (c->nblocks > 0) return batch_stage(c, g0, g1, beta, dt);
  if (batch_only(c)) return fail(c, GRMHD_E_INVALID, "context has no grid");
  if (!c->has_state) return fail(c, GRMHD_E_INVALID, "grmhd_set_prims has not been called");
  if (!(g0 == g0) || !(g1 == g1) || !(beta == beta) || !(dt == dt)) return fail(c, GRMHD_E_INVALID, "NaN stage coefficient");
  const bool first = g0 == 0.0;
  if (!first && c->s0 == c->sc) return fail(c, GRMHD_E_INVALID, "a stage with g0 != 0 needs a preceding stage with g0 == 0");
  int dst;
  if (first) {
    c->s0 = c->sc;
    dst = (c->sc + 1) % 3;
  } else {
    dst = 3 - c->s0 - c->sc;
  }
  const bool auto_dt = !(dt > 0.0);
  const bool track = auto_dt && first;
  const bool face = c->prm.ct == GRMHD_CT_FACE;
  if (face && !c->has_faces) return fail(c, GRMHD_E_INVALID, "grmhd_set_face_b has not been called");
  if (c->prm.scalar && !c->has_scalar) return fail(c, GRMHD_E_INVALID, "grmhd_set_scalar has not been called");
  const FormLaunchers& L = *c->L;
  const cudaStream_t s = c->stream;
  // this stage's parameters: with face-centred CT the flux kernels read the normal field of the faces
  DevParams dp = c->dp;
  if (face) dp.bface = c->Bslot[c->sc];
  if (c->timing) CK(collect_timing(c), "reading kernel timings");
#define TMARK(k) \
  if (c->timing) CK(cudaEventRecord(c->ev[k], s), "recording a timing event")
  unsigned long long* ms = c->scal;
  double* dt_dev = (double*)(c->scal + 3);
  unsigned long long* stats = c->scal + 8;
  CK(cudaMemsetAsync(stats, 0, 10 * sizeof(unsigned long long), s), "clearing stats and the worklist counts");
  if (track) CK(cudaMemsetAsync(ms, 0, 3 * sizeof(unsigned long long), s), "clearing speeds");
  TMARK(0);
  if (c->prm.bc == GRMHD_BC_PERIODIC) {
    CK(L.ghost(dp, c->P, s), "ghost fill");
    if (face) CK(L.ghost_faces(dp, c->Bslot[c->sc], s), "face ghost fill");
  } else if (c->prm.bc == GRMHD_BC_SPHERICAL) {
    CK(L.ghost(dp, c->P, s), "polar and azimuthal ghost fill");
  }
  for (int d = 0; d < 3; ++d) {
    TMARK(1 + d);
    CK(L.flux(dp, c->P, c->F[d], ms, d, track ? 1 : 0, s), "flux");
  }
  if (track) CK(launch_finalize_dt(ms, dt_dev, dp, s), "time step");
  TMARK(4);
  StageArgs a{};
  a.U0 = c->Uslot[c->s0];
  a.Ucur = c->Uslot[c->sc];
  a.Unew = c->Uslot[dst];
  a.status = c->status;
  a.dt_dev = dt_dev;
  a.stats = stats;
  a.g0 = g0;
  a.g1 = g1;
  a.beta = beta;
  a.dt = dt;
  a.use_dev_dt = auto_dt ? 1 : 0;
  a.worklist = c->worklist;
  a.wl_count = (unsigned int*)(c->scal + 16);
  a.wl_mu = c->wl_mu;
  if (c->worklist) {  // mixed form: floored cells re-derived in place; the list holds the full solves
    a.solvelist = c->floorlist;
    a.sl_count = (unsigned int*)(c->scal + 17);
  } else {
    a.floorlist = c->floorlist;
    a.fl_count = (unsigned int*)(c->scal + 17);
  }
  if (face) {
    CK(L.emf_face(dp, c->P, c->F[0], c->F[1], c->F[2], c->Ecc, c->E, s), "upwind EMF");
    CK(L.face_update(dp, c->Bslot[c->s0], c->Bslot[c->sc], c->Bslot[dst], c->E, a, s), "face update");
    a.bface_new = c->Bslot[dst];
  } else {
    CK(L.emf(dp, c->F[0], c->F[1], c->F[2], c->E, s), "EMF");
  }
  if (join_load) CK(cudaStreamWaitEvent(s, c->load_ev[kLoadChunks], 0), "joining the load's prim->cons");
  TMARK(5);
  if (!host_out) {
    CK(L.update(dp, c->P, c->F[0], c->F[1], c->F[2], c->E, a, s), "update");
    TMARK(6);
    CK(L.cell_passes(dp, c->P, a, s), "floored and deferred cells");
  } else {
    // In kLoadChunks slabs of interior z rows: a slab's update and its passes over deferred cells on the
    // context's stream, then the copy of its ghosted rows of P to the host on the loading stream, beside the
    // next slab's update (a 256^3 read-back: 0.6 GB at ~190 GB/s, 3.1 ms, against ~6 ms of update). A cell's
    // update and passes read and write only its own primitives, so the slabs' rows are final when copied.
    CK(ensure_load_stream(c), "creating the loading stream");
    if (!c->out_ev_made) {
      for (cudaEvent_t& e : c->out_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "creating an event");
      c->out_ev_made = true;
    }
    const long long plane = (long long)dp.nx * dp.ny, row = (long long)dp.gx * dp.gy, G = dp.gsize;
    const int nz = dp.nz, ng = dp.ng, gz = dp.gz;
    const int nch = nz < kLoadChunks ? nz : kLoadChunks;
    for (int ch = 0; ch < nch; ++ch) {
      const int k0 = (int)((long long)nz * ch / nch), k1 = (int)((long long)nz * (ch + 1) / nch);
      if (ch > 0 && c->worklist)
        CK(cudaMemsetAsync(c->scal + 16, 0, 2 * sizeof(unsigned long long), s), "clearing the list counts");
      a.t_begin = k0 * plane;
      a.t_end = k1 * plane;
      CK(L.update(dp, c->P, c->F[0], c->F[1], c->F[2], c->E, a, s), "update");
      CK(L.cell_passes(dp, c->P, a, s), "floored and deferred cells");
      CK(cudaEventRecord(c->out_ev[ch], s), "recording a read-back event");
      CK(cudaStreamWaitEvent(c->load_stream, c->out_ev[ch], 0), "ordering the loading stream");
      const int r0 = ch == 0 ? 0 : k0 + ng, r1 = ch == nch - 1 ? gz : k1 + ng;  // ghosted z rows of the slab
      for (int q = 0; q < NV; ++q)
        CK(cudaMemcpyAsync(host_out + q * G + r0 * row, (const float*)c->P + q * G + r0 * row,
                           sizeof(float) * (r1 - r0) * row, cudaMemcpyDeviceToHost, c->load_stream),
           "copying P to the host");
    }
    a.t_begin = a.t_end = 0;
    TMARK(6);  // the timing groups count these updates and passes together as the update
  }
  if (c->prm.scalar) {
    // the passive scalar: X of the stage's start, the stage's mass fluxes, its final D
    if (c->prm.bc == GRMHD_BC_PERIODIC) CK(L.scalar_ghost(dp, c->X, s), "scalar ghost fill");
    for (int d = 0; d < 3; ++d) CK(L.scalar_flux(dp, c->X, c->F[d], c->FX, d, s), "scalar flux");
    CK(L.scalar_update(dp, c->X, c->FX, c->DXslot[c->s0], c->DXslot[c->sc], c->DXslot[dst], c->Uslot[dst], a, s),
       "scalar update");
  }
  TMARK(7);
#undef TMARK
  if (c->timing) c->t_pending = true;
  c->sc = dst;
  if (host_out) {
    // later work on the context's stream (a load into P) waits for the copies; the call returns once they are done
    CK(cudaEventRecord(c->out_ev[kLoadChunks], c->load_stream), "recording a read-back event");
    CK(cudaStreamWaitEvent(s, c->out_ev[kLoadChunks], 0), "ordering the context's stream");
    CK(cudaEventSynchronize(c->out_ev[kLoadChunks]), "synchronising");
  }
  return GRMHD_OK;
}

int grmhd_stage(grmhd_ctx* c, double g0, double g1, double beta, double dt) {
  return stage_impl(c, g0, g1, beta, dt, nullptr);
}

int grmhd_stage_host_f32(grmhd_ctx* c, const float* P_in, float* P_out, double g0, double g1, double beta,
                         double dt) {
  if (!c) return GRMHD_E_INVALID;
  if (c->nblocks > 0 || batch_only(c)) return fail(c, GRMHD_E_INVALID, "context has no single-block grid");
  if (c->L->p_bytes != 4) return fail(c, GRMHD_E_INVALID, "single-precision primitives need a GRMHD_MIXED context");
  if (P_in) {
    const int r = set_prims_f32(c, P_in, GRMHD_HOST, false);
    if (r != GRMHD_OK) return r;
  }
  const int r = stage_impl(c, g0, g1, beta, dt, P_out, P_in != nullptr);
  if (P_in) {
    // P_in has been read when the call returns, whatever the stage did
    if (r != GRMHD_OK) cudaStreamWaitEvent(c->stream, c->load_ev[kLoadChunks], 0);
    const cudaError_t e = cudaEventSynchronize(c->load_ev[c->load_last]);
    if (r == GRMHD_OK && e != cudaSuccess) return fail(c, GRMHD_E_CUDA, "synchronising", e);
  }
  return r;
}

int grmhd_rk2_step(grmhd_ctx* c, double dt) {
  int r = grmhd_stage(c, 0.0, 1.0, 1.0, dt);
  if (r) return r;
  return grmhd_stage(c, 0.5, 0.5, 0.5, dt);
}

int grmhd_c2p(grmhd_ctx* c, long long n, const double* U, double* P, uint8_t* status, int* iters, int flags) {
  if (!c) return GRMHD_E_INVALID;
  if (n < 0 || (n > 0 && (!U || !P))) return fail(c, GRMHD_E_INVALID, "bad batch arguments");
  unsigned long long* stats = c->scal + 8;
  CK(cudaMemsetAsync(stats, 0, sizeof(unsigned long long), c->stream), "clearing stats");
  CK(launch_c2p_batch(U, P, status, iters, n, flags, c->dp, stats, c->stream), "con2prim batch");
  return GRMHD_OK;
}

static int grmhd_get_scalars(grmhd_ctx* c, int what, void* dst, int where) {
  const cudaMemcpyKind kind = where == GRMHD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (what == GRMHD_GET_STATS)
    CK(cudaMemcpyAsync(dst, c->scal + 8, 8 * sizeof(unsigned long long), kind, c->stream), "copying stats");
  else
    CK(cudaMemcpyAsync(dst, c->scal + 3, sizeof(double), kind, c->stream), "copying dt");
  if (where == GRMHD_HOST) CK(cudaStreamSynchronize(c->stream), "synchronising");
  return GRMHD_OK;
}

// Enqueue one batched stage on stream s (slot indices, coefficients and dt already fixed).
static int batch_enqueue(grmhd_ctx* c, const BatchArgs& a, bool track, cudaStream_t s) {
  const FormLaunchers& L = *c->L;
  unsigned long long* ms = c->scal;
  unsigned int* ctr = (unsigned int*)(c->scal + 20);
  CK(cudaMemsetAsync(c->scal + 8, 0, 10 * sizeof(unsigned long long), s), "clearing stats and list counts");
  CK(cudaMemsetAsync(ctr, 0, 4 * sizeof(unsigned int), s), "clearing work counters");
  if (track) CK(cudaMemsetAsync(ms, 0, sizeof(unsigned long long), s), "clearing speeds");
  const WorkItem* flux_items = c->ditems;
  const WorkItem* emf_items = flux_items + c->n_items[0];
  const WorkItem* upd_items = emf_items + c->n_items[1];
  const int grid = c->grid_persist;
  if (c->lattice_on)
    CK(L.batch_exchange(c->dblocks, c->nblocks, c->total_ghosted, c->lattice, s), "ghost exchange");
  if (c->mesh_on) {
    CK(L.mesh_exchange(c->dblocks, c->nblocks, c->mesh, 1, s), "mesh ghost exchange (pass 1)");
    CK(L.mesh_exchange(c->dblocks, c->nblocks, c->mesh, 2, s), "mesh ghost exchange (pass 2)");
  }
  CK(L.batch_flux(c->dblocks, flux_items, c->n_items[0], ctr + 0, ms, track ? 1 : 0, c->prm.metric, c->prm.recon,
                   c->grid_flux, s),
     "batched flux");
  if (track) CK(launch_batch_finalize_dt(ms, (double*)(c->scal + 3), c->prm.cfl, s), "time step");
  CK(L.batch_emf(c->dblocks, emf_items, c->n_items[1], ctr + 1, grid, s), "batched EMF");
  CK(L.batch_update(c->dblocks, upd_items, c->n_items[2], ctr + 2, a, c->prm.metric, grid, s), "batched update");
  CK(L.batch_floors(c->dblocks, c->nblocks, a, c->prm.metric, grid, s), "batched floor re-derivation");
  if (c->worklist) CK(L.batch_deferred(c->dblocks, c->nblocks, a, c->prm.metric, grid, s), "batched deferred con2prim");
  if (c->mesh_on && c->n_reflux > 0)
    CK(L.mesh_reflux(c->dblocks, c->dreflux, c->n_reflux, a, c->prm.metric, s), "refluxing");
  if (c->prm.scalar) {
    // the passive scalar of every block: X of the stage's start (its ghosts exchanged with P's), the stage's
    // mass fluxes, the blocks' final D
    for (int d = 0; d < 3; ++d)
      CK(L.batch_scalar_flux(c->dblocks, c->nblocks, c->max_runs, c->prm.recon, d, s), "batched scalar flux");
    CK(L.batch_scalar_update(c->dblocks, c->nblocks, c->max_cells, a, s), "batched scalar update");
    if (c->mesh_on && c->n_reflux > 0)
      CK(L.mesh_reflux_scalar(c->dblocks, c->dreflux, c->n_reflux, a, s), "scalar refluxing");
  }
  return GRMHD_OK;
}

static int batch_stage(grmhd_ctx* c, double g0, double g1, double beta, double dt) {
  if (!c->has_state) return fail(c, GRMHD_E_INVALID, "grmhd_batch_set_prims has not been called");
  if (c->prm.scalar)
    for (int b = 0; b < c->nblocks; ++b)
      if (!c->block_scalar[b]) return fail(c, GRMHD_E_INVALID, "grmhd_batch_set_scalar has not been called for every block");
  if (!(g0 == g0) || !(g1 == g1) || !(beta == beta) || !(dt == dt)) return fail(c, GRMHD_E_INVALID, "NaN stage coefficient");
  const bool first = g0 == 0.0;
  if (!first && c->s0 == c->sc) return fail(c, GRMHD_E_INVALID, "a stage with g0 != 0 needs a preceding stage with g0 == 0");
  const int s0 = first ? c->sc : c->s0;
  const int dst = first ? (c->sc + 1) % 3 : 3 - c->s0 - c->sc;
  const bool auto_dt = !(dt > 0.0);
  const bool track = auto_dt && first;
  BatchArgs a{};
  a.g0 = g0; a.g1 = g1; a.beta = beta; a.dt = dt;
  a.use_dev_dt = auto_dt ? 1 : 0;
  a.s0 = s0; a.sc = c->sc; a.dst = dst;
  a.dt_dev = (const double*)(c->scal + 3);
  a.stats = c->scal + 8;
  a.worklist = c->worklist;
  a.wl_count = (unsigned int*)(c->scal + 16);
  a.wl_mu = c->wl_mu;
  if (c->worklist) {  // mixed form: floored cells re-derived in place; the list holds the full solves
    a.solvelist = c->floorlist;
    a.sl_count = (unsigned int*)(c->scal + 17);
  } else {
    a.floorlist = c->floorlist;
    a.fl_count = (unsigned int*)(c->scal + 17);
  }
  if (c->use_graph) {
    const std::vector<double> key = {g0, g1, beta, dt, (double)s0, (double)c->sc, (double)dst, (double)c->tile};
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
      CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "starting the graph capture");
      const int rc = batch_enqueue(c, a, track, c->cap_stream);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
      if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      CK(e, "ending the graph capture");
      cudaGraphExec_t ex = nullptr;
      const cudaError_t e2 = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      CK(e2, "instantiating the stage graph");
      it = c->graphs.emplace(key, ex).first;
    }
    CK(cudaGraphLaunch(it->second, c->stream), "launching the stage graph");
  } else {
    const int rc = batch_enqueue(c, a, track, c->stream);
    if (rc) return rc;
  }
  c->s0 = s0;
  c->sc = dst;
  return GRMHD_OK;
}

int grmhd_bounds_fault(grmhd_ctx* c, unsigned long long out[2]) {
  if (!c || !out) return c ? fail(c, GRMHD_E_INVALID, "out is NULL") : GRMHD_E_INVALID;
  CK(cudaMemcpyAsync(out, c->scal + kFaultSlot, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream),
     "copying the fault word");
  CK(cudaStreamSynchronize(c->stream), "synchronising");
#ifdef GRMHD_BOUNDS_CHECK
  out[1] = 1;
#else
  out[1] = 0;
#endif
  return GRMHD_OK;
}

int grmhd_max_speed(grmhd_ctx* c, double out[3]) {
  if (!c || !out) return c ? fail(c, GRMHD_E_INVALID, "out is NULL") : GRMHD_E_INVALID;
  if (c->nblocks > 0 || batch_only(c)) return fail(c, GRMHD_E_INVALID, "context has no single-block grid");
  unsigned long long bits[3];
  CK(cudaMemcpyAsync(bits, c->scal, sizeof bits, cudaMemcpyDeviceToHost, c->stream), "copying the speeds");
  CK(cudaStreamSynchronize(c->stream), "synchronising");
  for (int d = 0; d < 3; ++d) {
    double v;
    std::memcpy(&v, &bits[d], sizeof v);  // non-negative doubles are kept as their bit patterns
    out[d] = v;
  }
  return GRMHD_OK;
}

int grmhd_get(grmhd_ctx* c, int what, void* dst, int where) {
  if (!c || !dst) return c ? fail(c, GRMHD_E_INVALID, "dst is NULL") : GRMHD_E_INVALID;
  if (c->nblocks > 0) {
    if (what == GRMHD_GET_STATS || what == GRMHD_GET_DT) return grmhd_get_scalars(c, what, dst, where);
    return fail(c, GRMHD_E_INVALID, "per-block data of a batch: use grmhd_batch_get");
  }
  if (where != GRMHD_HOST && where != GRMHD_DEVICE) return fail(c, GRMHD_E_INVALID, "bad where");
  const cudaMemcpyKind kind = where == GRMHD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  const cudaStream_t s = c->stream;
  if (what != GRMHD_GET_STATS && batch_only(c)) return fail(c, GRMHD_E_INVALID, "context has no grid");
  switch (what) {
    case GRMHD_GET_PRIMS: {
      const size_t bytes = sizeof(double) * NV * (size_t)c->dp.gsize;
      if (c->L->p_bytes == 8) {
        CK(cudaMemcpyAsync(dst, c->P, bytes, kind, s), "copying P");
      } else if (where == GRMHD_DEVICE) {
        CK(c->L->store_prims(c->dp, c->P, (double*)dst, s), "converting P");
      } else {
        // widen into the flux buffers (together >= 8 G doubles) and copy out
        CK(c->L->store_prims(c->dp, c->P, (double*)c->F[0], s), "converting P");
        CK(cudaMemcpyAsync(dst, c->F[0], bytes, kind, s), "copying P");
      }
      break;
    }
    case GRMHD_GET_CONS:
      CK(cudaMemcpyAsync(dst, c->Uslot[c->sc], sizeof(double) * NV * (size_t)c->dp.isize, kind, s), "copying U");
      break;
    case GRMHD_GET_PRIMS_F32:
      if (c->L->p_bytes != 4) return fail(c, GRMHD_E_INVALID, "single-precision primitives need a GRMHD_MIXED context");
      CK(cudaMemcpyAsync(dst, c->P, sizeof(float) * NV * (size_t)c->dp.gsize, kind, s), "copying P");
      break;
    case GRMHD_GET_STATUS:
      CK(cudaMemcpyAsync(dst, c->status, (size_t)c->dp.isize, kind, s), "copying status");
      break;
    case GRMHD_GET_STATS:
      CK(cudaMemcpyAsync(dst, c->scal + 8, 8 * sizeof(unsigned long long), kind, s), "copying stats");
      break;
    case GRMHD_GET_DT:
      CK(cudaMemcpyAsync(dst, c->scal + 3, sizeof(double), kind, s), "copying dt");
      break;
    case GRMHD_GET_SCALAR:
    case GRMHD_GET_SCALAR_CONS:
      if (!c->prm.scalar || !c->has_scalar) return fail(c, GRMHD_E_INVALID, "no passive scalar set");
      if (what == GRMHD_GET_SCALAR_CONS) {
        CK(cudaMemcpyAsync(dst, c->DXslot[c->sc], sizeof(double) * (size_t)c->dp.isize, kind, s), "copying D X");
      } else if (where == GRMHD_DEVICE) {
        CK(c->L->scalar_store(c->dp, c->X, (double*)dst, s), "converting X");
      } else {
        CK(c->L->scalar_store(c->dp, c->X, (double*)c->F[0], s), "converting X");
        CK(cudaMemcpyAsync(dst, c->F[0], sizeof(double) * (size_t)c->dp.gsize, kind, s), "copying X");
      }
      break;
    case GRMHD_GET_FACE_B:
      if (c->prm.ct != GRMHD_CT_FACE) return fail(c, GRMHD_E_INVALID, "not a face-centred CT context");
      CK(cudaMemcpyAsync(dst, c->Bslot[c->sc], sizeof(double) * 3 * (size_t)c->dp.gsize, kind, s), "copying faces");
      break;
    default:
      return fail(c, GRMHD_E_INVALID, "unknown GRMHD_GET_* selector");
  }
  if (where == GRMHD_HOST) CK(cudaStreamSynchronize(s), "synchronising");
  return GRMHD_OK;
}

int grmhd_set_timing(grmhd_ctx* c, int on) {
  if (!c) return GRMHD_E_INVALID;
  if (on && !c->timing) {
    for (int k = 0; k < 8; ++k) CK(cudaEventCreate(&c->ev[k]), "creating timing events");
  }
  if (!on && c->timing) {
    CK(collect_timing(c), "reading kernel timings");
    for (int k = 0; k < 8; ++k) cudaEventDestroy(c->ev[k]);
  }
  c->timing = on != 0;
  return GRMHD_OK;
}

int grmhd_get_timing(grmhd_ctx* c, double* ms, int* stages) {
  if (!c || !ms) return GRMHD_E_INVALID;
  if (c->timing) CK(collect_timing(c), "reading kernel timings");
  for (int k = 0; k < 7; ++k) {
    ms[k] = c->t_ms[k];
    c->t_ms[k] = 0.0;
  }
  if (stages) *stages = c->t_stages;
  c->t_stages = 0;
  return GRMHD_OK;
}

const char* grmhd_last_error(const grmhd_ctx* c) { return c ? c->err : g_create_err; }

void grmhd_destroy(grmhd_ctx* c) {
  if (c && c->timing)
    for (int k = 0; k < 8; ++k) cudaEventDestroy(c->ev[k]);
  if (c && c->out_ev_made)
    for (cudaEvent_t e : c->out_ev) cudaEventDestroy(e);
  if (c && c->load_stream) {
    for (cudaEvent_t e : c->load_ev) cudaEventDestroy(e);
    cudaStreamDestroy(c->load_stream);
  }
  if (c) {
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  }
  delete c;
}

// ------------------------------------------------------------------ batches of meshblocks

size_t grmhd_batch_workspace_bytes(const grmhd_params* p, int nblocks, const grmhd_block* blocks) {
  char msg[256];
  if (!p || nblocks < 1 || !blocks) return 0;
  grmhd_params q = *p;
  q.nx = blocks[0].nx; q.ny = blocks[0].ny; q.nz = blocks[0].nz;
  for (int i = 0; i < 3; ++i) q.dx[i] = blocks[0].dx[i];
  if (!valid_params(&q, msg, sizeof msg)) return 0;
  if (p->metric == GRMHD_KERR_SCHILD_SPHERICAL) return 0;
  for (int b = 0; b < nblocks; ++b)
    if (!valid_block(blocks[b], p->ng, msg, sizeof msg)) return 0;
  return batch_layout(p, nblocks, blocks).total;
}

int grmhd_batch_create(const grmhd_params* p, int nblocks, const grmhd_block* blocks, void* workspace, size_t bytes,
                       void* stream, grmhd_ctx** out) {
  if (!out) {
    snprintf(g_create_err, sizeof g_create_err, "out is NULL");
    return GRMHD_E_INVALID;
  }
  *out = nullptr;
  if (!p || nblocks < 1 || !blocks) {
    snprintf(g_create_err, sizeof g_create_err, "need params and at least one block");
    return GRMHD_E_INVALID;
  }
  grmhd_params q = *p;
  q.nx = blocks[0].nx; q.ny = blocks[0].ny; q.nz = blocks[0].nz;
  for (int i = 0; i < 3; ++i) q.dx[i] = blocks[0].dx[i];
  if (!valid_params(&q, g_create_err, sizeof g_create_err)) return GRMHD_E_INVALID;
  if (p->metric == GRMHD_KERR_SCHILD_SPHERICAL) {
    snprintf(g_create_err, sizeof g_create_err, "batches run the Cartesian metrics (spherical Kerr-Schild: grmhd_create)");
    return GRMHD_E_UNSUPPORTED;
  }
  if (p->bc != GRMHD_BC_FIXED) {
    snprintf(g_create_err, sizeof g_create_err, "batched blocks take their ghosts as given (GRMHD_BC_FIXED)");
    return GRMHD_E_UNSUPPORTED;
  }
  if (p->ct != GRMHD_CT_FLUX) {
    snprintf(g_create_err, sizeof g_create_err, "batches use flux-CT (GRMHD_CT_FLUX)");
    return GRMHD_E_UNSUPPORTED;
  }
  if (p->scalar && nblocks > 65535) {
    snprintf(g_create_err, sizeof g_create_err, "a batch with a passive scalar holds at most 65535 blocks");
    return GRMHD_E_UNSUPPORTED;
  }
  for (int b = 0; b < nblocks; ++b)
    if (!valid_block(blocks[b], p->ng, g_create_err, sizeof g_create_err)) return GRMHD_E_INVALID;
  const BatchLayout l = batch_layout(p, nblocks, blocks);
  if (bytes < l.total || !workspace) {
    snprintf(g_create_err, sizeof g_create_err, "workspace of %zu bytes is smaller than the %zu bytes needed", bytes,
             l.total);
    return GRMHD_E_WORKSPACE;
  }
  if (((uintptr_t)workspace) % kAlign != 0) {
    snprintf(g_create_err, sizeof g_create_err, "workspace must be 256-byte aligned");
    return GRMHD_E_WORKSPACE;
  }
  grmhd_ctx* c = new (std::nothrow) grmhd_ctx();
  if (!c) {
    snprintf(g_create_err, sizeof g_create_err, "host allocation failed");
    return GRMHD_E_INVALID;
  }
  c->prm = *p;
  c->dp = dev_params(&q);
  c->L = p->precision == GRMHD_MIXED ? &mixed_launchers() : &fp64_launchers();
  c->stream = (cudaStream_t)stream;
  c->ws = (char*)workspace;
  c->ws_bytes = bytes;
  c->scal = (unsigned long long*)(c->ws + l.scal);
  c->nblocks = nblocks;
  c->dblocks = (BlockDesc*)(c->ws + l.blocks);
  c->ditems = (WorkItem*)(c->ws + l.items);
  c->worklist = p->precision == GRMHD_MIXED ? (int*)(c->ws + l.worklist) : nullptr;
  c->wl_mu = p->precision == GRMHD_MIXED ? (double*)(c->ws + l.wl_mu) : nullptr;
  c->floorlist = (int*)(c->ws + l.floorlist);
  c->hblocks.resize(nblocks);
  c->max_runs = 0;
  c->max_cells = 0;
  c->block_scalar.assign(p->scalar ? nblocks : 0, 0);
  long long off = 0;
  for (int b = 0; b < nblocks; ++b) {
    BlockDesc& d = c->hblocks[b];
    d.p = block_params(p, blocks[b]);
    d.p.fault = c->scal + kFaultSlot;
    d.P = c->ws + l.P[b];
    for (int k = 0; k < 3; ++k) {
      d.U[k] = (double*)(c->ws + l.U[3 * b + k]);
      d.F[k] = c->ws + l.F[3 * b + k];
    }
    d.E = c->ws + l.E[b];
    d.status = (uint8_t*)(c->ws + l.status[b]);
    if (p->metric == GRMHD_KERR_SCHILD) d.p.geo = (const double*)(c->ws + l.geo[b]);
    d.X = nullptr;
    d.FX = nullptr;
    for (int k = 0; k < 3; ++k) d.DX[k] = nullptr;
    if (p->scalar) {
      d.X = c->ws + l.X[b];
      for (int k = 0; k < 3; ++k) d.DX[k] = (double*)(c->ws + l.DX[3 * b + k]);
      d.FX = c->ws + l.FX[b];
      c->max_runs = std::max(c->max_runs, (long long)d.p.gsize);
      c->max_cells = std::max(c->max_cells, d.p.isize);
    }
    d.cell_offset = off;
    off += d.p.isize;
  }
  c->total_cells = off;
  c->total_ghosted = (long long)nblocks * c->hblocks[0].p.gsize;
  c->lattice_on = false;
  c->mesh_on = false;
  c->dleaf = (int*)(c->ws + l.leaf);
  c->dreflux = (RefluxCell*)(c->ws + l.reflux);
  c->dghost = (unsigned*)(c->ws + l.ghost);
  c->dfine = (int*)(c->ws + l.fine);
  c->ghost_cap = l.ghost_cap;
  c->leaf_cap = l.leaf_cap;
  c->reflux_cap = l.reflux_cap;
  c->n_reflux = 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  c->grid_persist = (sms > 0 ? sms : 152) * c->L->batch_ctas_per_sm(p->metric);
  c->grid_flux = (sms > 0 ? sms : 152) * c->L->batch_flux_ctas_per_sm(p->metric, p->recon);
  cudaError_t e = cudaMemsetAsync(c->ws, 0, l.total, c->stream);
  for (int b = 0; b < nblocks && e == cudaSuccess; ++b)
    if (c->hblocks[b].p.geo) e = c->L->geometry(c->hblocks[b].p, (double*)c->hblocks[b].p.geo, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->dblocks, c->hblocks.data(), sizeof(BlockDesc) * nblocks, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    snprintf(g_create_err, sizeof g_create_err, "initialising the batch failed: %s", cudaGetErrorString(e));
    delete c;
    return GRMHD_E_CUDA;
  }
  *out = c;
  const int rc = grmhd_batch_set_tile(c, 512);
  if (rc) {
    snprintf(g_create_err, sizeof g_create_err, "%s", c->err);
    delete c;
    *out = nullptr;
    return rc;
  }
  return GRMHD_OK;
}

int grmhd_batch_set_tile(grmhd_ctx* c, int tile) {
  if (!c || c->nblocks < 1) return c ? fail(c, GRMHD_E_INVALID, "not a batch context") : GRMHD_E_INVALID;
  if (tile < kMinTile || tile > (1 << 20)) return fail(c, GRMHD_E_INVALID, "tile must be in [128, 2^20]");
  const std::vector<WorkItem> items = build_items(c->hblocks, tile, c->n_items);
  // items are built from a smaller minimum tile, so they always fit the reserved region
  CK(cudaMemcpyAsync(c->ditems, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice, c->stream),
     "uploading work items");
  CK(cudaStreamSynchronize(c->stream), "synchronising");
  c->tile = tile;
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
  return GRMHD_OK;
}

int grmhd_batch_set_lattice(grmhd_ctx* c, int nbx, int nby, int nbz, int periodic) {
  if (!c || c->nblocks < 1) return c ? fail(c, GRMHD_E_INVALID, "not a batch context") : GRMHD_E_INVALID;
  if (nbx == 0 && nby == 0 && nbz == 0) {
    c->lattice_on = false;
  } else {
    if (nbx < 1 || nby < 1 || nbz < 1 || (long long)nbx * nby * nbz != c->nblocks)
      return fail(c, GRMHD_E_INVALID, "the lattice must hold exactly the batch's blocks");
    const DevParams& a = c->hblocks[0].p;
    const int nb[3] = {nbx, nby, nbz};
    for (int b = 0; b < c->nblocks; ++b) {
      const DevParams& q = c->hblocks[b].p;
      if (q.nx != a.nx || q.ny != a.ny || q.nz != a.nz) return fail(c, GRMHD_E_INVALID, "lattice blocks differ in size");
      const int bc[3] = {b % nbx, (b / nbx) % nby, b / (nbx * nby)};
      const int n[3] = {a.nx, a.ny, a.nz};
      for (int d = 0; d < 3; ++d) {
        if (q.dx[d] != a.dx[d]) return fail(c, GRMHD_E_INVALID, "lattice blocks differ in cell width");
        const double want = a.x0[d] + (double)bc[d] * n[d] * a.dx[d];
        if (std::fabs(q.x0[d] - want) > 1e-9 * (std::fabs(want) + nb[d] * n[d] * a.dx[d]))
          return fail(c, GRMHD_E_INVALID, "block corners do not follow the lattice order");
      }
    }
    c->lattice.nb[0] = nbx;
    c->lattice.nb[1] = nby;
    c->lattice.nb[2] = nbz;
    c->lattice.periodic = periodic ? 1 : 0;
    c->lattice_on = true;
    c->mesh_on = false;
  }
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
  return GRMHD_OK;
}

int grmhd_batch_set_mesh(grmhd_ctx* c, int nbx, int nby, int nbz, int periodic, const int* level, const int* pos) {
  if (!c || c->nblocks < 1) return c ? fail(c, GRMHD_E_INVALID, "not a batch context") : GRMHD_E_INVALID;
  if (nbx == 0 && nby == 0 && nbz == 0) {
    c->mesh_on = false;
  } else {
    if (nbx < 1 || nby < 1 || nbz < 1 || !level || !pos) return fail(c, GRMHD_E_INVALID, "bad mesh arguments");
    if (8LL * nbx * nby * nbz > c->leaf_cap) return fail(c, GRMHD_E_INVALID, "more root blocks than the batch's leaves can tile");
    std::vector<DevParams> bp(c->nblocks);
    for (int b = 0; b < c->nblocks; ++b) bp[b] = c->hblocks[b].p;
    std::vector<int> leaf, fine;
    std::vector<RefluxCell> cells;
    std::vector<unsigned> ghost;
    const char* why =
        build_mesh_tables(bp.data(), c->nblocks, nbx, nby, nbz, periodic, level, pos, leaf, cells, ghost, fine);
    if (why) return fail(c, GRMHD_E_INVALID, why);
    if ((long long)ghost.size() > c->ghost_cap) return fail(c, GRMHD_E_INVALID, "ghost table larger than reserved");
    const long long units = (long long)leaf.size();
    if ((long long)cells.size() > c->reflux_cap) return fail(c, GRMHD_E_INVALID, "too many coarse-fine cells");
    for (int b = 0; b < c->nblocks; ++b) {
      c->hblocks[b].level = level[b];
      for (int d = 0; d < 3; ++d) c->hblocks[b].pos[d] = pos[3 * b + d];
    }
    CK(cudaMemcpyAsync(c->dleaf, leaf.data(), sizeof(int) * units, cudaMemcpyHostToDevice, c->stream), "mesh leaf map");
    if (!cells.empty())
      CK(cudaMemcpyAsync(c->dreflux, cells.data(), sizeof(RefluxCell) * cells.size(), cudaMemcpyHostToDevice, c->stream),
         "mesh reflux cells");
    CK(cudaMemcpyAsync(c->dghost, ghost.data(), sizeof(unsigned) * ghost.size(), cudaMemcpyHostToDevice, c->stream),
       "mesh ghost table");
    if (!fine.empty())
      CK(cudaMemcpyAsync(c->dfine, fine.data(), sizeof(int) * fine.size(), cudaMemcpyHostToDevice, c->stream),
         "mesh fine blocks");
    CK(cudaMemcpyAsync(c->dblocks, c->hblocks.data(), sizeof(BlockDesc) * c->nblocks, cudaMemcpyHostToDevice, c->stream),
       "mesh block descriptors");
    CK(cudaStreamSynchronize(c->stream), "mesh upload");
    c->mesh.nb[0] = nbx;
    c->mesh.nb[1] = nby;
    c->mesh.nb[2] = nbz;
    c->mesh.periodic = periodic ? 1 : 0;
    c->mesh.leaf = c->dleaf;
    c->mesh.ghost = c->dghost;
    c->mesh.nghost = (int)ghost.size();
    c->mesh.fine = c->dfine;
    c->mesh.nfine = (int)fine.size();
    c->n_reflux = (int)cells.size();
    c->mesh_on = true;
    c->lattice_on = false;
  }
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
  return GRMHD_OK;
}

int grmhd_batch_set_prims(grmhd_ctx* c, int block, const double* P, int where) {
  if (!c || c->nblocks < 1) return c ? fail(c, GRMHD_E_INVALID, "not a batch context") : GRMHD_E_INVALID;
  if (block < 0 || block >= c->nblocks || !P) return fail(c, GRMHD_E_INVALID, "bad block index or P");
  const BlockDesc& b = c->hblocks[block];
  const size_t bytes = sizeof(double) * NV * (size_t)b.p.gsize;
  const double* src = P;
  if (where == GRMHD_HOST) {
    // stage through the block's flux region (at least 8 G doubles in both forms)
    CK(cudaMemcpyAsync(b.F[0], P, bytes, cudaMemcpyHostToDevice, c->stream), "copying P to the device");
    CK(cudaStreamSynchronize(c->stream), "synchronising");  // a host P is read before the call returns
    src = (const double*)b.F[0];
  } else if (where != GRMHD_DEVICE) {
    return fail(c, GRMHD_E_INVALID, "where must be GRMHD_HOST or GRMHD_DEVICE");
  }
  CK(c->L->load_prims(b.p, src, b.P, c->stream), "loading primitives");
  CK(c->L->prim2con(b.p, b.P, b.U[0], 0, b.p.isize, c->stream), "prim->cons");
  c->s0 = c->sc = 0;
  c->has_state = true;
  if (!c->block_scalar.empty()) c->block_scalar[block] = 0;
  return GRMHD_OK;
}

int grmhd_batch_set_scalar(grmhd_ctx* c, int block, const double* X, int where) {
  if (!c || c->nblocks < 1) return c ? fail(c, GRMHD_E_INVALID, "not a batch context") : GRMHD_E_INVALID;
  if (block < 0 || block >= c->nblocks || !X) return fail(c, GRMHD_E_INVALID, "bad block index or X");
  if (!c->prm.scalar) return fail(c, GRMHD_E_INVALID, "the batch was created without a passive scalar");
  if (!c->has_state) return fail(c, GRMHD_E_INVALID, "grmhd_batch_set_prims has not been called");
  const BlockDesc& b = c->hblocks[block];
  const double* src = X;
  if (where == GRMHD_HOST) {
    CK(cudaMemcpyAsync(b.F[0], X, sizeof(double) * (size_t)b.p.gsize, cudaMemcpyHostToDevice, c->stream),
       "copying X to the device");
    src = (const double*)b.F[0];
  } else if (where != GRMHD_DEVICE) {
    return fail(c, GRMHD_E_INVALID, "where must be GRMHD_HOST or GRMHD_DEVICE");
  }
  CK(c->L->scalar_load(b.p, src, b.X, b.U[c->sc], b.DX[c->sc], c->stream), "loading X");
  if (where == GRMHD_HOST) CK(cudaStreamSynchronize(c->stream), "synchronising");
  c->block_scalar[block] = 1;
  return GRMHD_OK;
}

int grmhd_batch_get(grmhd_ctx* c, int block, int what, void* dst, int where) {
  if (!c || c->nblocks < 1) return c ? fail(c, GRMHD_E_INVALID, "not a batch context") : GRMHD_E_INVALID;
  if (!dst) return fail(c, GRMHD_E_INVALID, "dst is NULL");
  if (where != GRMHD_HOST && where != GRMHD_DEVICE) return fail(c, GRMHD_E_INVALID, "bad where");
  const cudaMemcpyKind kind = where == GRMHD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  const cudaStream_t s = c->stream;
  if (what == GRMHD_GET_STATS || what == GRMHD_GET_DT) return grmhd_get_scalars(c, what, dst, where);
  if (block < 0 || block >= c->nblocks) return fail(c, GRMHD_E_INVALID, "bad block index");
  const BlockDesc& b = c->hblocks[block];
  switch (what) {
    case GRMHD_GET_PRIMS: {
      const size_t bytes = sizeof(double) * NV * (size_t)b.p.gsize;
      if (c->L->p_bytes == 8) {
        CK(cudaMemcpyAsync(dst, b.P, bytes, kind, s), "copying P");
      } else if (where == GRMHD_DEVICE) {
        CK(c->L->store_prims(b.p, b.P, (double*)dst, s), "converting P");
      } else {
        CK(c->L->store_prims(b.p, b.P, (double*)b.F[0], s), "converting P");
        CK(cudaMemcpyAsync(dst, b.F[0], bytes, kind, s), "copying P");
      }
      break;
    }
    case GRMHD_GET_CONS:
      CK(cudaMemcpyAsync(dst, b.U[c->sc], sizeof(double) * NV * (size_t)b.p.isize, kind, s), "copying U");
      break;
    case GRMHD_GET_STATUS:
      CK(cudaMemcpyAsync(dst, b.status, (size_t)b.p.isize, kind, s), "copying status");
      break;
    case GRMHD_GET_SCALAR:
    case GRMHD_GET_SCALAR_CONS:
      if (!c->prm.scalar || !c->block_scalar[block]) return fail(c, GRMHD_E_INVALID, "no passive scalar set");
      if (what == GRMHD_GET_SCALAR_CONS) {
        CK(cudaMemcpyAsync(dst, b.DX[c->sc], sizeof(double) * (size_t)b.p.isize, kind, s), "copying D X");
      } else if (where == GRMHD_DEVICE) {
        CK(c->L->scalar_store(b.p, b.X, (double*)dst, s), "converting X");
      } else {
        CK(c->L->scalar_store(b.p, b.X, (double*)b.F[0], s), "converting X");
        CK(cudaMemcpyAsync(dst, b.F[0], sizeof(double) * (size_t)b.p.gsize, kind, s), "copying X");
      }
      break;
    default:
      return fail(c, GRMHD_E_INVALID, "unknown GRMHD_GET_* selector");
  }
  if (where == GRMHD_HOST) CK(cudaStreamSynchronize(s), "synchronising");
  return GRMHD_OK;
}

int grmhd_set_graph(grmhd_ctx* c, int on) {
  if (!c || c->nblocks < 1) return c ? fail(c, GRMHD_E_INVALID, "graphs are built for batch contexts") : GRMHD_E_INVALID;
  if (on && !c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "creating the capture stream");
  c->use_graph = on != 0;
  return GRMHD_OK;
}

int grmhd_batch_autotune(grmhd_ctx* c, int* best_tile, double* best_ms) {
  if (!c || c->nblocks < 1) return c ? fail(c, GRMHD_E_INVALID, "not a batch context") : GRMHD_E_INVALID;
  if (!c->has_state) return fail(c, GRMHD_E_INVALID, "load the blocks' primitives first");
  const int tiles[] = {128, 256, 512, 1024, 2048, 4096};
  int best = c->tile;
  float best_t = 1e30f;
  c->n_tuned = 0;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "creating events");
  CK(cudaEventCreate(&e1), "creating events");
  const bool graph = c->use_graph;
  c->use_graph = false;
  int rc = GRMHD_OK;
  for (int t : tiles) {
    rc = grmhd_batch_set_tile(c, t);
    if (rc) break;
    CK(cudaEventRecord(e0, c->stream), "recording");
    rc = grmhd_rk2_step(c, 0.0);  // one real step of the batch per candidate
    if (rc) break;
    CK(cudaEventRecord(e1, c->stream), "recording");
    CK(cudaEventSynchronize(e1), "synchronising");
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1), "reading events");
    c->tuned_tile[c->n_tuned] = t;
    c->tuned_ms[c->n_tuned] = 0.5 * ms;
    ++c->n_tuned;
    if (ms < best_t) {
      best_t = ms;
      best = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->use_graph = graph;
  if (rc) return rc;
  rc = grmhd_batch_set_tile(c, best);
  if (best_tile) *best_tile = best;
  if (best_ms) *best_ms = 0.5 * best_t;
  return rc;
}

int grmhd_batch_autotune_table(grmhd_ctx* c, int* tiles, double* ms, int cap, int* n) {
  if (!c || !n || cap < 0 || (cap > 0 && (!tiles || !ms))) return c ? fail(c, GRMHD_E_INVALID, "bad arguments") : GRMHD_E_INVALID;
  if (c->nblocks < 1) return fail(c, GRMHD_E_INVALID, "not a batch context");
  *n = c->n_tuned;
  for (int k = 0; k < c->n_tuned && k < cap; ++k) {
    tiles[k] = c->tuned_tile[k];
    ms[k] = c->tuned_ms[k];
  }
  return GRMHD_OK;
}

}  // extern "C"
