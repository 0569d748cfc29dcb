// C-ABI entry points of libgrmhd.so (declared and documented in include/grmhd.h).
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/grmhd.h"
#include "grmhd_device.cuh"
#include "grmhd_launch.h"

using namespace grmhd;

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
  unsigned long long* scal;  // [0..2] max speed bits, [3] dt (double), [8..15] stats, [16] worklist count
  int s0, sc;                // slot of U0 and of the current state
  bool has_state;
  bool timing;               // record CUDA events around each kernel group
  cudaEvent_t ev[8];         // ghost | flux x | flux y | flux z | emf | update | end
  double t_ms[6];            // accumulated ms per kernel group since the last read
  int t_stages;              // stages accumulated
  bool t_pending;            // events of the last stage not yet read
  char err[256];
};

namespace {

thread_local char g_create_err[256] = "";

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct Layout {
  size_t P, U[3], F[3], E, status, worklist, scal, total;
};

bool valid_params(const grmhd_params* p, char* msg, size_t n) {
  if (!p) { snprintf(msg, n, "params is NULL"); return false; }
  const bool batch_only = p->nx == 0 && p->ny == 0 && p->nz == 0;
  if (!batch_only) {
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) { snprintf(msg, n, "nx, ny, nz must be >= 1"); return false; }
    const int need = p->recon == GRMHD_RECON_WENO5Z_AOAH ? 3 : (p->recon == GRMHD_RECON_CONSTANT ? 1 : 2);
    if (p->ng < need) { snprintf(msg, n, "ng = %d too small for the reconstruction (needs %d)", p->ng, need); return false; }
    if (p->ng > 16) { snprintf(msg, n, "ng = %d too large", p->ng); return false; }
    for (int d = 0; d < 3; ++d)
      if (!(p->dx[d] > 0.0)) { snprintf(msg, n, "dx[%d] must be > 0", d); return false; }
    const double cells = (double)(p->nx + 2 * p->ng) * (p->ny + 2 * p->ng) * (p->nz + 2 * p->ng);
    if (cells > 4.0e9) { snprintf(msg, n, "block too large"); return false; }
  }
  if (p->metric != GRMHD_MINKOWSKI && p->metric != GRMHD_KERR_SCHILD) { snprintf(msg, n, "unknown metric"); return false; }
  if (p->recon < 0 || p->recon > 3) { snprintf(msg, n, "unknown reconstruction"); return false; }
  if (p->riemann != GRMHD_RIEMANN_LLF && p->riemann != GRMHD_RIEMANN_HLL) { snprintf(msg, n, "unknown Riemann solver"); return false; }
  if (p->precision != GRMHD_FP64 && p->precision != GRMHD_MIXED) { snprintf(msg, n, "unknown precision"); return false; }
  if (p->bc != GRMHD_BC_PERIODIC && p->bc != GRMHD_BC_FIXED) { snprintf(msg, n, "unknown boundary condition"); return false; }
  if (!(p->gamma_eos > 1.0)) { snprintf(msg, n, "gamma_eos must be > 1"); return false; }
  if (!(p->c2p_tol > 0.0) || p->c2p_max_iter < 1) { snprintf(msg, n, "bad con2prim tolerance / iteration cap"); return false; }
  if (!(p->w_max > 1.0)) { snprintf(msg, n, "w_max must be > 1"); return false; }
  if (p->metric == GRMHD_KERR_SCHILD && !(p->mass > 0.0)) { snprintf(msg, n, "mass must be > 0"); return false; }
  return true;
}

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
    l.E = take(3 * G * pb);
    l.status = take(I);
    if (p->precision == GRMHD_MIXED) l.worklist = take(I * sizeof(int));
  }
  l.total = off;
  return l;
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
  d.c2p_tol = p->c2p_tol; d.c2p_max_iter = p->c2p_max_iter;
  d.cfl = p->cfl; d.weno_eps = p->weno_eps;
  return d;
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
  cudaError_t e = cudaEventSynchronize(c->ev[6]);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < 6; ++k) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]);
    if (e != cudaSuccess) return e;
    c->t_ms[k] += ms;
  }
  c->t_stages += 1;
  c->t_pending = false;
  return cudaSuccess;
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
  c->L = p->precision == GRMHD_MIXED ? &mixed_launchers() : &fp64_launchers();
  c->stream = (cudaStream_t)stream;
  c->ws = (char*)workspace;
  c->ws_bytes = bytes;
  c->scal = (unsigned long long*)(c->ws + l.scal);
  if (!batch_only(c)) {
    c->P = c->ws + l.P;
    for (int s = 0; s < 3; ++s) c->Uslot[s] = (double*)(c->ws + l.U[s]);
    for (int d = 0; d < 3; ++d) c->F[d] = c->ws + l.F[d];
    c->E = c->ws + l.E;
    c->status = (uint8_t*)(c->ws + l.status);
    c->worklist = p->precision == GRMHD_MIXED ? (int*)(c->ws + l.worklist) : nullptr;
  }
  c->s0 = c->sc = 0;
  c->has_state = false;
  cudaError_t e = cudaMemsetAsync(c->ws, 0, l.total, c->stream);
  if (e != cudaSuccess) {
    snprintf(g_create_err, sizeof g_create_err, "clearing the workspace failed: %s", cudaGetErrorString(e));
    delete c;
    return GRMHD_E_CUDA;
  }
  *out = c;
  return GRMHD_OK;
}

int grmhd_set_prims(grmhd_ctx* c, const double* P, int where) {
  if (!c || !P) return c ? fail(c, GRMHD_E_INVALID, "P is NULL") : GRMHD_E_INVALID;
  if (batch_only(c)) return fail(c, GRMHD_E_INVALID, "context has no grid");
  const size_t bytes = sizeof(double) * NV * (size_t)c->dp.gsize;
  const double* src = P;
  if (where == GRMHD_HOST) {
    // Stage through the flux region: it spans at least 8 G doubles in both forms (one double flux
    // buffer, or three contiguous float flux buffers).
    void* tmp = c->F[0];
    CK(cudaMemcpyAsync(tmp, P, bytes, cudaMemcpyHostToDevice, c->stream), "copying P to the device");
    src = (const double*)tmp;
  } else if (where != GRMHD_DEVICE) {
    return fail(c, GRMHD_E_INVALID, "where must be GRMHD_HOST or GRMHD_DEVICE");
  }
  CK(c->L->load_prims(c->dp, src, c->P, c->stream), "loading primitives");
  c->s0 = c->sc = 0;
  CK(c->L->prim2con(c->dp, c->P, c->Uslot[0], c->stream), "prim->cons");
  c->has_state = true;
  return GRMHD_OK;
}

int grmhd_set_cons(grmhd_ctx* c, const double* U, int where) {
  if (!c || !U) return c ? fail(c, GRMHD_E_INVALID, "U is NULL") : GRMHD_E_INVALID;
  if (batch_only(c)) return fail(c, GRMHD_E_INVALID, "context has no grid");
  if (where != GRMHD_HOST && where != GRMHD_DEVICE) return fail(c, GRMHD_E_INVALID, "bad where");
  const size_t bytes = sizeof(double) * NV * (size_t)c->dp.isize;
  CK(cudaMemcpyAsync(c->Uslot[c->sc], U, bytes, where == GRMHD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                     c->stream),
     "copying U");
  if (where == GRMHD_HOST) CK(cudaStreamSynchronize(c->stream), "synchronising");
  c->has_state = true;
  return GRMHD_OK;
}

int grmhd_stage(grmhd_ctx* c, double g0, double g1, double beta, double dt) {
  if (!c) return GRMHD_E_INVALID;
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
  const FormLaunchers& L = *c->L;
  const cudaStream_t s = c->stream;
  if (c->timing) CK(collect_timing(c), "reading kernel timings");
#define TMARK(k) \
  if (c->timing) CK(cudaEventRecord(c->ev[k], s), "recording a timing event")
  unsigned long long* ms = c->scal;
  double* dt_dev = (double*)(c->scal + 3);
  unsigned long long* stats = c->scal + 8;
  CK(cudaMemsetAsync(stats, 0, 9 * sizeof(unsigned long long), s), "clearing stats and the worklist count");
  if (track) CK(cudaMemsetAsync(ms, 0, 3 * sizeof(unsigned long long), s), "clearing speeds");
  TMARK(0);
  if (c->prm.bc == GRMHD_BC_PERIODIC) CK(L.ghost(c->dp, c->P, s), "ghost fill");
  for (int d = 0; d < 3; ++d) {
    TMARK(1 + d);
    CK(L.flux(c->dp, c->P, c->F[d], ms, d, track ? 1 : 0, s), "flux");
  }
  if (track) CK(launch_finalize_dt(ms, dt_dev, c->dp, s), "time step");
  TMARK(4);
  CK(L.emf(c->dp, c->F[0], c->F[1], c->F[2], c->E, s), "EMF");
  TMARK(5);
  StageArgs a;
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
  CK(L.update(c->dp, c->P, c->F[0], c->F[1], c->F[2], c->E, a, s), "update");
  TMARK(6);
#undef TMARK
  if (c->timing) c->t_pending = true;
  c->sc = dst;
  return GRMHD_OK;
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

int grmhd_get(grmhd_ctx* c, int what, void* dst, int where) {
  if (!c || !dst) return c ? fail(c, GRMHD_E_INVALID, "dst is NULL") : GRMHD_E_INVALID;
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
    case GRMHD_GET_STATUS:
      CK(cudaMemcpyAsync(dst, c->status, (size_t)c->dp.isize, kind, s), "copying status");
      break;
    case GRMHD_GET_STATS:
      CK(cudaMemcpyAsync(dst, c->scal + 8, 8 * sizeof(unsigned long long), kind, s), "copying stats");
      break;
    case GRMHD_GET_DT:
      CK(cudaMemcpyAsync(dst, c->scal + 3, sizeof(double), kind, s), "copying dt");
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
    for (int k = 0; k < 7; ++k) CK(cudaEventCreate(&c->ev[k]), "creating timing events");
  }
  if (!on && c->timing) {
    CK(collect_timing(c), "reading kernel timings");
    for (int k = 0; k < 7; ++k) cudaEventDestroy(c->ev[k]);
  }
  c->timing = on != 0;
  return GRMHD_OK;
}

int grmhd_get_timing(grmhd_ctx* c, double* ms, int* stages) {
  if (!c || !ms) return GRMHD_E_INVALID;
  if (c->timing) CK(collect_timing(c), "reading kernel timings");
  for (int k = 0; k < 6; ++k) {
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
    for (int k = 0; k < 7; ++k) cudaEventDestroy(c->ev[k]);
  delete c;
}

}  // extern "C"
