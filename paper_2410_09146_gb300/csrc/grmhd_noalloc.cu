// grmhd_stage_noalloc: one all-FP64 Runge-Kutta stage that allocates nothing.
//
// Some callers cannot allocate device memory at all: code running inside a CUDA-graph capture,
// frameworks that own every allocation through their own pool, or embedded hosts without a
// device allocator. For them this entry point keeps its scratch (face fluxes, edge EMFs, the
// speed / time-step scalars) in one file-scope __device__ array of fixed size. The caller still
// passes the state arrays (inputs and outputs). The array exists on every device that loads the
// library and stays allocated until the process exits.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/grmhd.h"
#include "grmhd_device.cuh"
#include "grmhd_launch.h"

namespace grmhd {
char* create_error_buffer();  // thread-local message buffer read by grmhd_last_error(NULL)
// the checks and the kernel-side parameters of grmhd_create (grmhd_api.cu)
bool valid_params(const grmhd_params* p, char* msg, size_t n);
DevParams dev_params(const grmhd_params* p);
}

namespace {

using namespace grmhd;

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr size_t kScalarBytes = 512;                 // [0..2] max-speed bits, [3] dt, [8..15] stats
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_lock;
void* g_scratch_addr[kMaxDevices];  // device address of g_noalloc_scratch, per device

int fail(int code, const char* msg) {
  snprintf(create_error_buffer(), 256, "grmhd_stage_noalloc: %s", msg);
  return code;
}

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> guard(g_lock);
  if (g_scratch_addr[dev] == nullptr) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int grmhd_stage_noalloc(const grmhd_params* p, double* P, const double* U0, const double* Ucur,
                                   double* Unew, uint8_t* status, double g0, double g1, double beta, double dt,
                                   void* stream) {
  if (!p || !P || !Ucur || !Unew || !status) return fail(GRMHD_E_INVALID, "a required pointer is NULL");
  if (g0 != 0.0 && !U0) return fail(GRMHD_E_INVALID, "U0 is NULL but g0 != 0");
  if (!(g0 == g0) || !(g1 == g1) || !(beta == beta) || !(dt == dt)) return fail(GRMHD_E_INVALID, "NaN stage coefficient");
  char why[200];
  if (!valid_params(p, why, sizeof why)) return fail(GRMHD_E_INVALID, why);
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail(GRMHD_E_INVALID, "nx, ny, nz must be >= 1");
  if (p->precision != GRMHD_FP64) return fail(GRMHD_E_INVALID, "only the all-FP64 form is available");
  if (p->ct != GRMHD_CT_FLUX) return fail(GRMHD_E_INVALID, "face-centred CT needs a context (grmhd_create)");
  if (p->scalar) return fail(GRMHD_E_INVALID, "the passive scalar needs a context (grmhd_create)");
  if (p->metric == GRMHD_KERR_SCHILD_SPHERICAL) return fail(GRMHD_E_INVALID, "spherical Kerr-Schild needs a context (grmhd_create)");
  const double G = (double)(p->nx + 2 * p->ng) * (p->ny + 2 * p->ng) * (p->nz + 2 * p->ng);
  // scratch: scalars, three flux arrays [8][G] and the EMFs [3][G], all double
  const double need_bytes = (double)kScalarBytes + (3.0 * 8.0 + 3.0) * 8.0 * G;
  if (need_bytes > (double)kScratchBytes) {
    char msg[200];
    snprintf(msg, sizeof msg, "block of %.0f ghosted cells needs %.0f bytes of scratch, more than the %zu-byte maximum "
             "(at most %zu ghosted cells)", G, need_bytes, kScratchBytes, (kScratchBytes - kScalarBytes) / 216);
    return fail(GRMHD_E_INVALID, msg);
  }

  DevParams d = dev_params(p);

  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return fail(GRMHD_E_CUDA, cudaGetErrorString(e));
  char* sc = (char*)base;
  unsigned long long* ms = (unsigned long long*)sc;
  double* dt_dev = (double*)(ms + 3);
  unsigned long long* stats = ms + 8;
  d.fault = ms + 32;  // the bounds-check build's fault word (cleared below with the other scalars)
  double* F[3];
  for (int k = 0; k < 3; ++k) F[k] = (double*)(sc + kScalarBytes) + (size_t)k * 8 * d.gsize;
  double* E = (double*)(sc + kScalarBytes) + (size_t)24 * d.gsize;

  const cudaStream_t s = (cudaStream_t)stream;
  const FormLaunchers& L = fp64_launchers();
  const bool auto_dt = !(dt > 0.0);
  // as in grmhd_stage: the CFL step is taken on a first stage (g0 == 0); a later stage of the step with
  // dt <= 0 reuses the step the last first-stage call left in the array
  const bool track = auto_dt && g0 == 0.0;
  // the array keeps the previous call's contents: clear the reductions this call accumulates into
  e = cudaMemsetAsync(stats, 0, kScalarBytes - 8 * sizeof(unsigned long long), s);
  if (e == cudaSuccess && track) e = cudaMemsetAsync(ms, 0, 3 * sizeof(unsigned long long), s);
  if (e == cudaSuccess && p->bc == GRMHD_BC_PERIODIC) e = L.ghost(d, P, s);
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = L.flux(d, P, F[k], ms, k, track ? 1 : 0, s);
  if (e == cudaSuccess && track) e = launch_finalize_dt(ms, dt_dev, d, s);
  if (e == cudaSuccess) e = L.emf(d, F[0], F[1], F[2], E, s);
  if (e == cudaSuccess) {
    StageArgs a{};
    a.U0 = U0;
    a.Ucur = Ucur;
    a.Unew = Unew;
    a.status = status;
    a.dt_dev = dt_dev;
    a.stats = stats;
    a.g0 = g0;
    a.g1 = g1;
    a.beta = beta;
    a.dt = dt;
    a.use_dev_dt = auto_dt ? 1 : 0;
    a.worklist = nullptr;
    a.wl_count = nullptr;
    e = L.update(d, P, F[0], F[1], F[2], E, a, s);
  }
  if (e != cudaSuccess) return fail(GRMHD_E_CUDA, cudaGetErrorString(e));
  return GRMHD_OK;
}
