/* C ABI of the GB300 GRMHD stage library (libgrmhd.so).
 *
 * The library advances the Valencia-formulation GRMHD equations of Barker et al., "Phoebus:
 * Performance Portable GRRMHD for Relativistic Astrophysics" (arXiv:2410.09146) by one explicit
 * Runge-Kutta stage of the conservative finite-volume update on one logically Cartesian
 * meshblock with ghost zones:
 *   (sqrt(gamma) U)_t + (sqrt(-g) F^i)_i = sqrt(-g) S          Sec. 2.1, eq. (conservation law)
 * in the fixed order: reconstruction (PLM minmod / MC, WENO5-Z-AOAH; Sec. 3.1, App. B), LLF or
 * HLL Riemann fluxes (Sec. 3.1), Toth flux-CT of the cell-centred field (Sec. 3.1), flux
 * divergence plus geometric sources (Sec. 2.1 eq. (source vector)) with an analytic Minkowski or
 * Kerr-Schild metric (Sec. 2.3), and per-cell con2prim (Kastaun et al. 2021, Sec. 3.1) with
 * floors (Sec. 3.2) and an ideal-gas EOS (Sec. 2.2).
 *
 * Conventions shared by every entry point:
 *  - Return 0 on success, a negative GRMHD_E* code on error; grmhd_last_error() then holds a
 *    message. A con2prim failure in a cell is NOT a call error: it is reported per cell in the
 *    status array and summed in the statistics.
 *  - The library allocates no device memory. The caller passes one device workspace of at least
 *    grmhd_workspace_bytes() bytes (256-byte aligned) and a CUDA stream; both are borrowed for the
 *    lifetime of the context. All other pointers are borrowed for the call only.
 *  - Calls are asynchronous on the context's stream, except those that write host memory, which
 *    synchronise the stream before returning.
 *  - No global state besides a thread-local message buffer for failed grmhd_create calls: contexts
 *    are independent; one context must not be used from two threads at the same time.
 *  - Array layouts are C order with x fastest. Primitives P = (rho, W v^1, W v^2, W v^3, rho eps,
 *    B^1, B^2, B^3) (Sec. 2.1 eq. (primitive vector)) are [8][nz+2ng][ny+2ng][nx+2ng] including
 *    ghosts; conserved states U = sqrt(gamma) (D, S_1, S_2, S_3, tau, B^1, B^2, B^3)
 *    (Sec. 2.1 eq. (conserved vector), densitized) are [8][nz][ny][nx] over the interior.
 */
#ifndef GRMHD_H
#define GRMHD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define GRMHD_OK 0
#define GRMHD_E_INVALID (-1)     /* bad parameter, size or pointer */
#define GRMHD_E_CUDA (-2)        /* a CUDA call or kernel launch failed */
#define GRMHD_E_WORKSPACE (-3)   /* workspace too small or misaligned */
#define GRMHD_E_UNSUPPORTED (-4) /* option combination not built */

/* options */
#define GRMHD_MINKOWSKI 0     /* flat space, optionally with a constant shift (params.shift) */
#define GRMHD_KERR_SCHILD 1 /* Cartesian Kerr-Schild, spin a = spin * mass along z */
/* Kerr-Schild in spherical coordinates (x^1, x^2, x^3) = (ln r, theta, phi) (Sec. 2.3; the coordinates of the
 * paper's accretion set-ups, Sec. 3.2): r and the angles of the Cartesian form through x + i y = (r + i a)
 * e^{i phi} sin(theta), z = r cos(theta). Single-block contexts (both forms), flux-CT, no passive scalar;
 * GRMHD_BC_FIXED or GRMHD_BC_SPHERICAL. Theta faces on the polar axis carry no flux, sin(theta) times the phi
 * components of W v and B is reconstructed, and on the axis the EMF along phi is zero and the EMF along r is
 * its mean over phi. mass >= 0 (0: flat space in spherical coordinates). */
#define GRMHD_KERR_SCHILD_SPHERICAL 2

#define GRMHD_RECON_CONSTANT 0
#define GRMHD_RECON_PLM_MINMOD 1
#define GRMHD_RECON_PLM_MC 2
#define GRMHD_RECON_WENO5Z_AOAH 3
#define GRMHD_RECON_MP5 4        /* Suresh & Huynh's monotonicity-preserving fifth order (Sec. 3.1) */

#define GRMHD_RIEMANN_LLF 0
#define GRMHD_RIEMANN_HLL 1

#define GRMHD_BC_PERIODIC 0     /* ghosts refilled from the interior at the start of every stage */
#define GRMHD_BC_FIXED 1        /* ghosts keep the values given to grmhd_set_prims */
/* GRMHD_KERR_SCHILD_SPHERICAL over theta in [0, pi] and phi in [0, 2 pi) with nz even: phi periodic, a ghost
 * beyond a pole the cell mirrored across it and turned by pi in phi (the theta components of W v and B
 * negated), refilled at the start of every stage; the radial ghosts keep their given values. */
#define GRMHD_BC_SPHERICAL 2

#define GRMHD_FP64 0            /* every step in double precision */
#define GRMHD_MIXED 1           /* reconstruction, fluxes, EMFs and sources in float; P stored in float;
                                   state accumulation and con2prim in double */

/* constrained transport of the magnetic field */
#define GRMHD_CT_FLUX 0         /* Toth flux-CT of the cell-centred field (Sec. 3.1) */
#define GRMHD_CT_FACE 1         /* face-centred field, upwind edge EMFs (Sec. 5 names face-centred CT as
                                   planned work; scheme: the "contact" CT of Gardiner & Stone 2005) */

#define GRMHD_HOST 0
#define GRMHD_DEVICE 1

/* what grmhd_get returns */
#define GRMHD_GET_PRIMS 0       /* double [8][nz+2ng][ny+2ng][nx+2ng] */
#define GRMHD_GET_CONS 1        /* double [8][nz][ny][nx], the current state */
#define GRMHD_GET_STATUS 2      /* uint8 [nz][ny][nx], last stage's con2prim/floor bits (GRMHD_ST_*) */
#define GRMHD_GET_STATS 3       /* uint64 [8] of the last stage (or batch): con2prim iterations, cells with
                                   rho floor, eps floor, W cap, not converged, bad input, max iterations
                                   of a cell, cells the mixed form's float con2prim phase handed to the
                                   double iteration */
#define GRMHD_GET_DT 4          /* double [1]: the time step of the last first stage (CFL rule) */
#define GRMHD_GET_FACE_B 5      /* double [3][nz+2ng][ny+2ng][nx+2ng]: the current face field (GRMHD_CT_FACE) */
#define GRMHD_GET_SCALAR 6      /* double [nz+2ng][ny+2ng][nx+2ng]: the passive scalar X (params.scalar) */
#define GRMHD_GET_SCALAR_CONS 7 /* double [nz][ny][nx]: its conserved sqrt(gamma) D X, the current state */
#define GRMHD_GET_PRIMS_F32 8   /* float [8][nz+2ng][ny+2ng][nx+2ng]: the primitives as the mixed form stores them
                                   (GRMHD_MIXED contexts only) */

/* per-cell status bits */
#define GRMHD_ST_RHO_FLOOR 1
#define GRMHD_ST_EPS_FLOOR 2
#define GRMHD_ST_W_CAP 4
#define GRMHD_ST_NOT_CONVERGED 8
#define GRMHD_ST_BAD_INPUT 16

typedef struct grmhd_ctx grmhd_ctx;

typedef struct {
  int nx, ny, nz, ng;         /* interior cells per direction (0,0,0 for a con2prim-only context); ghosts */
  double x0[3];               /* coordinate of the interior's lower corner */
  double dx[3];               /* cell widths */
  int metric;                 /* GRMHD_MINKOWSKI | GRMHD_KERR_SCHILD | GRMHD_KERR_SCHILD_SPHERICAL (Sec. 2.3) */
  double spin, mass;          /* Kerr-Schild a/M and M */
  double gamma_eos;           /* ideal-gas index, P = (gamma_eos - 1) rho eps (Sec. 2.2) */
  int recon, riemann, precision, bc;
  double rho_floor0;          /* rho >= rho_floor0 r^-floor_r_exp (Kerr-Schild r) or rho_floor0 (Sec. 3.2) */
  double eps_floor0;          /* rho eps >= rho eps_floor0 r^-floor_r_exp */
  double floor_r_exp;
  double w_max;               /* Lorentz-factor ceiling */
  double c2p_tol;             /* relative tolerance of the con2prim root in mu = 1/(h W) */
  int c2p_max_iter;           /* iteration cap of the root solve */
  double cfl;                 /* dt = cfl / max_d(max |lambda_d| / dx_d) when the stage picks dt */
  double weno_eps;            /* epsilon of the WENO5-Z weights (App. B eq. (nonlinear weights)) */
  int ct;                     /* GRMHD_CT_FLUX | GRMHD_CT_FACE (single-block contexts only) */
  double shift[3];            /* GRMHD_MINKOWSKI only: constant shift beta^i, i.e. flat space in coordinates moving
                                 at velocity -beta (Sec. 4.1.1's boosted linear waves; |beta| < 1); ignored by
                                 Kerr-Schild */
  int scalar;                 /* 1: also evolve one passive scalar X, e.g. the electron fraction (Sec. 2.1,
                                 (X rho u^mu)_{;mu} = 0; see grmhd_set_scalar); single-block contexts, batches,
                                 lattices and two-level meshes, with flux-CT and ng >= 3 */
} grmhd_params;

/* Bytes of device workspace a context with these parameters needs (0 on invalid parameters). */
size_t grmhd_workspace_bytes(const grmhd_params* p);

/* The primitives in single precision, for the mixed form (which stores P in float): P is float
 * [8][nz+2ng][ny+2ng][nx+2ng], host or device (where), read during the call, copied into the context's P
 * without conversion; otherwise as grmhd_set_prims (U formed, a previous scalar or face field discarded).
 * The same state as grmhd_set_prims with these values in double (its load rounds to float), at half the
 * bytes. A host P is copied in slabs of z rows whose prim->cons overlaps the next slab's copy (on a stream the
 * context creates on its first host load and destroys with the context); the call returns once P has been
 * read, and later work on the context's stream waits for the prim->cons. Errors: GRMHD_E_INVALID (an
 * all-FP64 or batch context, P NULL, bad where), GRMHD_E_CUDA. */
int grmhd_set_prims_f32(grmhd_ctx* c, const float* P, int where);

/* Passive scalar (params.scalar = 1; Sec. 2.1: Phoebus evolves passive scalars X, the electron fraction
 * among them, by (X rho u^mu)_{;mu} = S; here S = 0, no radiation). Set X after grmhd_set_prims or
 * grmhd_set_cons (each discards a previous scalar): X is double [nz+2ng][ny+2ng][nx+2ng] (ghosts as for P: read when the
 * boundary is fixed, filled periodically otherwise), host or device (where), read during the call;
 * the conserved sqrt(gamma) D X of the interior is formed from the current state. Every stage then also
 * advances it: the face flux of sqrt(gamma) D X is the stage's face mass flux times X reconstructed (with
 * the stage's reconstruction) on the upwind side of that flux, the update takes the stage's RK weights,
 * and X = (sqrt(gamma) D X) / (sqrt(gamma) D) with the stage's final D (so a density floor dilutes X while
 * sqrt(gamma) D X stays conserved). Both forms: X stored like P, D X in double.
 * Errors: GRMHD_E_INVALID (no scalar in the params, no state yet, X NULL, bad where), GRMHD_E_CUDA. */
int grmhd_set_scalar(grmhd_ctx* c, const double* X, int where);

/* Create a context on the current CUDA device. `workspace` is a device pointer to at least
 * grmhd_workspace_bytes(p) bytes, 256-byte aligned (may be NULL when that is 0); `stream` is a
 * cudaStream_t (NULL = default stream). Both stay owned by the caller and must outlive the context.
 * Errors: GRMHD_E_INVALID (bad parameters), GRMHD_E_WORKSPACE, GRMHD_E_UNSUPPORTED. */
int grmhd_create(const grmhd_params* p, void* workspace, size_t bytes, void* stream, grmhd_ctx** out);

/* Load primitives P (double, [8][nz+2ng][ny+2ng][nx+2ng] including ghosts; `where` = GRMHD_HOST or
 * GRMHD_DEVICE) and derive the conserved state of the interior (Sec. 2.1 eq. (conserved vector)).
 * A host P is read before the call returns; a device P must stay unchanged until the stream has run
 * the load. Resets the Runge-Kutta slot bookkeeping. */
int grmhd_set_prims(grmhd_ctx* c, const double* P, int where);

/* Overwrite the current conserved state with U (double [8][nz][ny][nx]) without touching P; used
 * with grmhd_set_prims to restore a checkpoint taken with grmhd_get. */
int grmhd_set_cons(grmhd_ctx* c, const double* U, int where);

/* Face-centred CT (p->ct == GRMHD_CT_FACE): load the face field Bf (double [3][nz+2ng][ny+2ng][nx+2ng],
 * `where` = GRMHD_HOST or GRMHD_DEVICE): entry (i,j,k) of component d is sqrt(gamma) B^d on the lower
 * d-face of ghosted cell (i,j,k), i.e. the densitized field whose face divergence
 * sum_d (Bf_d(upper) - Bf_d(lower)) / dx_d the stage keeps. Call after grmhd_set_prims: the faces replace
 * the cell field of P (B^d = mean of the two d-faces / sqrt(gamma) at the cell centre, for every cell
 * whose two d-faces are stored: all but the last ghost layer along d; periodic blocks get their ghost
 * faces filled first) and the conserved state is derived again. Fixed ghost faces keep these values.
 * In this mode the stage advances the faces by the discrete Stokes theorem on upwind edge EMFs and
 * the cell field is the mean of its faces; the B components of U0 / Ucur are not read.
 * Errors: GRMHD_E_INVALID (no grid, not a face-CT context, bad `where`), GRMHD_E_CUDA. */
int grmhd_set_face_b(grmhd_ctx* c, const double* Bf, int where);

/* One Runge-Kutta stage (a0..a6 of the stage; Sec. 3.1):
 *   Unew = g0 U0 + g1 Ucur + beta dt L(Ucur)
 * where U0 is the state at the start of the step (the input of the last stage with g0 == 0) and
 * L = -sum_d dF^d/dx^d + sqrt(-g) S with CT fluxes for B; then con2prim + floors update P.
 * A stage with g0 == 0 starts a new step. dt > 0 is used as given; dt <= 0 takes the CFL time step,
 * computed on the device from this stage's face speeds when g0 == 0 and reused by later stages of
 * the step. Asynchronous. Errors: GRMHD_E_INVALID, GRMHD_E_CUDA. */
int grmhd_stage(grmhd_ctx* c, double g0, double g1, double beta, double dt);

/* One SSP-RK2 (Heun) step: stages (0, 1, 1) and (1/2, 1/2, 1/2) with the same dt (dt <= 0: CFL). */
int grmhd_rk2_step(grmhd_ctx* c, double dt);

/* One stage from host primitives to host primitives, for single-block GRMHD_MIXED contexts (float primitives,
 * the layout of grmhd_set_prims_f32: float [8][nz+2ng][ny+2ng][nx+2ng], host memory, page-locked for the
 * copies to overlap). Equivalent to
 *   grmhd_set_prims_f32(c, P_in, GRMHD_HOST)                  (skipped when P_in is NULL)
 *   grmhd_stage(c, g0, g1, beta, dt)
 *   grmhd_get(c, GRMHD_GET_PRIMS_F32, P_out, GRMHD_HOST)      (skipped when P_out is NULL)
 * with the same results bit for bit, but the copies overlap the device work: the load's copies run beside its
 * prim -> cons (as in grmhd_set_prims_f32), whose last part runs beside the stage's ghost fill and fluxes
 * (which read only P; the update waits for it), and the update and its passes over deferred cells run in 8
 * slabs of interior z rows, each slab's ghosted rows of P copied to P_out while the next slab is updated.
 * P_in is read and P_out written when the call returns, also when it fails. P_in given: the
 * stage starts a step (g0 == 0) and, for face-centred CT, needs grmhd_set_face_b, as after any load; P_in
 * NULL: the stage continues from the context's state (e.g. the second stage of an RK2 step). Returns when
 * P_out holds the stage's primitives (the device work that follows them, a passive scalar's update, may still
 * run). The caller owns both buffers; P_out must not overlap P_in. With timing on, the slabs' updates and
 * passes are counted together in the update group. Errors: GRMHD_E_INVALID (no single-block grid, not a
 * GRMHD_MIXED context, the errors of the three calls above), GRMHD_E_CUDA. */
int grmhd_stage_host_f32(grmhd_ctx* c, const float* P_in, float* P_out, double g0, double g1, double beta,
                         double dt);

/* Con2prim of a flat-space batch (a6 on its own; Sec. 3.1, the Kastaun et al. solve, and the Sec. 3.2
 * floors in their Minkowski form): U and P are device arrays [8][n] (structure of arrays) of densitized
 * conserved / primitive variables; status (uint8 [n]) and iters (int [n]) may be NULL. flags bit 0: P holds
 * a warm-start guess on entry. Uses the context's gamma_eos, floors, tolerance and stream. Asynchronous.
 * Two narrowings of the general interface, both deliberate: the states are given in the local orthonormal
 * frame (any metric reduces to it point by point, which is how the stage itself calls the same solve with
 * its cell's metric), and the arrays are device memory only (a caller with host arrays copies them with one
 * cudaMemcpyAsync each; the library allocates no staging buffer). Errors: GRMHD_E_INVALID, GRMHD_E_CUDA. */
int grmhd_c2p(grmhd_ctx* c, long long n, const double* U, double* P, uint8_t* status, int* iters, int flags);

/* Prim->cons of a flat-space batch (Sec. 2.1 eq. (conserved vector) with the Minkowski metric): P and U
 * are device arrays [8][n] (structure of arrays), the layouts of grmhd_c2p; uses the context's gamma_eos
 * and stream. Asynchronous. Errors: GRMHD_E_INVALID, GRMHD_E_CUDA. */
int grmhd_p2c(grmhd_ctx* c, long long n, const double* P, double* U);

/* ---- Learned initial guess for con2prim -------------------------------------------------------
 * The paper's con2prim (Sec. 3.1: the Kastaun et al. 2021 master function f(mu), root mu = 1/(h W) in
 * the bracket (0, mu_+]) starts its iteration from a fixed point of the bracket. These entry points
 * add a small network that predicts where the root lies: an 8 -> 64 -> 64 -> 64 -> 2 multilayer
 * perceptron with SiLU activations, BF16 weights and FP32 arithmetic, trained on the GPU by the
 * library's own forward, backward and Adam kernels. The paper has no counterpart.
 *
 * Network: raw features x = (log1p(q), log1p(r^2)/2, log1p(b^2)/2, log1p((r.b)^2)/4, r/(1+q), b^2/(1+q),
 * ln(max(eps_+, 1e-30))/10, ln W_+) of the invariants q = tau/D (clamped at 0), r^2 = S^2/D^2,
 * b^2 = B^2/D, (r.b)^2 and of eps_+, W_+ (the master-function intermediates at mu_+), standardised
 * (x - mean_x) * invstd_x; outputs o de-standardised y = o * std_y + mean_y with
 *   y0 = -ln(1 - mu/mu_+)  (clipped to [0, 30]),   y1 = ln W at the root (auxiliary).
 * The guess is mu_0 = mu_+ (1 - e^{-y0}); the safeguarded Newton iteration keeps its full bracket, so a
 * poor guess costs iterations, never the root.
 * Parameters theta (float [GRMHD_MLP_NPARAM]): W1 [64][8], b1 [64], W2 [64][64], b2 [64], W3 [64][64],
 * b3 [64], W4 [2][64], b4 [2], row-major [out][in]. Standardisation norm (float [GRMHD_MLP_NNORM]):
 * mean_x [8], invstd_x [8], mean_y [2], std_y [2].
 * Loss of a batch of n samples (X raw features [n][8], T raw targets [n][2], device float):
 *   L = (1/n) sum_s [(o0 - t0)^2 + aux (o1 - t1)^2],  t = (T - mean_y) / std_y.
 * Every forward pass, in training too, uses the BF16 copy of the weights; gradients are taken with
 * respect to that copy and applied to FP32 master weights by Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 * State: one device workspace of grmhd_mlp_workspace_bytes() bytes, 256-byte aligned, owned by the
 * caller (master weights, Adam moments, gradient, standardisation, BF16 weights). Functions without a
 * context report errors through grmhd_last_error(NULL) (thread-local). */
#define GRMHD_MLP_NPARAM 9026
#define GRMHD_MLP_NNORM 20

size_t grmhd_mlp_workspace_bytes(void);

/* Load theta and norm (host float arrays) into the workspace, clear the Adam state and the gradient,
 * and make the BF16 copy. Synchronises `stream`. Errors: GRMHD_E_INVALID, GRMHD_E_WORKSPACE (alignment),
 * GRMHD_E_CUDA. */
int grmhd_mlp_set_weights(void* ws, const float* theta, const float* norm, void* stream);

/* Copy the FP32 master weights to theta (host) and, when theta_bf16 is not NULL, the BF16 weights used
 * by the forward pass (as float) to theta_bf16. Synchronises `stream`. */
int grmhd_mlp_get_weights(const void* ws, float* theta, float* theta_bf16, void* stream);

/* Network outputs Y [n][2] (device float, raw units) for raw features X [n][8] (device float).
 * Asynchronous. */
int grmhd_mlp_forward(const void* ws, long long n, const float* X, float* Y, void* stream);

/* Loss and gradient of one batch (n >= 1): the gradient accumulates in the workspace (cleared first) and
 * is copied to grad (host float [GRMHD_MLP_NPARAM]) and the loss to *loss when those are not NULL; the
 * call synchronises `stream`. Computed in FP32 on the CUDA cores. */
int grmhd_mlp_grad(void* ws, long long n, const float* X, const float* T, double aux, float* grad, float* loss,
                   void* stream);

/* The same on the fifth-generation tensor cores (the training form of the learned guess, the paper has no
 * network): per tile of 128 samples the two 64 x 64 layers forward, the two products that carry the deltas
 * back through them and (accumulated over tiles) their weight and bias gradients are tcgen05 MMAs of BF16
 * operands with FP32 accumulation; the back-propagated deltas of layers 3 and 2 are rounded to BF16 where
 * they enter a product, the first and output layers and their gradients stay FP32. Errors: as
 * grmhd_mlp_grad, and GRMHD_E_CUDA when a tensor-core completion was not observed within the kernel's
 * wait limit (the gradient is then incomplete). */
int grmhd_mlp_grad_tc(void* ws, long long n, const float* X, const float* T, double aux, float* grad, float* loss,
                      void* stream);

/* One Adam update with the gradient held in the workspace (step counts from 1; learning rate lr);
 * refreshes the BF16 copy and clears the gradient. Asynchronous. */
int grmhd_mlp_adam(void* ws, double lr, int step, void* stream);

/* `steps` Adam steps over contiguous minibatches of `batch` samples of (X, T) (n samples, i.i.d.
 * order assumed; the window wraps to the start when it would pass the end), learning rate decaying
 * from lr to lr_end on a cosine; Adam's step count starts at first_step (>= 1). loss_dev (device
 * float [steps], or NULL) receives the loss of each minibatch. Asynchronous. */
int grmhd_mlp_train(void* ws, long long n, const float* X, const float* T, long long batch, int steps, double lr,
                    double lr_end, double aux, int first_step, float* loss_dev, void* stream);

/* grmhd_mlp_train with the tensor-core gradient of grmhd_mlp_grad_tc. Asynchronous; a tensor-core wait that
 * timed out is counted in the workspace and reported by the next grmhd_mlp_grad / grmhd_mlp_grad_tc. */
int grmhd_mlp_train_tc(void* ws, long long n, const float* X, const float* T, long long batch, int steps, double lr,
                       double lr_end, double aux, int first_step, float* loss_dev, void* stream);

/* Flat-space con2prim batch like grmhd_c2p (same U, P, status, iters layouts; the context's gamma_eos,
 * floors, tolerance and stream) with the initial guess chosen by mlp_ws and flags:
 *   mlp_ws == NULL: the standard start mu_+/2 (guess ignored);
 *   mlp_ws != NULL: the network's start mu_0 = mu_+ (1 - e^{-y0}). The solve runs at most 8 Newton
 *                   iterations from mu_0; if they do not converge (or mu_0 is not inside (0, mu_+)) it
 *                   falls back to the standard start with the full iteration budget. Network, flags 0:
 *                   one fused kernel per tile of 128 states, the two 64 x 64 layers as tcgen05 MMAs
 *                   (BF16 operands in shared memory, FP32 accumulators in tensor memory); guess (device
 *                   double [2][n], may be NULL) receives (mu_0, mu_+). flags GRMHD_GUESS_FP32: the
 *                   network on the FP32 cores in a separate kernel that writes guess (then required),
 *                   then the solve.
 * X (device float [n][8]) and T (device float [n][2]), when not NULL, receive the raw features and the
 * targets (y0, ln W) of the solved root: training pairs from the library's own FP64 solve (standard
 * start or GRMHD_GUESS_FP32 only; GRMHD_E_INVALID otherwise).
 * GRMHD_GET_STATS then holds [0] iterations (master-function evaluations, all attempts), [4] states not
 * converged, [6] tiles of the fused kernel abandoned because an MMA completion was not observed within
 * its wait limit (0 in normal operation; the states of such tiles are not written) and [7] fallbacks
 * to the standard start. Asynchronous. Errors: GRMHD_E_INVALID, GRMHD_E_WORKSPACE, GRMHD_E_CUDA. */
#define GRMHD_GUESS_FP32 1
int grmhd_c2p_guess(grmhd_ctx* c, const void* mlp_ws, long long n, const double* U, double* P, uint8_t* status,
                    int* iters, double* guess, float* X, float* T, int flags);

/* Copy `what` (GRMHD_GET_*) to dst (`where` = GRMHD_HOST synchronises the stream). */
int grmhd_get(grmhd_ctx* c, int what, void* dst, int where);

/* Per-kernel timing (tracing aid, off by default): with `on` != 0 every later stage records CUDA events
 * on the context's stream around its kernel groups. Creating the events is the only host-side cost;
 * the records are asynchronous. */
int grmhd_set_timing(grmhd_ctx* c, int on);

/* Accumulated device milliseconds per kernel group since the last call, ms[7] = ghost fill, flux x,
 * flux y, flux z (each including its share of the CFL reduction), EMF, update (divergence + sources +
 * RK + con2prim + floors), cell passes (re-derived hydro state of floored cells; the mixed form's
 * double con2prim of cells whose float phase did not settle), and the number of stages they cover;
 * resets the totals. Synchronises on the last recorded event. */
int grmhd_get_timing(grmhd_ctx* c, double* ms, int* stages);

/* Bounds-check build (compiled with -DGRMHD_BOUNDS_CHECK; a testing aid, the paper has no counterpart): the
 * stage kernels compare every global-memory index with its array's extent; the first out-of-range access of
 * a context's stages is recorded and skipped (loads read 0) and nothing traps. out[0] = 0 when no access was
 * out of range, else (source line << 48 | sign << 47 | |index|) + 1 of the first one; out[1] = 1 when the
 * library was built with the checks (0: out[0] is always 0). Synchronises the context's stream.
 * Errors: GRMHD_E_INVALID (NULL), GRMHD_E_CUDA. */
int grmhd_bounds_fault(grmhd_ctx* c, unsigned long long out[2]);

/* The a7 helper (CFL rule; the paper does not state one): out[d] = the largest characteristic speed |lambda+-|
 * over the interior faces of direction d, from the last stage of this single-block context that took its
 * time step from the face speeds (a first stage, g0 == 0, with dt <= 0); dt = cfl / max_d(out[d] / dx[d]) is
 * the step GRMHD_GET_DT returns. Zero before such a stage. Synchronises the context's stream.
 * Errors: GRMHD_E_INVALID (NULL, or a batch / con2prim-only context), GRMHD_E_CUDA. */
int grmhd_max_speed(grmhd_ctx* c, double out[3]);

/* Roofline denominators of the ALU-bound kernels (measurement aid; the paper has no counterpart): the dense
 * fused multiply-add rates of the current device in TFLOP/s (2 flops per FMA), FP64 and FP32, each timed
 * with CUDA events on `stream` over one launch of eight independent FMA chains per thread on every SM
 * (about 40 ms and 10 ms on a GB300). The double-precision update and con2prim of the stage are bound by
 * the FP64 pipe on GB300, whose FP64 rate is about 1/74 of its FP32 rate. `sink` is a caller-owned device
 * buffer of at least 8 bytes that the kernels may write (they do not in practice); blocks the calling
 * thread until the measurement ends. Errors: GRMHD_E_INVALID (a NULL pointer), GRMHD_E_CUDA. */
int grmhd_fp_peaks(double* sink, void* stream, double* fp64_tflops, double* fp32_tflops);

/* One all-FP64 Runge-Kutta stage, like grmhd_stage, for callers that cannot allocate device memory
 * (code inside a CUDA-graph capture, hosts whose framework owns every device allocation, embedded
 * hosts without a device allocator). The paper has no counterpart: this is a packaging of the same
 * stage. No context and no workspace: the caller passes the state, all device pointers --
 *   P      double [8][nz+2ng][ny+2ng][nx+2ng], primitives in; interior (and periodic ghosts) out
 *   U0     double [8][nz][ny][nx], state at the start of the step (read only when g0 != 0)
 *   Ucur   double [8][nz][ny][nx], the stage's input state
 *   Unew   double [8][nz][ny][nx], the stage's output state (may not alias Ucur or U0)
 *   status uint8  [nz][ny][nx]
 * -- and the coefficients of Unew = g0 U0 + g1 Ucur + beta dt L(Ucur). dt <= 0 on a first stage (g0 == 0)
 * takes the CFL step of this call's face speeds; dt <= 0 on a later stage (g0 != 0) reuses the step that
 * the last first-stage call on this device left in the shared array, as grmhd_stage reuses its first
 * stage's (a two-call RK2 step with dt <= 0 on both calls advances like grmhd_rk2_step, provided no
 * other call runs in between). p is checked as by grmhd_create (GRMHD_E_INVALID with the reason in
 * grmhd_last_error(NULL)); p->precision must be GRMHD_FP64 and p->ct GRMHD_CT_FLUX, without a scalar.
 * Scratch (face fluxes, edge EMFs, speed and time-step scalars) lives in a 16 MiB array of device
 * memory built into the library (every GPU that loads the library holds it until the process exits),
 * which bounds the block to floor((16 MiB - 512 B) / 216 B) = 77,669 ghosted cells, e.g. 34^3 interior cells
 * with 4 ghosts; larger blocks are rejected with GRMHD_E_INVALID and a message in
 * grmhd_last_error(NULL). The first call on each device looks up the array's device address; make
 * that first call before any stream capture. Every call shares the array and the array keeps the
 * previous call's contents (the call clears what it accumulates into): calls that overlap on the GPU,
 * on one stream or several, race on it. Asynchronous on `stream` (a cudaStream_t, NULL = default).
 * Errors: GRMHD_E_INVALID, GRMHD_E_CUDA. */
int grmhd_stage_noalloc(const grmhd_params* p, double* P, const double* U0, const double* Ucur, double* Unew,
                        uint8_t* status, double g0, double g1, double beta, double dt, void* stream);

/* ---- Batches of meshblocks (many uneven blocks advanced together) ----
 * A batch holds nblocks independent meshblocks that share the physics options of `p` (its nx..nz,
 * x0, dx fields are ignored; each block brings its own). Ghost zones are taken as given
 * (p->bc must be GRMHD_BC_FIXED), unless grmhd_batch_set_lattice declares the blocks a lattice, whose
 * ghosts are then exchanged on the device at the start of every stage. grmhd_stage and
 * grmhd_rk2_step advance every block: each phase (fluxes of all directions, EMFs, cell update, deferred
 * con2prim) is one persistent launch whose CTAs take fixed-size work items (`tile` faces, edges or
 * cells of one block) from a device counter. With dt <= 0 the CFL step is the minimum over the batch. */
typedef struct {
  int nx, ny, nz;  /* interior cells */
  double x0[3];    /* coordinate of the block's interior lower corner */
  double dx[3];    /* cell widths */
} grmhd_block;

/* Workspace bytes of a batch (0 on invalid input). */
size_t grmhd_batch_workspace_bytes(const grmhd_params* p, int nblocks, const grmhd_block* blocks);

/* Create a batch context (workspace and stream borrowed as for grmhd_create); the tile starts at 512.
 * Errors: GRMHD_E_INVALID, GRMHD_E_WORKSPACE, GRMHD_E_UNSUPPORTED (periodic blocks, face-centred CT),
 * GRMHD_E_CUDA. */
int grmhd_batch_create(const grmhd_params* p, int nblocks, const grmhd_block* blocks, void* workspace, size_t bytes,
                       void* stream, grmhd_ctx** out);

/* Declare that the batch's blocks tile an nbx x nby x nbz lattice of one meshblock grid: block b sits at
 * lattice position (b % nbx, (b / nbx) % nby, b / (nbx nby)); all blocks have the same cell counts and
 * widths and block b's interior corner is block 0's plus its lattice position times the block size.
 * Every later stage then starts with a same-level ghost exchange on the device: each ghost cell of each
 * block takes the primitives of the cell with the same global index in the block that owns it (across
 * the lattice edge: wrapped when `periodic`, else kept as loaded -- a fixed outer boundary). The result
 * is the stage of the one large block the lattice tiles. (0, 0, 0) switches the exchange off.
 * Errors: GRMHD_E_INVALID (not a batch, block count, sizes, widths or corners off the lattice). */
int grmhd_batch_set_lattice(grmhd_ctx* c, int nbx, int nby, int nbz, int periodic);

/* Passive scalar of block `block` of a batch created with params.scalar = 1 (as grmhd_set_scalar: X double
 * [gz][gy][gx] of that block, ghosts included, host or device, read during the call; the block's
 * sqrt(gamma) D X formed from its current state; grmhd_batch_set_prims of the block discards it). Every
 * block needs one before a stage; the stage then advances each block's scalar as grmhd_stage does, and
 * a lattice exchange (grmhd_batch_set_lattice) copies X's ghosts with P's; a two-level mesh
 * (grmhd_batch_set_mesh) exchanges X like a primitive and refluxes sqrt(gamma) D X with the scalar's face
 * fluxes after its update (then X = DX / D with the refluxed D). Read back per block with
 * grmhd_batch_get(GRMHD_GET_SCALAR / GRMHD_GET_SCALAR_CONS).
 * Errors: GRMHD_E_INVALID (not a batch, bad block, no scalar in the params, no state yet), GRMHD_E_CUDA. */
int grmhd_batch_set_scalar(grmhd_ctx* c, int block, const double* X, int where);

/* Declare that the batch's blocks are the leaves of a two-level block mesh over an nbx x nby x nbz grid of
 * root blocks (the meshblock AMR the method runs on, Sec. 3; one time step for both levels). level[b] is 0
 * for a root block and 1 for one of the 8 children of a refined root block (half the cell width);
 * pos[3b..3b+2] is block b's position in its level's block lattice (0 <= pos < nb, or < 2 nb on level 1).
 * All blocks have the same cell counts, each even and >= 4; block 0 fixes the level-0 cell width and the
 * mesh corner; every block's width and interior corner must follow its level and position, and the
 * leaves must tile the mesh once. Both arrays are read during the call only (host memory).
 * Every later stage then:
 *  - starts with a two-pass ghost exchange of the primitives: a ghost over a leaf of its own level copies
 *    that leaf's cell; a coarse ghost over a fine leaf takes the mean of the 8 fine cells under it; then a
 *    fine ghost over a coarse leaf takes the coarse cell plus, per direction, the minmod-limited slope
 *    (of the coarse cell and its two neighbours) times +-1/4 (prolongation). Outside the mesh the
 *    coordinates wrap when `periodic`; otherwise those ghosts keep their loaded values;
 *  - ends by refluxing every coarse cell with a face on a fine leaf: that face's flux (for B the flux-CT
 *    face flux from the edge EMFs) is replaced by the mean of the 4 fine face fluxes covering it,
 *    U += beta dt s (F_coarse - F_fine) / dx (s = +1 on the cell's upper face, -1 on its lower), and the
 *    cell takes con2prim (the double solver in both forms), floors and the re-derived hydro state again.
 * The mesh then conserves every variable to roundoff when periodic (floors aside). A passive scalar
 * (params.scalar) is exchanged and refluxed the same way (see grmhd_batch_set_scalar). (0, 0, 0) switches the
 * mesh off; declaring a lattice (grmhd_batch_set_lattice) replaces it and vice versa.
 * Errors: GRMHD_E_INVALID (not a batch, bad arguments, sizes, levels, widths, corners, overlapping or
 * missing leaves), GRMHD_E_CUDA (upload). */
int grmhd_batch_set_mesh(grmhd_ctx* c, int nbx, int nby, int nbz, int periodic, const int* level, const int* pos);

/* Load one block's primitives (double, [8][nz+2ng][ny+2ng][nx+2ng]) and derive its conserved state;
 * every block must be loaded before the first stage. */
int grmhd_batch_set_prims(grmhd_ctx* c, int block, const double* P, int where);

/* grmhd_get for one block (PRIMS, CONS, STATUS); STATS and DT are batch-wide. */
int grmhd_batch_get(grmhd_ctx* c, int block, int what, void* dst, int where);

/* Work-item size in faces / edges / cells (128 .. 2^20); results do not depend on it. */
int grmhd_batch_set_tile(grmhd_ctx* c, int tile);

/* Time tiles 128 .. 4096 with one real RK2 step each (the batch advances by 6 steps with the CFL time
 * step) and keep the fastest; returns it and its milliseconds per stage (either pointer may be NULL). */
int grmhd_batch_autotune(grmhd_ctx* c, int* best_tile, double* best_ms);

/* The timing table of the last grmhd_batch_autotune of this batch: *n candidates (0 before any), the first
 * min(*n, cap) written to tiles[] (work-item size) and ms[] (device milliseconds per stage, CUDA events on the
 * batch's stream). The tile the autotuner kept is the one with the smallest ms. Errors: GRMHD_E_INVALID. */
int grmhd_batch_autotune_table(grmhd_ctx* c, int* tiles, double* ms, int cap, int* n);

/* Batch contexts only: with `on` != 0 each distinct stage (coefficients, dt, state slots, tile) is
 * captured once into a CUDA graph on a library-owned capture stream and replayed on the context's
 * stream afterwards. Timing events are not recorded in graph mode. */
int grmhd_set_graph(grmhd_ctx* c, int on);

/* Last error message of the context (or of the last failed grmhd_create when c is NULL). */
const char* grmhd_last_error(const grmhd_ctx* c);

/* Release the context (the workspace and stream stay with the caller). */
void grmhd_destroy(grmhd_ctx* c);

#ifdef __cplusplus
}
#endif

#endif /* GRMHD_H */
