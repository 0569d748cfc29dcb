"""Python binding of libgrmhd.so: argument marshalling only, same names as the C ABI (include/grmhd.h).

Every step of the stage runs in the library's CUDA kernels; PyTorch only supplies the device
workspace and the stream. There is no CPU fallback: if the library is missing or cannot be loaded,
every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgrmhd.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "grmhd.h")

GRMHD_OK, GRMHD_E_INVALID, GRMHD_E_CUDA, GRMHD_E_WORKSPACE, GRMHD_E_UNSUPPORTED = 0, -1, -2, -3, -4
GRMHD_HOST, GRMHD_DEVICE = 0, 1
GRMHD_GET_PRIMS, GRMHD_GET_CONS, GRMHD_GET_STATUS, GRMHD_GET_STATS, GRMHD_GET_DT = 0, 1, 2, 3, 4
GRMHD_GET_FACE_B = 5
GRMHD_GET_SCALAR = 6
GRMHD_GET_SCALAR_CONS = 7
GRMHD_GET_PRIMS_F32 = 8
RECON = {"constant": 0, "plm_minmod": 1, "plm_mc": 2, "weno5z_aoah": 3, "mp5": 4}
RIEMANN = {"llf": 0, "hll": 1}
METRIC = {"minkowski": 0, "kerr_schild": 1, "kerr_schild_spherical": 2}
BC = {"periodic": 0, "fixed": 1, "spherical": 2}
PRECISION = {"fp64": 0, "mixed": 1}
CT = {"flux": 0, "face": 1}
ST_RHO_FLOOR, ST_EPS_FLOOR, ST_W_CAP, ST_NOT_CONVERGED, ST_BAD_INPUT = 1, 2, 4, 8, 16
GRMHD_MLP_NPARAM, GRMHD_MLP_NNORM = 9026, 20
GRMHD_GUESS_FP32 = 1


class GrmhdError(RuntimeError):
    pass


class grmhd_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("ng", ctypes.c_int),
        ("x0", ctypes.c_double * 3), ("dx", ctypes.c_double * 3),
        ("metric", ctypes.c_int), ("spin", ctypes.c_double), ("mass", ctypes.c_double),
        ("gamma_eos", ctypes.c_double),
        ("recon", ctypes.c_int), ("riemann", ctypes.c_int), ("precision", ctypes.c_int), ("bc", ctypes.c_int),
        ("rho_floor0", ctypes.c_double), ("eps_floor0", ctypes.c_double), ("floor_r_exp", ctypes.c_double),
        ("w_max", ctypes.c_double), ("c2p_tol", ctypes.c_double), ("c2p_max_iter", ctypes.c_int),
        ("cfl", ctypes.c_double), ("weno_eps", ctypes.c_double), ("ct", ctypes.c_int),
        ("shift", ctypes.c_double * 3), ("scalar", ctypes.c_int),
    ]


class grmhd_block(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("x0", ctypes.c_double * 3), ("dx", ctypes.c_double * 3)]


_lib = None


def exported_names():
    """Function names declared in include/grmhd.h."""
    src = open(HEADER).read()
    return sorted(set(re.findall(r"\b(grmhd_[a-z0-9_]+)\s*\(", src)))


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise GrmhdError(f"{LIB_PATH} is not built: run paper_2410_09146_gb300.build.build() "
                             "(the CUDA library has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        vp, P = ctypes.c_void_p, ctypes.POINTER(grmhd_params)
        L.grmhd_workspace_bytes.argtypes = [P]
        L.grmhd_workspace_bytes.restype = ctypes.c_size_t
        L.grmhd_create.argtypes = [P, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
        L.grmhd_set_prims.argtypes = [vp, vp, ctypes.c_int]
        L.grmhd_set_cons.argtypes = [vp, vp, ctypes.c_int]
        L.grmhd_set_face_b.argtypes = [vp, vp, ctypes.c_int]
        L.grmhd_set_scalar.argtypes = [vp, vp, ctypes.c_int]
        L.grmhd_set_prims_f32.argtypes = [vp, vp, ctypes.c_int]
        L.grmhd_batch_set_scalar.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int]
        L.grmhd_stage.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.grmhd_rk2_step.argtypes = [vp, ctypes.c_double]
        L.grmhd_stage_host_f32.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double]
        L.grmhd_c2p.argtypes = [vp, ctypes.c_longlong, vp, vp, vp, vp, ctypes.c_int]
        L.grmhd_get.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int]
        L.grmhd_set_timing.argtypes = [vp, ctypes.c_int]
        L.grmhd_get_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
        L.grmhd_stage_noalloc.argtypes = [P, vp, vp, vp, vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, vp]
        B = ctypes.POINTER(grmhd_block)
        L.grmhd_batch_workspace_bytes.argtypes = [P, ctypes.c_int, B]
        L.grmhd_batch_workspace_bytes.restype = ctypes.c_size_t
        L.grmhd_batch_create.argtypes = [P, ctypes.c_int, B, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
        L.grmhd_batch_set_prims.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int]
        L.grmhd_batch_get.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int]
        L.grmhd_batch_set_tile.argtypes = [vp, ctypes.c_int]
        L.grmhd_batch_set_lattice.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        ip = ctypes.POINTER(ctypes.c_int)
        L.grmhd_batch_set_mesh.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ip]
        L.grmhd_batch_autotune.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
        L.grmhd_set_graph.argtypes = [vp, ctypes.c_int]
        L.grmhd_batch_autotune_table.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                                 ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        fp = ctypes.POINTER(ctypes.c_float)
        L.grmhd_mlp_workspace_bytes.argtypes = []
        L.grmhd_mlp_workspace_bytes.restype = ctypes.c_size_t
        L.grmhd_mlp_set_weights.argtypes = [vp, fp, fp, vp]
        L.grmhd_mlp_get_weights.argtypes = [vp, fp, fp, vp]
        L.grmhd_mlp_forward.argtypes = [vp, ctypes.c_longlong, vp, vp, vp]
        L.grmhd_mlp_grad.argtypes = [vp, ctypes.c_longlong, vp, vp, ctypes.c_double, fp, fp, vp]
        L.grmhd_mlp_grad_tc.argtypes = [vp, ctypes.c_longlong, vp, vp, ctypes.c_double, fp, fp, vp]
        L.grmhd_mlp_adam.argtypes = [vp, ctypes.c_double, ctypes.c_int, vp]
        L.grmhd_mlp_train.argtypes = [vp, ctypes.c_longlong, vp, vp, ctypes.c_longlong, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_int, vp, vp]
        L.grmhd_mlp_train_tc.argtypes = [vp, ctypes.c_longlong, vp, vp, ctypes.c_longlong, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_int, vp, vp]
        L.grmhd_p2c.argtypes = [vp, ctypes.c_longlong, vp, vp]
        L.grmhd_c2p_guess.argtypes = [vp, vp, ctypes.c_longlong, vp, vp, vp, vp, vp, vp, vp, ctypes.c_int]
        L.grmhd_max_speed.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        L.grmhd_bounds_fault.argtypes = [vp, ctypes.POINTER(ctypes.c_ulonglong)]
        L.grmhd_fp_peaks.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        L.grmhd_last_error.argtypes = [vp]
        L.grmhd_last_error.restype = ctypes.c_char_p
        L.grmhd_destroy.argtypes = [vp]
        L.grmhd_destroy.restype = None
        _lib = L
    return _lib


def params(setup) -> grmhd_params:
    """Parameter struct from an ``inputs.Setup`` (or any object with the same fields)."""
    p = grmhd_params()
    p.nx, p.ny, p.nz = setup.n
    p.ng = setup.ng
    p.x0[:] = list(setup.x0)
    p.dx[:] = list(setup.dx)
    p.metric = METRIC[setup.metric]
    p.spin, p.mass, p.gamma_eos = setup.spin, setup.mass, setup.gamma_eos
    p.recon, p.riemann = RECON[setup.recon], RIEMANN[setup.riemann]
    p.precision, p.bc = PRECISION[setup.precision], BC[setup.bc]
    p.rho_floor0, p.eps_floor0, p.floor_r_exp, p.w_max = (setup.rho_floor0, setup.eps_floor0, setup.floor_r_exp,
                                                          setup.w_max)
    p.c2p_tol, p.c2p_max_iter, p.cfl, p.weno_eps = setup.c2p_tol, setup.c2p_max_iter, setup.cfl, setup.weno_eps
    p.ct = CT[getattr(setup, "ct", "flux")]
    p.shift[:] = list(getattr(setup, "shift", (0.0, 0.0, 0.0)))
    p.scalar = int(bool(getattr(setup, "scalar", False)))
    return p


def _check(rc, ctx=None):
    if rc != GRMHD_OK:
        msg = lib().grmhd_last_error(ctx)
        raise GrmhdError(f"libgrmhd error {rc}: {msg.decode() if msg else ''}")


def _ptr(a):
    """(pointer, where) of a numpy array (host) or a torch tensor (device)."""
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data, GRMHD_HOST
    assert a.is_contiguous()
    return a.data_ptr(), (GRMHD_DEVICE if a.is_cuda else GRMHD_HOST)


# ------------------------------------------------------------------ thin wrappers with the C names
def grmhd_workspace_bytes(p: grmhd_params) -> int:
    return int(lib().grmhd_workspace_bytes(ctypes.byref(p)))


def grmhd_create(p: grmhd_params, workspace_ptr: int, nbytes: int, stream_ptr: int) -> int:
    out = ctypes.c_void_p()
    _check(lib().grmhd_create(ctypes.byref(p), ctypes.c_void_p(workspace_ptr), nbytes, ctypes.c_void_p(stream_ptr),
                              ctypes.byref(out)))
    return out.value


def grmhd_set_prims(ctx: int, P) -> None:
    ptr, where = _ptr(P)
    _check(lib().grmhd_set_prims(ctx, ctypes.c_void_p(ptr), where), ctx)


def grmhd_set_cons(ctx: int, U) -> None:
    ptr, where = _ptr(U)
    _check(lib().grmhd_set_cons(ctx, ctypes.c_void_p(ptr), where), ctx)


def grmhd_set_face_b(ctx: int, Bf) -> None:
    ptr, where = _ptr(Bf)
    _check(lib().grmhd_set_face_b(ctx, ctypes.c_void_p(ptr), where), ctx)


def grmhd_set_prims_f32(ctx: int, P) -> None:
    ptr, where = _ptr(P)
    _check(lib().grmhd_set_prims_f32(ctx, ctypes.c_void_p(ptr), where), ctx)


def grmhd_set_scalar(ctx: int, X) -> None:
    ptr, where = _ptr(X)
    _check(lib().grmhd_set_scalar(ctx, ctypes.c_void_p(ptr), where), ctx)


def grmhd_stage(ctx: int, g0: float, g1: float, beta: float, dt: float) -> None:
    _check(lib().grmhd_stage(ctx, g0, g1, beta, dt), ctx)


def grmhd_rk2_step(ctx: int, dt: float) -> None:
    _check(lib().grmhd_rk2_step(ctx, dt), ctx)


def grmhd_stage_host_f32(ctx: int, P_in, P_out, g0: float, g1: float, beta: float, dt: float) -> None:
    """One stage from host float primitives P_in (None: continue from the context's state) to host float
    primitives P_out (None: no read-back), the read-back overlapped with the stage (C ABI grmhd_stage_host_f32).
    P_in / P_out: CPU tensors or arrays of float32 in the layout of grmhd_set_prims_f32."""
    def host_ptr(a):
        if a is None:
            return None
        ptr, where = _ptr(a)
        if where != GRMHD_HOST or "float32" not in str(a.dtype):
            raise GrmhdError("grmhd_stage_host_f32 takes float32 host buffers")
        return ptr
    _check(lib().grmhd_stage_host_f32(ctx, ctypes.c_void_p(host_ptr(P_in)), ctypes.c_void_p(host_ptr(P_out)), g0,
                                      g1, beta, dt), ctx)


def grmhd_c2p(ctx: int, n: int, U_ptr: int, P_ptr: int, status_ptr: int = 0, iters_ptr: int = 0,
              flags: int = 0) -> None:
    vp = ctypes.c_void_p
    _check(lib().grmhd_c2p(ctx, n, vp(U_ptr), vp(P_ptr), vp(status_ptr or None), vp(iters_ptr or None), flags), ctx)


def grmhd_p2c(ctx: int, n: int, P_ptr: int, U_ptr: int) -> None:
    vp = ctypes.c_void_p
    _check(lib().grmhd_p2c(ctx, n, vp(P_ptr), vp(U_ptr)), ctx)


def grmhd_c2p_guess(ctx: int, mlp_ws: int, n: int, U_ptr: int, P_ptr: int, status_ptr: int = 0, iters_ptr: int = 0,
                    guess_ptr: int = 0, X_ptr: int = 0, T_ptr: int = 0, flags: int = 0) -> None:
    vp = ctypes.c_void_p
    _check(lib().grmhd_c2p_guess(ctx, vp(mlp_ws or None), n, vp(U_ptr), vp(P_ptr), vp(status_ptr or None),
                                 vp(iters_ptr or None), vp(guess_ptr or None), vp(X_ptr or None), vp(T_ptr or None),
                                 flags), ctx)


def _fp(a):
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def grmhd_mlp_workspace_bytes() -> int:
    return int(lib().grmhd_mlp_workspace_bytes())


def grmhd_mlp_set_weights(ws: int, theta, norm, stream_ptr: int) -> None:
    theta = np.ascontiguousarray(theta, dtype=np.float32)
    norm = np.ascontiguousarray(norm, dtype=np.float32)
    assert theta.size == GRMHD_MLP_NPARAM and norm.size == GRMHD_MLP_NNORM
    _check(lib().grmhd_mlp_set_weights(ctypes.c_void_p(ws), _fp(theta), _fp(norm), ctypes.c_void_p(stream_ptr)))


def grmhd_mlp_get_weights(ws: int, stream_ptr: int):
    """(FP32 master weights, BF16 weights as float32)."""
    theta = np.zeros(GRMHD_MLP_NPARAM, np.float32)
    wb = np.zeros(GRMHD_MLP_NPARAM, np.float32)
    _check(lib().grmhd_mlp_get_weights(ctypes.c_void_p(ws), _fp(theta), _fp(wb), ctypes.c_void_p(stream_ptr)))
    return theta, wb


def grmhd_mlp_forward(ws: int, n: int, X_ptr: int, Y_ptr: int, stream_ptr: int) -> None:
    vp = ctypes.c_void_p
    _check(lib().grmhd_mlp_forward(vp(ws), n, vp(X_ptr), vp(Y_ptr), vp(stream_ptr)))


def grmhd_mlp_grad(ws: int, n: int, X_ptr: int, T_ptr: int, aux: float, stream_ptr: int, tc: bool = False):
    """(loss, gradient [NPARAM] float32) of one batch; tc: grmhd_mlp_grad_tc (tensor cores)."""
    vp = ctypes.c_void_p
    g = np.zeros(GRMHD_MLP_NPARAM, np.float32)
    loss = np.zeros(1, np.float32)
    fn = lib().grmhd_mlp_grad_tc if tc else lib().grmhd_mlp_grad
    _check(fn(vp(ws), n, vp(X_ptr), vp(T_ptr), aux, _fp(g), _fp(loss), vp(stream_ptr)))
    return float(loss[0]), g


def grmhd_mlp_adam(ws: int, lr: float, step: int, stream_ptr: int) -> None:
    _check(lib().grmhd_mlp_adam(ctypes.c_void_p(ws), lr, step, ctypes.c_void_p(stream_ptr)))


def grmhd_mlp_train(ws: int, n: int, X_ptr: int, T_ptr: int, batch: int, steps: int, lr: float, lr_end: float,
                    aux: float, first_step: int, loss_ptr: int, stream_ptr: int, tc: bool = False) -> None:
    """grmhd_mlp_train, or grmhd_mlp_train_tc (tensor-core gradient) with tc."""
    vp = ctypes.c_void_p
    fn = lib().grmhd_mlp_train_tc if tc else lib().grmhd_mlp_train
    _check(fn(vp(ws), n, vp(X_ptr), vp(T_ptr), batch, steps, lr, lr_end, aux, first_step, vp(loss_ptr or None),
              vp(stream_ptr)))


def grmhd_get(ctx: int, what: int, dst) -> None:
    ptr, where = _ptr(dst)
    _check(lib().grmhd_get(ctx, what, ctypes.c_void_p(ptr), where), ctx)


def grmhd_set_timing(ctx: int, on: bool) -> None:
    _check(lib().grmhd_set_timing(ctx, int(on)), ctx)


KERNEL_GROUPS = ("ghost", "flux_x", "flux_y", "flux_z", "emf", "update", "cell_passes")


def grmhd_get_timing(ctx: int):
    ms = (ctypes.c_double * 7)()
    n = ctypes.c_int(0)
    _check(lib().grmhd_get_timing(ctx, ms, ctypes.byref(n)), ctx)
    return dict(zip(KERNEL_GROUPS, list(ms))), n.value


def grmhd_bounds_fault(ctx: int):
    """(fault word, built with checks) of the bounds-check build (see include/grmhd.h)."""
    out = (ctypes.c_ulonglong * 2)()
    _check(lib().grmhd_bounds_fault(ctypes.c_void_p(ctx), out), ctx)
    return int(out[0]), bool(out[1])


def use_library(path):
    """Load the entry points from another build of the library (e.g. the bounds-check build) for the
    contexts created from now on; returns the previous (path, handle) for restore_library."""
    global _lib, LIB_PATH
    prev = (LIB_PATH, _lib)
    LIB_PATH, _lib = path, None
    lib()
    return prev


def restore_library(prev):
    global _lib, LIB_PATH
    LIB_PATH, _lib = prev


def grmhd_max_speed(ctx: int):
    """Largest |lambda| per direction over the interior faces of the last CFL stage (see include/grmhd.h)."""
    out = (ctypes.c_double * 3)()
    _check(lib().grmhd_max_speed(ctypes.c_void_p(ctx), out), ctx)
    return np.array(out[:])


def grmhd_fp_peaks(sink_ptr: int, stream_ptr: int = 0):
    """(FP64, FP32) dense FMA rates of the current device in TFLOP/s (see include/grmhd.h)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().grmhd_fp_peaks(ctypes.c_void_p(sink_ptr), ctypes.c_void_p(stream_ptr or None), ctypes.byref(a),
                                ctypes.byref(b)))
    return a.value, b.value


def grmhd_stage_noalloc(p: grmhd_params, P_ptr: int, U0_ptr: int, Ucur_ptr: int, Unew_ptr: int, status_ptr: int,
                        g0: float, g1: float, beta: float, dt: float, stream_ptr: int = 0) -> None:
    """Allocation-free all-FP64 stage on caller-owned device arrays (see include/grmhd.h)."""
    vp = ctypes.c_void_p
    _check(lib().grmhd_stage_noalloc(ctypes.byref(p), vp(P_ptr), vp(U0_ptr or None), vp(Ucur_ptr), vp(Unew_ptr),
                                     vp(status_ptr), g0, g1, beta, dt, vp(stream_ptr or None)))


def grmhd_destroy(ctx: int) -> None:
    lib().grmhd_destroy(ctx)


def grmhd_batch_workspace_bytes(p: grmhd_params, blocks) -> int:
    arr = (grmhd_block * len(blocks))(*blocks)
    return int(lib().grmhd_batch_workspace_bytes(ctypes.byref(p), len(blocks), arr))


def grmhd_batch_create(p: grmhd_params, blocks, workspace_ptr: int, nbytes: int, stream_ptr: int) -> int:
    arr = (grmhd_block * len(blocks))(*blocks)
    out = ctypes.c_void_p()
    _check(lib().grmhd_batch_create(ctypes.byref(p), len(blocks), arr, ctypes.c_void_p(workspace_ptr), nbytes,
                                    ctypes.c_void_p(stream_ptr), ctypes.byref(out)))
    return out.value


def grmhd_batch_set_lattice(ctx: int, nbx: int, nby: int, nbz: int, periodic: bool) -> None:
    _check(lib().grmhd_batch_set_lattice(ctx, nbx, nby, nbz, int(periodic)), ctx)


def grmhd_batch_set_mesh(ctx: int, nbx: int, nby: int, nbz: int, periodic: bool, level, pos) -> None:
    lv = np.ascontiguousarray(level, dtype=np.int32).ravel()
    ps = np.ascontiguousarray(pos, dtype=np.int32).ravel()
    ip = ctypes.POINTER(ctypes.c_int)
    _check(lib().grmhd_batch_set_mesh(ctx, nbx, nby, nbz, int(periodic), lv.ctypes.data_as(ip), ps.ctypes.data_as(ip)),
           ctx)


def grmhd_batch_set_scalar(ctx: int, block: int, X) -> None:
    ptr, where = _ptr(X)
    _check(lib().grmhd_batch_set_scalar(ctx, block, ctypes.c_void_p(ptr), where), ctx)


def grmhd_batch_set_prims(ctx: int, block: int, P) -> None:
    ptr, where = _ptr(P)
    _check(lib().grmhd_batch_set_prims(ctx, block, ctypes.c_void_p(ptr), where), ctx)


def grmhd_batch_get(ctx: int, block: int, what: int, dst) -> None:
    ptr, where = _ptr(dst)
    _check(lib().grmhd_batch_get(ctx, block, what, ctypes.c_void_p(ptr), where), ctx)


def grmhd_batch_set_tile(ctx: int, tile: int) -> None:
    _check(lib().grmhd_batch_set_tile(ctx, tile), ctx)


def grmhd_batch_autotune(ctx: int):
    t = ctypes.c_int(0)
    ms = ctypes.c_double(0.0)
    _check(lib().grmhd_batch_autotune(ctx, ctypes.byref(t), ctypes.byref(ms)), ctx)
    return t.value, ms.value


def grmhd_batch_autotune_table(ctx: int):
    """[(tile, ms per stage)] of the last autotune of the batch (see include/grmhd.h)."""
    tiles = (ctypes.c_int * 8)()
    ms = (ctypes.c_double * 8)()
    n = ctypes.c_int()
    _check(lib().grmhd_batch_autotune_table(ctypes.c_void_p(ctx), tiles, ms, 8, ctypes.byref(n)), ctx)
    return [(tiles[k], ms[k]) for k in range(min(n.value, 8))]


def grmhd_set_graph(ctx: int, on: bool) -> None:
    _check(lib().grmhd_set_graph(ctx, int(on)), ctx)


def block_of(setup) -> grmhd_block:
    b = grmhd_block()
    b.nx, b.ny, b.nz = setup.n
    b.x0[:] = list(setup.x0)
    b.dx[:] = list(setup.dx)
    return b


class BatchContext:
    """Many meshblocks advanced together (one persistent launch per phase); `setups` give each block's
    size and placement, the first one the shared physics options."""

    def __init__(self, setups, device: int = 0, stream=None):
        import torch
        self.setups = list(setups)
        self.p = params(self.setups[0])
        self.blocks = [block_of(s) for s in self.setups]
        nbytes = grmhd_batch_workspace_bytes(self.p, self.blocks)
        if nbytes == 0:
            raise GrmhdError("invalid batch parameters")
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        self.ws_ptr = (self._ws.data_ptr() + 255) // 256 * 256
        self.ctx = grmhd_batch_create(self.p, self.blocks, self.ws_ptr, nbytes, self.stream.cuda_stream)

    def __del__(self):
        if getattr(self, "ctx", None):
            grmhd_destroy(self.ctx)
            self.ctx = None

    def set_prims(self, block, P):
        grmhd_batch_set_prims(self.ctx, block, P)

    def set_scalar(self, block, X):
        """Passive scalar X of one block (ghosted, double; params.scalar): ``grmhd_batch_set_scalar``."""
        grmhd_batch_set_scalar(self.ctx, block, X)

    def stage(self, g0, g1, beta, dt=0.0):
        grmhd_stage(self.ctx, g0, g1, beta, dt)

    def rk2_step(self, dt=0.0):
        grmhd_rk2_step(self.ctx, dt)

    def get(self, block, what):
        s = self.setups[block]
        shape, dt = {GRMHD_GET_PRIMS: (s.prim_shape(), np.float64), GRMHD_GET_CONS: (s.cons_shape(), np.float64),
                     GRMHD_GET_STATUS: (s.cons_shape()[1:], np.uint8),
                     GRMHD_GET_SCALAR: (s.prim_shape()[1:], np.float64),
                     GRMHD_GET_SCALAR_CONS: (s.cons_shape()[1:], np.float64)}[what]
        out = np.empty(shape, dt)
        grmhd_batch_get(self.ctx, block, what, out)
        return out

    def stats(self):
        out = np.empty(8, np.uint64)
        grmhd_get(self.ctx, GRMHD_GET_STATS, out)
        return out

    def dt(self):
        out = np.empty(1, np.float64)
        grmhd_get(self.ctx, GRMHD_GET_DT, out)
        return float(out[0])

    def set_tile(self, tile):
        grmhd_batch_set_tile(self.ctx, tile)

    def set_lattice(self, nb, periodic):
        grmhd_batch_set_lattice(self.ctx, nb[0], nb[1], nb[2], periodic)

    def set_mesh(self, nb, periodic, level, pos):
        """Declare the blocks the leaves of a two-level mesh (``grmhd_batch_set_mesh``)."""
        grmhd_batch_set_mesh(self.ctx, nb[0], nb[1], nb[2], periodic, level, pos)

    def autotune(self):
        return grmhd_batch_autotune(self.ctx)

    def autotune_table(self):
        return grmhd_batch_autotune_table(self.ctx)

    def set_graph(self, on=True):
        grmhd_set_graph(self.ctx, on)


# ------------------------------------------------------------------ convenience object
class Context:
    """One meshblock context: owns a torch workspace tensor and borrows a torch stream."""

    def __init__(self, setup, device: int = 0, stream=None):
        import torch
        self.setup = setup
        self.p = params(setup)
        nbytes = grmhd_workspace_bytes(self.p)
        if nbytes == 0 and setup.n != (0, 0, 0):
            raise GrmhdError("invalid parameters: " + lib().grmhd_last_error(None).decode())
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self._ws.data_ptr()
        self.ws_ptr = (base + 255) // 256 * 256
        self.ws_bytes = nbytes
        self.ctx = grmhd_create(self.p, self.ws_ptr, nbytes, self.stream.cuda_stream)

    def __del__(self):
        if getattr(self, "ctx", None):
            grmhd_destroy(self.ctx)
            self.ctx = None

    def set_prims(self, P):
        grmhd_set_prims(self.ctx, P)

    def set_cons(self, U):
        grmhd_set_cons(self.ctx, U)

    def set_face_b(self, Bf):
        grmhd_set_face_b(self.ctx, Bf)

    def set_scalar(self, X):
        """Passive scalar X (ghosted, double; params.scalar): ``grmhd_set_scalar``."""
        grmhd_set_scalar(self.ctx, X)

    def stage(self, g0, g1, beta, dt=0.0):
        grmhd_stage(self.ctx, g0, g1, beta, dt)

    def rk2_step(self, dt=0.0):
        grmhd_rk2_step(self.ctx, dt)

    def get(self, what, out=None):
        s = self.setup
        shapes = {GRMHD_GET_PRIMS: (s.prim_shape(), np.float64), GRMHD_GET_CONS: (s.cons_shape(), np.float64),
                  GRMHD_GET_STATUS: (s.cons_shape()[1:], np.uint8), GRMHD_GET_STATS: ((8,), np.uint64),
                  GRMHD_GET_DT: ((1,), np.float64), GRMHD_GET_FACE_B: ((3,) + s.prim_shape()[1:], np.float64),
                  GRMHD_GET_SCALAR: (s.prim_shape()[1:], np.float64),
                  GRMHD_GET_SCALAR_CONS: (s.cons_shape()[1:], np.float64),
                  GRMHD_GET_PRIMS_F32: (s.prim_shape(), np.float32)}
        if out is None:
            shape, dt = shapes[what]
            out = np.empty(shape, dt)
        grmhd_get(self.ctx, what, out)
        return out

    def prims(self):
        return self.get(GRMHD_GET_PRIMS)

    def cons(self):
        return self.get(GRMHD_GET_CONS)

    def status(self):
        return self.get(GRMHD_GET_STATUS)

    def stats(self):
        return self.get(GRMHD_GET_STATS)

    def dt(self):
        return float(self.get(GRMHD_GET_DT)[0])

    def max_speed(self):
        return grmhd_max_speed(self.ctx)

    def face_b(self):
        return self.get(GRMHD_GET_FACE_B)

    def scalar(self):
        return self.get(GRMHD_GET_SCALAR)

    def scalar_cons(self):
        return self.get(GRMHD_GET_SCALAR_CONS)

    def set_timing(self, on=True):
        grmhd_set_timing(self.ctx, on)

    def timing(self):
        """(ms per kernel group accumulated since the last call, number of stages)."""
        return grmhd_get_timing(self.ctx)

    def c2p(self, U, P, status=None, iters=None, flags=0):
        """Flat-space con2prim batch of torch device tensors U, P of shape [8][n] (float64)."""
        n = U.shape[1]
        grmhd_c2p(self.ctx, n, U.data_ptr(), P.data_ptr(), 0 if status is None else status.data_ptr(),
                  0 if iters is None else iters.data_ptr(), flags)

    def p2c(self, P, U):
        """Flat-space prim->cons batch of torch device tensors P, U of shape [8][n] (float64)."""
        grmhd_p2c(self.ctx, P.shape[1], P.data_ptr(), U.data_ptr())

    def c2p_guess(self, U, P, status=None, iters=None, net=None, guess=None, X=None, T=None, fp32=False):
        """Flat-space con2prim batch [8][n] from the network's start (net: GuessNet) or the standard start
        (net None). Network on the tensor cores (fused kernel) unless fp32; guess (float64 [2][n]) receives
        (mu_0, mu_+) and is required with fp32. X [n][8] and T [n][2] (float32) receive training pairs
        (standard start or fp32 only)."""
        n = U.shape[1]
        if net is not None and fp32 and guess is None:
            raise GrmhdError("the FP32-core guess needs a guess buffer")
        ptr = lambda a: 0 if a is None else a.data_ptr()
        grmhd_c2p_guess(self.ctx, 0 if net is None else net.ws_ptr, n, U.data_ptr(), P.data_ptr(), ptr(status),
                        ptr(iters), ptr(guess) if net is not None else 0, ptr(X), ptr(T),
                        GRMHD_GUESS_FP32 if fp32 else 0)


class GuessNet:
    """The learned con2prim guess: a device workspace with weights, Adam state and standardisation.

    Initialisation (He-uniform hidden layers, small output layer, zero biases) and the standardisation
    statistics are host-side set-up; forward, backward and Adam run in the library's kernels.
    """

    def __init__(self, device: int = 0, stream=None, seed: int = 0):
        import torch
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = grmhd_mlp_workspace_bytes()
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        self.ws_ptr = (self._ws.data_ptr() + 255) // 256 * 256
        self.step = 0
        self.norm = np.zeros(GRMHD_MLP_NNORM, np.float32)
        self.norm[8:16] = 1.0
        self.norm[18:20] = 1.0
        self.set_weights(init_weights(seed), self.norm)

    def set_weights(self, theta, norm):
        self.norm = np.asarray(norm, np.float32).copy()
        grmhd_mlp_set_weights(self.ws_ptr, theta, self.norm, self.stream.cuda_stream)
        self.step = 0

    def weights(self):
        return grmhd_mlp_get_weights(self.ws_ptr, self.stream.cuda_stream)

    def fit_norm(self, X, T, sample: int = 1 << 20):
        """Standardisation from (a leading sample of) raw features X [n][8] and targets T [n][2]
        (device float32); keeps the weights and resets Adam."""
        Xs = X[:sample].double().cpu().numpy()
        Ts = T[:sample].double().cpu().numpy()
        norm = np.zeros(GRMHD_MLP_NNORM)
        norm[0:8] = Xs.mean(0)
        norm[8:16] = 1.0 / np.maximum(Xs.std(0), 1e-6)
        norm[16:18] = Ts.mean(0)
        norm[18:20] = np.maximum(Ts.std(0), 1e-6)
        theta, _ = self.weights()
        self.set_weights(theta, norm)

    def forward(self, X, Y=None):
        import torch
        n = X.shape[0]
        if Y is None:
            Y = torch.empty((n, 2), dtype=torch.float32, device=X.device)
        grmhd_mlp_forward(self.ws_ptr, n, X.data_ptr(), Y.data_ptr(), self.stream.cuda_stream)
        return Y

    def grad(self, X, T, aux: float = 0.1, tc: bool = False):
        return grmhd_mlp_grad(self.ws_ptr, X.shape[0], X.data_ptr(), T.data_ptr(), aux, self.stream.cuda_stream, tc)

    def adam(self, lr: float):
        self.step += 1
        grmhd_mlp_adam(self.ws_ptr, lr, self.step, self.stream.cuda_stream)

    def train(self, X, T, batch: int, steps: int, lr: float, lr_end: float = 0.0, aux: float = 0.1, losses=None,
              tc: bool = False):
        """Adam over contiguous minibatches (see grmhd_mlp_train); losses: device float32 [steps] or None;
        tc: the tensor-core gradient (grmhd_mlp_train_tc)."""
        grmhd_mlp_train(self.ws_ptr, X.shape[0], X.data_ptr(), T.data_ptr(), batch, steps, lr, lr_end, aux,
                        self.step + 1, 0 if losses is None else losses.data_ptr(), self.stream.cuda_stream, tc)
        self.step += steps


def init_weights(seed: int = 0):
    """He-uniform hidden layers, output layer scaled by 0.1, zero biases (float32 [GRMHD_MLP_NPARAM])."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in, scale in ((64, 8, 1.0), (64, 64, 1.0), (64, 64, 1.0), (2, 64, 0.1)):
        bound = scale * np.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-bound, bound, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    theta = np.concatenate(parts).astype(np.float32)
    assert theta.size == GRMHD_MLP_NPARAM
    return theta
