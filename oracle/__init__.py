"""Serial FP64 oracle for one Runge-Kutta stage of the Valencia GRMHD update.

TEST INFRASTRUCTURE. This package is the correctness reference for the CUDA
library and nothing else: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it. The product path never routes
through it. It shares no code with the CUDA path; the two meet only through the
seeded input generators in ``paper_2410_09146_gb300/inputs.py``.

The arithmetic lives in ``grmhd_oracle.cpp`` (compiled with
``-O2 -ffp-contract=off``); this module compiles it on first use and wraps its
C entry points with numpy marshalling.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants or brute force (see each test's docstring).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# GRMHD_ORACLE_SRC / GRMHD_ORACLE_BUILD point the package at another copy of the source (the planted-mistake
# tests compile copies with one mistake each and run the pins against them)
_SRC = os.environ.get("GRMHD_ORACLE_SRC") or os.path.join(_HERE, "grmhd_oracle.cpp")
_BUILD = os.environ.get("GRMHD_ORACLE_BUILD") or os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

RECON = {"constant": 0, "plm_minmod": 1, "plm_mc": 2, "weno5z_aoah": 3, "mp5": 4}
RIEMANN = {"llf": 0, "hll": 1}
METRIC = {"minkowski": 0, "kerr_schild": 1, "kerr_schild_spherical": 2}
BC = {"periodic": 0, "fixed": 1, "spherical": 2}

ST_RHO_FLOOR, ST_EPS_FLOOR, ST_W_CAP, ST_NOT_CONVERGED, ST_BAD_INPUT = 1, 2, 4, 8, 16


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, -O2 -ffp-contract=off)."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _SO + f".tmp{os.getpid()}"
            cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                   "-o", tmp, _SRC]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _SO)
    return _SO


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("ng", ctypes.c_int),
        ("x0", ctypes.c_double * 3), ("dx", ctypes.c_double * 3),
        ("metric", ctypes.c_int), ("spin", ctypes.c_double), ("mass", ctypes.c_double),
        ("gamma_eos", ctypes.c_double),
        ("recon", ctypes.c_int), ("riemann", ctypes.c_int), ("bc", ctypes.c_int),
        ("rho_floor0", ctypes.c_double), ("eps_floor0", ctypes.c_double), ("floor_r_exp", ctypes.c_double),
        ("w_max", ctypes.c_double), ("c2p_tol", ctypes.c_double), ("c2p_max_iter", ctypes.c_int),
        ("cfl", ctypes.c_double), ("weno_eps", ctypes.c_double), ("shift", ctypes.c_double * 3),
    ]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        P = ctypes.POINTER(OrcParams)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        ip = ctypes.POINTER(ctypes.c_int)
        L = ctypes.c_long
        lib.orc_geom_points.argtypes = [P, L, dp, dp]
        lib.orc_prim2con_points.argtypes = [P, L, dp, dp, dp, dp, dp, dp, dp]
        lib.orc_c2p_points.argtypes = [P, L, dp, dp, dp, u8p, ip, ctypes.c_int]
        lib.orc_c2p_mu_points.argtypes = [P, L, dp, dp, dp, dp, dp]
        lib.orc_recon_points.argtypes = [ctypes.c_int, L, dp, ctypes.c_double, dp, dp]
        lib.orc_weno5z_points.argtypes = [L, dp, ctypes.c_double, dp, dp, dp]
        lib.orc_riemann_points.argtypes = [P, L, dp, dp, dp, ctypes.c_int, dp, dp]
        lib.orc_prim2con_grid.argtypes = [P, dp, dp]
        lib.orc_ghost_fill.argtypes = [P, dp]
        lib.orc_stage.argtypes = [P, dp, dp, dp, dp, u8p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, dp, dp, ip, dp, dp]
        lib.orc_stage_face_ct.argtypes = lib.orc_stage.argtypes + [dp, dp, dp]
        lib.orc_face_b_to_cells.argtypes = [P, dp, dp]
        lib.orc_face_fluxes_used.argtypes = [P, dp, dp, dp]
        lib.orc_stage_scalar.argtypes = [P, dp, dp, dp, dp, u8p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, dp, dp, ip, dp, dp, dp, dp, dp, dp, dp]
        lib.orc_finish_points.argtypes = [P, L, dp, dp, dp, u8p]
        _lib = lib
    return _lib


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def params(setup) -> OrcParams:
    """Build the oracle's parameter struct from an ``inputs.Setup``."""
    p = OrcParams()
    p.nx, p.ny, p.nz = setup.n
    p.ng = setup.ng
    p.x0[:] = list(setup.x0)
    p.dx[:] = list(setup.dx)
    p.metric = METRIC[setup.metric]
    p.spin, p.mass, p.gamma_eos = setup.spin, setup.mass, setup.gamma_eos
    p.recon, p.riemann, p.bc = RECON[setup.recon], RIEMANN[setup.riemann], BC[setup.bc]
    p.rho_floor0, p.eps_floor0, p.floor_r_exp, p.w_max = (setup.rho_floor0, setup.eps_floor0, setup.floor_r_exp,
                                                          setup.w_max)
    p.c2p_tol, p.c2p_max_iter = setup.c2p_tol, setup.c2p_max_iter
    p.cfl, p.weno_eps = setup.cfl, setup.weno_eps
    p.shift[:] = list(getattr(setup, "shift", (0.0, 0.0, 0.0)))
    return p


def geom_points(p: OrcParams, xyz):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((len(xyz), 101))
    _load().orc_geom_points(ctypes.byref(p), len(xyz), _dp(xyz), _dp(out))
    pr = [(1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]
    gam = np.zeros((len(xyz), 3, 3))
    gamu = np.zeros((len(xyz), 3, 3))
    for t, (a, b) in enumerate(pr):
        gam[:, a - 1, b - 1] = gam[:, b - 1, a - 1] = out[:, 4 + t]
        gamu[:, a - 1, b - 1] = gamu[:, b - 1, a - 1] = out[:, 10 + t]
    return {
        "alpha": out[:, 0], "beta": out[:, 1:4], "gam": gam, "gamu": gamu,
        "sqrtgam": out[:, 16], "sqrtmg": out[:, 17], "dlnalpha": out[:, 18:21],
        "g": out[:, 21:37].reshape(-1, 4, 4), "gu": out[:, 37:53].reshape(-1, 4, 4),
        "dg": out[:, 53:101].reshape(-1, 3, 4, 4),
    }


def prim2con_points(p: OrcParams, xyz, P):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    P = np.ascontiguousarray(P, dtype=np.float64).reshape(-1, 8)
    n = len(P)
    U = np.zeros((n, 8)); F = np.zeros((n, 3, 8)); lam = np.zeros((n, 3, 2))
    T = np.zeros((n, 4, 4)); S = np.zeros((n, 8))
    _load().orc_prim2con_points(ctypes.byref(p), n, _dp(xyz), _dp(P), _dp(U), _dp(F), _dp(lam), _dp(T), _dp(S))
    return {"U": U, "F": F, "lam": lam, "T": T, "S": S}


def c2p_points(p: OrcParams, xyz, U, floors: bool = True):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(-1, 8)
    n = len(U)
    P = np.zeros((n, 8)); st = np.zeros(n, np.uint8); it = np.zeros(n, np.int32)
    _load().orc_c2p_points(ctypes.byref(p), n, _dp(xyz), _dp(U), _dp(P),
                           st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                           it.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(floors))
    return P, st, it


def c2p_mu_points(p: OrcParams, xyz, U, aux: bool = False):
    """Root mu = 1/(h W) and bracket end mu_+ of the con2prim master function at points; with
    aux=True also eps and W of the master-function intermediates at mu_+."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(-1, 8)
    mu = np.zeros(len(U)); mup = np.zeros(len(U)); ax = np.zeros((len(U), 2))
    _load().orc_c2p_mu_points(ctypes.byref(p), len(U), _dp(xyz), _dp(U), _dp(mu), _dp(mup), _dp(ax))
    if aux:
        return mu, mup, ax[:, 0].copy(), ax[:, 1].copy()
    return mu, mup


def recon_points(method: str, f, weno_eps: float = 1e-26):
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1, 5)
    qm = np.zeros(len(f)); qp = np.zeros(len(f))
    _load().orc_recon_points(RECON[method], len(f), _dp(f), weno_eps, _dp(qm), _dp(qp))
    return qm, qp


def weno5z_points(f, eps: float = 1e-26):
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1, 5)
    n = len(f)
    val = np.zeros(n); w = np.zeros((n, 3)); sig = np.zeros(n)
    _load().orc_weno5z_points(n, _dp(f), eps, _dp(val), _dp(w), _dp(sig))
    return val, w, sig


def riemann_points(p: OrcParams, xyz, PL, PR, d: int):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    PL = np.ascontiguousarray(PL, dtype=np.float64).reshape(-1, 8)
    PR = np.ascontiguousarray(PR, dtype=np.float64).reshape(-1, 8)
    n = len(PL)
    Fh = np.zeros((n, 8)); cm = np.zeros(n)
    _load().orc_riemann_points(ctypes.byref(p), n, _dp(xyz), _dp(PL), _dp(PR), d, _dp(Fh), _dp(cm))
    return Fh, cm


def prim2con_grid(p: OrcParams, P):
    P = np.ascontiguousarray(P, dtype=np.float64)
    U = np.zeros((8, p.nz, p.ny, p.nx))
    _load().orc_prim2con_grid(ctypes.byref(p), _dp(P), _dp(U))
    return U


def ghost_fill(p: OrcParams, P):
    assert P.dtype == np.float64 and P.flags.c_contiguous
    _load().orc_ghost_fill(ctypes.byref(p), _dp(P))
    return P


def stage(p: OrcParams, P, U0, Ucur, g0: float, g1: float, beta: float, dt: float, debug: bool = False):
    """One RK stage. ``P`` is updated in place (ghosts when periodic, interior by con2prim).

    Returns dict(U=Unew, status, dt, maxspeed, iters[, F, E]).
    """
    assert P.dtype == np.float64 and P.flags.c_contiguous
    Ucur = np.ascontiguousarray(Ucur, dtype=np.float64)
    U0 = None if U0 is None else np.ascontiguousarray(U0, dtype=np.float64)
    Unew = np.zeros_like(Ucur)
    st = np.zeros(Ucur.shape[1:], np.uint8)
    dt_used = ctypes.c_double(0.0)
    ms = np.zeros(3)
    it = ctypes.c_int(0)
    gsz = P.shape[1] * P.shape[2] * P.shape[3]
    F = np.zeros((3, 8) + P.shape[1:]) if debug else None
    E = np.zeros((3,) + P.shape[1:]) if debug else None
    _load().orc_stage(ctypes.byref(p), _dp(P), _dp(U0), _dp(Ucur), _dp(Unew),
                      st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), g0, g1, beta, dt,
                      ctypes.byref(dt_used), _dp(ms), ctypes.byref(it), _dp(F), _dp(E))
    del gsz
    out = {"U": Unew, "status": st, "dt": dt_used.value, "maxspeed": ms, "iters": it.value}
    if debug:
        out["F"], out["E"] = F, E
    return out


def stage_scalar(p: OrcParams, P, X, U0, Ucur, DX0, DXcur, g0: float, g1: float, beta: float, dt: float,
                 debug: bool = False):
    """One flux-CT stage that also advances a passive scalar X (ghosted [gz][gy][gx], updated in place like P)
    with conserved sqrt(gamma) D X (DX0 / DXcur interior arrays; DX0 may be None when g0 = 0).
    Returns dict(U, DX, status, dt, maxspeed, iters[, F, E, FX])."""
    assert P.dtype == np.float64 and P.flags.c_contiguous and X.dtype == np.float64 and X.flags.c_contiguous
    Unew = np.zeros_like(Ucur)
    DXnew = np.zeros_like(DXcur)
    st = np.zeros(Ucur.shape[1:], np.uint8)
    dt_used = ctypes.c_double(0.0)
    ms = np.zeros(3)
    it = ctypes.c_int(0)
    DX0 = None if DX0 is None else np.ascontiguousarray(DX0, dtype=np.float64)
    DXcur = np.ascontiguousarray(DXcur, dtype=np.float64)
    F = np.zeros((3, 8) + P.shape[1:]) if debug else None
    E = np.zeros((3,) + P.shape[1:]) if debug else None
    FX = np.zeros((3,) + P.shape[1:]) if debug else None
    _load().orc_stage_scalar(ctypes.byref(p), _dp(P), _dp(None if U0 is None else np.ascontiguousarray(U0)),
                             _dp(np.ascontiguousarray(Ucur)), _dp(Unew),
                             st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), g0, g1, beta, dt,
                             ctypes.byref(dt_used), _dp(ms), ctypes.byref(it), _dp(X), _dp(DX0), _dp(DXcur), _dp(DXnew),
                             _dp(F), _dp(E), _dp(FX))
    out = dict(U=Unew, DX=DXnew, status=st, dt=dt_used.value, maxspeed=ms, iters=it.value)
    if debug:
        out["F"], out["E"], out["FX"] = F, E, FX
    return out


def rk2_step_scalar(p: OrcParams, P, X, U, DX, dt: float = 0.0):
    """SSP-RK2 step of the fluid and the passive scalar (stage coefficients as ``rk2_step``).
    Returns (U, DX, status, dt)."""
    s1 = stage_scalar(p, P, X, None, U, None, DX, 0.0, 1.0, 1.0, dt)
    s2 = stage_scalar(p, P, X, U, s1["U"], DX, s1["DX"], 0.5, 0.5, 0.5, s1["dt"])
    return s2["U"], s2["DX"], s2["status"], s1["dt"]


def face_fluxes_used(p: OrcParams, F, E):
    """Fluxes the flux-CT update uses on every interior face, [3][8] + grid shape: the hydro components of
    the stage's face fluxes ``F`` and the CT fluxes of B formed from its edge EMFs ``E`` (both from
    ``stage(..., debug=True)``)."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    out = np.zeros_like(F)
    _load().orc_face_fluxes_used(ctypes.byref(p), _dp(F), _dp(E), _dp(out))
    return out


def finish_points(p: OrcParams, xyz, Un):
    """The stage's last step at points: con2prim of the densitized conserved states ``Un`` [n][8], floors,
    and the hydro part re-derived from the floored primitives when a status bit is set.
    Returns (Un after, P, status)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    Un = np.array(Un, dtype=np.float64, order="C").reshape(-1, 8)
    n = len(Un)
    P = np.zeros((n, 8)); st = np.zeros(n, np.uint8)
    _load().orc_finish_points(ctypes.byref(p), n, _dp(xyz), _dp(Un), _dp(P),
                              st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return Un, P, st


def rk2_step(p: OrcParams, P, U, dt: float = 0.0):
    """One SSP-RK2 (Heun) step: stage coefficients (0, 1, 1) then (1/2, 1/2, 1/2).

    ``dt <= 0`` takes the CFL time step from the first stage. Returns (U, status, dt).
    """
    s1 = stage(p, P, None, U, 0.0, 1.0, 1.0, dt)
    s2 = stage(p, P, U, s1["U"], 0.5, 0.5, 0.5, s1["dt"])
    return s2["U"], s2["status"] | s1["status"], s1["dt"]


def face_b_to_cells(p: OrcParams, Bf, P):
    """Cell-centred B of ``P`` from the face field ``Bf`` [3][gz][gy][gx] (densitized sqrt(gamma) B^d on the
    lower d-face of each ghosted cell): B^d = mean of the cell's two d-faces / sqrt(gamma), for every cell
    whose two d-faces are stored. Periodic blocks get their ghost faces filled first (``Bf`` in place)."""
    assert P.dtype == np.float64 and P.flags.c_contiguous
    assert Bf.dtype == np.float64 and Bf.flags.c_contiguous and Bf.shape == (3,) + P.shape[1:]
    _load().orc_face_b_to_cells(ctypes.byref(p), _dp(Bf), _dp(P))
    return P


def stage_face_ct(p: OrcParams, P, Bf0, Bf, U0, Ucur, g0: float, g1: float, beta: float, dt: float,
                  debug: bool = False):
    """One RK stage with face-centred upwind CT. ``P`` is updated in place; ``Bf`` (this stage's faces)
    gets its ghost faces filled when periodic. Returns dict(U, Bf (new faces), status, dt, maxspeed,
    iters[, F, E])."""
    assert P.dtype == np.float64 and P.flags.c_contiguous
    assert Bf.dtype == np.float64 and Bf.flags.c_contiguous and Bf.shape == (3,) + P.shape[1:]
    Ucur = np.ascontiguousarray(Ucur, dtype=np.float64)
    U0 = None if U0 is None else np.ascontiguousarray(U0, dtype=np.float64)
    Bf0 = None if Bf0 is None else np.ascontiguousarray(Bf0, dtype=np.float64)
    Unew = np.zeros_like(Ucur)
    Bfn = np.zeros_like(Bf)
    st = np.zeros(Ucur.shape[1:], np.uint8)
    dt_used = ctypes.c_double(0.0)
    ms = np.zeros(3)
    it = ctypes.c_int(0)
    F = np.zeros((3, 8) + P.shape[1:]) if debug else None
    E = np.zeros((3,) + P.shape[1:]) if debug else None
    rc = _load().orc_stage_face_ct(ctypes.byref(p), _dp(P), _dp(U0), _dp(Ucur), _dp(Unew),
                                   st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), g0, g1, beta, dt,
                                   ctypes.byref(dt_used), _dp(ms), ctypes.byref(it), _dp(F), _dp(E),
                                   _dp(Bf0), _dp(Bf), _dp(Bfn))
    assert rc == 0
    out = {"U": Unew, "Bf": Bfn, "status": st, "dt": dt_used.value, "maxspeed": ms, "iters": it.value}
    if debug:
        out["F"], out["E"] = F, E
    return out


def rk2_step_face_ct(p: OrcParams, P, Bf, U, dt: float = 0.0):
    """SSP-RK2 step with face-centred upwind CT (stage coefficients as ``rk2_step``).
    Returns (U, Bf, status, dt)."""
    s1 = stage_face_ct(p, P, None, Bf, None, U, 0.0, 1.0, 1.0, dt)
    s2 = stage_face_ct(p, P, Bf, s1["Bf"], U, s1["U"], 0.5, 0.5, 0.5, s1["dt"])
    return s2["U"], s2["Bf"], s2["status"] | s1["status"], s1["dt"]


def face_divergence(p: OrcParams, Bf):
    """Face divergence sum_d (Bf_d(upper) - Bf_d(lower)) / dx_d of every interior cell, [nz][ny][nx]."""
    ng = p.ng
    nx, ny, nz = p.nx, p.ny, p.nz
    sl = (slice(ng, ng + nz), slice(ng, ng + ny), slice(ng, ng + nx))
    out = np.zeros((nz, ny, nx))
    for d, ax in ((0, 2), (1, 1), (2, 0)):
        up = list(sl)
        up[ax] = slice(sl[ax].start + 1, sl[ax].stop + 1)
        out += (Bf[d][tuple(up)] - Bf[d][sl]) / p.dx[d]
    return out
