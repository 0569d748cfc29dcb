"""Comparison helpers for the CUDA path against the oracle (test infrastructure).

FP64 parity is judged per stage: both sides start the stage from the same state (the CUDA
path's state before the stage), so an ill-conditioned cell cannot carry its roundoff into later
stages. Errors are relative, per cell:
  * conserved U: against the magnitudes that enter the cell's update, i.e. the largest over the
    cell and its six face neighbours of |D| (for D), max(tau + D, |S|) (for S_j and tau) and |B|
    (for B^k), floored at 1e-3 of the grid maximum of each;
  * primitives: rho against max(rho, 1e-3 max rho); W v^i against max(|W v|, 1) (the Lorentz-factor
    scale); rho eps against (tau + D)/sqrt(gamma) (con2prim recovers it from tau + D by
    cancellation); B^k against |B|. The bound is tol * max(1, kappa) with kappa the cell's
    con2prim condition number, measured on the oracle by perturbing its conserved state;
  * backward: the CUDA primitives must reproduce the CUDA conserved state (prim->cons of the oracle)
    to tol under the same U scales.
Cells whose status bits differ between the two sides are excluded and counted. Cells where a
floor or the Lorentz-factor cap fired hold unphysical pre-floor states whose values are set by
roundoff; they are compared separately.

The characteristic speeds of the Riemann solver (Sec. 3.1; Valencia fast-speed formula) are formed on
both sides from 1 - v^2 = 1/W^2 and 1 - c^2 = (1 - vA^2)(1 - cs^2), not by the differences whose rounding
W^2 would amplify next to ultra-relativistic cells, so the conserved-state bound is the flat tolerance
everywhere, capped cells' neighbours included.
"""
import numpy as np


def _vnorm(a):
    return np.sqrt(np.sum(a * a, axis=0))


def _nbr_max(a):
    """Max over each cell and its six face neighbours (edges clamped)."""
    out = a.copy()
    for ax in range(3):
        lo = np.concatenate([np.take(a, [0], axis=ax), np.take(a, range(a.shape[ax] - 1), axis=ax)], axis=ax)
        hi = np.concatenate([np.take(a, range(1, a.shape[ax]), axis=ax), np.take(a, [a.shape[ax] - 1], axis=ax)], axis=ax)
        out = np.maximum(out, np.maximum(lo, hi))
    return out


def cons_scales(Ub):
    D = np.abs(Ub[0])
    E = np.maximum(np.abs(Ub[4] + Ub[0]), _vnorm(Ub[1:4]))
    B = _vnorm(Ub[5:8])
    sc = np.empty_like(Ub)
    sc[0] = np.maximum(_nbr_max(D), 1e-3 * D.max())
    sc[1:5] = np.maximum(_nbr_max(E), 1e-3 * E.max())[None]
    sc[5:8] = np.maximum(_nbr_max(B), 1e-3 * B.max() + 1e-300)[None]
    return np.maximum(sc, 1e-300)




def rel_err_cons(a, b):
    return np.abs(a - b) / cons_scales(b)


def rel_err_prims(Pa, Pb, Ub, sqrtgam, ng):
    """Errors of interior primitives; Ub is the (reference) conserved state of the same cells."""
    sl = (slice(None),) + tuple(slice(ng, -ng) for _ in range(3))
    a, b = Pa[sl], Pb[sl]
    out = np.zeros_like(a)
    rs = np.maximum(np.abs(b[0]), 1e-3 * np.abs(b[0]).max())
    out[0] = np.abs(a[0] - b[0]) / rs
    us = np.maximum(_vnorm(b[1:4]), 1.0)
    out[1:4] = np.abs(a[1:4] - b[1:4]) / us[None]
    escale = np.abs(Ub[4] + Ub[0]) / sqrtgam
    out[4] = np.abs(a[4] - b[4]) / np.maximum(escale, 1e-300)
    bs = np.maximum(_vnorm(b[5:8]), 1e-3 * _vnorm(b[5:8]).max() + 1e-300)
    out[5:8] = np.abs(a[5:8] - b[5:8]) / bs[None]
    return out


def l1_rel(a, b):
    """Per-variable L1 error sum|a - b| / sum|b|."""
    return np.array([np.abs(a[v] - b[v]).sum() / max(np.abs(b[v]).sum(), 1e-300) for v in range(a.shape[0])])


def interior_sqrtgam(orc, p, s):
    x = [s.cell_centres(d, ghosts=False) for d in range(3)]
    Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    return orc.geom_points(p, np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1))["sqrtgam"].reshape(X.shape)


def interior_points(s):
    x = [s.cell_centres(d, ghosts=False) for d in range(3)]
    Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)


def c2p_condition(orc, p, xyz, U, sg, rel=1e-9, seed=0, ndir=3):
    """Per-cell con2prim condition number: the largest scaled primitive change over `ndir` random sign
    perturbations of relative size `rel` of the conserved state, divided by `rel`."""
    Un = U.reshape(8, -1).T.copy()
    P0, _, _ = orc.c2p_points(p, xyz, Un, floors=False)
    shp = U.shape[1:]
    inner = (slice(None),) + (slice(1, -1),) * 3
    b = np.zeros((8,) + tuple(d + 2 for d in shp))
    b[inner] = P0.T.reshape((8,) + shp)
    rng = np.random.default_rng(seed)
    kappa = np.zeros(shp)
    for _ in range(ndir):
        r = rng.choice([-1.0, 1.0], size=Un.shape)
        P1, _, _ = orc.c2p_points(p, xyz, Un * (1.0 + rel * r), floors=False)
        a = np.zeros_like(b)
        a[inner] = P1.T.reshape((8,) + shp)
        kappa = np.maximum(kappa, np.max(rel_err_prims(a, b, U, sg, 1), axis=0) / rel)
    return kappa


def interior_faces(s, Bf):
    """The faces a stage advances, flattened: component d over face indices [0, n_d] along d and the
    interior cells along the other two directions."""
    ng = s.ng
    nx, ny, nz = s.n
    out = []
    for d, ax in ((0, 2), (1, 1), (2, 0)):
        sl = [slice(ng, ng + nz), slice(ng, ng + ny), slice(ng, ng + nx)]
        sl[ax] = slice(sl[ax].start, sl[ax].stop + 1)
        out.append(Bf[d][tuple(sl)].ravel())
    return np.concatenate(out)


def compare_stage(orc, s, p, P_in, U0, U_in, g0, g1, beta, dt, P_out, U_out, st_out, sg=None, faces=None):
    """Oracle stage from (P_in, U0, U_in) against the CUDA outputs; returns the worst scaled errors.

    U:        CUDA conserved state against the oracle stage (neighbour-scaled, see module docstring);
    P:        CUDA primitives against the oracle's con2prim of the CUDA conserved state, divided by
              max(1, kappa) -- the con2prim parity, separated from the update's;
    backward: oracle prim->cons of the CUDA primitives against the CUDA conserved state.
    faces:    face-centred CT: (Bf0, Bf_in, Bf_out), the step-start, input and CUDA output faces; adds
              "Bf", the largest difference of the advanced faces relative to the largest face field.
    """
    Po = P_in.copy()
    if faces is None:
        r = orc.stage(p, Po, U0, U_in, g0, g1, beta, dt)
    else:
        Bf0, Bf_in, Bf_out = faces
        r = orc.stage_face_ct(p, Po, Bf0, Bf_in.copy(), U0, U_in, g0, g1, beta, dt)
    ok = st_out == r["status"]
    if sg is None:
        sg = interior_sqrtgam(orc, p, s)
    xyz = interior_points(s)
    plain = ok & (r["status"] == 0)
    floored = ok & (r["status"] != 0)
    ng = s.ng
    eu = rel_err_cons(U_out, r["U"])
    inner = (slice(None),) + (slice(ng, -ng),) * 3
    Pc, stc, _ = orc.c2p_points(p, xyz, U_out.reshape(8, -1).T.copy(), floors=True)
    Pref = np.zeros_like(P_out)
    Pref[inner] = Pc.T.reshape(U_out.shape)
    ep = rel_err_prims(P_out, Pref, U_out, sg, ng)
    kappa = c2p_condition(orc, p, xyz, U_out, sg)
    epk = ep / np.maximum(1.0, kappa)[None]
    Pin = P_out[inner].reshape(8, -1).T.copy()
    Ub = orc.prim2con_points(p, xyz, Pin)["U"].T.reshape(U_out.shape)
    eb = rel_err_cons(Ub, U_out)
    ep_stage = rel_err_prims(P_out, Po, r["U"], sg, ng)
    mx = lambda a, m: float(a[:, m].max()) if m.any() else 0.0
    extra = {}
    if faces is not None:
        ref = interior_faces(s, r["Bf"])
        extra["Bf"] = float(np.abs(interior_faces(s, faces[2]) - ref).max() / max(np.abs(ref).max(), 1e-300))
    return {**extra,
        "dt": r["dt"],
        "mismatch": 1.0 - ok.mean(),
        "floored_frac": float(np.mean(r["status"] != 0)),
        "U": mx(eu, plain),
        "P": mx(epk, plain),
        "kappa_max": float(kappa[plain].max()) if plain.any() else 0.0,
        "backward": mx(eb, plain),
        "P_vs_stage": mx(ep_stage, plain),
        "U_floored": mx(eu, floored),
        "P_floored": mx(ep_stage, floored),
    }
