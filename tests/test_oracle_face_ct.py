"""Pins of the oracle's face-centred upwind constrained transport (the stage with the field on the faces).

The scheme (oracle ``stage_impl``): the normal field of every face comes from the face array, edge EMFs
are the upwind "contact" interpolation of Gardiner & Stone (2005), faces advance by the discrete Stokes
theorem and the cell field is the mean of its faces. Each test pins a property the mathematics fixes,
independent of the oracle's own formulas:

* plane reduction: on a state that varies along one direction only, the face-CT update equals the plain
  finite-volume update with the same face fluxes (all 8 variables by their own flux divergence), which
  the upwind EMF reproduces exactly for such states (and Toth's averaged EMF does not);
* the face divergence keeps its initial (roundoff) value, on anisotropic cells and curved space;
* the normal-field flux of each face vanishes (both Riemann states share the face's normal field);
* a periodic run is equivariant under cyclic shifts (bitwise) and mirror reflections (to rounding);
* on smooth Kerr-Schild data the face-CT EMFs and fluxes approach Toth's at second order;
* the cell field derived from the faces maps back (through the pinned prim->cons map) to the face mean;
* an advected field loop never gains magnetic energy (the upwind choice is dissipative).

``test_planted_mistakes_fail_a_pin`` compiles copies of the oracle with one plausible mistake each
(a sign, an index, a missing sqrt(gamma), the upwind direction, a missing ghost fill) and checks that
every copy fails at least one of these pins.
"""
import importlib.util
import os
import tempfile

import numpy as np
import pytest

import oracle as orc
from paper_2410_09146_gb300 import inputs as I


def _ready(o, s, P, Bf):
    p = o.params(s)
    o.face_b_to_cells(p, Bf, P)
    return p, o.prim2con_grid(p, P)


def _interior(s, A):
    ng = s.ng
    nx, ny, nz = s.n
    return A[..., ng:ng + nz, ng:ng + ny, ng:ng + nx]


def _flux_divergence(s, F):
    """Sum over directions of (F(upper face) - F(lower face)) / dx of every interior cell, [8][nz][ny][nx]."""
    ng = s.ng
    nx, ny, nz = s.n
    sl = (slice(ng, ng + nz), slice(ng, ng + ny), slice(ng, ng + nx))
    out = np.zeros((8, nz, ny, nx))
    for e, ax in ((0, 2), (1, 1), (2, 0)):
        up = list(sl)
        up[ax] = slice(sl[ax].start + 1, sl[ax].stop + 1)
        out += (F[e][(slice(None),) + tuple(up)] - F[e][(slice(None),) + sl]) / s.dx[e]
    return out


# ----------------------------------------------------------------------------- pin functions
# Each returns a number whose bound is stated in the test that calls it (used again on the planted copies).
def plane_reduction(o, d, recon="weno5z_aoah", riemann="hll"):
    n = [2, 2, 2]
    n[d] = 16
    s = I.Setup(n=tuple(n), dx=(1 / 16,) * 3, recon=recon, riemann=riemann)
    P, Bf = I.plane_random_prims(s, d, seed=7 + d)
    p, U = _ready(o, s, P, Bf)
    dt = 0.2 / 16
    plain = o.stage(p, P.copy(), None, U, 0.0, 1.0, 1.0, dt, debug=True)
    Uplain = U - dt * _flux_divergence(s, plain["F"])
    r = o.stage_face_ct(p, P.copy(), None, Bf.copy(), None, U, 0.0, 1.0, 1.0, dt)
    scale = np.abs(U).max(axis=(1, 2, 3))[:, None, None, None] + 1e-300
    return float(np.max(np.abs(r["U"] - Uplain) / scale)), float(np.max(np.abs(plain["U"] - Uplain) / scale))


def divergence_growth(o):
    """Max over two blocks of |face divergence| x dx / max|Bf| after one RK2 step."""
    worst = 0.0
    s1 = I.kerr_schild_setup(8, recon="weno5z_aoah", riemann="hll", lo=4.0, hi=12.0)
    s2 = I.Setup(n=(8, 6, 5), dx=(1 / 8, 1 / 6, 1 / 5), recon="plm_mc", riemann="llf")
    for s, seed in ((s1, 3), (s2, 4)):
        P, Bf = I.kerr_schild_random_prims(s, seed=seed, kmax=1, faces=True)
        p, U = _ready(o, s, P, Bf)
        U, Bf, st, dt = o.rk2_step_face_ct(p, P, Bf, U)
        worst = max(worst, float(np.abs(o.face_divergence(p, Bf)).max() * min(s.dx) / np.abs(Bf).max()))
    return worst


def normal_flux(o):
    """Max |F^d of B^d| over all faces relative to the largest flux."""
    s = I.kerr_schild_setup(8, recon="weno5z_aoah", riemann="hll", lo=4.0, hi=12.0)
    P, Bf = I.kerr_schild_random_prims(s, seed=3, kmax=1, faces=True)
    p, U = _ready(o, s, P, Bf)
    r = o.stage_face_ct(p, P, None, Bf, None, U, 0.0, 1.0, 1.0, 0.0, debug=True)
    return max(float(np.abs(r["F"][d][5 + d]).max()) for d in range(3)) / float(np.abs(r["F"]).max())


def _periodic_state(o, seed=4):
    s = I.Setup(n=(8, 6, 5), dx=(1 / 8, 1 / 6, 1 / 5), recon="weno5z_aoah", riemann="hll")
    P, Bf = I.kerr_schild_random_prims(s, seed=seed, kmax=1, faces=True)
    p = o.params(s)
    o.face_b_to_cells(p, Bf, P)
    return s, p, P, Bf


def _run(o, p, P, Bf, steps):
    U = o.prim2con_grid(p, P)
    for _ in range(steps):
        U, Bf, st, dt = o.rk2_step_face_ct(p, P, Bf, U)
    return U


def shift_equivariance(o):
    s, p, P, Bf = _periodic_state(o)
    U1 = _run(o, p, P.copy(), Bf.copy(), 2)
    sh = (3, 1, 2)  # z, y, x
    ng = s.ng
    Ps, Bs = P.copy(), Bf.copy()
    Ps[:, ng:-ng, ng:-ng, ng:-ng] = np.roll(_interior(s, P), sh, axis=(1, 2, 3))
    Bs[:, ng:-ng, ng:-ng, ng:-ng] = np.roll(_interior(s, Bf), sh, axis=(1, 2, 3))
    o.face_b_to_cells(p, Bs, Ps)
    U2 = _run(o, p, Ps, Bs, 2)
    return float(np.max(np.abs(np.roll(U1, sh, axis=(1, 2, 3)) - U2)) / np.abs(U1).max())


def mirror_equivariance(o, d):
    """Reflect direction d (x_d -> -x_d: W v^d, B^d change sign, faces swap sides) and compare."""
    s, p, P, Bf = _periodic_state(o)
    U1 = _run(o, p, P.copy(), Bf.copy(), 1)
    ax = 3 - d
    Pm = np.flip(P, axis=ax).copy()
    Pm[1 + d] *= -1
    Pm[5 + d] *= -1
    Bm = np.flip(Bf, axis=ax).copy()
    Bm[d] = -np.roll(Bm[d], 1, axis=ax - 1)  # the lower d-face of a mirrored cell is its old upper face
    o.face_b_to_cells(p, Bm, Pm)
    U2 = np.flip(_run(o, p, Pm, Bm, 1), axis=ax).copy()
    U2[1 + d] *= -1
    U2[5 + d] *= -1
    return float(np.max(np.abs(U1 - U2)) / np.abs(U1).max())


def smooth_toth_distance(o, n):
    """Mean |EMF difference| / mean |EMF| and mean |hydro flux difference| / mean |flux| between face-CT
    and Toth's flux-CT on a smooth Kerr-Schild block of n^3 cells."""
    s = I.kerr_schild_setup(n, recon="weno5z_aoah", riemann="hll", lo=6.0, hi=10.0)
    P, Bf = I.smooth_random_prims(s, seed=11)
    p, U = _ready(o, s, P, Bf)
    dt = 0.1 * s.dx[0]
    r1 = o.stage(p, P.copy(), None, U, 0.0, 1.0, 1.0, dt, debug=True)
    r2 = o.stage_face_ct(p, P.copy(), None, Bf.copy(), None, U, 0.0, 1.0, 1.0, dt, debug=True)
    E1, E2 = _interior(s, r1["E"]), _interior(s, r2["E"])
    F1, F2 = _interior(s, r1["F"][:, :5]), _interior(s, r2["F"][:, :5])
    return float(np.abs(E1 - E2).mean() / np.abs(E1).mean()), float(np.abs(F1 - F2).mean() / np.abs(F1).mean())


def field_loop_energy(o, steps=40):
    """(largest step-to-step increase of sum B~^2, final / initial) of the advected field loop."""
    s = I.field_loop_setup(32)
    P, Bf = I.field_loop_prims(s)
    p, U = _ready(o, s, P, Bf)
    e = [float(np.sum(U[5:8] ** 2))]
    for _ in range(steps):
        U, Bf, st, dt = o.rk2_step_face_ct(p, P, Bf, U)
        e.append(float(np.sum(U[5:8] ** 2)))
    return float(np.max(np.diff(e)) / e[0]), e[-1] / e[0]


def cells_from_faces(o):
    s = I.kerr_schild_setup(6, lo=4.0, hi=10.0)
    P, Bf = I.kerr_schild_random_prims(s, seed=2, kmax=1, faces=True)
    p, U = _ready(o, s, P, Bf)
    ng = s.ng
    worst = 0.0
    for d, ax in ((0, 2), (1, 1), (2, 0)):
        lo = [slice(ng, -ng)] * 3
        up = list(lo)
        up[ax] = slice(ng + 1, -ng + 1 if ng > 1 else None)
        mean = 0.5 * (Bf[d][tuple(lo)] + Bf[d][tuple(up)])
        worst = max(worst, float(np.max(np.abs(U[5 + d] - mean)) / np.abs(mean).max()))
    return worst


# ----------------------------------------------------------------------------- tests
@pytest.mark.parametrize("recon,riemann", [("weno5z_aoah", "hll"), ("plm_mc", "llf"), ("constant", "hll")])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_plane_state_reduces_to_plain_fv(d, recon, riemann):
    err, toth = plane_reduction(orc, d, recon, riemann)
    assert err < 1e-14
    assert toth > 1e-3  # Toth's averaged EMFs do not reduce: the test tells the two schemes apart


def test_face_divergence_is_kept():
    assert divergence_growth(orc) < 1e-14


def test_normal_field_flux_vanishes():
    assert normal_flux(orc) < 1e-14


def test_periodic_run_is_shift_equivariant():
    assert shift_equivariance(orc) == 0.0


@pytest.mark.parametrize("d", [0, 1, 2])
def test_periodic_run_is_mirror_equivariant(d):
    assert mirror_equivariance(orc, d) < 1e-12


def test_second_order_agreement_with_flux_ct_on_smooth_data():
    e8, f8 = smooth_toth_distance(orc, 8)
    e16, f16 = smooth_toth_distance(orc, 16)
    assert e8 / e16 > 3.2 and f8 / f16 > 3.2


def test_cell_field_is_face_mean():
    assert cells_from_faces(orc) < 1e-14


def test_field_loop_never_gains_energy():
    incr, ratio = field_loop_energy(orc)
    assert incr < 0.0
    assert 0.5 < ratio < 1.0


# ----------------------------------------------------------------------------- planted mistakes
_MUTANTS = {
    "upwind direction reversed": ("return m > 0.0 ? lo_cell : (m < 0.0 ? hi_cell",
                                  "return m < 0.0 ? lo_cell : (m > 0.0 ? hi_cell"),
    "no upwind correction": ("0.25 * (xb_lo - xb_hi) + 0.25 * (xa_lo - xa_hi);", "0.0;"),
    "wrong cell in a b half-face": ("OB(fa - 1) - Oc(fa - 1, fb - 1), OB(fa) - Oc(fa, fb - 1));",
                                    "OB(fa - 1) - Oc(fa - 1, fb), OB(fa) - Oc(fa, fb - 1));"),
    "wrong face in an a half-face": ("Oc(fa, fb - 1) - OA(fb - 1), Oc(fa, fb) - OA(fb));",
                                     "Oc(fa, fb - 1) - OA(fb), Oc(fa, fb) - OA(fb));"),
    "upwind by the wrong b-face": ("const double xa_lo = pick(DB(fa - 1)", "const double xa_lo = pick(DB(fa)"),
    "upwind by the wrong a-face": ("const double xb_hi = pick(DA(fb),", "const double xb_hi = pick(DA(fb - 1),"),
    "a-face EMF sign": ("auto OA = [&](int ib) { return -F[", "auto OA = [&](int ib) { return F["),
    "cell EMF sign": ("G.sqrtgam * (Fl.Bcon[a] * Fl.vt[b] - Fl.Bcon[b] * Fl.vt[a]);",
                      "G.sqrtgam * (Fl.Bcon[b] * Fl.vt[a] - Fl.Bcon[a] * Fl.vt[b]);"),
    "cell EMF without sqrt(gamma)": ("G.sqrtgam * (Fl.Bcon[a] * Fl.vt[b]", "(Fl.Bcon[a] * Fl.vt[b]"),
    "Stokes sign (x faces)": ("/ p->dx[1] + (Ev(1, i, j, k + 1) - Ev(1, i, j, k)) / p->dx[2];\n            else if",
                              "/ p->dx[1] - (Ev(1, i, j, k + 1) - Ev(1, i, j, k)) / p->dx[2];\n            else if"),
    "Stokes spacing (y faces)": ("curl = (Ev(2, i + 1, j, k) - Ev(2, i, j, k)) / p->dx[0]",
                                 "curl = (Ev(2, i + 1, j, k) - Ev(2, i, j, k)) / p->dx[1]"),
    "Stokes index (z faces)": ("+ (Ev(0, i, j + 1, k) - Ev(0, i, j, k)) / p->dx[1];",
                               "+ (Ev(0, i + 1, j, k) - Ev(0, i, j, k)) / p->dx[1];"),
    "normal field on one side only": ("PL[5 + d] = bn;\n            PR[5 + d] = bn;", "PL[5 + d] = bn;"),
    "normal field without sqrt(gamma)": ("const double bn = Bfcur[d * gn + g.gi(i, j, k)] / G.sqrtgam;",
                                         "const double bn = Bfcur[d * gn + g.gi(i, j, k)];"),
    "cell field from one face": ("Un[5 + d] = 0.5 * (Bfnew[d * gn + gc] + Bfnew[d * gn + gc + st[d]]);",
                                 "Un[5 + d] = Bfnew[d * gn + gc];"),
    "RK weight of the step start dropped": ("Bfnew[f] = g0 * b0 + g1 * Bfcur[f] + beta * dt * curl;",
                                            "Bfnew[f] = g1 * Bfcur[f] + beta * dt * curl;"),
    "no periodic fill of the faces": ("if (face_ct) ghost_fill_faces_periodic(g, Bfcur);", ""),
    "cell field without sqrt(gamma)": (
        "P[(5 + d) * gn + gc] = 0.5 * (Bf[d * gn + gc] + Bf[d * gn + gc + st[d]]) / G.sqrtgam;",
        "P[(5 + d) * gn + gc] = 0.5 * (Bf[d * gn + gc] + Bf[d * gn + gc + st[d]]);"),
}


def _caught(o):
    """True as soon as one pin fails (cheapest first)."""
    for d in range(3):
        if plane_reduction(o, d)[0] >= 1e-14:
            return True
    if normal_flux(o) >= 1e-14 or cells_from_faces(o) >= 1e-14 or divergence_growth(o) >= 1e-14:
        return True
    if shift_equivariance(o) != 0.0:
        return True
    if any(mirror_equivariance(o, d) >= 1e-12 for d in range(3)):
        return True
    e8, f8 = smooth_toth_distance(o, 8)
    e16, f16 = smooth_toth_distance(o, 16)
    if not (e8 / e16 > 3.2 and f8 / f16 > 3.2):
        return True
    incr, ratio = field_loop_energy(o)
    return not (incr < 0.0 and 0.5 < ratio < 1.0)


def _oracle_copy(src, workdir, tag):
    """A separate instance of the oracle package built from the given C++ source."""
    d = os.path.join(workdir, tag)
    os.makedirs(d)
    path = os.path.join(d, "grmhd_oracle.cpp")
    with open(path, "w") as f:
        f.write(src)
    spec = importlib.util.spec_from_file_location(f"oracle_planted_{tag}", orc.__file__)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._SRC, mod._BUILD, mod._SO = path, d, os.path.join(d, "liboracle.so")
    return mod


def test_planted_mistakes_fail_a_pin():
    with open(orc._SRC) as f:
        src = f.read()
    missed = []
    with tempfile.TemporaryDirectory() as tmp:
        for k, (name, (a, b)) in enumerate(_MUTANTS.items()):
            assert src.count(a) == 1, name
            o = _oracle_copy(src.replace(a, b), tmp, f"m{k}")
            if not _caught(o):
                missed.append(name)
    assert not missed, f"planted mistakes no pin catches: {missed}"
