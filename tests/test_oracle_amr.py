"""Pins of the two-level mesh oracle (oracle/amr.py): ghost exchange between levels (restriction and
prolongation of the primitives), refluxing at coarse-fine faces, one time step for both levels.

Fixed by the mathematics or by the single-block oracle, not by amr.py's own formulas:
* a uniform state is a fixed point of the mesh stage;
* on primitives linear in the coordinates every ghost the exchange fills equals the linear function at
  its centre (copies, the mean of 8 children and the limited linear prolongation are all exact there);
* prolongation conserves: the 8 fine ghosts of each coarse cell average to that cell; and it is limited:
  no fine ghost leaves the range of its coarse cell and that cell's 6 face neighbours (per-direction
  minmod slopes add up to at most 3/4 of the distance to either end of that range);
* the periodic mesh conserves every variable (sum of cell volume x densitized state) to roundoff, and
  does not without refluxing;
* a mesh of one level everywhere (all roots, or all their children) is the single large block, bit for bit;
* the state stays consistent: every leaf's primitives are the con2prim of its conserved state;
* a passive scalar on the mesh: the sum of sqrt(gamma) D X is conserved to roundoff (and is not without
  the scalar's refluxing), X = DX / D on every leaf, and a uniform X stays uniform across the levels;
* a fast magnetosonic wave on a partly refined mesh ends with an error between those of the coarse and
  the fine uniform grids.
``test_planted_mistakes_fail_a_pin`` plants wrong prolongation offsets, an unlimited one-sided prolongation
slope, wrong restriction weights and child offsets, reflux signs, fine-face indices and weights, and a
missing con2prim after refluxing, each in a copy of amr.py.
"""
import importlib.util
import json
import math
import os
import sys
import tempfile

import numpy as np
import pytest

import oracle as orc
from oracle import amr
from paper_2410_09146_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fast_wave_minkowski.json")


def _mesh(periodic=True, refined=((1, 0, 0),), nb=(2, 2, 2), n=8, recon="plm_mc", riemann="hll"):
    root = I.Setup(n=(n, n, n), dx=(1 / 16, 1 / 16, 1 / 16), recon=recon, riemann=riemann, bc="fixed")
    return I.two_level_mesh(root, nb, list(refined), periodic)


def _interior(P, ng=4):
    return P[:, ng:-ng, ng:-ng, ng:-ng]


def test_leaf_map_tiles_the_mesh():
    m = _mesh(nb=(3, 2, 2), refined=[(1, 0, 0), (2, 1, 1)])
    lm = amr.leaf_map(m)
    assert lm.shape == (4, 4, 6) and m.nblocks == 10 + 16
    assert np.array_equal(np.bincount(lm.ravel()), [8] * 10 + [1] * 16)


def test_uniform_state_is_a_fixed_point(A=amr):
    m = _mesh()
    P0 = np.array([1.0, 0.2, -0.1, 0.05, 1.5, 0.3, 0.1, -0.2])
    Ps = [np.broadcast_to(P0[:, None, None, None], m.setup(b).prim_shape()).copy() for b in range(m.nblocks)]
    Us = A.mesh_prim2con(m, Ps)
    U1, st, _ = A.mesh_stage(m, Ps, None, Us, 0.0, 1.0, 1.0, 0.01)
    for b in range(m.nblocks):
        assert np.all(st[b] == 0)
        assert np.max(np.abs(U1[b] - Us[b])) < 1e-14
        assert np.max(np.abs(_interior(Ps[b]) - P0[:, None, None, None])) < 1e-13


def _linear_mesh_prims(m, seed=3):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(8, 4))
    out = []
    for b in range(m.nblocks):
        s = m.setup(b)
        x = [s.cell_centres(d) for d in range(3)]
        Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
        out.append(a[:, 0, None, None, None] + a[:, 1, None, None, None] * X + a[:, 2, None, None, None] * Y
                   + a[:, 3, None, None, None] * Z)
    return out


def linear_fill_error(A=amr):
    """Largest ghost error after the exchange on linear data (ghosts inside the mesh scrambled first)."""
    m = _mesh(periodic=False, nb=(3, 2, 2), refined=[(1, 0, 0), (2, 1, 1)])
    exact = _linear_mesh_prims(m)
    Ps = [e.copy() for e in exact]
    ng = m.root.ng
    for b, P in enumerate(Ps):
        mask = np.ones(P.shape[1:], bool)
        mask[ng:-ng, ng:-ng, ng:-ng] = False
        # scramble only the ghosts that lie inside the mesh (the others are the fixed outer boundary)
        s = m.setup(b)
        ext = m.extent()
        inside = np.ones(P.shape[1:], bool)
        for d, ax in ((0, 2), (1, 1), (2, 0)):
            x = s.cell_centres(d)
            ok = (x > m.root.x0[d]) & (x < m.root.x0[d] + ext[d])
            shape = [1, 1, 1]
            shape[ax] = -1
            inside &= ok.reshape(shape)
        P[:, mask & inside] = 1e3
    A.fill_ghosts(m, Ps)
    return max(np.max(np.abs(P - e)) for P, e in zip(Ps, exact))


def test_ghost_fill_exact_on_linear_data():
    assert linear_fill_error() < 1e-12


def prolongation_mean_error(A=amr):
    return _prolongation_errors(A)[0]


def prolongation_range_excess(A=amr):
    return _prolongation_errors(A)[1]


def _prolongation_errors(A=amr):
    """Over complete sets of 8 fine ghosts filled from a coarse cell: the largest |mean of the 8 - the coarse
    cell|, and the largest excursion of a fine ghost outside [min, max] of the coarse cell and its 6 face
    neighbours (a limited prolongation creates no new extrema)."""
    m = _mesh(periodic=True, refined=[(1, 0, 0)])
    Ps = I.two_level_prims(m, seed=4, amp=0.4)
    A.fill_ghosts(m, Ps)
    n, ng = m.root.n[0], m.root.ng
    lm = A.leaf_map(m)
    worst, excess = 0.0, -np.inf
    for b in range(m.nblocks):
        if m.levels[b] != 1:
            continue
        p = m.pos[b]
        # complete child pairs along each axis: ghost index pairs (-4,-3), (-2,-1), (n, n+1), (n+2, n+3)
        pairs = [-4, -2, n, n + 2]
        rng_ = [pairs + list(range(0, n, 2))] * 3
        for k0 in rng_[2]:
            for j0 in rng_[1]:
                for i0 in rng_[0]:
                    if 0 <= i0 < n and 0 <= j0 < n and 0 <= k0 < n:
                        continue
                    g = [(p[0] * n + i0) % (2 * m.nb[0] * n), (p[1] * n + j0) % (2 * m.nb[1] * n),
                         (p[2] * n + k0) % (2 * m.nb[2] * n)]
                    src = lm[g[2] // n, g[1] // n, g[0] // n]
                    if m.levels[src] != 0:
                        continue
                    ps = m.pos[src]
                    c = [g[d] // 2 - ps[d] * n + ng for d in range(3)]
                    kids = Ps[b][:, k0 + ng:k0 + ng + 2, j0 + ng:j0 + ng + 2, i0 + ng:i0 + ng + 2].reshape(8, 8)
                    C = Ps[src]
                    worst = max(worst, np.max(np.abs(kids.mean(1) - C[:, c[2], c[1], c[0]])))
                    nbrs = [C[:, c[2], c[1], c[0]]]
                    for e in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
                        for sg in (1, -1):
                            nbrs.append(C[:, c[2] + sg * e[2], c[1] + sg * e[1], c[0] + sg * e[0]])
                    nbrs = np.stack(nbrs, 1)
                    lo, hi = nbrs.min(1)[:, None], nbrs.max(1)[:, None]
                    excess = max(excess, float(np.max(np.maximum(kids - hi, lo - kids))))
    return worst, excess


def test_prolongation_conserves_the_coarse_value_and_creates_no_extrema():
    mean_err, excess = _prolongation_errors()
    assert mean_err < 1e-14
    assert excess <= 1e-15 and excess > -np.inf


def _two_steps(m, A=amr, dt=0.02, seed=8):
    Ps = I.two_level_prims(m, seed=seed)
    Us = A.mesh_prim2con(m, Ps)
    t0 = A.mesh_totals(m, Us)
    scale = sum(np.abs(U).reshape(8, -1).sum(1) * np.prod(m.setup(b).dx) for b, U in enumerate(Us))
    for _ in range(2):
        U1, st, _ = A.mesh_stage(m, Ps, None, Us, 0.0, 1.0, 1.0, dt)
        Us, st, _ = A.mesh_stage(m, Ps, Us, U1, 0.5, 0.5, 0.5, dt)
        assert all(np.all(s == 0) for s in st)
    return Ps, Us, np.abs(A.mesh_totals(m, Us) - t0) / scale


def conservation_error(A=amr):
    m = _mesh(periodic=True, nb=(2, 2, 2), refined=[(1, 0, 0), (0, 1, 1)])
    return _two_steps(m, A)[2].max()


def test_periodic_mesh_conserves_every_variable():
    assert conservation_error() < 1e-14


def test_without_refluxing_the_mesh_does_not_conserve(monkeypatch):
    monkeypatch.setattr(amr, "_reflux", lambda mesh, lm, Fu: [dict() for _ in range(mesh.nblocks)])
    assert conservation_error() > 1e-7


def consistency_error(A=amr):
    """Largest |P - con2prim(U)| over every leaf after two steps (relative to the variable's scale)."""
    m = _mesh(periodic=True, refined=[(1, 0, 0)])
    Ps, Us, _ = _two_steps(m, A)
    worst = 0.0
    for b in range(m.nblocks):
        s = m.setup(b)
        x = [s.cell_centres(d, ghosts=False) for d in range(3)]
        Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
        xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
        _, P, _ = orc.finish_points(orc.params(s), xyz, Us[b].reshape(8, -1).T)
        worst = max(worst, np.max(np.abs(P.T - _interior(Ps[b]).reshape(8, -1))))
    return worst


def test_state_stays_consistent():
    assert consistency_error() < 1e-12


@pytest.mark.parametrize("level", [0, 1])
def test_one_level_everywhere_is_the_large_block(level):
    nb = (2, 2, 1)
    refined = [(x, y, z) for z in range(nb[2]) for y in range(nb[1]) for x in range(nb[0])] if level else []
    m = _mesh(periodic=True, nb=nb, refined=refined, recon="weno5z_aoah")
    Ps = I.two_level_prims(m, seed=2)
    n = m.root.n[0]
    f = 2 ** level
    big = I.Setup(n=(nb[0] * n * f, nb[1] * n * f, nb[2] * n * f), dx=m.setup(m.nblocks - 1).dx, recon="weno5z_aoah",
                  riemann="hll", bc="periodic")
    PB = np.zeros(big.prim_shape())
    ng = big.ng
    for b in range(m.nblocks):
        p = m.pos[b]
        PB[:, ng + p[2] * n:ng + (p[2] + 1) * n, ng + p[1] * n:ng + (p[1] + 1) * n, ng + p[0] * n:ng + (p[0] + 1) * n] = \
            _interior(Ps[b])
    pb = orc.params(big)
    UB = orc.prim2con_grid(pb, PB)
    Us = amr.mesh_prim2con(m, Ps)
    dt = 0.01
    U1B = orc.stage(pb, PB, None, UB, 0.0, 1.0, 1.0, dt)["U"]
    U2B = orc.stage(pb, PB, UB, U1B, 0.5, 0.5, 0.5, dt)["U"]
    U1, _, _ = amr.mesh_stage(m, Ps, None, Us, 0.0, 1.0, 1.0, dt)
    U2, _, _ = amr.mesh_stage(m, Ps, Us, U1, 0.5, 0.5, 0.5, dt)
    for b in range(m.nblocks):
        p = m.pos[b]
        sl = (slice(None), slice(p[2] * n, (p[2] + 1) * n), slice(p[1] * n, (p[1] + 1) * n), slice(p[0] * n, (p[0] + 1) * n))
        assert np.array_equal(U2[b], U2B[sl])


def _wave_error(setup_or_mesh, gw, t_end, dt):
    amp = 1e-6
    if isinstance(setup_or_mesh, I.Setup):
        s = setup_or_mesh
        p = orc.params(s)
        P = I.linear_wave_prims(s, gw["background_prims"], gw["eigvec_prims"], amplitude=amp)
        P0 = P.copy()
        U = orc.prim2con_grid(p, P)
        for _ in range(int(round(t_end / dt))):
            U, st, _ = orc.rk2_step(p, P, U, dt)
        exact = 2.0 * gw["background_prims"][0] - _interior(P0)[0]  # half a period: the mode inverted
        return np.mean(np.abs(_interior(P)[0] - exact)) / amp
    m = setup_or_mesh
    Ps = I.two_level_wave_prims(m, gw["background_prims"], gw["eigvec_prims"], amp)
    P0 = [P.copy() for P in Ps]
    Us = amr.mesh_prim2con(m, Ps)
    for _ in range(int(round(t_end / dt))):
        U1, st, _ = amr.mesh_stage(m, Ps, None, Us, 0.0, 1.0, 1.0, dt)
        Us, st, _ = amr.mesh_stage(m, Ps, Us, U1, 0.5, 0.5, 0.5, dt)
    err = vol = 0.0
    for b in range(m.nblocks):
        dv = float(np.prod(m.setup(b).dx))
        e = np.abs(_interior(Ps[b])[0] - (2.0 * gw["background_prims"][0] - _interior(P0[b])[0]))
        err += e.sum() * dv
        vol += e.size * dv
    return err / vol / amp


def test_fast_wave_on_a_partly_refined_mesh():
    gw = json.load(open(GOLDEN))
    t_end = 0.5 / gw["fast_speed"]
    lam = max(abs(v) for v in gw["all_speeds"])
    steps = int(math.ceil(t_end / (0.4 * (1 / 64) / lam)))
    dt = t_end / steps
    root = I.Setup(n=(8, 4, 4), dx=(1 / 32, 1 / 32, 1 / 32), recon="plm_mc", riemann="hll", bc="fixed")
    m = I.two_level_mesh(root, (4, 1, 1), [(1, 0, 0)], True)
    coarse = I.Setup(n=(32, 4, 4), dx=(1 / 32,) * 3, recon="plm_mc", riemann="hll", bc="periodic")
    fine = I.Setup(n=(64, 8, 8), dx=(1 / 64,) * 3, recon="plm_mc", riemann="hll", bc="periodic")
    ec, e2, ef = (_wave_error(x, gw, t_end, dt) for x in (coarse, m, fine))
    assert ef < e2 < ec, (ef, e2, ec)


_MUTANTS = {
    "prolongation offset sign": ("np.where(glob[d][m] % 2 == 1, 0.25, -0.25)", "np.where(glob[d][m] % 2 == 1, -0.25, 0.25)"),
    "restriction weight": ("Ps[b][dsel] = acc / 8.0", "Ps[b][dsel] = acc / 7.0"),
    "restriction child offset": ("f0 = [2 * glob[d][m] - ps[d] * n[d] + ng for d in range(3)]",
                                 "f0 = [2 * glob[d][m] - ps[d] * n[d] + ng - 1 for d in range(3)]"),
    "prolongation one-sided slope": ("val = val + off[d] * _minmod(up - pc, pc - dn)", "val = val + off[d] * (up - pc)"),
    "reflux sign": ("dU = side * (Fc - Ff / 4.0) / s.dx[d]", "dU = -side * (Fc - Ff / 4.0) / s.dx[d]"),
    "reflux fine face index": ("ff[d] = 0 if side > 0 else n[d]", "ff[d] = n[d] if side > 0 else 0"),
    "reflux fine weight": ("dU = side * (Fc - Ff / 4.0) / s.dx[d]", "dU = side * (Fc - Ff / 2.0) / s.dx[d]"),
    "no con2prim after refluxing": ("Ps[b][:, k + ng, j + ng, i + ng] = P[q]", "pass"),
}


def _planted(tmp, k, a, b):
    with open(amr.__file__) as f:
        src = f.read()
    assert src.count(a) == 1, a
    path = os.path.join(tmp, f"amr_planted_{k}.py")
    with open(path, "w") as f:
        f.write(src.replace(a, b))
    name = f"oracle.amr_planted_{k}"
    spec = importlib.util.spec_from_file_location(name, path)
    mod = importlib.util.module_from_spec(spec)
    sys.modules[name] = mod
    spec.loader.exec_module(mod)
    return mod


def test_planted_mistakes_fail_a_pin():
    missed = []
    with tempfile.TemporaryDirectory() as tmp:
        for k, (name, (a, b)) in enumerate(_MUTANTS.items()):
            A = _planted(tmp, k, a, b)
            caught = (linear_fill_error(A) >= 1e-12 or prolongation_mean_error(A) >= 1e-14
                      or prolongation_range_excess(A) > 1e-15
                      or conservation_error(A) >= 1e-14 or consistency_error(A) >= 1e-12)
            if not caught:
                missed.append(name)
    assert not missed, missed


def _scalar_mesh_steps(m, A=amr, dt=0.02, X0=None, steps=2):
    Ps = I.two_level_prims(m, seed=8)
    Us = A.mesh_prim2con(m, Ps)
    rng = np.random.default_rng(12)
    Xs = [(np.full(m.setup(b).prim_shape()[1:], X0) if X0 is not None
           else rng.uniform(0.0, 1.0, m.setup(b).prim_shape()[1:])) for b in range(m.nblocks)]
    DXs = [Us[b][0] * _interior(Xs[b][None])[0] for b in range(m.nblocks)]
    t0 = sum(DX.sum() * np.prod(m.setup(b).dx) for b, DX in enumerate(DXs))
    for _ in range(steps):
        U1, st, _, DX1 = A.mesh_stage(m, Ps, None, Us, 0.0, 1.0, 1.0, dt, Xs, None, DXs)
        Us, st, _, DXs = A.mesh_stage(m, Ps, Us, U1, 0.5, 0.5, 0.5, dt, Xs, DXs, DX1)
    t1 = sum(DX.sum() * np.prod(m.setup(b).dx) for b, DX in enumerate(DXs))
    scale = sum(np.abs(DX).sum() * np.prod(m.setup(b).dx) for b, DX in enumerate(DXs))
    return Ps, Us, Xs, DXs, abs(t1 - t0) / scale


def test_mesh_scalar_is_conserved_and_consistent():
    m = _mesh(periodic=True, nb=(2, 2, 2), refined=[(1, 0, 0), (0, 1, 1)])
    Ps, Us, Xs, DXs, err = _scalar_mesh_steps(m)
    assert err < 1e-14
    for b in range(m.nblocks):
        np.testing.assert_allclose(_interior(Xs[b][None])[0], DXs[b] / Us[b][0], rtol=1e-15)


def test_mesh_uniform_scalar_stays_uniform():
    m = _mesh(periodic=True, nb=(2, 2, 2), refined=[(1, 0, 0), (0, 1, 1)])
    Ps, Us, Xs, DXs, _ = _scalar_mesh_steps(m, X0=0.3)
    assert max(np.max(np.abs(_interior(X[None]) - 0.3)) for X in Xs) < 1e-15


def test_mesh_scalar_needs_its_refluxing(monkeypatch):
    m = _mesh(periodic=True, nb=(2, 2, 2), refined=[(1, 0, 0), (0, 1, 1)])
    orig = amr._reflux
    monkeypatch.setattr(amr, "_reflux", lambda mesh, lm, Fu: orig(mesh, lm, Fu) if Fu[0][0].shape[0] == 8
                        else [dict() for _ in range(mesh.nblocks)])
    assert _scalar_mesh_steps(m)[-1] > 1e-8
