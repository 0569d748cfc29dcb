"""Two-level block meshes on the GPU (grmhd_batch_set_mesh): the two-pass ghost exchange between levels and
the refluxing of coarse cells at coarse-fine faces, against the two-level mesh oracle (oracle/amr.py,
pinned in tests/test_oracle_amr.py), through the C ABI.

* All-FP64 form: after two RK2 steps every conserved variable and primitive of every leaf within 1e-12 of
  the oracle's (relative to that variable's largest magnitude on the mesh; smooth moderate states, no
  floors): periodic Minkowski meshes (a refined root block; two refined roots meeting at an edge and a
  corner; PLM-MC and WENO5-Z-AOAH) and a Kerr-Schild mesh with fixed outer ghosts refined next to the
  hole. Status bits identical.
* The periodic mesh conserves every variable to roundoff on the device too.
* Replaying the stage as a CUDA graph gives the same bits.
* Mixed form: per-variable L1 of U and P against the oracle within 1e-6 (the mixed form's bound on
  smooth data).
* A mesh of root blocks only is the lattice exchange, bit for bit; bad meshes are refused.
* With a passive scalar (exchanged like a primitive, refluxed after its update): X and sqrt(gamma) D X of
  every leaf within 1e-12 of the oracle (FP64) and the sum of sqrt(gamma) D X conserved on a periodic mesh.
The time step is passed in (both sides take the same dt).
"""
import dataclasses

import numpy as np
import pytest

from paper_2410_09146_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_09146_gb300 import build
    build.build()
    from paper_2410_09146_gb300 import grmhd
    return grmhd


def _minkowski_mesh(refined, recon="plm_mc", nb=(2, 2, 2), n=8):
    root = I.Setup(n=(n, n, n), dx=(1 / 16, 1 / 16, 1 / 16), recon=recon, riemann="hll", bc="fixed")
    return I.two_level_mesh(root, nb, refined, True)


def _kerr_schild_mesh(recon="weno5z_aoah"):
    root = I.Setup(n=(8, 8, 8), x0=(2.0, 2.0, 2.0), dx=(0.5, 0.5, 0.5), metric="kerr_schild", spin=0.9, mass=1.0,
                   recon=recon, riemann="hll", bc="fixed")
    return I.two_level_mesh(root, (2, 2, 2), [(0, 0, 0)], False)


def _gpu(G, m, Ps, dt, steps, precision="fp64", graph=False, lattice=False):
    setups = [dataclasses.replace(m.setup(b), precision=precision) for b in range(m.nblocks)]
    bc = G.BatchContext(setups)
    for b in range(m.nblocks):
        bc.set_prims(b, Ps[b].copy())
    if lattice:
        bc.set_lattice(m.nb, m.periodic)
    else:
        bc.set_mesh(m.nb, m.periodic, m.levels, m.pos)
    if graph:
        bc.set_graph(True)
    for _ in range(steps):
        bc.stage(0.0, 1.0, 1.0, dt)
        bc.stage(0.5, 0.5, 0.5, dt)
    ng = m.root.ng
    U = [bc.get(b, G.GRMHD_GET_CONS) for b in range(m.nblocks)]
    P = [bc.get(b, G.GRMHD_GET_PRIMS)[:, ng:-ng, ng:-ng, ng:-ng] for b in range(m.nblocks)]
    st = [bc.get(b, G.GRMHD_GET_STATUS) for b in range(m.nblocks)]
    return U, P, st


def _oracle(m, Ps, dt, steps):
    from oracle import amr
    Ps = [P.copy() for P in Ps]
    Us = amr.mesh_prim2con(m, Ps)
    for _ in range(steps):
        U1, st, _ = amr.mesh_stage(m, Ps, None, Us, 0.0, 1.0, 1.0, dt)
        Us, st, _ = amr.mesh_stage(m, Ps, Us, U1, 0.5, 0.5, 0.5, dt)
    ng = m.root.ng
    return Us, [P[:, ng:-ng, ng:-ng, ng:-ng] for P in Ps], st


def _max_rel(A, B):
    """Largest |A - B| per variable over all leaves, relative to the variable's largest |B|."""
    diff = np.max([np.abs(a - b).reshape(8, -1).max(1) for a, b in zip(A, B)], axis=0)
    scale = np.max([np.abs(b).reshape(8, -1).max(1) for b in B], axis=0)
    return diff / np.maximum(scale, 1e-300)


CASES = [("one refined root, PLM-MC", lambda: _minkowski_mesh([(1, 0, 0)])),
         ("two refined roots, WENO5-Z-AOAH", lambda: _minkowski_mesh([(0, 0, 0), (1, 1, 1)], recon="weno5z_aoah")),
         ("Kerr-Schild, refined next to the hole", _kerr_schild_mesh)]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_fp64_mesh_matches_the_oracle(G, name, make):
    m = make()
    Ps = I.two_level_prims(m, seed=5)
    dt = 0.4 * min(m.setup(b).dx[0] for b in range(m.nblocks)) / 1.5
    U, P, st = _gpu(G, m, Ps, dt, 2)
    Uo, Po, sto = _oracle(m, Ps, dt, 2)
    for b in range(m.nblocks):
        assert np.array_equal(st[b], sto[b]), b
    eu, ep = _max_rel(U, Uo), _max_rel(P, Po)
    assert eu.max() < 1e-12 and ep.max() < 1e-12, (eu, ep)


def test_fp64_mesh_conserves_and_replays_as_a_graph(G):
    from oracle import amr
    m = _minkowski_mesh([(1, 0, 0), (0, 1, 1)])
    Ps = I.two_level_prims(m, seed=8)
    t0 = amr.mesh_totals(m, amr.mesh_prim2con(m, [P.copy() for P in Ps]))
    U, P, st = _gpu(G, m, Ps, 0.02, 2)
    scale = sum(np.abs(u).reshape(8, -1).sum(1) * np.prod(m.setup(b).dx) for b, u in enumerate(U))
    assert np.max(np.abs(amr.mesh_totals(m, U) - t0) / scale) < 1e-14
    Ug, Pg, stg = _gpu(G, m, Ps, 0.02, 2, graph=True)
    for b in range(m.nblocks):
        assert np.array_equal(U[b], Ug[b]) and np.array_equal(P[b], Pg[b])


@pytest.mark.parametrize("name,make", CASES[::2], ids=[c[0] for c in CASES[::2]])
def test_mixed_mesh_within_the_mixed_bound(G, name, make):
    from tests.parity import l1_rel
    m = make()
    Ps = I.two_level_prims(m, seed=5)
    dt = 0.4 * min(m.setup(b).dx[0] for b in range(m.nblocks)) / 1.5
    U, P, st = _gpu(G, m, Ps, dt, 2, precision="mixed")
    Uo, Po, _ = _oracle(m, Ps, dt, 2)
    lu = l1_rel(np.concatenate([u.reshape(8, -1) for u in U], 1), np.concatenate([u.reshape(8, -1) for u in Uo], 1))
    lp = l1_rel(np.concatenate([p.reshape(8, -1) for p in P], 1), np.concatenate([p.reshape(8, -1) for p in Po], 1))
    assert lu.max() < 1e-6 and lp.max() < 1e-6, (lu, lp)


def test_root_blocks_only_is_the_lattice(G):
    m = _minkowski_mesh([], recon="weno5z_aoah")
    Ps = I.two_level_prims(m, seed=3)
    a = _gpu(G, m, Ps, 0.02, 1)
    b = _gpu(G, m, Ps, 0.02, 1, lattice=True)
    for x, y in zip(a[0] + a[1], b[0] + b[1]):
        assert np.array_equal(x, y)


def test_mesh_refusals(G):
    m = _minkowski_mesh([(1, 0, 0)])
    bc = G.BatchContext([m.setup(b) for b in range(m.nblocks)])
    lv, ps = list(m.levels), [list(p) for p in m.pos]
    with pytest.raises(G.GrmhdError):
        bc.set_mesh((2, 2, 2), True, lv[:-1] + [0], ps)            # a fine block declared coarse: width
    bad = [list(p) for p in ps]
    bad[-1] = list(bad[-2])
    with pytest.raises(G.GrmhdError):
        bc.set_mesh((2, 2, 2), True, lv, bad)                      # two leaves on one spot
    with pytest.raises(G.GrmhdError):
        bc.set_mesh((3, 2, 2), True, lv, ps)                       # leaves do not cover the mesh
    bc.set_mesh((2, 2, 2), True, lv, ps)
    bc.set_mesh((0, 0, 0), True, lv, ps)                           # switched off
    odd = I.two_level_mesh(I.Setup(n=(6, 6, 5), dx=(0.1,) * 3, bc="fixed"), (1, 1, 1), [], True)
    bo = G.BatchContext([odd.setup(0)])
    with pytest.raises(G.GrmhdError):
        bo.set_mesh((1, 1, 1), True, odd.levels, odd.pos)


@pytest.mark.parametrize("name,make", [CASES[1], CASES[2]], ids=[CASES[1][0], CASES[2][0]])
def test_fp64_mesh_scalar_matches_the_oracle(G, name, make):
    from oracle import amr
    m = make()
    m.root = dataclasses.replace(m.root, scalar=True)
    Ps = I.two_level_prims(m, seed=5)
    rng = np.random.default_rng(6)
    Xs = [rng.uniform(0.2, 0.8, m.setup(b).prim_shape()[1:]) for b in range(m.nblocks)]
    dt = 0.4 * min(m.setup(b).dx[0] for b in range(m.nblocks)) / 1.5
    bc = G.BatchContext([m.setup(b) for b in range(m.nblocks)])
    for b in range(m.nblocks):
        bc.set_prims(b, Ps[b].copy())
        bc.set_scalar(b, Xs[b].copy())
    bc.set_mesh(m.nb, m.periodic, m.levels, m.pos)
    Po, Xo = [P.copy() for P in Ps], [X.copy() for X in Xs]
    Us = amr.mesh_prim2con(m, Po)
    ng = m.root.ng
    DXs = [Us[b][0] * Xo[b][ng:-ng, ng:-ng, ng:-ng] for b in range(m.nblocks)]
    t0 = sum(DX.sum() * np.prod(m.setup(b).dx) for b, DX in enumerate(DXs))
    for _ in range(2):
        bc.stage(0.0, 1.0, 1.0, dt)
        bc.stage(0.5, 0.5, 0.5, dt)
        U1, _, _, DX1 = amr.mesh_stage(m, Po, None, Us, 0.0, 1.0, 1.0, dt, Xo, None, DXs)
        Us, _, _, DXs = amr.mesh_stage(m, Po, Us, U1, 0.5, 0.5, 0.5, dt, Xo, DXs, DX1)
    Xg = [bc.get(b, G.GRMHD_GET_SCALAR)[ng:-ng, ng:-ng, ng:-ng] for b in range(m.nblocks)]
    DXg = [bc.get(b, G.GRMHD_GET_SCALAR_CONS) for b in range(m.nblocks)]
    ex = max(np.max(np.abs(a - b_[ng:-ng, ng:-ng, ng:-ng])) for a, b_ in zip(Xg, Xo)) / max(np.abs(X).max() for X in Xo)
    ed = max(np.max(np.abs(a - b_)) for a, b_ in zip(DXg, DXs)) / max(np.abs(D).max() for D in DXs)
    assert ex < 1e-12 and ed < 1e-12, (ex, ed)
    if m.periodic:
        t1 = sum(DX.sum() * np.prod(m.setup(b).dx) for b, DX in enumerate(DXg))
        scale = sum(np.abs(DX).sum() * np.prod(m.setup(b).dx) for b, DX in enumerate(DXg))
        assert abs(t1 - t0) < 1e-14 * scale
