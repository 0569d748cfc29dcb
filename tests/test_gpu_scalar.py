"""The passive scalar on the GPU (params.scalar, grmhd_set_scalar) against the oracle's (orc_stage_scalar,
pinned in tests/test_oracle_scalar.py), through the C ABI.

* All-FP64 form: every stage of two RK2 steps, from the GPU's own state, the oracle's stage gives X and
  sqrt(gamma) D X within 1e-12 (relative to their largest magnitude): smooth Kerr-Schild (WENO5-Z-AOAH +
  HLL), periodic Minkowski (PLM-MC + LLF, MP5 + HLL) and a ragged periodic 13 x 7 x 5 block (WENO).
* The periodic block conserves the sum of sqrt(gamma) D X on the device (FP64 to 1e-14; mixed to 1e-9,
  its flux divergence being formed in float like the fluid's); a uniform X stays uniform (FP64 to 1e-15,
  mixed to 1e-6: the scalar's flux is formed in float there).
* Mixed form: per-variable L1 of X and D X against the FP64 oracle within 1e-6 after two steps.
* Refusals: no scalar in the params, no prior grmhd_set_prims, a stage before grmhd_set_scalar, ng < 3.
* Batches: uneven Kerr-Schild blocks in one batch (and its CUDA-graph replay) bit for bit each block's own
  context in both forms; a periodic lattice (X's ghosts exchanged with P's) bit for bit the large block.
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


def _ks(precision="fp64"):
    s = dataclasses.replace(I.kerr_schild_setup(12, recon="weno5z_aoah", riemann="hll"), scalar=True,
                            precision=precision)
    P = I.kerr_schild_random_prims(s, seed=5, rho_range=(0.1, 1.0), w_range=(1.0, 2.0), sigma_range=(0.01, 1.0),
                                   p_coef=0.5, kmax=1)
    return s, P


def _mink(n=(16, 16, 16), recon="plm_mc", riemann="llf", precision="fp64"):
    s = dataclasses.replace(I.linear_wave_setup(n[0], ny=n[1], nz=n[2], recon=recon, riemann=riemann), scalar=True,
                            precision=precision)
    P, _ = I.smooth_random_prims(s, seed=3, amp=0.3, b_amp=0.3, kmax=1)
    return s, P


def _scalar_field(s, seed=4):
    rng = np.random.default_rng(seed)
    x = [s.cell_centres(d) for d in range(3)]
    span = [s.n[d] * s.dx[d] for d in range(3)]
    Z, Y, X = np.meshgrid(*[(x[d] - s.x0[d]) / span[d] for d in (2, 1, 0)], indexing="ij")
    ph = rng.uniform(0, 2 * np.pi, 3)
    f = 0.5 + 0.3 * np.sin(2 * np.pi * X + ph[0]) * np.cos(2 * np.pi * Y + ph[1]) + 0.1 * np.sin(2 * np.pi * Z + ph[2])
    return f + np.where(X > 0.5, 0.2, 0.0)  # and a jump


CASES = [("kerr_schild weno hll", _ks), ("minkowski plm llf", lambda: _mink()),
         ("minkowski mp5 hll", lambda: _mink(recon="mp5", riemann="hll")),
         ("ragged weno", lambda: _mink(n=(13, 7, 5), recon="weno5z_aoah", riemann="hll"))]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_fp64_scalar_matches_the_oracle(G, orc, name, make):
    s, P = make()
    p = orc.params(s)
    ctx = G.Context(s)
    ctx.set_prims(P.copy())
    X = _scalar_field(s)
    ctx.set_scalar(X)
    U0 = ctx.cons()
    DX0 = ctx.scalar_cons()
    np.testing.assert_allclose(DX0, U0[0] * X[4:-4, 4:-4, 4:-4], rtol=1e-15)
    worst = 0.0
    for _ in range(2):
        for g0, g1, beta in ((0.0, 1.0, 1.0), (0.5, 0.5, 0.5)):
            P_in, U_in, X_in, DX_in = ctx.prims(), ctx.cons(), ctx.scalar(), ctx.scalar_cons()
            if g0 == 0.0:
                Ustep, DXstep = U_in, DX_in
                ctx.stage(g0, g1, beta, 0.0)  # the CFL step, passed to the oracle too
                dtv = ctx.dt()
            else:
                ctx.stage(g0, g1, beta, dtv)
            Xo = X_in.copy()
            r = orc.stage_scalar(p, P_in.copy(), Xo, None if g0 == 0.0 else Ustep, U_in,
                                 None if g0 == 0.0 else DXstep, DX_in, g0, g1, beta, dtv)
            Xg, DXg = ctx.scalar(), ctx.scalar_cons()
            ex = np.max(np.abs(Xg[4:-4, 4:-4, 4:-4] - Xo[4:-4, 4:-4, 4:-4])) / np.max(np.abs(Xo))
            ed = np.max(np.abs(DXg - r["DX"])) / np.max(np.abs(r["DX"]))
            worst = max(worst, ex, ed)
    assert worst < 1e-12, worst


@pytest.mark.parametrize("precision,tol,ctol", [("fp64", 1e-15, 1e-14), ("mixed", 1e-6, 1e-9)])
def test_uniform_scalar_and_conservation_on_the_device(G, precision, tol, ctol):
    """The mixed form forms the divergence of its float face fluxes in float, like the fluid's: the flux
    differences then telescope only to float rounding (measured 2e-11 of the total after three steps)."""
    s, P = _ks(precision)
    ctx = G.Context(s)
    ctx.set_prims(P.copy())
    ctx.set_scalar(np.full(s.prim_shape()[1:], 0.3))
    for _ in range(2):
        ctx.rk2_step()
    assert np.max(np.abs(ctx.scalar()[4:-4, 4:-4, 4:-4] - 0.3)) < tol
    s, P = _mink(precision=precision)
    ctx = G.Context(s)
    ctx.set_prims(P.copy())
    ctx.set_scalar(_scalar_field(s))
    t0 = ctx.scalar_cons().sum()
    for _ in range(3):
        ctx.rk2_step()
    DX = ctx.scalar_cons()
    assert abs(DX.sum() - t0) < ctol * np.abs(DX).sum()


@pytest.mark.parametrize("name,make", CASES[:2], ids=[c[0] for c in CASES[:2]])
def test_mixed_scalar_within_the_mixed_bound(G, orc, name, make):
    s, P = make()
    p = orc.params(s)
    X0 = _scalar_field(s)
    ctx = G.Context(dataclasses.replace(s, precision="mixed"))
    ctx.set_prims(P.copy())
    ctx.set_scalar(X0)
    Po, Xo = P.copy(), X0.copy()
    U = orc.prim2con_grid(p, Po.copy())
    DX = U[0] * Xo[4:-4, 4:-4, 4:-4]
    dt = None
    for _ in range(2):
        U, DX, st, dt_o = orc.rk2_step_scalar(p, Po, Xo, U, DX, 0.0 if dt is None else dt)
        ctx.rk2_step(dt_o)
        dt = dt_o
    Xg, DXg = ctx.scalar()[4:-4, 4:-4, 4:-4], ctx.scalar_cons()
    lx = np.abs(Xg - Xo[4:-4, 4:-4, 4:-4]).sum() / np.abs(Xo[4:-4, 4:-4, 4:-4]).sum()
    ld = np.abs(DXg - DX).sum() / np.abs(DX).sum()
    assert lx < 1e-6 and ld < 1e-6, (lx, ld)


def test_scalar_refusals(G):
    s, P = _mink(n=(8, 8, 8))
    plain = G.Context(dataclasses.replace(s, scalar=False))
    plain.set_prims(P.copy())
    with pytest.raises(G.GrmhdError):
        plain.set_scalar(np.zeros(s.prim_shape()[1:]))          # no scalar in the params
    ctx = G.Context(s)
    with pytest.raises(G.GrmhdError):
        ctx.set_scalar(np.zeros(s.prim_shape()[1:]))            # no state yet
    ctx.set_prims(P.copy())
    with pytest.raises(G.GrmhdError):
        ctx.stage(0.0, 1.0, 1.0, 0.001)                         # the scalar was not set
    with pytest.raises(G.GrmhdError):
        G.Context(dataclasses.replace(s, ng=2, recon="plm_mc"))  # the scalar's stencil needs ng >= 3
    bc = G.BatchContext([dataclasses.replace(s, bc="fixed")])
    bc.set_prims(0, P.copy())
    with pytest.raises(G.GrmhdError):
        bc.stage(0.0, 1.0, 1.0, 0.001)                          # a block without its scalar


def _batch_blocks(precision):
    layout = [((8, 8, 8), (3.0, 3.0, 3.0), 0.5), ((12, 10, 6), (8.0, 3.0, 3.0), 0.4),
              ((16, 16, 16), (3.0, 10.0, 10.0), 0.3), ((5, 7, 9), (14.0, 14.0, 4.0), 0.6)]
    setups = [I.Setup(n=n3, x0=lo, dx=(h, h, h), metric="kerr_schild", spin=0.9, recon="weno5z_aoah", riemann="hll",
                      bc="fixed", precision=precision, scalar=True) for n3, lo, h in layout]
    prims = [I.kerr_schild_random_prims(s, seed=3 + b, rho_range=(0.1, 1.0), w_range=(1.0, 2.0),
                                        sigma_range=(0.01, 1.0), p_coef=0.5, kmax=1) for b, s in enumerate(setups)]
    return setups, prims


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_scalar_is_each_blocks_own_context(G, precision):
    """Uneven Kerr-Schild blocks in one batch (also replayed as a CUDA graph): each block's X and D X bit
    for bit those of the block advanced in its own context."""
    setups, prims = _batch_blocks(precision)
    Xs = [_scalar_field(s, seed=7 + b) for b, s in enumerate(setups)]
    ref = []
    for s, P, X in zip(setups, prims, Xs):
        c = G.Context(s)
        c.set_prims(P.copy())
        c.set_scalar(X)
        for _ in range(2):
            c.stage(0.0, 1.0, 1.0, 0.02)
            c.stage(0.5, 0.5, 0.5, 0.02)
        ref.append((c.scalar(), c.scalar_cons(), c.cons()))
    for graph in (False, True):
        bc = G.BatchContext(setups)
        for b, (P, X) in enumerate(zip(prims, Xs)):
            bc.set_prims(b, P.copy())
            bc.set_scalar(b, X)
        if graph:
            bc.set_graph(True)
        for _ in range(2):
            bc.stage(0.0, 1.0, 1.0, 0.02)
            bc.stage(0.5, 0.5, 0.5, 0.02)
        for b, (Xr, DXr, Ur) in enumerate(ref):
            assert np.array_equal(bc.get(b, G.GRMHD_GET_SCALAR), Xr), (precision, graph, b)
            assert np.array_equal(bc.get(b, G.GRMHD_GET_SCALAR_CONS), DXr), (precision, graph, b)
            assert np.array_equal(bc.get(b, G.GRMHD_GET_CONS), Ur), (precision, graph, b)


def test_lattice_scalar_is_the_large_block(G):
    """A periodic lattice of blocks exchanges X's ghosts with P's: all-FP64, bit for bit the large block."""
    s = dataclasses.replace(I.linear_wave_setup(32, ny=24, nz=16, recon="weno5z_aoah", riemann="hll"), scalar=True)
    P, _ = I.smooth_random_prims(s, seed=9, amp=0.3, b_amp=0.3, kmax=1)
    X = _scalar_field(s, seed=2)
    big = G.Context(s)
    big.set_prims(P.copy())
    big.set_scalar(X)
    nb = (4, 3, 2)
    n = [s.n[d] // nb[d] for d in range(3)]
    ng = s.ng
    bc_setups, sl = [], []
    for bz in range(nb[2]):
        for by in range(nb[1]):
            for bx in range(nb[0]):
                b3 = (bx, by, bz)
                x0 = tuple(s.x0[d] + b3[d] * n[d] * s.dx[d] for d in range(3))
                bc_setups.append(dataclasses.replace(s, n=tuple(n), x0=x0, bc="fixed"))
                sl.append(tuple(slice(b3[d] * n[d], b3[d] * n[d] + n[d] + 2 * ng) for d in (2, 1, 0)))
    bc = G.BatchContext(bc_setups)
    for b, q in enumerate(sl):
        bc.set_prims(b, np.ascontiguousarray(P[(slice(None),) + q]))
        bc.set_scalar(b, np.ascontiguousarray(X[q]))
    bc.set_lattice(nb, True)
    for _ in range(2):
        big.stage(0.0, 1.0, 1.0, 0.01)
        big.stage(0.5, 0.5, 0.5, 0.01)
        bc.stage(0.0, 1.0, 1.0, 0.01)
        bc.stage(0.5, 0.5, 0.5, 0.01)
    Xb, DXb = big.scalar(), big.scalar_cons()
    for b, q in enumerate(sl):
        inner = tuple(slice(t.start + ng, t.stop - ng) for t in q)
        assert np.array_equal(bc.get(b, G.GRMHD_GET_SCALAR)[ng:-ng, ng:-ng, ng:-ng], Xb[inner]), b
        assert np.array_equal(bc.get(b, G.GRMHD_GET_SCALAR_CONS),
                              DXb[tuple(slice(t.start, t.stop - 2 * ng) for t in q)]), b

