"""Batched form: many uneven meshblocks advanced by one persistent launch per phase (optionally replayed
from a CUDA graph) give the same result, bit for bit, as each block advanced on its own, for any work
item size; the batch's CFL time step is the minimum over its blocks."""
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


def _blocks(precision, recon="weno5z_aoah"):
    layout = [((8, 8, 8), (3.0, 3.0, 3.0), 0.5), ((12, 10, 6), (8.0, 3.0, 3.0), 0.4),
              ((16, 16, 16), (3.0, 10.0, 10.0), 0.3), ((5, 7, 9), (14.0, 14.0, 4.0), 0.6)]
    setups = [I.Setup(n=n3, x0=lo, dx=(h, h, h), metric="kerr_schild", spin=0.9, recon=recon, riemann="hll",
                      bc="fixed", precision=precision) for n3, lo, h in layout]
    prims = [I.kerr_schild_random_prims(s, seed=3 + b) for b, s in enumerate(setups)]
    return setups, prims


def _run(G, setups, prims, graph=False, tile=None, steps=2, dt=0.02):
    bc = G.BatchContext(setups)
    for b, P in enumerate(prims):
        bc.set_prims(b, P.copy())
    if tile:
        bc.set_tile(tile)
    if graph:
        bc.set_graph(True)
    for _ in range(steps):
        bc.stage(0.0, 1.0, 1.0, dt)
        bc.stage(0.5, 0.5, 0.5, dt)
    return [(bc.get(b, G.GRMHD_GET_CONS), bc.get(b, G.GRMHD_GET_PRIMS), bc.get(b, G.GRMHD_GET_STATUS))
            for b in range(len(setups))]


@pytest.mark.parametrize("precision,recon", [("fp64", "weno5z_aoah"), ("mixed", "weno5z_aoah"), ("mixed", "mp5")])
def test_batch_matches_single_blocks(G, precision, recon):
    setups, prims = _blocks(precision, recon)
    ref = []
    for s, P in zip(setups, prims):
        c = G.Context(s)
        c.set_prims(P.copy())
        for _ in range(2):
            c.stage(0.0, 1.0, 1.0, 0.02)
            c.stage(0.5, 0.5, 0.5, 0.02)
        ref.append((c.cons(), c.prims(), c.status()))
    for graph, tile in ((False, None), (True, None), (False, 128), (True, 4096)):
        got = _run(G, setups, prims, graph=graph, tile=tile)
        for b, ((U, P, st), (Ur, Pr, str_)) in enumerate(zip(got, ref)):
            assert np.array_equal(U, Ur), (precision, graph, tile, b)
            assert np.array_equal(P, Pr), (precision, graph, tile, b)
            assert np.array_equal(st, str_), (precision, graph, tile, b)


def test_batch_cfl_is_minimum_over_blocks(G):
    setups, prims = _blocks("fp64", recon="plm_mc")
    dts = []
    for s, P in zip(setups, prims):
        c = G.Context(s)
        c.set_prims(P.copy())
        c.stage(0.0, 1.0, 1.0, 0.0)
        dts.append(c.dt())
    bc = G.BatchContext(setups)
    for b, P in enumerate(prims):
        bc.set_prims(b, P.copy())
    bc.stage(0.0, 1.0, 1.0, 0.0)
    assert abs(bc.dt() - min(dts)) <= 1e-14 * min(dts)


def test_batch_autotune(G):
    """The autotuner times every candidate work-item size with a real RK2 step and keeps the fastest: the
    tile it returns is the argmin of its own timing table, with that entry's time."""
    setups, prims = _blocks("mixed")
    bc = G.BatchContext(setups)
    for b, P in enumerate(prims):
        bc.set_prims(b, P.copy())
    assert bc.autotune_table() == []
    tile, ms = bc.autotune()
    table = bc.autotune_table()
    assert [t for t, _ in table] == [128, 256, 512, 1024, 2048, 4096]
    assert all(m > 0 for _, m in table)
    t_best, m_best = min(table, key=lambda e: e[1])
    assert tile == t_best and ms == m_best, (tile, ms, table)
    bc.set_graph(True)
    bc.rk2_step(0.0)
    assert np.all(np.isfinite(bc.get(0, G.GRMHD_GET_CONS)))
