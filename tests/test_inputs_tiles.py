"""Tiles of the seeded Kerr-Schild generator (the input recipe, no method arithmetic): a tile made by
kerr_schild_tile carries exactly the parent block's primitives and face field on its ghosted cells, so a
small tile of the 256^3 workload stands for that workload in the oracle parity tests."""
import dataclasses

import numpy as np
import pytest

from paper_2410_09146_gb300 import inputs as I


def test_tile_equals_parent_sub_block():
    par = I.kerr_schild_setup(32, recon="weno5z_aoah")
    P, Bf = I.kerr_schild_random_prims(par, seed=2, faces=True)
    off, n = (5, 9, 13), (12, 10, 14)
    t = dataclasses.replace(I.kerr_schild_tile(par, off, n), precision="mixed")
    Pt, Bft = I.kerr_schild_random_prims(t, seed=2, faces=True)
    g = par.ng
    sl = (slice(None), slice(off[2], off[2] + n[2] + 2 * g), slice(off[1], off[1] + n[1] + 2 * g),
          slice(off[0], off[0] + n[0] + 2 * g))
    assert np.array_equal(Pt, P[sl])
    assert np.array_equal(Bft, Bf[sl])
    assert t.x0 == tuple(par.x0[d] + off[d] * par.dx[d] for d in range(3)) and t.dx == par.dx


def test_slab_scale_matches_whole_block():
    par = I.kerr_schild_setup(24)
    a = I._ks_b_scale(par, 3, (1e-6, 1.0), (1.0, 10.0), (1e-2, 50.0), 3, slab=5)
    I._SCALE_CACHE.clear()
    b = I._ks_b_scale(par, 3, (1e-6, 1.0), (1.0, 10.0), (1e-2, 50.0), 3, slab=1000)
    assert a == b


def test_tile_outside_parent_refused():
    par = I.kerr_schild_setup(16)
    with pytest.raises(ValueError):
        I.kerr_schild_tile(par, (10, 0, 0), (8, 8, 8))
