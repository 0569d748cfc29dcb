"""The bounds-check build (-DGRMHD_BOUNDS_CHECK): the stage kernels compare every global-memory index with its
array's extent and record the first out-of-range access (grmhd_bounds_fault) instead of making it. Here the
small parity cases run through that build: they must match the oracle as in the normal build, and no access
may be recorded, in either form, for every reconstruction (face-centric and cell-centric flux kernels,
ragged blocks whose sizes are not multiples of the kernels' tiles)."""
import dataclasses
import json
import os

import numpy as np
import pytest

from paper_2410_09146_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fast_wave_minkowski.json")


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_09146_gb300 import build
    build.build()
    path = build.build(bounds_check=True)
    from paper_2410_09146_gb300 import grmhd
    prev = grmhd.use_library(path)
    yield grmhd
    grmhd.restore_library(prev)


def _cases():
    gw = json.load(open(GOLDEN))
    out = []
    for n3, recon, riemann in (((12, 12, 12), "plm_mc", "llf"), ((13, 7, 5), "weno5z_aoah", "hll"),
                               ((11, 9, 7), "mp5", "hll"), ((8, 6, 5), "constant", "llf")):
        s = I.linear_wave_setup(*n3, recon=recon, riemann=riemann)
        out.append((s, I.linear_wave_prims(s, gw["background_prims"], gw["eigvec_prims"], amplitude=1e-3)))
    for recon in ("weno5z_aoah", "plm_mc"):
        s = I.kerr_schild_setup(12, recon=recon, riemann="hll")
        out.append((s, I.kerr_schild_random_prims(s, seed=1)))
    return out


def test_bounds_check_build_is_loaded(G):
    ctx = G.Context(I.linear_wave_setup(8))
    word, checked = G.grmhd_bounds_fault(ctx.ctx)
    assert checked and word == 0


@pytest.mark.parametrize("k", range(6))
def test_parity_cases_under_bounds_checks(G, orc, k):
    from tests.test_gpu_parity import _step_compare
    s, P = _cases()[k]
    ctx, worst = _step_compare(G, orc, s, P, nsteps=1, max_mismatch=2e-3)
    word, checked = G.grmhd_bounds_fault(ctx.ctx)
    assert checked and word == 0, hex(word)
    # the mixed form's kernels (float fluxes, the tiled y / z sweep, the mixed update and cell passes)
    m = G.Context(dataclasses.replace(s, precision="mixed"))
    m.set_prims(P.copy())
    m.rk2_step(0.0)
    m.rk2_step(0.0)
    word, checked = G.grmhd_bounds_fault(m.ctx)
    assert checked and word == 0, hex(word)
    assert np.all(np.isfinite(m.cons()))
