"""Single-precision transfer of the primitives for the mixed form (grmhd_set_prims_f32,
GRMHD_GET_PRIMS_F32), through the C ABI: loading float P gives the same state, bit for bit, as loading the
double P (whose load rounds to float), and reading P back in float gives the double read-back rounded to
float; all-FP64 contexts refuse both."""
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


def test_float_primitives_give_the_same_state(G):
    s = I.kerr_schild_setup(16, recon="weno5z_aoah", riemann="hll", precision="mixed")
    P = I.kerr_schild_random_prims(s, seed=2)
    a = G.Context(s)
    a.set_prims(P.copy())
    b = G.Context(s)
    G.grmhd_set_prims_f32(b.ctx, np.ascontiguousarray(P.astype(np.float32)))
    assert np.array_equal(a.cons(), b.cons())
    for c in (a, b):
        c.rk2_step(0.01)
    assert np.array_equal(a.cons(), b.cons())
    Pf = b.get(G.GRMHD_GET_PRIMS_F32)
    assert Pf.dtype == np.float32 and np.array_equal(Pf, b.prims().astype(np.float32))
    assert np.array_equal(b.prims(), Pf.astype(np.float64))


def test_fp64_context_refuses_float_primitives(G):
    s = dataclasses.replace(I.kerr_schild_setup(8), precision="fp64")
    c = G.Context(s)
    with pytest.raises(G.GrmhdError):
        G.grmhd_set_prims_f32(c.ctx, np.zeros(s.prim_shape(), np.float32))
    c.set_prims(I.kerr_schild_random_prims(s, seed=1))
    with pytest.raises(G.GrmhdError):
        c.get(G.GRMHD_GET_PRIMS_F32)
