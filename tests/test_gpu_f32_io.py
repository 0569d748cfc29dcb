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


@pytest.mark.parametrize("n", [(40, 24, 20), (24, 16, 5)])
def test_stage_host_f32_equals_load_stage_get(G, n):
    """grmhd_stage_host_f32 (the update in z slabs, each slab's rows read back beside the next slab's update)
    gives the results of grmhd_set_prims_f32 + grmhd_stage + grmhd_get bit for bit: the primitives it writes
    to the host, the conserved state, the status bits and the deferred-cell count; over a first stage (with
    the load) and a second stage (continuing, P_in = None), on a grid with more z rows than slabs and on one
    with fewer (5 rows: one slab per row)."""
    import torch
    nx, ny, nz = n
    s = I.kerr_schild_setup(nx, recon="weno5z_aoah", riemann="hll", precision="mixed")
    s = dataclasses.replace(s, n=(nx, ny, nz))
    P = np.ascontiguousarray(I.kerr_schild_random_prims(s, seed=3).astype(np.float32))
    a, b = G.Context(s), G.Context(s)
    Pin = torch.from_numpy(P).pin_memory()
    out = torch.empty_like(Pin).pin_memory()
    G.grmhd_set_prims_f32(a.ctx, P)
    for g0, g1, beta in ((0.0, 1.0, 1.0), (0.5, 0.5, 0.5)):
        a.stage(g0, g1, beta, 0.0)
        G.grmhd_stage_host_f32(b.ctx, Pin if g0 == 0.0 else None, out, g0, g1, beta, 0.0)
        ref = a.get(G.GRMHD_GET_PRIMS_F32)
        assert np.array_equal(out.numpy(), ref)
        assert np.array_equal(b.cons(), a.cons())
        assert np.array_equal(b.status(), a.status())
        sa, sb = a.stats(), b.stats()
        assert sa[7] == sb[7] and sa[2] == sb[2] and sa[0] == sb[0], (sa, sb)


def test_stage_host_f32_refusals(G):
    s = dataclasses.replace(I.kerr_schild_setup(8), precision="fp64")
    c = G.Context(s)
    c.set_prims(I.kerr_schild_random_prims(s, seed=1))
    with pytest.raises(G.GrmhdError):
        G.grmhd_stage_host_f32(c.ctx, None, np.zeros(s.prim_shape(), np.float32), 0.0, 1.0, 1.0, 0.0)
    sm = I.kerr_schild_setup(8, precision="mixed")
    m = G.Context(sm)
    with pytest.raises(G.GrmhdError):  # a second stage needs a first one
        G.grmhd_stage_host_f32(m.ctx, np.zeros(sm.prim_shape(), np.float32), None, 0.5, 0.5, 0.5, 0.0)
    with pytest.raises(G.GrmhdError):  # float32 host buffers only
        G.grmhd_stage_host_f32(m.ctx, np.zeros(sm.prim_shape(), np.float64), None, 0.0, 1.0, 1.0, 0.0)
