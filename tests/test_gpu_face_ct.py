"""Face-centred upwind CT on the GPU against the oracle, through the C ABI (GB300, sm_103a).

All-FP64 form: every stage within 1e-12 under the measures of tests/parity.py (conserved state,
con2prim, backward error) plus the advanced faces within 1e-12 of the oracle's, on Kerr-Schild random
blocks (fixed ghosts), anisotropic periodic Minkowski blocks and the field loop, at sizes that span
several thread blocks with ragged tails. Mixed form: per-variable L1 <= 1e-6 against the FP64 oracle
on smooth data. At any size: the face divergence keeps its initial roundoff value (the faces advance by
a curl differenced in double). The C ABI refuses the combinations the mode does not support.
"""
import numpy as np
import pytest

from paper_2410_09146_gb300 import inputs as I
from tests.parity import compare_stage, interior_sqrtgam, l1_rel, rel_err_cons

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


def _context(G, orc, s, P, Bf):
    s.ct = "face"
    ctx = G.Context(s)
    ctx.set_prims(P.copy())
    ctx.set_face_b(Bf.copy())
    return ctx


def _fct_compare(G, orc, s, P, Bf, nsteps=2, tol=1e-12, tol_floored=1e-5, max_mismatch=0.0):
    p = orc.params(s)
    ctx = _context(G, orc, s, P, Bf)
    Po, Bo = P.copy(), Bf.copy()
    orc.face_b_to_cells(p, Bo, Po)
    assert rel_err_cons(ctx.cons(), orc.prim2con_grid(p, Po)).max() <= tol
    sg = interior_sqrtgam(orc, p, s)
    worst = {}
    for _ in range(nsteps):
        P_in, U0, B0 = ctx.prims(), ctx.cons(), ctx.face_b()
        ctx.stage(0.0, 1.0, 1.0, 0.0)
        dt = ctx.dt()
        r1 = compare_stage(orc, s, p, P_in, None, U0, 0.0, 1.0, 1.0, 0.0, ctx.prims(), ctx.cons(), ctx.status(), sg,
                           faces=(None, B0, ctx.face_b()))
        assert abs(r1["dt"] - dt) <= 1e-13 * dt, (r1["dt"], dt)
        P_in, U_in, B_in = ctx.prims(), ctx.cons(), ctx.face_b()
        ctx.stage(0.5, 0.5, 0.5, 0.0)
        r2 = compare_stage(orc, s, p, P_in, U0, U_in, 0.5, 0.5, 0.5, dt, ctx.prims(), ctx.cons(), ctx.status(), sg,
                           faces=(B0, B_in, ctx.face_b()))
        for r in (r1, r2):
            for k, v in r.items():
                worst[k] = max(worst.get(k, 0.0), v)
    assert worst["mismatch"] <= max_mismatch, worst
    assert worst["U"] <= tol and worst["P"] <= tol and worst["backward"] <= tol, worst
    assert worst["Bf"] <= tol, worst
    assert worst["U_floored"] <= tol_floored and worst["P_floored"] <= tol_floored, worst
    return ctx, worst


@pytest.mark.parametrize("n,recon", [(12, "weno5z_aoah"), (10, "plm_mc")])
def test_face_ct_kerr_schild_parity(G, orc, n, recon):
    s = I.kerr_schild_setup(n, recon=recon, riemann="hll")
    P, Bf = I.kerr_schild_random_prims(s, seed=1, faces=True)
    _fct_compare(G, orc, s, P, Bf, nsteps=2, max_mismatch=2e-3)


@pytest.mark.parametrize("n3,recon,riemann", [((13, 7, 5), "weno5z_aoah", "hll"), ((11, 9, 6), "plm_mc", "llf")])
def test_face_ct_periodic_parity(G, orc, n3, recon, riemann):
    s = I.Setup(n=n3, dx=tuple(1.0 / k for k in n3), recon=recon, riemann=riemann)
    P, Bf = I.smooth_random_prims(s, seed=8)
    _fct_compare(G, orc, s, P, Bf, nsteps=2)


def test_face_ct_field_loop_parity(G, orc):
    s = I.field_loop_setup(24, recon="weno5z_aoah")
    P, Bf = I.field_loop_prims(s)
    _fct_compare(G, orc, s, P, Bf, nsteps=3)


def test_face_ct_mixed_l1_smooth(G, orc):
    """Mixed form against the FP64 oracle after one RK2 step of smooth Kerr-Schild data."""
    s = I.kerr_schild_setup(32, recon="weno5z_aoah", riemann="hll", lo=6.0, hi=14.0)
    P, Bf = I.smooth_random_prims(s, seed=12)
    p = orc.params(s)
    Po, Bo = P.copy(), Bf.copy()
    orc.face_b_to_cells(p, Bo, Po)
    Uo, Bn, _, _ = orc.rk2_step_face_ct(p, Po, Bo, orc.prim2con_grid(p, Po.copy()))
    s.precision = "mixed"
    ctx = _context(G, orc, s, P, Bf)
    ctx.rk2_step(0.0)
    ng = s.ng
    inner = (slice(None),) + (slice(ng, -ng),) * 3
    l1u, l1p = l1_rel(ctx.cons(), Uo), l1_rel(ctx.prims()[inner], Po[inner])
    from tests.parity import interior_faces
    fb = interior_faces(s, ctx.face_b())
    l1b = np.abs(fb - interior_faces(s, Bn)).sum() / np.abs(interior_faces(s, Bn)).sum()
    assert l1u.max() <= 1e-6, l1u
    assert l1p.max() <= 1e-6, l1p
    assert l1b <= 1e-6, l1b


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_face_ct_divergence_kept(G, orc, precision):
    """Cold random Kerr-Schild block of 64^3: after three RK2 steps the face divergence is still at the
    roundoff of the initial faces (relative to the largest face field over a cell width)."""
    s = I.kerr_schild_setup(64, recon="weno5z_aoah", riemann="hll", precision=precision)
    P, Bf = I.kerr_schild_random_prims(s, seed=3, faces=True)
    p = orc.params(s)
    div0 = np.abs(orc.face_divergence(p, Bf)).max() * min(s.dx) / np.abs(Bf).max()
    ctx = _context(G, orc, s, P, Bf)
    for _ in range(3):
        ctx.rk2_step(0.0)
    B = ctx.face_b()
    div = np.abs(orc.face_divergence(p, B)).max() * min(s.dx) / np.abs(B).max()
    assert np.isfinite(B).all()
    assert div <= max(1e-13, 10 * div0), (div, div0)


def test_face_ct_api_refusals(G, orc):
    import torch
    s = I.linear_wave_setup(8)
    P, Bf = I.smooth_random_prims(s, seed=1)
    flux_ctx = G.Context(s)
    flux_ctx.set_prims(P.copy())
    with pytest.raises(G.GrmhdError):
        flux_ctx.set_face_b(Bf.copy())            # not a face-CT context
    with pytest.raises(G.GrmhdError):
        flux_ctx.face_b()
    s.ct = "face"
    ctx = G.Context(s)
    with pytest.raises(G.GrmhdError):
        ctx.set_face_b(Bf.copy())                 # before set_prims
    ctx.set_prims(P.copy())
    with pytest.raises(G.GrmhdError):
        ctx.stage(0.0, 1.0, 1.0, 0.0)             # faces not loaded
    ctx.set_face_b(Bf.copy())
    ctx.stage(0.0, 1.0, 1.0, 0.0)
    torch.cuda.synchronize()
    # the all-FP64 allocation-free stage has no face arrays, and batches use flux-CT
    dev = lambda a: torch.tensor(a, device="cuda")
    Pd, Ud = dev(P), dev(np.zeros(s.cons_shape()))
    Un, st = torch.zeros_like(Ud), torch.zeros(s.cons_shape()[1:], dtype=torch.uint8, device="cuda")
    with pytest.raises(G.GrmhdError):
        G.grmhd_stage_noalloc(G.params(s), Pd.data_ptr(), 0, Ud.data_ptr(), Un.data_ptr(), st.data_ptr(),
                              0.0, 1.0, 1.0, 1e-3)
    ks = I.kerr_schild_setup(8)
    ks.ct = "face"
    with pytest.raises(G.GrmhdError):
        G.BatchContext([ks, ks])
