"""CUDA path against the oracle, element by element, through the C ABI (GB300, sm_103a).

All-FP64 form: within 1e-12 per cell, per variable, per stage under the condition-aware measure
of tests/parity.py: the conserved update against the oracle stage, the con2prim against the
oracle's con2prim of the same conserved state (scaled by its measured condition number), and the
backward error of the primitives. Cells where a floor or the Lorentz-factor cap fired hold
unphysical pre-floor states set by roundoff; they must carry identical status bits and agree to 1e-5. Mixed form: per-variable L1 <= 1e-6 against the FP64 oracle. Inputs are the
seeded generators of paper_2410_09146_gb300/inputs.py at sizes that span several thread blocks
and ragged tails; the full 128^3 Kerr-Schild workload is compared on the whole grid.
"""
import json
import os

import numpy as np
import pytest

from paper_2410_09146_gb300 import inputs as I
from tests.parity import compare_stage, interior_sqrtgam, l1_rel, rel_err_cons

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fast_wave_minkowski.json")


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_09146_gb300 import build
    build.build()
    from paper_2410_09146_gb300 import grmhd
    return grmhd


def _step_compare(G, orc, s, P, nsteps=1, tol=1e-12, tol_floored=1e-5, max_mismatch=0.0):
    """Run RK2 steps on the GPU (CFL dt chosen on the device) and check every stage against the
    oracle started from the GPU's own state before that stage."""
    p = orc.params(s)
    ctx = G.Context(s)
    ctx.set_prims(P.copy())
    assert rel_err_cons(ctx.cons(), orc.prim2con_grid(p, P.copy())).max() <= tol
    sg = interior_sqrtgam(orc, p, s)
    worst = {}
    for _ in range(nsteps):
        P_in, U0 = ctx.prims(), ctx.cons()
        ctx.stage(0.0, 1.0, 1.0, 0.0)
        dt = ctx.dt()
        r1 = compare_stage(orc, s, p, P_in, None, U0, 0.0, 1.0, 1.0, 0.0, ctx.prims(), ctx.cons(), ctx.status(), sg)
        assert abs(r1["dt"] - dt) <= 1e-13 * dt, (r1["dt"], dt)
        P_in, U_in = ctx.prims(), ctx.cons()
        ctx.stage(0.5, 0.5, 0.5, 0.0)
        r2 = compare_stage(orc, s, p, P_in, U0, U_in, 0.5, 0.5, 0.5, dt, ctx.prims(), ctx.cons(), ctx.status(), sg)
        for r in (r1, r2):
            for k, v in r.items():
                worst[k] = max(worst.get(k, 0.0), v)
    assert worst["mismatch"] <= max_mismatch, worst
    assert worst["U"] <= tol and worst["P"] <= tol and worst["backward"] <= tol, worst
    assert worst["U_floored"] <= tol_floored and worst["P_floored"] <= tol_floored, worst
    return ctx, worst


def test_c2p_batch_parity(G, orc):
    import torch
    s = I.linear_wave_setup(8)
    p = orc.params(s)
    Ps = I.c2p_states(20000, seed=4)
    x = np.zeros((len(Ps), 3))
    U = orc.prim2con_points(p, x, Ps)["U"]
    Po, sto, _ = orc.c2p_points(p, x, U, floors=True)
    ctx = G.Context(I.Setup(n=(0, 0, 0)))
    Ud = torch.tensor(U.T.copy(), device="cuda")
    Pd = torch.zeros_like(Ud)
    st = torch.zeros(len(Ps), dtype=torch.uint8, device="cuda")
    it = torch.zeros(len(Ps), dtype=torch.int32, device="cuda")
    ctx.c2p(Ud, Pd, st, it)
    torch.cuda.synchronize()
    Pg = Pd.cpu().numpy().T
    assert np.array_equal(st.cpu().numpy(), sto)
    assert it.cpu().numpy().max() <= s.c2p_max_iter
    # backward error of the GPU solution against the given U (the conditioning-free measure), on the
    # states no floor or cap modified
    plain = sto == 0
    assert plain.mean() > 0.5
    Ug = orc.prim2con_points(p, x, Pg)["U"]
    scale = np.abs(U[:, 0]) + np.abs(U[:, 4]) + np.linalg.norm(U[:, 1:4], axis=1)
    be = (np.max(np.abs(Ug - U), axis=1) / scale)[plain]
    assert be.max() < 1e-11 and np.median(be) < 1e-14
    # forward parity on the well-conditioned part (W <= 10, sigma <= 10, p/rho >= 1e-4)
    W = np.sqrt(1 + np.sum(Ps[:, 1:4] ** 2, 1))
    sig = np.sum(Ps[:, 5:8] ** 2, 1) / (Ps[:, 0] * W * W)
    good = (W <= 10) & (sig <= 10) & (Ps[:, 4] * (2.0 / 3.0) / Ps[:, 0] >= 1e-4)
    assert good.sum() > 100
    rel = np.abs(Pg[good, 0] - Po[good, 0]) / Po[good, 0]
    assert rel.max() < 1e-12
    esc = (U[good, 4] + U[good, 0])
    assert (np.abs(Pg[good, 4] - Po[good, 4]) / esc).max() < 1e-13


@pytest.mark.parametrize("n3,recon,riemann", [((16, 16, 16), "plm_mc", "llf"), ((13, 7, 5), "plm_mc", "llf"),
                                               ((12, 10, 9), "weno5z_aoah", "hll"), ((9, 9, 9), "plm_minmod", "hll"),
                                               ((8, 6, 5), "constant", "llf"), ((11, 9, 7), "mp5", "hll")])
def test_stage_linear_wave_parity(G, orc, n3, recon, riemann):
    gw = json.load(open(GOLDEN))
    s = I.linear_wave_setup(n3[0], n3[1], n3[2], recon=recon, riemann=riemann)
    P = I.linear_wave_prims(s, gw["background_prims"], gw["eigvec_prims"], amplitude=1e-3)
    ctx, worst = _step_compare(G, orc, s, P, nsteps=2)
    assert worst["floored_frac"] == 0.0


@pytest.mark.parametrize("n,recon", [(16, "weno5z_aoah"), (12, "plm_mc"), (12, "mp5")])
def test_stage_kerr_schild_parity(G, orc, n, recon):
    s = I.kerr_schild_setup(n, recon=recon, riemann="hll")
    P = I.kerr_schild_random_prims(s, seed=1)
    _step_compare(G, orc, s, P, nsteps=2, max_mismatch=2e-3)


def test_stage_kerr_schild_moderate_parity(G, orc):
    """Smooth Kerr-Schild data where no floor fires: every cell compared."""
    s = I.kerr_schild_setup(20, recon="weno5z_aoah", riemann="hll")
    P = I.kerr_schild_random_prims(s, seed=5, rho_range=(0.1, 1.0), w_range=(1.0, 2.0), sigma_range=(0.01, 1.0),
                                   p_coef=0.5, kmax=1)
    ctx, worst = _step_compare(G, orc, s, P, nsteps=2)
    assert worst["floored_frac"] < 0.02


def _mixed_l1(G, orc, s, P):
    p = orc.params(s)
    Po = P.copy()
    Uo, _, _ = orc.rk2_step(p, Po, orc.prim2con_grid(p, Po.copy()), 0.0)
    s.precision = "mixed"
    ctx = G.Context(s)
    ctx.set_prims(P.copy())
    ctx.rk2_step(0.0)
    ng = s.ng
    inner = (slice(None),) + (slice(ng, -ng),) * 3
    return l1_rel(ctx.cons(), Uo), l1_rel(ctx.prims()[inner], Po[inner])


def test_mixed_precision_l1_smooth(G, orc):
    """Mixed form (float reconstruction, fluxes, EMFs, sources; double update and con2prim): per-variable
    L1 <= 1e-6 against the FP64 oracle after one RK2 step of smooth Kerr-Schild data (no floor fires; where
    floors fire the pre-floor state is unphysical and its recovered values are set by roundoff)."""
    s = I.kerr_schild_setup(32, recon="weno5z_aoah", riemann="hll")
    P = I.kerr_schild_random_prims(s, seed=2, rho_range=(0.1, 1.0), w_range=(1.0, 1.5), sigma_range=(0.01, 0.5),
                                   p_coef=1.0, kmax=1)
    l1u, l1p = _mixed_l1(G, orc, s, P)
    assert l1u.max() <= 1e-6, l1u
    assert l1p.max() <= 1e-6, l1p


@pytest.mark.parametrize("offset", [(96, 96, 96), (0, 0, 0)])
def test_mixed_precision_l1_c2_tile(G, orc, offset):
    """The precision contract on the 256^3 workload itself (Kerr-Schild a = 0.9, seed 2, WENO5-Z-AOAH + HLL):
    a 64^3 tile of that block (kerr_schild_tile: the block's own primitives, ghosts included, so the same
    cell widths, roughness, magnetisation and coldness), one RK2 step of the mixed form against the FP64
    oracle. The conserved state must meet per-variable L1 <= 1e-6. The primitives are reported: rho eps on
    the scale con2prim recovers it from, (tau + D)/sqrt(gamma) (its L1 there also <= 1e-6); rho and W v on
    their own scale, where the con2prim condition number of these cold, magnetised cells (up to ~W^2)
    multiplies the conserved-state error (bound 1e-4, measured ~1e-5). The tile at the origin sits next to
    the hole (W > 7 in half its cells); the central one has twice the block's share of cells with W > 5 and
    sigma > 5, where the float fluxes' error concentrates."""
    parent = I.kerr_schild_setup(256, recon="weno5z_aoah", riemann="hll")
    s = I.kerr_schild_tile(parent, offset, (64, 64, 64))
    P = I.kerr_schild_random_prims(s, seed=2)
    p = orc.params(s)
    Po = P.copy()
    Uo, _, _ = orc.rk2_step(p, Po, orc.prim2con_grid(p, Po.copy()), 0.0)
    s.precision = "mixed"
    ctx = G.Context(s)
    ctx.set_prims(P.copy())
    ctx.rk2_step(0.0)
    ng = s.ng
    inner = (slice(None),) + (slice(ng, -ng),) * 3
    U, Pm = ctx.cons(), ctx.prims()[inner]
    l1u = l1_rel(U, Uo)
    l1p = l1_rel(Pm, Po[inner])
    sg = interior_sqrtgam(orc, p, s)
    l1e = np.abs(Pm[4] - Po[inner][4]).sum() / (np.abs(Uo[4] + Uo[0]) / sg).sum()
    maxu = [float(np.abs(U[v] - Uo[v]).max() / np.abs(Uo[v]).max()) for v in range(8)]
    print(f"tile {offset}: L1 U {l1u}, max U {np.array(maxu)}, L1 P {l1p}, L1 rho eps / ((tau + D)/sqrt(gamma)) {l1e:.2e}")
    assert l1u.max() <= 1e-6, l1u
    assert l1e <= 1e-6, l1e
    assert l1p[[0, 1, 2, 3, 5, 6, 7]].max() <= 1e-4, l1p


def test_conservation_divb_determinism_checkpoint(G, orc):
    s = I.linear_wave_setup(16, recon="weno5z_aoah", riemann="hll")
    P = I.kerr_schild_random_prims(s, seed=7, rho_range=(0.3, 1.0), w_range=(1.0, 1.3), sigma_range=(0.01, 0.1),
                                   p_coef=1.0, kmax=1)
    a = G.Context(s)
    a.set_prims(P.copy())
    U0 = a.cons()
    for _ in range(2):
        a.rk2_step(0.0)
    Ua = a.cons()
    assert np.all(a.status() == 0)
    for v in range(8):
        assert abs(Ua[v].sum() - U0[v].sum()) <= 1e-13 * np.abs(U0[v]).sum()
    from tests.test_oracle_stage import _corner_div
    assert np.abs(_corner_div(Ua, s) - _corner_div(U0, s)).max() < 1e-13 * np.abs(U0[5:8]).max() / s.dx[0]
    # checkpoint after one step, restore into a fresh context, continue: bitwise equal
    b = G.Context(s)
    b.set_prims(P.copy())
    b.rk2_step(0.0)
    Pck, Uck = b.prims(), b.cons()
    c = G.Context(s)
    c.set_prims(Pck)
    c.set_cons(Uck)
    c.rk2_step(0.0)
    assert np.array_equal(c.cons(), Ua)
    assert np.array_equal(c.prims(), a.prims())


def test_bad_input_flags_only_that_cell(G, orc):
    s = I.linear_wave_setup(8)
    gw = json.load(open(GOLDEN))
    P = I.linear_wave_prims(s, gw["background_prims"], gw["eigvec_prims"], amplitude=1e-3)
    P_bad = P.copy()
    g = s.ng
    P_bad[0, g + 3, g + 4, g + 5] = -1.0   # negative density -> D < 0 after prim->cons
    ref = G.Context(s)
    ref.set_prims(P.copy())
    ref.stage(0.0, 1.0, 1.0, 1e-3)
    ctx = G.Context(s)
    ctx.set_prims(P_bad)
    ctx.stage(0.0, 1.0, 1.0, 1e-3)
    st = ctx.status()
    assert st[3, 4, 5] & G.ST_BAD_INPUT
    assert ctx.stats()[5] >= 1
    # cells outside the stencil reach of the bad cell are untouched (2 stages of radius 2)
    far = np.ones_like(st, bool)
    far[0:7, 1:8, 2:8] = False
    assert np.array_equal(ctx.cons()[:, far], ref.cons()[:, far])


def test_full_size_kerr_schild_128(G, orc):
    """The 128^3 Kerr-Schild workload (HLL, PLM-MC, FP64): one RK2 step, every cell against the oracle."""
    s = I.kerr_schild_setup(128, recon="plm_mc", riemann="hll")
    P = I.kerr_schild_random_prims(s, seed=1)
    _step_compare(G, orc, s, P, nsteps=1, max_mismatch=1e-3)


def test_max_speed_gives_the_cfl_step(G, orc):
    """grmhd_max_speed (the a7 helper): the per-direction largest |lambda| of the last CFL stage, from which
    dt = cfl / max_d(lambda_d / dx_d) is the step the stage took and the oracle's."""
    s = I.kerr_schild_setup(12, recon="plm_mc", riemann="hll")
    P = I.kerr_schild_random_prims(s, seed=5, rho_range=(0.1, 1.0), w_range=(1.0, 2.0), sigma_range=(0.01, 1.0),
                                   p_coef=0.5, kmax=1)
    ctx = G.Context(s)
    ctx.set_prims(P.copy())
    assert np.array_equal(ctx.max_speed(), np.zeros(3))
    ctx.stage(0.0, 1.0, 1.0, 0.0)
    lam = ctx.max_speed()
    assert np.all(lam > 0) and np.all(lam <= 1.0 + 1e-12)
    dt = s.cfl / max(lam[d] / s.dx[d] for d in range(3))
    assert dt == ctx.dt()
    p = orc.params(s)
    r = orc.stage(p, P.copy(), None, orc.prim2con_grid(p, P.copy()), 0.0, 1.0, 1.0, 0.0)
    assert abs(r["dt"] - dt) <= 1e-13 * dt
    # a later stage of the step does not retake the speeds
    ctx.stage(0.5, 0.5, 0.5, 0.0)
    assert np.array_equal(ctx.max_speed(), lam)


def test_fp_peaks_measures_both_fma_rates(G):
    import torch
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    f64, f32 = G.grmhd_fp_peaks(sink.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert 0.05 < f64 < 100.0 and 1.0 < f32 < 1000.0 and f32 > 4 * f64, (f64, f32)
