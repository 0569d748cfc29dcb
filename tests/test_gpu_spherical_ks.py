"""Spherical Kerr-Schild coordinates (x^1, x^2, x^3) = (ln r, theta, phi) on the GPU (single-block contexts,
flux-CT) against the oracle, stage by stage through the C ABI, within 1e-12 per cell under the
condition-aware measure of tests/parity.py (the GPU's own state before each stage is the oracle's input):

* a full sphere with the spherical boundary (polar ghosts mirrored across the axis and turned by pi in phi,
  phi periodic): axis faces without flux, sin(theta)-weighted reconstruction of the phi components, the axis
  EMFs (zero along phi, the phi mean along r), the general geometric sources with sqrt(-g) != 1;
* a torus block away from the axis with fixed ghosts (the set-up of the paper's accretion runs), with
  a perturbed state and a field so the stage is far from stationary;
* the time step from the device's speeds equals the oracle's.

The mixed form (float reconstruction, fluxes, EMFs, sources; double update and con2prim, the latter with
the metric's full 3-matrices) on the same two blocks after one RK2 step against the oracle: the conserved
state within per-variable L1 <= 1e-6 (the precision contract; measured <= 7.7e-7); the primitives within
1e-5 (measured <= 1.8e-6, in the r and theta velocity components: small velocities recovered from momenta
that the rotation dominates, so the con2prim's conditioning multiplies the conserved-state error there).
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


def _steps(G, orc, s, P, nsteps=2, tol=1e-12):
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
    assert worst["mismatch"] == 0.0, worst
    assert worst["U"] <= tol and worst["P"] <= tol and worst["backward"] <= tol, worst
    assert worst["U_floored"] <= 1e-5 and worst["P_floored"] <= 1e-5, worst
    return worst


@pytest.mark.parametrize("recon", ["weno5z_aoah", "plm_mc"])
def test_full_sphere_with_polar_ghosts(G, orc, recon):
    s = I.full_sphere_setup(8, 12, 16, recon=recon)
    _steps(G, orc, s, I.spherical_random_prims(s, seed=21))


def test_flat_space_full_sphere(G, orc):
    """mass = 0: flat space in spherical coordinates (the metric's M -> 0 limit; all sources from the
    coordinates alone)."""
    s = I.full_sphere_setup(6, 10, 12, mass=0.0, spin=0.0)
    _steps(G, orc, s, I.spherical_random_prims(s, seed=22))


def test_torus_block_fixed_ghosts(G, orc):
    s, P = _torus_perturbed()
    _steps(G, orc, s, P)


def _torus_perturbed(seed=23):
    """The stationary torus with its density and energy perturbed by 10%, velocities along r and theta of
    ~1% of light (contravariant in ln r and theta: divided by r) and a weak field, so every conserved
    component is of its own size (in equilibrium S_r and S_theta would be ~0 and an L1 relative to them
    would measure nothing but the float rounding of the balancing forces)."""
    s = I.torus_setup(16, 4.0, 24.0, 0.5, np.pi - 0.5, nphi=6, dphi=0.05)
    P = I.torus_prims(s)
    rng = np.random.default_rng(seed)
    r = np.exp(s.cell_centres(0))[None, None, :]
    P[0] *= 1.0 + 0.1 * rng.uniform(-1.0, 1.0, P[0].shape)
    P[4] *= 1.0 + 0.1 * rng.uniform(-1.0, 1.0, P[4].shape)
    P[1] += 0.01 * rng.uniform(-1.0, 1.0, P[1].shape) / r
    P[2] += 0.01 * rng.uniform(-1.0, 1.0, P[2].shape) / r
    P[5] = 1e-3 * rng.uniform(-1.0, 1.0, P[5].shape)
    P[6] = 1e-3 * rng.uniform(-1.0, 1.0, P[6].shape)
    return s, P


@pytest.mark.parametrize("block", ["full_sphere", "torus"])
def test_mixed_form_l1(G, orc, block):
    if block == "full_sphere":
        s = I.full_sphere_setup(8, 12, 16)
        P = I.spherical_random_prims(s, seed=21)
    else:
        s, P = _torus_perturbed()
    p = orc.params(s)
    Po = P.copy()
    Uo, _, _ = orc.rk2_step(p, Po, orc.prim2con_grid(p, Po.copy()), 0.0)
    s.precision = "mixed"
    ctx = G.Context(s)
    ctx.set_prims(P.copy())
    ctx.rk2_step(0.0)
    ng = s.ng
    inner = (slice(None),) + (slice(ng, -ng),) * 3
    l1u, l1p = l1_rel(ctx.cons(), Uo), l1_rel(ctx.prims()[inner], Po[inner])
    assert l1u.max() <= 1e-6, (l1u, l1p)
    assert l1p.max() <= 1e-5, (l1u, l1p)


def test_spherical_refusals(G):
    """What the spherical metric does not run with is refused at creation."""
    import dataclasses
    s = I.full_sphere_setup(8, 12, 16)
    for bad in (dataclasses.replace(s, ct="face"), dataclasses.replace(s, scalar=True)):
        with pytest.raises(G.GrmhdError):
            G.Context(bad)
