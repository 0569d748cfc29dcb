"""Spherical Kerr-Schild coordinates (x^1, x^2, x^3) = (ln r, theta, phi) on the GPU (all-FP64 form, single-block
contexts, flux-CT) against the oracle, stage by stage through the C ABI, within 1e-12 per cell under the
condition-aware measure of tests/parity.py (the GPU's own state before each stage is the oracle's input):

* a full sphere with the spherical boundary (polar ghosts mirrored across the axis and turned by pi in phi,
  phi periodic): axis faces without flux, sin(theta)-weighted reconstruction of the phi components, the axis
  EMFs (zero along phi, the phi mean along r), the general geometric sources with sqrt(-g) != 1;
* a torus block away from the axis with fixed ghosts (the set-up of the paper's accretion runs), with
  a perturbed state and a field so the stage is far from stationary;
* the time step from the device's speeds equals the oracle's.
"""
import numpy as np
import pytest

from paper_2410_09146_gb300 import inputs as I
from tests.parity import compare_stage, interior_sqrtgam, rel_err_cons

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
    s = I.torus_setup(16, 4.0, 24.0, 0.5, np.pi - 0.5, nphi=6, dphi=0.05)
    P = I.torus_prims(s)
    rng = np.random.default_rng(23)
    P[0] *= 1.0 + 0.1 * rng.uniform(-1.0, 1.0, P[0].shape)
    P[4] *= 1.0 + 0.1 * rng.uniform(-1.0, 1.0, P[4].shape)
    P[5] = 1e-3 * rng.uniform(-1.0, 1.0, P[5].shape)
    P[6] = 1e-3 * rng.uniform(-1.0, 1.0, P[6].shape)
    _steps(G, orc, s, P)


def test_spherical_refusals(G):
    """What the spherical metric does not run with is refused at creation."""
    import dataclasses
    s = I.full_sphere_setup(8, 12, 16)
    for bad in (dataclasses.replace(s, precision="mixed"), dataclasses.replace(s, ct="face"),
                dataclasses.replace(s, scalar=True)):
        with pytest.raises(G.GrmhdError):
            G.Context(bad)
