"""Pins of the oracle's passive scalar (Sec. 2.1: (X rho u^mu)_{;mu} = S, here S = 0; the electron fraction
Y_e is the paper's use): conserved sqrt(gamma) D X, face flux = the stage's mass flux times X on its upwind
side, X = (sqrt(gamma) D X) / (sqrt(gamma) D) after the stage.

Fixed by the mathematics, not by the oracle's scalar code:
* a uniform X stays uniform (the scalar's flux is then X times the mass flux, exactly);
* a periodic block conserves the sum of sqrt(gamma) D X to roundoff;
* in a uniform flow (D and the mass flux constant) the scheme is upwind linear advection of X at the
  fluid's coordinate velocity v^x = u^x / W, with the face values of the (separately pinned)
  reconstruction and SSP-RK2: equal to that scheme written out here;
* a 0 / 1 step carried by a smooth compressible flow (PLM-MC) stays within [0, 1].
"""
import numpy as np
import pytest

import oracle as orc
from paper_2410_09146_gb300 import inputs as I


def _interior(a, ng=4):
    return a[..., ng:-ng, ng:-ng, ng:-ng]


def test_uniform_scalar_stays_uniform():
    s = I.kerr_schild_setup(12, recon="weno5z_aoah", riemann="hll")
    P = I.kerr_schild_random_prims(s, seed=5, rho_range=(0.1, 1.0), w_range=(1.0, 2.0), sigma_range=(0.01, 1.0),
                                   p_coef=0.5, kmax=1)
    p = orc.params(s)
    U = orc.prim2con_grid(p, P.copy())
    X = np.full(s.prim_shape()[1:], 0.3)
    DX = U[0] * 0.3
    for _ in range(2):
        U, DX, st, _ = orc.rk2_step_scalar(p, P, X, U, DX)
        # an internal-energy floor keeps rho and W (D re-derived to roundoff); a density floor would dilute X
        assert not np.any(st & orc.ST_RHO_FLOOR)
    assert np.max(np.abs(_interior(X) - 0.3)) < 1e-15


@pytest.mark.parametrize("recon", ["plm_mc", "weno5z_aoah"])
def test_periodic_block_conserves_the_scalar(recon):
    s = I.linear_wave_setup(16, recon=recon, riemann="hll")
    P, _ = I.smooth_random_prims(s, seed=3, amp=0.3, b_amp=0.3, kmax=1)
    p = orc.params(s)
    U = orc.prim2con_grid(p, P.copy())
    rng = np.random.default_rng(4)
    X = rng.uniform(0.0, 1.0, s.prim_shape()[1:])
    DX = U[0] * _interior(X)
    t0 = DX.sum()
    for _ in range(3):
        U, DX, st, _ = orc.rk2_step_scalar(p, P, X, U, DX)
    assert abs(DX.sum() - t0) < 1e-14 * np.abs(DX).sum()
    np.testing.assert_allclose(_interior(X), DX / U[0], rtol=1e-15)


def test_uniform_flow_is_upwind_linear_advection():
    n = 32
    s = I.Setup(n=(n, 4, 4), dx=(1.0 / n, 1.0 / n, 1.0 / n), recon="plm_mc", riemann="hll", bc="periodic")
    p = orc.params(s)
    P0 = np.array([1.0, 0.3, 0.0, 0.0, 1.5, 0.2, 0.1, 0.0])
    P = np.broadcast_to(P0[:, None, None, None], s.prim_shape()).copy()
    U = orc.prim2con_grid(p, P.copy())
    x = s.cell_centres(0, ghosts=False)
    x0 = np.sin(2 * np.pi * x) + np.where((x > 0.4) & (x < 0.7), 1.0, 0.0)
    X = np.broadcast_to(np.concatenate([x0[-4:], x0, x0[:4]])[None, None, :], s.prim_shape()[1:]).copy()
    DX = U[0] * _interior(X)
    a = P0[1] / np.sqrt(1.0 + P0[1] ** 2)  # v^x = u^x / W (flat metric, no shift)
    dt = 0.4 / n

    def L(v):  # upwind face values (a > 0: the cell below each face), periodic
        st = np.stack([np.roll(v, -k) for k in (-2, -1, 0, 1, 2)], 1)
        qp = orc.recon_points("plm_mc", st)[1]            # value at each cell's upper face
        return -a * (qp - np.roll(qp, 1)) * n

    v = x0.copy()
    for _ in range(5):
        U, DX, st, _ = orc.rk2_step_scalar(p, P, X, U, DX, dt)
        v1 = v + dt * L(v)
        v = 0.5 * v + 0.5 * (v1 + dt * L(v1))
    assert np.all(st == 0)
    Xi = _interior(X)
    assert np.max(np.abs(Xi - Xi[:1, :1, :])) == 0.0  # transversally uniform
    assert np.max(np.abs(Xi[0, 0] - v)) < 1e-13


def test_step_carried_by_a_compressible_flow_stays_bounded():
    s = I.linear_wave_setup(24, recon="plm_mc", riemann="hll")
    P, _ = I.smooth_random_prims(s, seed=6, amp=0.3, b_amp=0.3, kmax=1)
    p = orc.params(s)
    U = orc.prim2con_grid(p, P.copy())
    x = s.cell_centres(0)
    X = np.broadcast_to(np.where((x > 0.3) & (x < 0.6), 1.0, 0.0)[None, None, :], s.prim_shape()[1:]).copy()
    DX = U[0] * _interior(X)
    for _ in range(30):
        U, DX, st, _ = orc.rk2_step_scalar(p, P, X, U, DX)
        assert np.all(st == 0)
        assert _interior(X).min() >= -1e-14 and _interior(X).max() <= 1.0 + 1e-14
