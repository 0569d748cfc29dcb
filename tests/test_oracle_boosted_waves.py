"""Pins of the oracle's flat metric with a constant shift (the coordinate boost of the paper's 2-D linear-wave
tests, Sec. 4.1.1) and of the boosted-wave fixture tests/golden/boosted_waves.json.

* The metric is flat space in coordinates moving at -beta: g_00 = -1 + beta^2, g_0i = beta_i, g_ij = delta_ij, so
  alpha = 1, the shift is beta and gamma_ij = delta_ij (closed form).
* The conserved vector does not depend on the shift (it cancels algebraically: equal to roundoff); the fluxes do.
* Characteristic speeds in the moving coordinates are the unshifted ones minus beta.n, for every mode that moves
  with the fluid (the normal-field mode keeps zero speed), recomputed from the oracle's flux Jacobians.
* The oracle converges at second order to the exact translated plane wave (PLM-MC, HLL).
"""
import json
import os

import numpy as np

import oracle as orc
from oracle import make_golden as MG
from paper_2410_09146_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "boosted_waves.json")


def test_shifted_metric_closed_form():
    s = I.boosted_wave_setup(8)
    b = np.array(s.shift)
    G = orc.geom_points(orc.params(s), np.array([[0.3, 0.7, 0.1]]))
    g = G["g"][0]
    assert abs(g[0, 0] - (-1.0 + b @ b)) < 1e-15
    assert np.allclose(g[0, 1:], b, atol=1e-15) and np.allclose(g[1:, 1:], np.eye(3), atol=1e-15)
    assert abs(G["alpha"][0] - 1.0) < 1e-14
    assert np.allclose(G["beta"][0], b, atol=1e-14)
    assert np.allclose(G["gam"][0], np.eye(3), atol=1e-14) and np.allclose(G["gamu"][0], np.eye(3), atol=1e-14)
    assert abs(G["sqrtmg"][0] - 1.0) < 1e-14


def test_conserved_state_does_not_depend_on_the_shift():
    rng = np.random.default_rng(3)
    Ps = I.c2p_states(200, seed=3)
    x = rng.uniform(size=(200, 3))
    s0, s1 = I.boosted_wave_setup(8, shift=(0.0, 0.0, 0.0)), I.boosted_wave_setup(8)
    o0, o1 = orc.prim2con_points(orc.params(s0), x, Ps), orc.prim2con_points(orc.params(s1), x, Ps)
    # the shift cancels algebraically; the roundoff left is relative to the cancelling terms (~ B^2 W^2)
    W2 = 1.0 + np.sum(Ps[:, 1:4] ** 2, axis=1)
    scale = (np.abs(o0["U"]).max(axis=1) + np.sum(Ps[:, 5:8] ** 2, axis=1) * W2)[:, None]
    assert np.all(np.abs(o0["U"] - o1["U"]) <= 1e-14 * scale)
    assert not np.allclose(o0["F"], o1["F"])


def test_mode_speeds_shift_by_beta_dot_n():
    bw = MG.boosted_waves()
    bn = bw["shift_dot_n"]
    assert abs(bn - np.dot(bw["shift"], bw["n"])) < 1e-15
    for name, w in bw["waves"].items():
        assert abs(w["speed"] - (w["speed_unshifted"] - bn)) < 1e-9, name
        lam, lam0 = np.array(w["spectrum"]), np.array(w["spectrum_unshifted"])
        # every unshifted speed but one zero (the normal field's) reappears shifted by -beta.n
        moved = np.sort(np.concatenate([lam0[np.argsort(np.abs(lam0))[1:]] - bn, [0.0]]))
        assert np.allclose(np.sort(lam), moved, atol=1e-8), name
    # the stored fixture is what the oracle writes
    stored = json.load(open(GOLDEN))
    for name, w in bw["waves"].items():
        assert abs(stored["waves"][name]["speed"] - w["speed"]) < 1e-12
        assert np.allclose(stored["waves"][name]["eigvec_prims"], w["eigvec_prims"], atol=1e-10)


def _l1_after(n, t_end, wave="fast", amp=1e-6):
    g = json.load(open(GOLDEN))
    w = g["waves"][wave]
    s = I.boosted_wave_setup(n)
    p = orc.params(s)
    P = I.boosted_wave_prims(s, w["background_prims"], w["eigvec_prims"], w["speed"], amp)
    U = orc.prim2con_grid(p, P.copy())
    vmax = max(abs(v) for v in w["spectrum"])
    steps = int(np.ceil(t_end / (0.4 * s.dx[0] / vmax)))
    dt = t_end / steps
    for _ in range(steps):
        U, st, _ = orc.rk2_step(p, P, U, dt)
    exact = I.boosted_wave_prims(s, w["background_prims"], w["eigvec_prims"], w["speed"], amp, t=t_end)
    ng = s.ng
    inner = (slice(None), slice(ng, -ng), slice(ng, -ng), slice(ng, -ng))
    return float(np.abs(P[inner] - exact[inner]).sum() / (amp * n * n))


def test_oracle_second_order_on_the_boosted_fast_wave():
    e16, e32 = _l1_after(16, 0.25), _l1_after(32, 0.25)
    assert e16 / e32 > 3.2, (e16, e32)
