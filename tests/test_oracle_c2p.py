"""Pins of the oracle's con2prim (paper Sec. 3.1, the Kastaun et al. 2021 recovery) and floors (Sec. 3.2).

The prim->cons map is pinned independently (test_oracle_fluid); con2prim is its inverse, so
* on well-conditioned states (W <= 10, b^2/rho <= 10, p/rho >= 1e-4) prim -> cons -> prim
  returns rho and W v to 1e-12 and rho eps to 1e-14 of the energy scale (tau + D), which is
  the conditioning of that cancellation;
* on the full sampled range the backward error |U(P') - U| / |U| stays at roundoff
  (forward errors there are bounded by the conditioning, not by the solver);
* B = 0, v = 0 has the closed form rho = D, rho eps = tau;
* floors and the W ceiling fire exactly when their conditions hold; bad input is flagged; the internal
  energy floor is one on the specific internal energy (Sec. 3.2 sets it like the density floor,
  eps >= eps0 r^-2), so u is raised to rho eps_flr, and a thin but warm cell is left alone;
* an energy below that of the cold state with the same D, S and B (no eps >= 0 solution) is corrected
  by raising eps to the validity bound eps = 0 (Kastaun et al. 2021): the result is that cold state,
  reproducing D and S to roundoff; only tau changes.
"""
import numpy as np

from paper_2410_09146_gb300 import inputs as I


def _wellcond(n, seed):
    rng = np.random.default_rng(seed)
    P = np.zeros((n, 8))
    P[:, 0] = 10 ** rng.uniform(-4, 0, n)
    W = 10 ** rng.uniform(0, 1, n)
    d = rng.normal(size=(n, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
    P[:, 1:4] = np.sqrt(W * W - 1)[:, None] * d
    P[:, 4] = P[:, 0] * 10 ** rng.uniform(-4, 0, n) / (2.0 / 3.0)
    sig = 10 ** rng.uniform(-3, 1, n)
    db = rng.normal(size=(n, 3)); db /= np.linalg.norm(db, axis=1, keepdims=True)
    P[:, 5:8] = np.sqrt(sig * P[:, 0])[:, None] * db
    return P


def test_roundtrip_wellconditioned_minkowski_and_ks(orc):
    for setup, lo, hi in ((I.linear_wave_setup(8), 0.0, 1.0), (I.kerr_schild_setup(8), 3.0, 23.0)):
        p = orc.params(setup)
        n = 3000
        P = _wellcond(n, 11)
        x = np.random.default_rng(12).uniform(lo, hi, (n, 3))
        U = orc.prim2con_points(p, x, P)["U"]
        P2, st, it = orc.c2p_points(p, x, U, floors=False)
        assert np.all(st == 0)
        np.testing.assert_allclose(P2[:, 0], P[:, 0], rtol=1e-12)
        # rho eps is recovered from tau + D by cancellation: its error scales with (tau + D), not u.
        sg = orc.geom_points(p, x)["sqrtgam"]
        escale = (U[:, 4] + U[:, 0]) / sg
        assert np.max(np.abs(P2[:, 4] - P[:, 4]) / escale) < 1e-14
        W = np.sqrt(1 + np.sum(P[:, 1:4] ** 2, 1))
        np.testing.assert_allclose(P2[:, 1:4], P[:, 1:4], rtol=0, atol=1e-12 * W.max())
        np.testing.assert_allclose(P2[:, 5:8], P[:, 5:8], rtol=4e-16)  # sqrt(gamma) round trip


def test_backward_error_full_range(orc):
    p = orc.params(I.linear_wave_setup(8))
    P = I.c2p_states(5000, seed=3)
    x = np.zeros((len(P), 3))
    U = orc.prim2con_points(p, x, P)["U"]
    P2, st, it = orc.c2p_points(p, x, U, floors=False)
    assert np.all(st == 0)
    U2 = orc.prim2con_points(p, x, P2)["U"]
    scale = np.abs(U[:, 0]) + np.abs(U[:, 4]) + np.linalg.norm(U[:, 1:4], axis=1)
    be = np.max(np.abs(U2 - U), axis=1) / scale
    assert np.max(be) < 1e-11
    assert np.median(be) < 1e-14


def test_static_unmagnetised_closed_form(orc):
    p = orc.params(I.linear_wave_setup(8))
    rng = np.random.default_rng(5)
    n = 100
    U = np.zeros((n, 8))
    U[:, 0] = 10 ** rng.uniform(-6, 0, n)
    U[:, 4] = U[:, 0] * 10 ** rng.uniform(-6, 2, n)
    P, st, it = orc.c2p_points(p, np.zeros((n, 3)), U, floors=False)
    np.testing.assert_allclose(P[:, 0], U[:, 0], rtol=1e-15)
    np.testing.assert_allclose(P[:, 4], U[:, 4], rtol=1e-13)
    assert np.all(P[:, 1:4] == 0)


def test_floors_and_bad_input(orc):
    s = I.kerr_schild_setup(8)
    p = orc.params(s)
    x = np.array([[5.0, 5.0, 5.0]] * 5)
    r = np.sqrt(75.0)  # a = 0.9 barely changes r at this distance; the oracle uses the Kerr-Schild r
    P = np.array([[1e-14, 0, 0, 0, 1e-30, 0, 0, 0],        # both floors
                  [1.0, 0, 0, 0, 1e-14, 0, 0, 0],          # eps floor only
                  [1.0, 300.0, 0, 0, 1.0, 0, 0, 0],         # W ceiling
                  [1.0, 0.1, 0, 0, 1.0, 0, 0, 0],           # untouched
                  [1.0, 0.1, 0, 0, 1.0, 0, 0, 0]])
    U = orc.prim2con_points(p, x, P)["U"]
    U[4, 0] = np.nan
    P2, st, it = orc.c2p_points(p, x, U, floors=True)
    g = orc.geom_points(p, x)
    assert st[0] & orc.ST_RHO_FLOOR and st[0] & orc.ST_EPS_FLOOR
    assert st[1] == orc.ST_EPS_FLOOR
    assert st[2] & orc.ST_W_CAP  # capped inside the solve, which can also reset the internal energy
    assert st[3] == 0
    assert st[4] & orc.ST_BAD_INPUT
    assert P2[0, 0] >= 1e-10 / r ** 2 * 0.99
    W = np.sqrt(1 + np.einsum("ni,nij,nj->n", P2[:, 1:4], g["gam"], P2[:, 1:4]))
    np.testing.assert_allclose(W[2], 100.0, rtol=1e-13)


def test_specific_internal_energy_floor(orc):
    s = I.kerr_schild_setup(8)
    p = orc.params(s)
    x = np.array([[5.0, 5.0, 5.0]] * 2)
    # Kerr-Schild radius: r^4 - (R^2 - a^2) r^2 - a^2 z^2 = 0 with R^2 = x^2 + y^2 + z^2
    a, R2, z = s.spin * s.mass, 75.0, 5.0
    r = np.sqrt(0.5 * (R2 - a * a) + np.sqrt(0.25 * (R2 - a * a) ** 2 + a * a * z * z))
    eps_flr = s.eps_floor0 * r ** -s.floor_r_exp
    rho = 1e-3  # far above rho0 r^-2
    P = np.array([[rho, 0, 0, 0, rho * 0.01 * eps_flr, 0, 0, 0],   # eps below the floor
                  [rho, 0, 0, 0, rho * 100 * eps_flr, 0, 0, 0]])   # warm, u below eps_flr itself
    assert P[1, 4] < eps_flr
    U = orc.prim2con_points(p, x, P)["U"]
    P2, st, it = orc.c2p_points(p, x, U, floors=True)
    g = orc.geom_points(p, x)
    assert st[0] == orc.ST_EPS_FLOOR and st[1] == 0
    assert abs(P2[0, 4] / (rho * eps_flr) - 1) < 1e-13
    assert abs(P2[1, 4] - P[1, 4]) < 1e-14 * (U[1, 4] + U[1, 0]) / g["sqrtgam"][1]  # roundoff of tau + D
    np.testing.assert_allclose(P2[:, 0], rho, rtol=1e-14)


def test_energy_below_the_cold_state(orc):
    for setup, lo, hi in ((I.linear_wave_setup(8), 0.0, 1.0), (I.kerr_schild_setup(8), 3.0, 23.0)):
        p = orc.params(setup)
        rng = np.random.default_rng(7)
        n = 400
        P = np.zeros((n, 8))
        P[:, 0] = 10 ** rng.uniform(-3, 0, n)
        W = 10 ** rng.uniform(0, 0.7, n)
        d = rng.normal(size=(n, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
        P[:, 1:4] = np.sqrt(W * W - 1)[:, None] * d
        sig = 10 ** rng.uniform(0, 4, n)  # b^2 / rho
        db = rng.normal(size=(n, 3)); db /= np.linalg.norm(db, axis=1, keepdims=True)
        P[:, 5:8] = np.sqrt(sig * P[:, 0])[:, None] * db
        x = rng.uniform(lo, hi, (n, 3))
        U = orc.prim2con_points(p, x, P)["U"]        # the cold state: u = 0
        U[:, 4] -= U[:, 4] * 10 ** rng.uniform(-4, -1, n)
        P2, st, it = orc.c2p_points(p, x, U, floors=False)
        assert np.all(st == 0) and np.all(P2[:, 4] == 0.0)
        U2 = orc.prim2con_points(p, x, P2)["U"]
        np.testing.assert_allclose(U2[:, 0], U[:, 0], rtol=1e-14)
        assert np.max(np.abs(U2[:, 1:4] - U[:, 1:4]).max(1) / (np.abs(U[:, 1:4]).max(1) + U[:, 0])) < 1e-12
        np.testing.assert_allclose(P2[:, 0], P[:, 0], rtol=1e-10)
        assert np.max(np.abs(P2[:, 1:4] - P[:, 1:4])) < 1e-10
