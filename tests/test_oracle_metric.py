"""Pins of the oracle's analytic metric (paper Sec. 2.3) against properties that fix it.

* a = 0 reduces to Schwarzschild in Cartesian ingoing Kerr-Schild form (textbook).
* Kerr is a vacuum solution: the Ricci tensor built from the oracle's Christoffel symbols
  (finite-differenced in space) vanishes. A wrong sign, index or factor in g, its analytic
  derivatives or Gamma breaks this.
* The analytic derivatives match 4th-order central differences of g.
* det g = -1 in Cartesian Kerr-Schild, so sqrt(-g) = alpha sqrt(gamma) = 1.
* 3+1 consistency: alpha^2 = -1/g^{00}, beta_i = g_{0i} = gamma_ij beta^j, gamma^{ij} gamma_jk = delta.
"""
import numpy as np
import pytest

from paper_2410_09146_gb300 import inputs as I


def _pts(n=40, seed=0):
    rng = np.random.default_rng(seed)
    return rng.uniform(3.0, 23.0, size=(n, 3))


def test_schwarzschild_limit(orc):
    s = I.kerr_schild_setup(8)
    s.spin = 0.0
    p = orc.params(s)
    x = _pts()
    g = orc.geom_points(p, x)
    R = np.linalg.norm(x, axis=1)
    l = np.concatenate([np.ones((len(x), 1)), x / R[:, None]], axis=1)
    eta = np.diag([-1.0, 1, 1, 1])
    expect = eta[None] + (2.0 / R)[:, None, None] * l[:, :, None] * l[:, None, :]
    np.testing.assert_allclose(g["g"], expect, rtol=0, atol=1e-15)


def test_minkowski_is_flat(orc):
    p = orc.params(I.linear_wave_setup(8))
    g = orc.geom_points(p, _pts(5))
    np.testing.assert_array_equal(g["g"], np.broadcast_to(np.diag([-1.0, 1, 1, 1]), g["g"].shape))
    assert np.all(g["dg"] == 0) and np.all(g["alpha"] == 1) and np.all(g["beta"] == 0)


def _fd(fun, x, h=1e-3):
    """4th-order central difference of fun(points) along each axis -> [n][3][...]."""
    outs = []
    for k in range(3):
        e = np.zeros(3); e[k] = h
        d = (-fun(x + 2 * e) + 8 * fun(x + e) - 8 * fun(x - e) + fun(x - 2 * e)) / (12 * h)
        outs.append(d)
    return np.stack(outs, axis=1)


def test_analytic_derivatives_match_fd(orc):
    p = orc.params(I.kerr_schild_setup(8))
    x = _pts(30, 1)
    g = orc.geom_points(p, x)
    fd = _fd(lambda y: orc.geom_points(p, y)["g"], x)
    np.testing.assert_allclose(g["dg"], fd, rtol=0, atol=1e-10)
    fd_la = _fd(lambda y: np.log(orc.geom_points(p, y)["alpha"]), x)
    np.testing.assert_allclose(g["dlnalpha"], fd_la, rtol=0, atol=1e-10)


def test_det_and_3p1_split(orc):
    p = orc.params(I.kerr_schild_setup(8))
    x = _pts(50, 2)
    g = orc.geom_points(p, x)
    np.testing.assert_allclose(np.linalg.det(g["g"]), -1.0, rtol=0, atol=1e-13)
    np.testing.assert_allclose(g["sqrtmg"], 1.0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(g["alpha"] ** 2, -1.0 / g["gu"][:, 0, 0], rtol=1e-14)
    beta_low = np.einsum("nij,nj->ni", g["gam"], g["beta"])
    np.testing.assert_allclose(beta_low, g["g"][:, 0, 1:], rtol=0, atol=1e-14)
    eye = np.einsum("nij,njk->nik", g["gamu"], g["gam"])
    np.testing.assert_allclose(eye, np.broadcast_to(np.eye(3), eye.shape), rtol=0, atol=1e-14)
    np.testing.assert_allclose(g["sqrtgam"] ** 2, np.linalg.det(g["gam"]), rtol=1e-14)
    # Kerr-Schild: the lapse is below 1 and the shift points inwards-ish (f > 0).
    assert np.all(g["alpha"] < 1.0)


def _christoffel(g, dg, gu):
    """Gamma^d_{ab} from metric derivatives; dg has time index 0 = 0 (stationary)."""
    n = len(g)
    D = np.zeros((n, 4, 4, 4))
    D[:, 1:] = dg
    t = D.transpose(0, 2, 1, 3) + D.transpose(0, 2, 3, 1) - D  # [n][c][a][b]: d_a g_cb + d_b g_ca - d_c g_ab
    return 0.5 * np.einsum("ndc,ncab->ndab", gu, t)


def test_ricci_flat(orc):
    """Kerr is a vacuum solution: R_{mu nu} = 0 (Christoffels from the oracle, d Gamma by FD)."""
    p = orc.params(I.kerr_schild_setup(8))
    x = _pts(12, 3)

    def gam_at(y):
        g = orc.geom_points(p, y)
        return _christoffel(g["g"], g["dg"], g["gu"])

    G = gam_at(x)
    dG = np.zeros((len(x), 4, 4, 4, 4))  # dG[n][m][d][a][b] = d_m Gamma^d_ab
    dG[:, 1:] = _fd(gam_at, x, h=1e-3)
    ricci = (np.einsum("nllab->nab", dG) - np.einsum("nblal->nab", dG)
             + np.einsum("nlls,nsab->nab", G, G) - np.einsum("nlbs,nsal->nab", G, G))
    # The individual terms are O(1e-5) at r ~ 10; their sum must cancel to FD accuracy.
    scale = max(np.max(np.abs(np.einsum("nllab->nab", dG))), np.max(np.abs(np.einsum("nlbs,nsal->nab", G, G))))
    assert scale > 1e-6
    assert np.max(np.abs(ricci)) < 1e-7 * scale
