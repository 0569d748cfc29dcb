"""Pins of the oracle's prim->cons map, fluxes, stress tensor, sources and speeds (paper Sec. 2.1).

* Flat space, B = 0: textbook special-relativistic hydrodynamics (D = rho W, S = rho h W^2 v,
  tau = rho h W^2 - p - D, fluxes U v + p terms).
* Flat space with B: the special-relativistic MHD closed forms
  S = (rho h W^2 + B^2) v - (B.v) B and tau = rho h W^2 - p + B^2 (1 + v^2)/2 - (B.v)^2/2 - D,
  induction flux B^k v^i - B^i v^k.
* Curved (Kerr-Schild): the conserved vector and fluxes against the stress tensor
  (tau + D = alpha^2 T^00, S_j = alpha T^0_j, F_Sj = T^i_j, F_tau + F_D = alpha T^{i0}),
  the trace T^mu_mu = 3p - rho - u, the orthogonality b.u = 0 and b^2 = b_mu b^mu.
* Sources: zero in Minkowski; S_j = 1/2 T^{mu nu} d_j g_{mu nu}; and the Killing-energy identity
  alpha S_tau - beta^j S_j + d_i alpha (F^i_tau + F^i_D) - d_i beta^j F^i_{S_j} = 0 of a stationary metric.
* Speeds: flat 1-D relativistic velocity addition (v +- c)/(1 +- v c); at rest with B
  perpendicular the exact fast speed vA^2 + cs^2 (1 - vA^2).
"""
import numpy as np

from paper_2410_09146_gb300 import inputs as I

G53 = 5.0 / 3.0


def _random_prims(n, seed, flat_B=True, wmax=5.0):
    rng = np.random.default_rng(seed)
    P = np.zeros((n, 8))
    P[:, 0] = 10 ** rng.uniform(-3, 0, n)
    P[:, 1:4] = rng.normal(size=(n, 3)) * rng.uniform(0, wmax, (n, 1)) / np.sqrt(3)
    P[:, 4] = P[:, 0] * 10 ** rng.uniform(-3, 1, n)
    if flat_B:
        P[:, 5:8] = rng.normal(size=(n, 3)) * np.sqrt(P[:, :1])
    return P


def _flat_fluid(P):
    rho, u = P[:, 0], P[:, 4]
    W = np.sqrt(1 + np.sum(P[:, 1:4] ** 2, 1))
    v = P[:, 1:4] / W[:, None]
    p = (G53 - 1) * u
    h = 1 + (u + p) / rho
    return rho, u, p, h, W, v


def test_flat_hydro_textbook(orc):
    p = orc.params(I.linear_wave_setup(8))
    P = _random_prims(200, 0, flat_B=False)
    out = orc.prim2con_points(p, np.zeros((200, 3)), P)
    rho, u, pr, h, W, v = _flat_fluid(P)
    U = out["U"]
    np.testing.assert_allclose(U[:, 0], rho * W, rtol=1e-14)
    np.testing.assert_allclose(U[:, 1:4], (rho * h * W * W)[:, None] * v, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(U[:, 4], rho * h * W * W - pr - rho * W, rtol=1e-12)
    for d in range(3):
        F = out["F"][:, d]
        np.testing.assert_allclose(F[:, 0], U[:, 0] * v[:, d], rtol=1e-13, atol=1e-16)
        mom = U[:, 1:4] * v[:, d:d + 1]
        mom[:, d] += pr
        np.testing.assert_allclose(F[:, 1:4], mom, rtol=1e-13, atol=1e-16)
        np.testing.assert_allclose(F[:, 4], (U[:, 4] + pr) * v[:, d], rtol=1e-12, atol=1e-16)


def test_flat_mhd_textbook(orc):
    p = orc.params(I.linear_wave_setup(8))
    P = _random_prims(300, 1)
    out = orc.prim2con_points(p, np.zeros((300, 3)), P)
    rho, u, pr, h, W, v = _flat_fluid(P)
    B = P[:, 5:8]
    B2 = np.sum(B * B, 1); Bv = np.sum(B * v, 1); v2 = np.sum(v * v, 1)
    U = out["U"]
    np.testing.assert_allclose(U[:, 1:4], (rho * h * W * W + B2)[:, None] * v - Bv[:, None] * B, rtol=1e-12,
                               atol=1e-14)
    tau = rho * h * W * W - pr + 0.5 * B2 * (1 + v2) - 0.5 * Bv ** 2 - rho * W
    np.testing.assert_allclose(U[:, 4], tau, rtol=1e-12)
    np.testing.assert_array_equal(U[:, 5:8], B)
    for d in range(3):
        Fb = out["F"][:, d, 5:8]
        expect = B * v[:, d:d + 1] - B[:, d:d + 1] * v
        np.testing.assert_allclose(Fb, expect, rtol=1e-13, atol=1e-15)


def _ks_points(n, seed):
    return np.random.default_rng(seed).uniform(3.0, 23.0, size=(n, 3))


def test_curved_cons_and_flux_vs_tmunu(orc):
    p = orc.params(I.kerr_schild_setup(8))
    n = 200
    x = _ks_points(n, 2)
    P = _random_prims(n, 3)
    out = orc.prim2con_points(p, x, P)
    g = orc.geom_points(p, x)
    T = out["T"]
    al, sg, smg = g["alpha"], g["sqrtgam"], g["sqrtmg"]
    U = out["U"] / sg[:, None]
    np.testing.assert_allclose(U[:, 4] + U[:, 0], al ** 2 * T[:, 0, 0], rtol=1e-12)
    T_mixed = np.einsum("nab,nbc->nac", T, g["g"])  # T^a_c
    np.testing.assert_allclose(U[:, 1:4], al[:, None] * T_mixed[:, 0, 1:], rtol=1e-11, atol=1e-12)
    for d in range(3):
        F = out["F"][:, d] / smg[:, None]
        np.testing.assert_allclose(F[:, 1:4], T_mixed[:, d + 1, 1:], rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(F[:, 4] + F[:, 0], al * T[:, d + 1, 0], rtol=1e-11, atol=1e-12)
    # trace and orthogonality
    tr = np.einsum("nab,nab->n", T, g["g"])
    pr = (G53 - 1) * P[:, 4]
    np.testing.assert_allclose(tr, 3 * pr - P[:, 0] - P[:, 4], rtol=1e-10, atol=1e-12)


def test_sources(orc):
    # Minkowski: identically zero.
    pm = orc.params(I.linear_wave_setup(8))
    P = _random_prims(50, 4)
    assert np.all(orc.prim2con_points(pm, np.zeros((50, 3)), P)["S"] == 0.0)
    # Kerr-Schild: S_j = 1/2 T^{mu nu} d_j g_{mu nu}; S_D = S_B = 0.
    p = orc.params(I.kerr_schild_setup(8))
    n = 200
    x = _ks_points(n, 5)
    P = _random_prims(n, 6)
    out = orc.prim2con_points(p, x, P)
    g = orc.geom_points(p, x)
    S = out["S"] / g["sqrtmg"][:, None]
    Sj = 0.5 * np.einsum("nab,njab->nj", out["T"], g["dg"])
    np.testing.assert_allclose(S[:, 1:4], Sj, rtol=1e-10, atol=1e-14)
    assert np.all(S[:, 0] == 0) and np.all(S[:, 5:] == 0)
    # Killing-energy identity with d alpha and d beta^j by 4th-order differences.
    h = 1e-3
    dal = np.zeros((n, 3)); dbe = np.zeros((n, 3, 3))
    for k in range(3):
        e = np.zeros(3); e[k] = h
        gs = [orc.geom_points(p, x + c * e) for c in (2, 1, -1, -2)]
        dal[:, k] = (-gs[0]["alpha"] + 8 * gs[1]["alpha"] - 8 * gs[2]["alpha"] + gs[3]["alpha"]) / (12 * h)
        dbe[:, k] = (-gs[0]["beta"] + 8 * gs[1]["beta"] - 8 * gs[2]["beta"] + gs[3]["beta"]) / (12 * h)
    F = out["F"] / g["sqrtmg"][:, None, None]
    lhs = (g["alpha"] * S[:, 4] - np.einsum("nj,nj->n", g["beta"], S[:, 1:4])
           + np.einsum("ni,ni->n", dal, F[:, :, 4] + F[:, :, 0])
           - np.einsum("nij,nij->n", dbe, F[:, :, 1:4]))
    scale = np.abs(g["alpha"] * S[:, 4]) + np.einsum("ni,ni->n", np.abs(dal), np.abs(F[:, :, 4]))
    assert np.max(np.abs(lhs) / scale) < 1e-8


def test_speeds_special_cases(orc):
    p = orc.params(I.linear_wave_setup(8))
    n = 100
    rng = np.random.default_rng(7)
    P = np.zeros((n, 8))
    P[:, 0] = 10 ** rng.uniform(-2, 0, n)
    P[:, 4] = P[:, 0] * 10 ** rng.uniform(-2, 1, n)
    vx = rng.uniform(-0.95, 0.95, n)
    P[:, 1] = vx / np.sqrt(1 - vx ** 2)
    out = orc.prim2con_points(p, np.zeros((n, 3)), P)
    pr = (G53 - 1) * P[:, 4]
    h = 1 + (P[:, 4] + pr) / P[:, 0]
    cs = np.sqrt(G53 * pr / (P[:, 0] * h))
    lam = out["lam"][:, 0]
    np.testing.assert_allclose(lam[:, 1], (vx + cs) / (1 + vx * cs), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(lam[:, 0], (vx - cs) / (1 - vx * cs), rtol=1e-13, atol=1e-15)
    # at rest, B along y, propagation along x: exact fast speed
    P2 = P.copy(); P2[:, 1:4] = 0; P2[:, 6] = rng.uniform(0.1, 3, n)
    lam2 = orc.prim2con_points(p, np.zeros((n, 3)), P2)["lam"][:, 0]
    b2 = P2[:, 6] ** 2
    va2 = b2 / (P2[:, 0] * h + b2)
    cf = np.sqrt(va2 + cs ** 2 * (1 - va2))
    np.testing.assert_allclose(lam2[:, 1], cf, rtol=1e-14)
    np.testing.assert_allclose(lam2[:, 0], -cf, rtol=1e-14)
