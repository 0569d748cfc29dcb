"""Pins of the oracle's reconstruction (paper Sec. 3.1, App. B) and Riemann solvers (Sec. 3.1).

* PLM (minmod and MC) is exact on linear data and returns the cell value at extrema.
* Every WENO5-Z candidate reproduces quadratic cell averages exactly, so any convex
  combination does: WENO5-Z is exact on quadratics, WENO5-Z-AOAH too (PLM part aside it
  mixes the same polynomial; on quadratics MC-PLM is not exact, so AOAH is checked on
  linear data and for sigma -> 1 on constants).
* WENO5-Z converges at fifth order on cell averages of sin(2 pi x); AOAH at >= 3.
* At a step, AOAH stays within the data range (no new extrema).
* AOAH mixes both faces of a cell with one weight sigma, a harmonic mean of the two face values
  sigma_{j+-1/2} (eq. def:sigma): it lies between the smaller side and their geometric mean (an
  arithmetic mean lies above the geometric one). The two sides share the three smoothness indicators
  (the mirrored face sees them with the linear weights reversed), so their ratio stays within [1/3, 3].
* Riemann: consistency F(U, U) = F(U) for LLF and HLL; HLL = upwind flux when all speeds > 0.
"""
import numpy as np

from paper_2410_09146_gb300 import inputs as I


def _stencils(vals):
    return np.stack([vals[j - 2:j + 3] for j in range(2, len(vals) - 2)])


def test_plm_exact_on_linear(orc):
    x = np.arange(12.0)
    f = 3.0 + 0.7 * x
    S = _stencils(f)
    for m in ("plm_minmod", "plm_mc", "weno5z_aoah"):
        qm, qp = orc.recon_points(m, S)
        np.testing.assert_allclose(qp, 3.0 + 0.7 * (x[2:-2] + 0.5), rtol=1e-14)
        np.testing.assert_allclose(qm, 3.0 + 0.7 * (x[2:-2] - 0.5), rtol=1e-14)
    # extremum: slopes vanish
    qm, qp = orc.recon_points("plm_mc", np.array([[0.0, 1.0, 2.0, 1.0, 0.0]]))
    assert qm[0] == 2.0 and qp[0] == 2.0


def test_mc_and_minmod_limiters(orc):
    qm, qp = orc.recon_points("plm_mc", np.array([[0, 0, 1.0, 4.0, 9.0]]))
    assert qp[0] == 1.0 + 0.5 * 2.0  # min(2*1, 2*3, 2) = 2
    qm, qp = orc.recon_points("plm_minmod", np.array([[0, 0, 1.0, 4.0, 9.0]]))
    assert qp[0] == 1.5


def _cell_avg(F, x0, h):
    return (F(x0 + h / 2) - F(x0 - h / 2)) / h


def test_weno_candidates_exact_on_quadratic_averages(orc):
    h = 0.1
    xc = np.arange(10) * h
    F = lambda x: 0.3 * x + 0.5 * x ** 2 - 0.4 * x ** 3  # primitive of 0.3 + x - 1.2 x^2
    f = _cell_avg(F, xc, h)
    exact = lambda x: 0.3 + x - 1.2 * x ** 2
    val, w, sig = orc.weno5z_points(_stencils(f))
    np.testing.assert_allclose(val, exact(xc[2:-2] + h / 2), rtol=1e-13)


def test_weno_fifth_order(orc):
    errs5, errs_ao = [], []
    for n in (32, 64, 128):
        h = 1.0 / n
        xc = (np.arange(-2, n + 2) + 0.5) * h
        f = (-np.cos(2 * np.pi * (xc + h / 2)) + np.cos(2 * np.pi * (xc - h / 2))) / (2 * np.pi * h)
        S = _stencils(f)
        exact = np.sin(2 * np.pi * (xc[2:-2] + h / 2))
        val, w, sig = orc.weno5z_points(S)
        errs5.append(np.max(np.abs(val - exact)))
        qm, qp = orc.recon_points("weno5z_aoah", S)
        errs_ao.append(np.max(np.abs(qp - exact)))
    r5 = np.log2(np.array(errs5[:-1]) / np.array(errs5[1:]))
    rao = np.log2(np.array(errs_ao[:-1]) / np.array(errs_ao[1:]))
    assert np.all(r5 > 4.5), r5
    assert np.all(rao > 3.0), rao


def test_aoah_sigma_limits(orc):
    # constant data: beta = 0 -> w = gamma -> sigma_side = 1
    val, w, sig = orc.weno5z_points(np.ones((1, 5)) * 2.0)
    np.testing.assert_allclose(w[0], [0.1, 0.6, 0.3], rtol=1e-15)
    np.testing.assert_allclose(sig[0], 1.0, rtol=1e-15)
    # step: no new extrema
    f = np.array([0, 0, 0, 0, 1.0, 1, 1, 1])
    qm, qp = orc.recon_points("weno5z_aoah", _stencils(f))
    assert np.all(qm >= -1e-15) and np.all(qm <= 1 + 1e-15)
    assert np.all(qp >= -1e-15) and np.all(qp <= 1 + 1e-15)


def test_riemann_consistency(orc):
    rng = np.random.default_rng(3)
    n = 50
    P = np.zeros((n, 8))
    P[:, 0] = 10 ** rng.uniform(-2, 0, n)
    P[:, 1:4] = rng.normal(size=(n, 3))
    P[:, 4] = P[:, 0] * rng.uniform(0.01, 2, n)
    P[:, 5:8] = rng.normal(size=(n, 3)) * 0.3
    for setup, lo, hi in ((I.linear_wave_setup(8), 0, 1), (I.kerr_schild_setup(8), 3, 23)):
        x = rng.uniform(lo, hi, (n, 3))
        for rs in ("llf", "hll"):
            setup.riemann = rs
            p = orc.params(setup)
            phys = orc.prim2con_points(p, x, P)
            for d in (1, 2, 3):
                Fh, cm = orc.riemann_points(p, x, P, P, d)
                np.testing.assert_allclose(Fh, phys["F"][:, d - 1], rtol=1e-13, atol=1e-13)


def test_hll_supersonic_is_upwind(orc):
    s = I.linear_wave_setup(8); s.riemann = "hll"
    p = orc.params(s)
    PL = np.array([[1.0, 5.0, 0, 0, 0.1, 0, 0, 0]])
    PR = np.array([[0.9, 4.8, 0, 0, 0.12, 0, 0, 0]])
    Fh, cm = orc.riemann_points(p, np.zeros((1, 3)), PL, PR, 1)
    phys = orc.prim2con_points(p, np.zeros((1, 3)), PL)
    np.testing.assert_allclose(Fh[0], phys["F"][0, 0], rtol=1e-14, atol=1e-16)


def test_aoah_sigma_is_a_harmonic_mean_of_the_sides(orc):
    rng = np.random.default_rng(2)
    n = 20000
    x = np.arange(5)[None, :] - 2.0
    f = rng.normal(size=(n, 1)) + rng.normal(size=(n, 1)) * x + 0.3 * rng.normal(size=(n, 1)) * x ** 2
    f += np.where(x >= rng.integers(0, 5, n)[:, None] - 1.5, rng.normal(size=(n, 1)) * 3, 0.0)  # a jump
    vp, _, sp = orc.weno5z_points(f)
    vm, _, sm = orc.weno5z_points(f[:, ::-1].copy())  # the j-1/2 face: the mirrored stencil
    ratio = np.maximum(sp, sm) / np.minimum(sp, sm)
    assert ratio.max() <= 3.0 * (1 + 1e-12) and ratio.max() > 2.9
    qm, qp = orc.recon_points("weno5z_aoah", f)
    lm, lp = orc.recon_points("plm_mc", f)
    scale = np.abs(f).max(1)
    use = (np.abs(vp - lp) > 1e-2 * scale) & (np.abs(vm - lm) > 1e-2 * scale) & (ratio > 1.5) & (np.maximum(sp, sm) < 1)
    assert use.sum() > 1000
    # the weight each face mixed with: q = sigma P5 + (1 - sigma) P_plm
    sig_p = ((qp - lp) / (vp - lp))[use]
    sig_m = ((qm - lm) / (vm - lm))[use]
    assert np.abs(sig_p - sig_m).max() < 1e-12
    lo, gm = np.minimum(sp, sm)[use], np.sqrt(sp * sm)[use]
    assert np.all(sig_p >= lo * (1 - 1e-12)) and np.all(sig_p <= gm * (1 + 1e-12))
