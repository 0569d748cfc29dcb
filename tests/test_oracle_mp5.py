"""Pins of the oracle's MP5 reconstruction (Sec. 3.1 names the fifth-order monotonicity-preserving scheme of
Suresh & Huynh 1997 without formulas; the oracle restates the published scheme).

Properties fixed by the mathematics, not by the oracle's formulas:
* cell averages of any quartic: both face values equal the polynomial's point values (fifth-order
  interpolant, limiter inactive on monotone smooth data);
* smooth periodic data with extrema: the face error falls at fifth order in the max norm (the
  accuracy-preserving limiter does not clip smooth extrema);
* a step a | b: the face of the cell before the step takes exactly a, the face after it exactly b;
* linear advection of a square wave and a triangle with SSP-RK3 at CFL 1/(1 + alpha) = 0.2 (alpha = 4):
  no new extrema at any step (the monotonicity-preserving property the scheme is built for).
The MP parameter alpha = 4 and the 4/3 large-curvature weight are readings of the published scheme;
the advection pin fails for alpha large enough to break the CFL bound, not for smaller ones.
``test_planted_mistakes_fail_a_pin`` checks that copies of the oracle with a wrong interpolation weight,
swapped limited curvatures, a wrong lower bound or a reversed acceptance test each fail a pin.
"""
import importlib.util
import os
import tempfile

import numpy as np
import pytest

import oracle as orc


def _smooth_error(o, N):
    h = 1.0 / N
    x = (np.arange(N) + 0.5) * h
    F = lambda t: -np.cos(2 * np.pi * t) / (2 * np.pi) + 0.3 * np.sin(6 * np.pi * t) / (6 * np.pi)
    f = lambda t: np.sin(2 * np.pi * t) + 0.3 * np.cos(6 * np.pi * t)
    avg = (F(x + h / 2) - F(x - h / 2)) / h
    st = np.stack([np.roll(avg, -k) for k in (-2, -1, 0, 1, 2)], 1)
    qm, qp = o.recon_points("mp5", st)
    return max(np.abs(qp - f(x + h / 2)).max(), np.abs(qm - f(x - h / 2)).max())


def quartic_error(o):
    rng = np.random.default_rng(0)
    worst = 0.0
    for _ in range(20):
        c = np.array([rng.uniform(-1, 1), rng.uniform(0.5, 1.5), *rng.uniform(-0.2, 0.2, 3)]) * rng.choice([-1, 1])
        P = np.polynomial.Polynomial(c)
        Pi = P.integ()
        h = 0.1
        xs = np.arange(-2, 3) * h
        avg = (Pi(xs + h / 2) - Pi(xs - h / 2)) / h
        qm, qp = o.recon_points("mp5", avg[None])
        worst = max(worst, abs(qp[0] - P(h / 2)), abs(qm[0] - P(-h / 2)))
    return worst


def order(o):
    return float(np.log2(_smooth_error(o, 160) / _smooth_error(o, 320)))


def step_error(o):
    rng = np.random.default_rng(1)
    worst = 0.0
    for _ in range(50):
        a, b = rng.normal(size=2)
        qm, qp = o.recon_points("mp5", np.array([[a, a, a, b, b], [a, a, b, b, b]]))
        worst = max(worst, abs(qp[0] - a), abs(qm[1] - b))
    return worst


def advection_overshoot(o, N=100, steps=250, cfl=0.2):
    """u_t + u_x = 0 on a periodic grid, face flux from the upwind (plus) side, SSP-RK3: the largest excursion
    outside [0, 1] over all steps."""
    x = (np.arange(N) + 0.5) / N
    u = np.where((x > 0.2) & (x < 0.45), 1.0, 0.0)
    u += np.where((x > 0.6) & (x < 0.8), np.clip(1 - np.abs(x - 0.7) * 20, 0, 1) * 0.7, 0.0)

    def L(v):
        st = np.stack([np.roll(v, -k) for k in (-2, -1, 0, 1, 2)], 1)
        qp = o.recon_points("mp5", st)[1]
        return -(qp - np.roll(qp, 1)) * N

    dt = cfl / N
    worst = 0.0
    for _ in range(steps):
        u1 = u + dt * L(u)
        u2 = 0.75 * u + 0.25 * (u1 + dt * L(u1))
        u = u / 3 + 2.0 / 3.0 * (u2 + dt * L(u2))
        worst = max(worst, u.max() - 1.0, -u.min())
    return worst


def test_mp5_exact_on_quartics():
    assert quartic_error(orc) < 1e-13


def test_mp5_fifth_order_with_extrema():
    assert order(orc) > 4.9


def test_mp5_step_keeps_cell_values():
    assert step_error(orc) < 1e-15


def test_mp5_advection_creates_no_extrema():
    assert advection_overshoot(orc) <= 1e-14


def test_mp5_constant():
    qm, qp = orc.recon_points("mp5", np.full((3, 5), 2.5))
    assert np.all(qm == 2.5) and np.all(qp == 2.5)


_MUTANTS = {
    "interpolation weight": ("+ 27.0 * f[3]", "+ 26.0 * f[3]"),
    "limited curvatures swapped": ("const double vmd = vav - 0.5 * dhp;", "const double vmd = vav - 0.5 * dhm;"),
    "lower bound term": ("std::min(std::min(f[2], vul), vlc));\n  const double vmax",
                         "std::min(std::min(f[2], vul), vmd));\n  const double vmax"),
    "acceptance test reversed": ("if ((v - f[2]) * (v - vmp) <= 0.0) return v;",
                                 "if ((v - f[2]) * (v - vmp) >= 0.0) return v;"),
}


def test_planted_mistakes_fail_a_pin():
    with open(orc._SRC) as f:
        src = f.read()
    missed = []
    with tempfile.TemporaryDirectory() as tmp:
        for k, (name, (a, b)) in enumerate(_MUTANTS.items()):
            assert src.count(a) == 1, name
            d = os.path.join(tmp, f"m{k}")
            os.makedirs(d)
            path = os.path.join(d, "grmhd_oracle.cpp")
            with open(path, "w") as f:
                f.write(src.replace(a, b))
            spec = importlib.util.spec_from_file_location(f"oracle_mp5_planted_{k}", orc.__file__)
            o = importlib.util.module_from_spec(spec)
            spec.loader.exec_module(o)
            o._SRC, o._BUILD, o._SO = path, d, os.path.join(d, "liboracle.so")
            caught = (quartic_error(o) >= 1e-13 or order(o) <= 4.9 or step_error(o) >= 1e-15
                      or advection_overshoot(o) > 1e-14)
            if not caught:
                missed.append(name)
    assert not missed, missed
