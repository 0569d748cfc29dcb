"""Exact solution of the 1-D special-relativistic hydrodynamic Riemann problem (gamma-law, v_t = 0, B = 0).

TEST INFRASTRUCTURE (part of the oracle): used only by the shock-tube tests.

The star pressure p* is found by bisection on v*_L(p) - v*_R(p) = 0. Each outer wave is
* a rarefaction when p* <= p_K: isentropic (p = K rho^Gamma) with the Riemann invariant
  artanh(v) +- (2/sqrt(Gamma-1)) artanh(c_s/sqrt(Gamma-1)) carried through the fan, the fan
  being self-similar with xi = (v -+ c_s)/(1 -+ v c_s);
* a shock when p* > p_K: the post-shock density from the Taub adiabat
  h_b^2 - h_a^2 = (h_a/rho_a + h_b/rho_b)(p_b - p_a), then the post-shock velocity and shock
  speed from the mass and energy jump conditions V_s [q] = [f(q)], found by bisection.
``shock_jump_residual`` reports the momentum jump condition, which the construction does not
impose, so the test of it is an independent check of the shock branch.
"""
from __future__ import annotations

import math

import numpy as np


def _bisect(f, a, b, tol=1e-15, maxit=300):
    fa, fb = f(a), f(b)
    if fa == 0:
        return a
    if fb == 0:
        return b
    assert fa * fb < 0, (a, b, fa, fb)
    for _ in range(maxit):
        m = 0.5 * (a + b)
        fm = f(m)
        if fm == 0 or (b - a) < tol * max(abs(m), 1e-300):
            return m
        if fa * fm < 0:
            b, fb = m, fm
        else:
            a, fa = m, fm
    return 0.5 * (a + b)


class State:
    def __init__(self, rho, p, v, gamma):
        self.rho, self.p, self.v, self.g = rho, p, v, gamma

    @property
    def h(self):
        return 1.0 + self.g / (self.g - 1.0) * self.p / self.rho

    @property
    def cs(self):
        return math.sqrt(self.g * self.p / (self.rho * self.h))

    @property
    def W(self):
        return 1.0 / math.sqrt(1.0 - self.v * self.v)

    def cons(self):
        W, h = self.W, self.h
        return np.array([self.rho * W, self.rho * h * W * W * self.v, self.rho * h * W * W - self.p])

    def flux(self):
        W, h = self.W, self.h
        return np.array([self.rho * W * self.v, self.rho * h * W * W * self.v ** 2 + self.p, self.rho * h * W * W * self.v])


def _inv(cs, g):
    return 2.0 / math.sqrt(g - 1.0) * math.atanh(cs / math.sqrt(g - 1.0))


def _rarefaction(a: State, p: float, sign: int) -> State:
    """State behind a rarefaction with pressure p; sign = -1 for the left wave, +1 for the right."""
    rho = a.rho * (p / a.p) ** (1.0 / a.g)
    s = State(rho, p, 0.0, a.g)
    # left wave (sign -1): artanh v + J(c) conserved; right wave: artanh v - J(c) conserved
    J = math.atanh(a.v) - sign * _inv(a.cs, a.g)
    s.v = math.tanh(J + sign * _inv(s.cs, a.g))
    return s


def _shock(a: State, p: float, sign: int):
    """Post-shock state and shock speed for post-shock pressure p > p_a (Taub adiabat + jumps)."""
    g = a.g
    k = g / (g - 1.0)
    dp = p - a.p
    # Taub adiabat as a quadratic in y = 1/rho_b with h_b = 1 + k p y
    A = k * k * p * p - k * p * dp
    B = 2.0 * k * p - dp
    C = 1.0 - a.h ** 2 - a.h * dp / a.rho
    if abs(A) < 1e-300:
        y = -C / B
    else:
        disc = math.sqrt(B * B - 4 * A * C)
        roots = [(-B + disc) / (2 * A), (-B - disc) / (2 * A)]
        y = max(r for r in roots if r > 0) if A > 0 else min(r for r in roots if r > 0)
    b = State(1.0 / y, p, 0.0, g)
    qa, fa = a.cons(), a.flux()

    def vs_of(v):
        b.v = v
        qb = b.cons()
        return (b.rho * b.W * v - fa[0]) / (qb[0] - qa[0])

    def energy(v):
        Vs = vs_of(v)
        qb, fb = b.cons(), b.flux()
        return Vs * (qb[2] - qa[2]) - (fb[2] - fa[2])

    eps = 1e-14
    if sign > 0:  # right-going shock: fluid behind it moves right relative to a
        lo, hi = a.v + eps * (1 - a.v), 1.0 - 1e-15
    else:
        lo, hi = -1.0 + 1e-15, a.v - eps * (1 + a.v)
    # energy(v) changes sign on (lo, hi); scan for a bracket
    vs = np.linspace(lo, hi, 2001)
    vals = [energy(v) for v in vs]
    br = None
    for i in range(len(vs) - 1):
        if vals[i] == 0 or vals[i] * vals[i + 1] < 0:
            br = (vs[i], vs[i + 1])
            if sign > 0:
                break
    assert br is not None
    v = _bisect(energy, *br)
    b.v = v
    return b, vs_of(v)


def shock_jump_residual(a: State, b: State, Vs: float):
    """|V_s [q] - [f]| / scale for (D, S, tau + D); the momentum row is not imposed by _shock."""
    dq = b.cons() - a.cons()
    df = b.flux() - a.flux()
    scale = np.abs(b.flux()) + np.abs(a.flux()) + np.abs(b.cons()) + np.abs(a.cons())
    return np.abs(Vs * dq - df) / scale


class RiemannSolution:
    def __init__(self, left: State, right: State):
        self.L, self.R = left, right
        g = left.g

        def star(p, side, sign):
            if p <= side.p:
                return _rarefaction(side, p, sign), None
            return _shock(side, p, sign)

        def gap(p):
            return star(p, left, -1)[0].v - star(p, right, +1)[0].v

        lo = 1e-8 * min(left.p, right.p)
        hi = 10.0 * max(left.p, right.p)
        self.pstar = _bisect(gap, lo, hi, tol=1e-15)
        self.starL, self.VsL = star(self.pstar, left, -1)
        self.starR, self.VsR = star(self.pstar, right, +1)
        self.vstar = 0.5 * (self.starL.v + self.starR.v)
        self.g = g

    def _fan(self, side: State, xi: float, sign: int) -> State:
        # inside a rarefaction: xi = (v + sign c)/(1 + sign v c) with the invariant of that family
        def f(p):
            s = _rarefaction(side, p, sign)
            return (s.v + sign * s.cs) / (1.0 + sign * s.v * s.cs) - xi
        p = _bisect(f, self.pstar, side.p) if self.pstar < side.p else self.pstar
        return _rarefaction(side, p, sign)

    def sample(self, xi: float) -> State:
        L, R, sL, sR = self.L, self.R, self.starL, self.starR
        if xi < self.vstar:
            if self.VsL is not None:  # shock
                return L if xi < self.VsL else sL
            head = (L.v - L.cs) / (1 - L.v * L.cs)
            tail = (sL.v - sL.cs) / (1 - sL.v * sL.cs)
            if xi < head:
                return L
            if xi > tail:
                return sL
            return self._fan(L, xi, -1)
        if self.VsR is not None:
            return R if xi > self.VsR else sR
        head = (R.v + R.cs) / (1 + R.v * R.cs)
        tail = (sR.v + sR.cs) / (1 + sR.v * sR.cs)
        if xi > head:
            return R
        if xi < tail:
            return sR
        return self._fan(R, xi, +1)

    def rho_at(self, x, t, x0=0.5):
        return np.array([self.sample((xx - x0) / t).rho for xx in np.atleast_1d(x)])
