"""Planted mistakes in the core oracle: copies of oracle/grmhd_oracle.cpp, each with one plausible error in
the metric, the fluid equations, reconstruction, the Riemann solvers, con2prim, the floors or the stage,
must each fail one of the oracle's pin files (run in a subprocess against that copy, selected through
GRMHD_ORACLE_SRC / GRMHD_ORACLE_BUILD). A mistake no pin notices would be a gap in the pins.

The planted mistakes, by the passage they break:
* Kerr-Schild metric (Sec. 2): the power of r in f = 2 M r^3 / (r^4 + a^2 z^2), the sign of a in the null
  vector l; the factor 1/2 of the Christoffel symbols;
* conserved variables and fluxes (Sec. 2, the Valencia form): the lapse in b^0 and in b^2, -D in tau, the
  total pressure in the momentum flux, the shift in the transport velocity, v^i in the tau flux;
* fast magnetosonic speed (the (1 - v_A^2) factor), geometric sources (the sign of the metric-derivative term
  and of the tau source);
* reconstruction (Sec. 3.1, App. B): the MC factor 2, the WENO linear weights in reverse, a wrong
  denominator in a candidate polynomial, the AOAH weight as an arithmetic instead of a harmonic mean;
* Riemann solvers: the sign of the dissipation term in LLF and in HLL;
* flux-CT: the 1/4 in the edge average of the EMF;
* the RK stage: the two state weights exchanged;
* con2prim (Kastaun et al. 2021): the sign of the B-term in qbar, the W factor of eps, min instead of max in
  nu; the floors (Sec. 3.2): the internal energy floor absolute instead of specific;
* the passive scalar (Sec. 2.1): X taken downwind, X from the old density, the RK weights exchanged, the
  ghosts not filled, the stencil of the face's left state shifted;
* spherical Kerr-Schild: the (1 + q) factor of g_{r phi}, the radial derivative of q, the ln r chain rule of
  the x^1 derivatives; the polar boundary: the sign change on the wrong component, no half turn in phi,
  flux through the axis faces, phi components reconstructed without the sin(theta) weight, the EMFs on the
  axis left as computed (along phi) or not averaged over phi (along r).
"""
import os
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import oracle as orc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_metric.py", "tests/test_oracle_fluid.py", "tests/test_oracle_recon_riemann.py",
        "tests/test_oracle_c2p.py", "tests/test_oracle_stage.py", "tests/test_oracle_boosted_waves.py",
        "tests/test_oracle_scalar.py", "tests/test_oracle_spherical_ks.py"]

MUTANTS = {
    "KS f power of r": ("const double f = 2.0 * M * r * r2 / Sig;", "const double f = 2.0 * M * r2 / Sig;"),
    "KS l_x sign of a": ("double l[4] = {1.0, (r * x + a * y) / ra,", "double l[4] = {1.0, (r * x - a * y) / ra,"),
    "Christoffel 1/2": ("G.Gam[d][a][b] = 0.5 * s;", "G.Gam[d][a][b] = s;"),
    "b^0 lapse": ("F.bcon[0] = F.W * Bv / G.alpha;", "F.bcon[0] = F.W * Bv;"),
    "b^2 lapse": ("F.b2 = (B2 + G.alpha * G.alpha * F.bcon[0] * F.bcon[0]) / (F.W * F.W);",
                  "F.b2 = (B2 + G.alpha * F.bcon[0] * F.bcon[0]) / (F.W * F.W);"),
    "tau without -D": ("F.bcon[0] * F.bcon[0] - U[0];", "F.bcon[0] * F.bcon[0];"),
    "momentum flux gas pressure": ("(i == j ? pstar : 0.0)", "(i == j ? F.p : 0.0)"),
    "tau flux velocity": ("Fl[4] = U[4] * vta + pstar * F.v[i]", "Fl[4] = U[4] * vta + pstar * vta"),
    "transport velocity shift sign": ("F.vt[i] = G.alpha * F.v[i] - G.beta[i];", "F.vt[i] = G.alpha * F.v[i] + G.beta[i];"),
    "fast speed factor": ("const double c2 = va2 + cs2 * (1.0 - va2);", "const double c2 = va2 + cs2;"),
    "source metric-derivative sign": ("s += T[m][n] * (G.dg[m][n][j] - gg);", "s += T[m][n] * (G.dg[m][n][j] + gg);"),
    "tau source sign": ("S[4] = G.alpha * (s1 - s2);", "S[4] = G.alpha * (s1 + s2);"),
    "MC factor 2": ("std::min(std::min(2.0 * std::fabs(dm), 2.0 * std::fabs(dp)), std::fabs(c));",
                    "std::min(std::min(std::fabs(dm), std::fabs(dp)), std::fabs(c));"),
    "WENO linear weights reversed": ("WENO_GAMMA[3] = {0.1, 0.6, 0.3};", "WENO_GAMMA[3] = {0.3, 0.6, 0.1};"),
    "WENO candidate denominator": ("const double P0 = (2.0 * f[0] - 7.0 * f[1] + 11.0 * f[2]) / 6.0;",
                                   "const double P0 = (2.0 * f[0] - 7.0 * f[1] + 11.0 * f[2]) / 5.0;"),
    "AOAH arithmetic mean": ("double sigma = 2.0 * sp * sm / (sp + sm);", "double sigma = 0.5 * (sp + sm);"),
    "LLF dissipation sign": ("0.5 * (L.F[v] + R.F[v]) - 0.5 * cmax * (R.U[v] - L.U[v]);",
                             "0.5 * (L.F[v] + R.F[v]) + 0.5 * cmax * (R.U[v] - L.U[v]);"),
    "HLL dissipation sign": ("(cr * L.F[v] - cl * R.F[v] + cr * cl * (R.U[v] - L.U[v])) / (cr - cl);",
                             "(cr * L.F[v] - cl * R.F[v] - cr * cl * (R.U[v] - L.U[v])) / (cr - cl);"),
    "EMF edge average": ("E[2 * gn + g.gi(fi, fj, k)] = 0.25 * (", "E[2 * gn + g.gi(fi, fj, k)] = 0.5 * ("),
    "RK state weights exchanged": ("Un[v] = g0 * u0 + g1 * Ucur[v * in + c] + beta * dt * L[v];",
                                   "Un[v] = g1 * u0 + g0 * Ucur[v * in + c] + beta * dt * L[v];"),
    "con2prim qbar B-term sign": ("const double qbar = c.q - 0.5 * c.b2 - 0.5 * mu * mu * x * x * (c.b2 * c.r2 - c.rb2);",
                                  "const double qbar = c.q - 0.5 * c.b2 + 0.5 * mu * mu * x * x * (c.b2 * c.r2 - c.rb2);"),
    "con2prim eps W factor": ("vh2 * Wh * Wh / (1.0 + Wh);", "vh2 * Wh / (1.0 + Wh);"),
    "con2prim nu min": ("const double nu = std::max(nuA, nuB);", "const double nu = std::min(nuA, nuB);"),
    "absolute internal energy floor": ("if (!(P[4] >= P[0] * eps_flr)) { P[4] = P[0] * eps_flr;",
                                       "if (!(P[4] >= eps_flr)) { P[4] = eps_flr;"),
    "scalar taken downwind": ("FX[d * gn + f] = mdot * (mdot >= 0.0 ? XL : XR);",
                              "FX[d * gn + f] = mdot * (mdot >= 0.0 ? XR : XL);"),
    "scalar from the old density": ("X[g.gi(i, j, k)] = DXnew[c] / Unew[c];", "X[g.gi(i, j, k)] = DXnew[c] / Ucur[c];"),
    "scalar RK weights exchanged": ("DXnew[c] = g0 * x0 + g1 * DXcur[c] + beta * dt * (-div);",
                                    "DXnew[c] = g1 * x0 + g0 * DXcur[c] + beta * dt * (-div);"),
    "scalar ghosts not filled": ("if (p->bc == 0) ghost_fill_periodic(g, X, 1);", "if (p->bc == 7) ghost_fill_periodic(g, X, 1);"),
    "spherical g_rphi factor": ("gs[1][3] = -a * s2 * (1.0 + q);", "gs[1][3] = -a * s2 * q;"),
    "spherical dq/dr": ("const double dqr = 2.0 * M * (Sig - r * dSr) / (Sig * Sig);",
                        "const double dqr = 2.0 * M * (Sig - 2.0 * r * dSr) / (Sig * Sig);"),
    "spherical ln r chain rule": ("G.dg[1][m][n] = k * fac * gs[m][n] + fac * r * gr[m][n];",
                                  "G.dg[1][m][n] = fac * r * gr[m][n];"),
    "polar sign on the radial component": ("const double f = (nvar == 8 && (v == 2 || v == 6)) ? sign : 1.0;",
                                           "const double f = (nvar == 8 && (v == 1 || v == 5)) ? sign : 1.0;"),
    "polar ghost without the half turn": ("          sk = wrap(sk + g.nz / 2, g.nz);\n", "          sk = wrap(sk, g.nz);\n"),
    "flux through the polar axis": ("if (p->metric == 2 && d == 1 && std::fabs(std::sin(xf[1])) < 1e-12) {",
                                    "if (p->metric == 2 && d == 1 && std::fabs(std::sin(xf[1])) < -1.0) {"),
    "phi components reconstructed unweighted": ("const bool reg = sph && (v == 3 || v == 7) && std::fabs(sfc) > 1e-12;",
                                                "const bool reg = false;"),
    "axis EMF along phi kept": ("if (p->metric == 2 && std::fabs(std::sin(g.xf(1, fj))) < 1e-12) {\n            E[2 * gn",
                                "if (p->metric == 7 && std::fabs(std::sin(g.xf(1, fj))) < 1e-12) {\n            E[2 * gn"),
    "axis EMF along r not averaged": ("    if (p->metric == 2)\n      for (int fj = 0; fj <= g.ny; fj += g.ny) {",
                                      "    if (p->metric == 7)\n      for (int fj = 0; fj <= g.ny; fj += g.ny) {"),
    "scalar left stencil": ("            cl[d] += q - 3;  // stencil of the cell below the face\n",
                            "            cl[d] += q - 2;  // stencil of the cell below the face\n"),
}


def _run(tmp, k, a, b, src):
    d = os.path.join(tmp, f"m{k}")
    os.makedirs(d)
    path = os.path.join(d, "grmhd_oracle.cpp")
    with open(path, "w") as f:
        f.write(src.replace(a, b))
    env = dict(os.environ, GRMHD_ORACLE_SRC=path, GRMHD_ORACLE_BUILD=d)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    summary = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else ""
    # caught: a pin test failed; a mutant that does not compile (an error, not a failure) is not a catch
    return r.returncode == 1 and " failed" in summary and " error" not in summary, summary


def test_planted_core_mistakes_fail_a_pin():
    with open(orc._SRC) as f:
        src = f.read()
    for name, (a, b) in MUTANTS.items():
        assert src.count(a) == 1, name
    with tempfile.TemporaryDirectory() as tmp:
        # an unchanged copy first: the pins must pass on it, or no failure below would mean anything
        d = os.path.join(tmp, "unchanged")
        os.makedirs(d)
        with open(os.path.join(d, "grmhd_oracle.cpp"), "w") as f:
            f.write(src)
        env = dict(os.environ, GRMHD_ORACLE_SRC=os.path.join(d, "grmhd_oracle.cpp"), GRMHD_ORACLE_BUILD=d)
        with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
            base = ex.submit(subprocess.run, [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                             cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
            res = list(ex.map(lambda kv: _run(tmp, kv[0], *kv[1][1], src), enumerate(MUTANTS.items())))
            base = base.result()
    assert base.returncode == 0, base.stdout[-2000:]
    missed = {name: summary for name, (caught, summary) in zip(MUTANTS, res) if not caught}
    assert not missed, missed
