// Serial FP64 oracle for one explicit Runge-Kutta stage of the Valencia GRMHD
// finite-volume update of Barker et al., "Phoebus: Performance Portable GRRMHD
// for Relativistic Astrophysics" (arXiv:2410.09146).
//
// TEST INFRASTRUCTURE ONLY. This file is the correctness reference for the CUDA
// library. Only the test suite, the package smoke check and the CPU-baseline leg
// of the benchmark may load it. It shares no code, header or constant table with
// the CUDA path, and it is built with -O2 -ffp-contract=off (no FMA contraction).
//
// Every routine follows the paper's equations in the paper's notation:
//   Sec. 2.1  eq. (conservation law), (conserved vector), (flux vector),
//             (source vector), (3-velocity), (densitized 3-velocity),
//             (Lorentz factor), (b-B relations), (T^{mu nu}), (primitive vector)
//   Sec. 2.3  analytic metric and its derivatives (Cartesian Kerr-Schild)
//   Sec. 3.1  second-order FV, Toth flux-CT on cell-centred B, LLF / HLL,
//             constant / PLM (minmod, MC) / WENO5-Z-AOAH / MP5 reconstruction,
//             Kastaun et al. (2021) con2prim
//   Sec. 5    face-centred constrained transport (named there as planned work; the
//             scheme is the upwind CT of Gardiner & Stone 2005, see stage_impl)
//   Sec. 3.2  density / specific-energy floors rho0 r^-alpha
//   App. B    WENO5-Z-AOAH
// Readings where the paper is silent are stated at the routine that takes them.
//
// Array layouts (all C order, i fastest):
//   P  [8][ngz][ngy][ngx]  primitives rho, W v^1..3, rho*eps, B^1..3 incl. ghosts
//   U  [8][nz][ny][nx]     densitized conserved sqrt(gamma)*(D,S_1..3,tau,B^1..3)
//   status [nz][ny][nx]    uint8 bit set (ORC_ST_*)
//   Bf [3][ngz][ngy][ngx]  face-centred densitized field sqrt(gamma) B^d; entry (i,j,k) of component d
//                          is the lower d-face of ghosted cell (i,j,k)

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>

extern "C" {

typedef struct {
  int nx, ny, nz, ng;
  double x0[3];          // coordinate of the interior's lower corner
  double dx[3];          // cell widths
  int metric;            // 0 Minkowski, 1 Cartesian Kerr-Schild
  double spin;           // a/M
  double mass;           // M
  double gamma_eos;      // ideal-gas adiabatic index
  int recon;             // 0 constant, 1 PLM minmod, 2 PLM MC, 3 WENO5-Z-AOAH, 4 MP5
  int riemann;           // 0 LLF, 1 HLL
  int bc;                // 0 periodic, 1 fixed ghosts
  double rho_floor0;     // rho_flr = rho_floor0 * r^-floor_r_exp (KS) or rho_floor0 (Minkowski)
  double eps_floor0;     // u >= rho * eps_floor0 * r^-floor_r_exp
  double floor_r_exp;
  double w_max;          // Lorentz-factor ceiling
  double c2p_tol;        // unused by the oracle (it always converges to roundoff)
  int c2p_max_iter;      // unused by the oracle
  double cfl;
  double weno_eps;
  double shift[3];       // Minkowski only: constant shift beta^i of coordinates moving at -beta (zero: at rest)
} orc_params;

}  // extern "C"

namespace {

enum { ST_RHO_FLOOR = 1, ST_EPS_FLOOR = 2, ST_W_CAP = 4, ST_NOT_CONVERGED = 8, ST_BAD_INPUT = 16 };

// ---------------------------------------------------------------- metric (Sec. 2.3)
// Indices 0..3 are (t, x, y, z); Latin indices use 1..3 of the same arrays.
struct Geom {
  double g[4][4];        // g_{mu nu}
  double gu[4][4];       // g^{mu nu}
  double dg[4][4][4];    // dg[m][a][b] = d_m g_{ab}; m = 0 is zero (stationary)
  double alpha;
  double beta[4];        // beta^i at [1..3]
  double gam[4][4];      // gamma_{ij} at [1..3][1..3]
  double gamu[4][4];     // gamma^{ij}
  double sqrtgam, sqrtmg;
  double dlnalpha[4];    // d_m ln(alpha)
  double Gam[4][4][4];   // Gamma^d_{ab}
  double r;              // Kerr-Schild radius (1 for Minkowski), used by the floors
};

// Gauss-Jordan inverse of a 4x4 matrix with partial pivoting.
static void invert4(const double a_in[4][4], double inv[4][4]) {
  double a[4][8];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 8; ++j) a[i][j] = j < 4 ? a_in[i][j] : (j - 4 == i ? 1.0 : 0.0);
  for (int c = 0; c < 4; ++c) {
    int piv = c;
    for (int r = c + 1; r < 4; ++r)
      if (std::fabs(a[r][c]) > std::fabs(a[piv][c])) piv = r;
    if (piv != c)
      for (int j = 0; j < 8; ++j) std::swap(a[c][j], a[piv][j]);
    double d = a[c][c];
    for (int j = 0; j < 8; ++j) a[c][j] /= d;
    for (int r = 0; r < 4; ++r) {
      if (r == c) continue;
      double m = a[r][c];
      for (int j = 0; j < 8; ++j) a[r][j] -= m * a[c][j];
    }
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) inv[i][j] = a[i][j + 4];
}

static double det3(const double m[4][4]) {  // determinant of the [1..3][1..3] block
  return m[1][1] * (m[2][2] * m[3][3] - m[2][3] * m[3][2]) -
         m[1][2] * (m[2][1] * m[3][3] - m[2][3] * m[3][1]) +
         m[1][3] * (m[2][1] * m[3][2] - m[2][2] * m[3][1]);
}

// Kerr-Schild in Cartesian coordinates: g_{ab} = eta_{ab} + f l_a l_b with
// f = 2 M r^3 / (r^4 + a^2 z^2), l = (1, (r x + a y)/(r^2+a^2), (r y - a x)/(r^2+a^2), z/r),
// r the positive root of r^4 - (R^2 - a^2) r^2 - a^2 z^2 = 0. Derivatives are analytic
// (chain rule through r), which the paper allows alongside finite differences.
static void metric_eval(const orc_params& p, double x, double y, double z, Geom& G) {
  std::memset(&G, 0, sizeof(G));
  double eta[4][4] = {{-1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}};
  if (p.metric == 0) {
    // flat space in coordinates moving at constant velocity -shift (Sec. 4.1.1's boosted linear waves):
    // ds^2 = -dt^2 + (dx^i + beta^i dt)^2, i.e. g_00 = -1 + beta^2, g_0i = beta_i, g_ij = delta_ij
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) G.g[a][b] = eta[a][b];
    double b2 = 0.0;
    for (int i = 1; i <= 3; ++i) {
      G.g[0][i] = G.g[i][0] = p.shift[i - 1];
      b2 += p.shift[i - 1] * p.shift[i - 1];
    }
    G.g[0][0] = -1.0 + b2;
    G.r = 1.0;
  } else if (p.metric == 2) {
    // Kerr-Schild in spherical coordinates with a logarithmic radius, (x^1, x^2, x^3) = (ln r, theta, phi):
    // the radius and angles of the Cartesian form below through x + i y = (r + i a) e^{i phi} sin(theta),
    // z = r cos(theta). With Sigma = r^2 + a^2 cos^2(theta) and q = 2 M r / Sigma, in (t, r, theta, phi):
    // g_tt = -(1 - q), g_tr = q, g_tphi = -a sin^2 q, g_rr = 1 + q, g_rphi = -a sin^2 (1 + q),
    // g_thth = Sigma, g_phph = sin^2 (Sigma + a^2 sin^2 (1 + q)); each r index then carries a factor r
    // (dr = r dx^1) and d/dx^1 = r d/dr. Stationary and axisymmetric: no t or phi derivatives.
    const double M = p.mass, a = p.spin * p.mass;
    const double r = std::exp(x), sn = std::sin(y), cs = std::cos(y), s2 = sn * sn;
    const double Sig = r * r + a * a * cs * cs;
    const double q = 2.0 * M * r / Sig;
    const double dSr = 2.0 * r, dSt = -2.0 * a * a * cs * sn;          // d Sigma / dr, d Sigma / dtheta
    const double dqr = 2.0 * M * (Sig - r * dSr) / (Sig * Sig);          // dq / dr
    const double dqt = -2.0 * M * r * dSt / (Sig * Sig);                 // dq / dtheta
    double gs[4][4] = {}, gr[4][4] = {}, gt[4][4] = {};                  // g, d_r g, d_theta g in (t, r, theta, phi)
    gs[0][0] = -(1.0 - q); gr[0][0] = dqr; gt[0][0] = dqt;
    gs[0][1] = q; gr[0][1] = dqr; gt[0][1] = dqt;
    gs[0][3] = -a * s2 * q; gr[0][3] = -a * s2 * dqr; gt[0][3] = -a * (2.0 * sn * cs * q + s2 * dqt);
    gs[1][1] = 1.0 + q; gr[1][1] = dqr; gt[1][1] = dqt;
    gs[1][3] = -a * s2 * (1.0 + q); gr[1][3] = -a * s2 * dqr; gt[1][3] = -a * (2.0 * sn * cs * (1.0 + q) + s2 * dqt);
    gs[2][2] = Sig; gr[2][2] = dSr; gt[2][2] = dSt;
    const double Ep = Sig + a * a * s2 * (1.0 + q);
    gs[3][3] = s2 * Ep;
    gr[3][3] = s2 * (dSr + a * a * s2 * dqr);
    gt[3][3] = 2.0 * sn * cs * Ep + s2 * (dSt + a * a * (2.0 * sn * cs * (1.0 + q) + s2 * dqt));
    for (int m = 0; m < 4; ++m)
      for (int n = m + 1; n < 4; ++n) {
        gs[n][m] = gs[m][n];
        gr[n][m] = gr[m][n];
        gt[n][m] = gt[m][n];
      }
    for (int m = 0; m < 4; ++m)
      for (int n = 0; n < 4; ++n) {
        const int k = (m == 1) + (n == 1);
        const double fac = k == 0 ? 1.0 : (k == 1 ? r : r * r);
        G.g[m][n] = fac * gs[m][n];
        G.dg[1][m][n] = k * fac * gs[m][n] + fac * r * gr[m][n];  // r d/dr (r^k g)
        G.dg[2][m][n] = fac * gt[m][n];
      }
    G.r = r;
  } else {
    const double M = p.mass, a = p.spin * p.mass;
    const double xs[4] = {0.0, x, y, z};
    const double R2 = x * x + y * y + z * z;
    const double A = R2 - a * a;
    const double sq = std::sqrt(A * A + 4.0 * a * a * z * z);
    const double r2 = 0.5 * (A + sq);
    const double r = std::sqrt(r2);
    G.r = r;
    // d_k r from implicit differentiation of r^4 - (R^2 - a^2) r^2 - a^2 z^2 = 0
    double dr[4] = {0, 0, 0, 0};
    for (int k = 1; k <= 3; ++k) dr[k] = (xs[k] * r2 + (k == 3 ? a * a * z : 0.0)) / (r * sq);
    const double Sig = r2 * r2 + a * a * z * z;
    const double f = 2.0 * M * r * r2 / Sig;
    double df[4] = {0, 0, 0, 0};
    for (int k = 1; k <= 3; ++k) {
      double dSig = 4.0 * r * r2 * dr[k] + (k == 3 ? 2.0 * a * a * z : 0.0);
      df[k] = 2.0 * M * (3.0 * r2 * dr[k] * Sig - r * r2 * dSig) / (Sig * Sig);
    }
    const double ra = r2 + a * a;
    double l[4] = {1.0, (r * x + a * y) / ra, (r * y - a * x) / ra, z / r};
    double dl[4][4];  // dl[k][mu]
    std::memset(dl, 0, sizeof(dl));
    for (int k = 1; k <= 3; ++k) {
      double d1 = (k == 1 ? 1.0 : 0.0), d2 = (k == 2 ? 1.0 : 0.0), d3 = (k == 3 ? 1.0 : 0.0);
      dl[k][1] = ((dr[k] * x + r * d1 + a * d2) * ra - (r * x + a * y) * 2.0 * r * dr[k]) / (ra * ra);
      dl[k][2] = ((dr[k] * y + r * d2 - a * d1) * ra - (r * y - a * x) * 2.0 * r * dr[k]) / (ra * ra);
      dl[k][3] = (d3 * r - z * dr[k]) / r2;
    }
    for (int m = 0; m < 4; ++m)
      for (int n = 0; n < 4; ++n) G.g[m][n] = eta[m][n] + f * l[m] * l[n];
    for (int k = 1; k <= 3; ++k)
      for (int m = 0; m < 4; ++m)
        for (int n = 0; n < 4; ++n)
          G.dg[k][m][n] = df[k] * l[m] * l[n] + f * (dl[k][m] * l[n] + l[m] * dl[k][n]);
  }
  invert4(G.g, G.gu);
  // 3+1 split: alpha = (-g^{00})^{-1/2}, beta^i = -g^{0i}/g^{00}, gamma_ij = g_ij
  G.alpha = 1.0 / std::sqrt(-G.gu[0][0]);
  for (int i = 1; i <= 3; ++i) G.beta[i] = -G.gu[0][i] / G.gu[0][0];
  for (int i = 1; i <= 3; ++i)
    for (int j = 1; j <= 3; ++j) {
      G.gam[i][j] = G.g[i][j];
      G.gamu[i][j] = G.gu[i][j] - G.gu[0][i] * G.gu[0][j] / G.gu[0][0];
    }
  G.sqrtgam = std::sqrt(det3(G.gam));
  G.sqrtmg = G.alpha * G.sqrtgam;
  // d_m ln alpha = -1/2 d_m g^{00} / g^{00}, d_m g^{00} = -g^{0a} g^{0b} d_m g_{ab}
  for (int m = 0; m < 4; ++m) {
    double dgu00 = 0.0;
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) dgu00 -= G.gu[0][a] * G.gu[0][b] * G.dg[m][a][b];
    G.dlnalpha[m] = -0.5 * dgu00 / G.gu[0][0];
  }
  // Gamma^d_{ab} = 1/2 g^{dc} (d_a g_{cb} + d_b g_{ca} - d_c g_{ab})
  for (int d = 0; d < 4; ++d)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        double s = 0.0;
        for (int c = 0; c < 4; ++c) s += G.gu[d][c] * (G.dg[a][c][b] + G.dg[b][c][a] - G.dg[c][a][b]);
        G.Gam[d][a][b] = 0.5 * s;
      }
}

// ---------------------------------------------------------------- fluid state (Sec. 2.1)
struct Fluid {
  double rho, u, p, h;   // h = 1 + eps + p/rho
  double W;
  double v[4];           // v^i (Eulerian 3-velocity), [1..3]
  double vl[4];          // v_i
  double vt[4];          // densitized 3-velocity  v~^i = alpha v^i - beta^i
  double ucon[4];        // u^mu
  double bcon[4];        // b^mu
  double bcov[4];        // b_mu
  double Bcon[4];        // B^i
  double b2;
};

static void fluid_from_prims(const orc_params& p, const Geom& G, const double* P, Fluid& F) {
  std::memset(&F, 0, sizeof(F));
  F.rho = P[0];
  F.u = P[4];
  double ut[4] = {0, P[1], P[2], P[3]};  // W v^i
  for (int i = 1; i <= 3; ++i) F.Bcon[i] = P[4 + i];
  double usq = 0.0;
  for (int i = 1; i <= 3; ++i)
    for (int j = 1; j <= 3; ++j) usq += G.gam[i][j] * ut[i] * ut[j];
  F.W = std::sqrt(1.0 + usq);
  for (int i = 1; i <= 3; ++i) F.v[i] = ut[i] / F.W;
  for (int i = 1; i <= 3; ++i) {
    F.vl[i] = 0.0;
    for (int j = 1; j <= 3; ++j) F.vl[i] += G.gam[i][j] * F.v[j];
  }
  for (int i = 1; i <= 3; ++i) F.vt[i] = G.alpha * F.v[i] - G.beta[i];       // eq. (densitized 3-velocity)
  F.ucon[0] = F.W / G.alpha;                                                   // eq. (Lorentz factor)
  for (int i = 1; i <= 3; ++i) F.ucon[i] = F.W * (F.v[i] - G.beta[i] / G.alpha);  // eq. (3-velocity) solved for u^i
  double Bv = 0.0, B2 = 0.0;
  for (int i = 1; i <= 3; ++i) Bv += F.Bcon[i] * F.vl[i];
  for (int i = 1; i <= 3; ++i)
    for (int j = 1; j <= 3; ++j) B2 += G.gam[i][j] * F.Bcon[i] * F.Bcon[j];
  F.bcon[0] = F.W * Bv / G.alpha;                                               // eq. (b^0)
  for (int i = 1; i <= 3; ++i) F.bcon[i] = (F.Bcon[i] + G.alpha * F.bcon[0] * F.ucon[i]) / F.W;  // eq. (b^i)
  F.b2 = (B2 + G.alpha * G.alpha * F.bcon[0] * F.bcon[0]) / (F.W * F.W);       // eq. (b^2)
  for (int m = 0; m < 4; ++m) {
    F.bcov[m] = 0.0;
    for (int n = 0; n < 4; ++n) F.bcov[m] += G.g[m][n] * F.bcon[n];
  }
  F.p = (p.gamma_eos - 1.0) * F.u;  // ideal gas P = (Gamma - 1) rho eps
  F.h = (F.rho + F.u + F.p) / F.rho;
}

// Conserved vector (eq. conserved vector), NOT densitized.
static void cons_from_fluid(const Geom& G, const Fluid& F, double* U) {
  const double pstar = F.p + 0.5 * F.b2;
  const double w = F.rho * F.h + F.b2;
  U[0] = F.rho * F.W;
  for (int j = 1; j <= 3; ++j) U[j] = w * F.W * F.W * F.vl[j] - G.alpha * F.bcon[0] * F.bcov[j];
  U[4] = w * F.W * F.W - pstar - G.alpha * G.alpha * F.bcon[0] * F.bcon[0] - U[0];
  for (int k = 1; k <= 3; ++k) U[4 + k] = F.Bcon[k];
}

// Flux vector in direction i (eq. flux vector), NOT densitized.
static void flux_from_fluid(const Geom& G, const Fluid& F, const double* U, int i, double* Fl) {
  const double pstar = F.p + 0.5 * F.b2;
  const double vta = F.vt[i] / G.alpha;
  Fl[0] = U[0] * vta;
  for (int j = 1; j <= 3; ++j) Fl[j] = U[j] * vta + (i == j ? pstar : 0.0) - F.bcov[j] * F.Bcon[i] / F.W;
  Fl[4] = U[4] * vta + pstar * F.v[i] - G.alpha * F.bcon[0] * F.Bcon[i] / F.W;
  for (int k = 1; k <= 3; ++k) Fl[4 + k] = F.Bcon[k] * vta - F.Bcon[i] * F.vt[k] / G.alpha;
}

// Characteristic speeds in direction d. The paper does not state them; this is the
// Valencia sound-speed formula (Banyuls et al. 1997) with the sound speed replaced by
// the approximate fast speed c^2 = vA^2 + cs^2 (1 - vA^2). Its factors 1 - v^2, 1 - c^2 and
// 1 - v^2 c^2 are taken in the equal forms 1/W^2 (the Lorentz factor's definition),
// (1 - vA^2)(1 - cs^2) with 1 - vA^2 = rho h/(rho h + b^2), and (1 - c^2) + c^2 (1 - v^2): the
// differences 1 - v^2 etc. would round with an error amplified by W^2 (1e4 at the W cap).
static void speeds_from_fluid(const orc_params& p, const Geom& G, const Fluid& F, int d, double& lm, double& lp) {
  const double rhoh = F.rho * F.h;
  const double cs2 = p.gamma_eos * F.p / rhoh;
  const double va2 = F.b2 / (rhoh + F.b2);
  const double c2 = va2 + cs2 * (1.0 - va2);
  const double one_v2 = 1.0 / (F.W * F.W);
  const double one_c2 = rhoh / (rhoh + F.b2) * (1.0 - cs2);
  const double one_v2c2 = one_c2 + c2 * one_v2;
  const double vd = F.v[d];
  double disc = one_v2 * (G.gamu[d][d] * one_v2c2 - vd * vd * one_c2);
  if (disc < 0.0) disc = 0.0;
  const double c = std::sqrt(c2);
  const double pre = G.alpha / one_v2c2;
  lp = pre * (vd * one_c2 + c * std::sqrt(disc)) - G.beta[d];
  lm = pre * (vd * one_c2 - c * std::sqrt(disc)) - G.beta[d];
}

// Stress-energy tensor (eq. T^{mu nu}).
static void tmunu(const Geom& G, const Fluid& F, double T[4][4]) {
  const double w = F.rho + F.u + F.p + F.b2;
  const double pt = F.p + 0.5 * F.b2;
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) T[m][n] = w * F.ucon[m] * F.ucon[n] + pt * G.gu[m][n] - F.bcon[m] * F.bcon[n];
}

// Source vector (eq. source vector) without the radiation four-force, NOT densitized.
static void sources(const Geom& G, const Fluid& F, double* S) {
  double T[4][4];
  tmunu(G, F, T);
  for (int v = 0; v < 8; ++v) S[v] = 0.0;
  for (int j = 1; j <= 3; ++j) {
    double s = 0.0;
    for (int m = 0; m < 4; ++m)
      for (int n = 0; n < 4; ++n) {
        double gg = 0.0;
        for (int d = 0; d < 4; ++d) gg += G.Gam[d][n][m] * G.g[d][j];
        s += T[m][n] * (G.dg[m][n][j] - gg);
      }
    S[j] = s;
  }
  double s1 = 0.0, s2 = 0.0;
  for (int m = 0; m < 4; ++m) s1 += T[m][0] * G.dlnalpha[m];
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) s2 += T[m][n] * G.Gam[0][n][m];
  S[4] = G.alpha * (s1 - s2);
}

// ---------------------------------------------------------------- reconstruction (Sec. 3.1, App. B)
static double sgn(double a) { return a > 0 ? 1.0 : (a < 0 ? -1.0 : 0.0); }

static double slope_minmod(double dm, double dp) {
  if (dm * dp <= 0.0) return 0.0;
  return sgn(dm) * std::min(std::fabs(dm), std::fabs(dp));
}

// Monotonized-central limiter: minmod(2 dm, 2 dp, (dm + dp)/2).
static double slope_mc(double dm, double dp) {
  if (dm * dp <= 0.0) return 0.0;
  double c = 0.5 * (dm + dp);
  return sgn(dm) * std::min(std::min(2.0 * std::fabs(dm), 2.0 * std::fabs(dp)), std::fabs(c));
}

// WENO5-Z value at the face to the right of the centre cell of f[0..4] = f_{j-2..j+2}
// (App. B, eqs. interp:linear, low:order:polynomials, nonlinear:weights, weno:beta).
// Readings: third-order candidates in the standard cell-average (Jiang-Shu) form,
// linear weights (1/10, 6/10, 3/10), tau_Z = |beta_2 - beta_0|, p = 2.
static const double WENO_GAMMA[3] = {0.1, 0.6, 0.3};

static double weno5z_face(const double* f, double eps, double w[3]) {
  const double P0 = (2.0 * f[0] - 7.0 * f[1] + 11.0 * f[2]) / 6.0;
  const double P1 = (-f[1] + 5.0 * f[2] + 2.0 * f[3]) / 6.0;
  const double P2 = (2.0 * f[2] + 5.0 * f[3] - f[4]) / 6.0;
  double t;
  double b[3];
  t = f[0] - 2.0 * f[1] + f[2];
  b[0] = 13.0 / 12.0 * t * t;
  t = f[0] - 4.0 * f[1] + 3.0 * f[2];
  b[0] += 0.25 * t * t;
  t = f[1] - 2.0 * f[2] + f[3];
  b[1] = 13.0 / 12.0 * t * t;
  t = f[1] - f[3];
  b[1] += 0.25 * t * t;
  t = f[2] - 2.0 * f[3] + f[4];
  b[2] = 13.0 / 12.0 * t * t;
  t = 3.0 * f[2] - 4.0 * f[3] + f[4];
  b[2] += 0.25 * t * t;
  const double tau = std::fabs(b[2] - b[0]);
  double a[3], asum = 0.0;
  for (int k = 0; k < 3; ++k) {
    double q = tau / (b[k] + eps);
    a[k] = WENO_GAMMA[k] * (1.0 + q * q);
    asum += a[k];
  }
  for (int k = 0; k < 3; ++k) w[k] = a[k] / asum;
  return w[0] * P0 + w[1] * P1 + w[2] * P2;
}

// eq. (def:sigma:side)
static double weno_sigma_side(const double w[3]) {
  const double g0 = WENO_GAMMA[0], g1 = WENO_GAMMA[1], g2 = WENO_GAMMA[2];
  return 3.0 * w[0] * w[1] * w[2] / (g2 * w[0] * w[1] + g1 * w[0] * w[2] + g0 * w[1] * w[2]);
}

// MP5 (Sec. 3.1 names the fifth-order monotonicity-preserving scheme of Suresh & Huynh 1997,
// J. Comput. Phys. 136, 83, without formulas): value at the right face of the centre cell of
// f[0..4] = f_{j-2..j+2}. The fifth-order interpolant is kept when it lies between f_j and the
// monotonicity-preserving bound f_j + minmod(f_{j+1} - f_j, alpha (f_j - f_{j-1})); otherwise it is
// moved to the nearest end of the accuracy-preserving interval, whose ends combine the upper and
// middle limits with the large-curvature limits built from the limited second differences d^M4.
// Readings: alpha = 4 and the 4/3 curvature weight of the published scheme; the acceptance test is
// (v - f_j)(v - f_MP) <= 0 (no absolute epsilon, so the test does not depend on the data's scale).
static double minmod2(double a, double b) { return 0.5 * (sgn(a) + sgn(b)) * std::min(std::fabs(a), std::fabs(b)); }

static double minmod4(double w, double x, double y, double z) {
  const double s = 0.125 * (sgn(w) + sgn(x)) * std::fabs((sgn(w) + sgn(y)) * (sgn(w) + sgn(z)));
  return s * std::min(std::min(std::fabs(w), std::fabs(x)), std::min(std::fabs(y), std::fabs(z)));
}

static double mp5_face(const double* f) {
  const double alpha = 4.0;
  const double v = (2.0 * f[0] - 13.0 * f[1] + 47.0 * f[2] + 27.0 * f[3] - 3.0 * f[4]) / 60.0;
  const double vmp = f[2] + minmod2(f[3] - f[2], alpha * (f[2] - f[1]));
  if ((v - f[2]) * (v - vmp) <= 0.0) return v;
  const double dm = f[0] - 2.0 * f[1] + f[2];  // second differences at j-1, j, j+1
  const double d0 = f[1] - 2.0 * f[2] + f[3];
  const double dp = f[2] - 2.0 * f[3] + f[4];
  const double dhp = minmod4(4.0 * d0 - dp, 4.0 * dp - d0, d0, dp);  // limited curvature at j+1/2
  const double dhm = minmod4(4.0 * d0 - dm, 4.0 * dm - d0, d0, dm);  // and at j-1/2
  const double vul = f[2] + alpha * (f[2] - f[1]);                   // upper limit
  const double vav = 0.5 * (f[2] + f[3]);
  const double vmd = vav - 0.5 * dhp;                                 // median
  const double vlc = f[2] + 0.5 * (f[2] - f[1]) + 4.0 / 3.0 * dhm;    // large curvature
  const double vmin = std::max(std::min(std::min(f[2], f[3]), vmd), std::min(std::min(f[2], vul), vlc));
  const double vmax = std::min(std::max(std::max(f[2], f[3]), vmd), std::max(std::max(f[2], vul), vlc));
  return v + minmod2(vmin - v, vmax - v);  // the median of v, vmin, vmax
}

// Reconstruct the two face values of cell j from f[0..4] = f_{j-2..j+2}.
// qm = value at x_{j-1/2}, qp = value at x_{j+1/2}.
static void recon_cell(int method, const double* f, double eps, double& qm, double& qp) {
  const double fj = f[2];
  if (method == 0) {
    qm = qp = fj;
    return;
  }
  if (method == 4) {  // MP5; the j-1/2 face from the mirrored stencil
    const double fr[5] = {f[4], f[3], f[2], f[1], f[0]};
    qp = mp5_face(f);
    qm = mp5_face(fr);
    return;
  }
  const double dm = f[2] - f[1], dp = f[3] - f[2];
  if (method == 1 || method == 2) {
    double s = method == 1 ? slope_minmod(dm, dp) : slope_mc(dm, dp);
    qm = fj - 0.5 * s;
    qp = fj + 0.5 * s;
    return;
  }
  // WENO5-Z-AOAH: the j-1/2 face uses the mirrored stencil x -> -x.
  double wp[3], wm[3];
  const double fr[5] = {f[4], f[3], f[2], f[1], f[0]};
  const double P5p = weno5z_face(f, eps, wp);
  const double P5m = weno5z_face(fr, eps, wm);
  const double sp = weno_sigma_side(wp), sm = weno_sigma_side(wm);
  double sigma = 2.0 * sp * sm / (sp + sm);   // eq. (def:sigma)
  if (sigma > 1.0) sigma = 1.0;                // the paper states 0 < sigma < 1
  const double s = slope_mc(dm, dp);          // MC-limited linear part
  qp = sigma * P5p + (1.0 - sigma) * (fj + 0.5 * s);   // eq. (weno:lin)
  qm = sigma * P5m + (1.0 - sigma) * (fj - 0.5 * s);
}

// ---------------------------------------------------------------- Riemann solvers (Sec. 3.1)
struct FaceSide {
  double U[8];    // sqrt(gamma) U
  double F[8];    // sqrt(-g) F^d
  double lm, lp;  // characteristic speeds
};

static void face_side(const orc_params& p, const Geom& G, const double* P, int d, FaceSide& s) {
  Fluid F;
  fluid_from_prims(p, G, P, F);
  double U[8], Fl[8];
  cons_from_fluid(G, F, U);
  flux_from_fluid(G, F, U, d, Fl);
  for (int v = 0; v < 8; ++v) {
    s.U[v] = G.sqrtgam * U[v];
    s.F[v] = G.sqrtmg * Fl[v];
  }
  speeds_from_fluid(p, G, F, d, s.lm, s.lp);
}

// Returns the face flux and the largest |speed| of the two sides.
static double riemann(const orc_params& p, const FaceSide& L, const FaceSide& R, double* Fhat) {
  const double cmax = std::max(std::max(std::fabs(L.lm), std::fabs(L.lp)), std::max(std::fabs(R.lm), std::fabs(R.lp)));
  if (p.riemann == 0) {  // local Lax-Friedrichs
    for (int v = 0; v < 8; ++v) Fhat[v] = 0.5 * (L.F[v] + R.F[v]) - 0.5 * cmax * (R.U[v] - L.U[v]);
  } else {               // HLL
    const double cl = std::min(0.0, std::min(L.lm, R.lm));
    const double cr = std::max(0.0, std::max(L.lp, R.lp));
    if (cr - cl == 0.0) {
      for (int v = 0; v < 8; ++v) Fhat[v] = 0.5 * (L.F[v] + R.F[v]);
    } else {
      for (int v = 0; v < 8; ++v) Fhat[v] = (cr * L.F[v] - cl * R.F[v] + cr * cl * (R.U[v] - L.U[v])) / (cr - cl);
    }
  }
  return cmax;
}

// ---------------------------------------------------------------- con2prim (Sec. 3.1: Kastaun et al. 2021)
// Restated from the published method: with q = tau/D, r_i = S_i/D, b^i = B^i/sqrt(D) and the
// unknown mu = 1/(h W), the master function f(mu) = mu - 1/(nu(mu) + mu rbar^2(mu)) has a
// unique root in [0, mu_+], mu_+ the root of f_a(mu) = mu sqrt(h0^2 + rbar^2(mu)) - 1 (h0 = 1).
// The oracle brackets both roots and runs Brent's method to roundoff.
struct C2PCtx {
  double D, q, r2, b2, rb2, gm1, v0sq;
};

static double rbar2_of(const C2PCtx& c, double mu, double& x) {
  x = 1.0 / (1.0 + mu * c.b2);
  return x * x * c.r2 + mu * x * (1.0 + x) * c.rb2;
}

static double fa_of(const C2PCtx& c, double mu) {
  double x;
  double rb = rbar2_of(c, mu, x);
  return mu * std::sqrt(1.0 + rb) - 1.0;
}

struct MasterOut {
  double f, x, rbar2, W, rho, eps;
};

static double master_f(const C2PCtx& c, double mu, MasterOut* o) {
  double x;
  const double rb = rbar2_of(c, mu, x);
  const double qbar = c.q - 0.5 * c.b2 - 0.5 * mu * mu * x * x * (c.b2 * c.r2 - c.rb2);
  double vh2 = mu * mu * rb;
  if (vh2 > c.v0sq) vh2 = c.v0sq;
  const double Wh = 1.0 / std::sqrt(1.0 - vh2);
  const double rhoh = c.D / Wh;
  double epsh = Wh * (qbar - mu * rb) + vh2 * Wh * Wh / (1.0 + Wh);
  if (epsh < 0.0) epsh = 0.0;  // ideal-gas validity range eps >= 0
  const double Ph = c.gm1 * rhoh * epsh;
  const double ah = Ph / (rhoh * (1.0 + epsh));
  const double nuA = (1.0 + ah) * (1.0 + epsh) / Wh;
  const double nuB = (1.0 + ah) * (1.0 + qbar - mu * rb);
  const double nu = std::max(nuA, nuB);
  const double f = mu - 1.0 / (nu + mu * rb);
  if (o) {
    o->f = f; o->x = x; o->rbar2 = rb; o->W = Wh; o->rho = rhoh; o->eps = epsh;
  }
  return f;
}

// Brent's method for a root of fn on [a, b] with fn(a) fn(b) <= 0, to roundoff.
template <class Fn>
static double brent(Fn fn, double a, double b, double fa, double fb, int* iters) {
  if (fa == 0.0) return a;
  if (fb == 0.0) return b;
  double c = a, fc = fa, d = b - a, e = d;
  int it = 0;
  for (; it < 400; ++it) {
    if ((fb > 0 && fc > 0) || (fb < 0 && fc < 0)) {
      c = a; fc = fa; d = b - a; e = d;
    }
    if (std::fabs(fc) < std::fabs(fb)) {
      a = b; b = c; c = a;
      fa = fb; fb = fc; fc = fa;
    }
    const double tol = 2.0 * 2.220446049250313e-16 * std::fabs(b) + 1e-300;
    const double m = 0.5 * (c - b);
    if (std::fabs(m) <= tol || fb == 0.0) break;
    if (std::fabs(e) >= tol && std::fabs(fa) > std::fabs(fb)) {
      double s = fb / fa, pp, qq;
      if (a == c) {
        pp = 2.0 * m * s;
        qq = 1.0 - s;
      } else {
        double qa = fa / fc, r = fb / fc;
        pp = s * (2.0 * m * qa * (qa - r) - (b - a) * (r - 1.0));
        qq = (qa - 1.0) * (r - 1.0) * (s - 1.0);
      }
      if (pp > 0) qq = -qq; else pp = -pp;
      if (2.0 * pp < std::min(3.0 * m * qq - std::fabs(tol * qq), std::fabs(e * qq))) {
        e = d; d = pp / qq;
      } else {
        d = m; e = m;
      }
    } else {
      d = m; e = m;
    }
    a = b; fa = fb;
    b += std::fabs(d) > tol ? d : (m > 0 ? tol : -tol);
    fb = fn(b);
  }
  if (iters) *iters += it;
  return b;
}

struct C2PResult {
  double P[8];
  int status;
  int iters;
  double mu, mup;  // root of the master function and the upper end of its bracket
  double eps_p, W_p;  // eps and W of the master-function intermediates at mu_+
};

// Undensitized conserved Uc = (D, S_j, tau, B^k) -> primitives, before floors.
static void con2prim_point(const orc_params& p, const Geom& G, const double* Uc, C2PResult& R) {
  R.status = 0;
  R.iters = 0;
  for (int v = 0; v < 8; ++v) R.P[v] = 0.0;
  bool finite = true;
  for (int v = 0; v < 8; ++v) finite = finite && std::isfinite(Uc[v]);
  R.mu = R.mup = R.eps_p = R.W_p = 0.0;
  if (!finite || !(Uc[0] > 0.0)) {
    R.status = ST_BAD_INPUT;
    for (int k = 1; k <= 3; ++k) R.P[4 + k] = std::isfinite(Uc[4 + k]) ? Uc[4 + k] : 0.0;
    return;
  }
  C2PCtx c;
  c.D = Uc[0];
  c.q = Uc[4] / c.D;
  double rl[4] = {0, Uc[1] / c.D, Uc[2] / c.D, Uc[3] / c.D};
  double ru[4] = {0, 0, 0, 0};
  for (int i = 1; i <= 3; ++i)
    for (int j = 1; j <= 3; ++j) ru[i] += G.gamu[i][j] * rl[j];
  const double sD = std::sqrt(c.D);
  double bu[4] = {0, Uc[5] / sD, Uc[6] / sD, Uc[7] / sD};
  c.r2 = 0.0; c.b2 = 0.0;
  double rb = 0.0;
  for (int i = 1; i <= 3; ++i) {
    c.r2 += rl[i] * ru[i];
    rb += rl[i] * bu[i];
    for (int j = 1; j <= 3; ++j) c.b2 += G.gam[i][j] * bu[i] * bu[j];
  }
  c.rb2 = rb * rb;
  c.gm1 = p.gamma_eos - 1.0;
  // Velocity bound inside the solve: the physical bound v^2 <= r^2/(h0^2 + r^2) (h0 = 1), and the
  // Lorentz-factor ceiling v^2 <= 1 - 1/w_max^2 (reading: it keeps W(mu) bounded for unphysical states).
  c.v0sq = std::min(c.r2 / (1.0 + c.r2), 1.0 - 1.0 / (p.w_max * p.w_max));
  // Upper bracket mu_+ from f_a on (0, 1/h0].
  double mup = 1.0;
  double fa1 = fa_of(c, 1.0);
  if (fa1 > 0.0) mup = brent([&](double m) { return fa_of(c, m); }, 0.0, 1.0, -1.0, fa1, nullptr);
  // Root of the master function on [0, mu_+]; f(0) = -1/nu(0) < 0.
  double f0 = master_f(c, 0.0, nullptr);
  MasterOut op;
  double fup = master_f(c, mup, &op);
  R.eps_p = op.eps;
  R.W_p = op.W;
  double mu;
  if (fup <= 0.0) {
    // Analytically f(mu_+) >= 0 (nu >= (1+a)(1+eps)/W >= sqrt(1 - v^2) there); a non-positive
    // value is roundoff at a root that sits on mu_+ itself.
    mu = mup;
  } else {
    mu = brent([&](double m) { return master_f(c, m, nullptr); }, 0.0, mup, f0, fup, &R.iters);
  }
  R.mu = mu;
  R.mup = mup;
  MasterOut o;
  master_f(c, mu, &o);
  const double W = o.W;
  R.P[0] = o.rho;
  for (int i = 1; i <= 3; ++i) {
    double vi = mu * o.x * (ru[i] + mu * rb * bu[i]);
    R.P[i] = W * vi;
  }
  R.P[4] = o.rho * o.eps;
  for (int k = 1; k <= 3; ++k) R.P[4 + k] = Uc[4 + k];
}

// Floors (Sec. 3.2) and the Lorentz-factor ceiling. Readings: rho_flr = rho0 r^-alpha
// (Kerr-Schild radius r; in the spherical coordinates x^1 = ln r this is the paper's rho0 e^{-alpha x^1})
// or rho0 (Minkowski); u >= rho eps0 r^-alpha; W <= w_max.
static int apply_floors(const orc_params& p, const Geom& G, double* P) {
  int st = 0;
  double fr = p.metric >= 1 ? std::pow(G.r, -p.floor_r_exp) : 1.0;
  const double rho_flr = p.rho_floor0 * fr;
  const double eps_flr = p.eps_floor0 * fr;
  if (!(P[0] >= rho_flr)) { P[0] = rho_flr; st |= ST_RHO_FLOOR; }
  if (!(P[4] >= P[0] * eps_flr)) { P[4] = P[0] * eps_flr; st |= ST_EPS_FLOOR; }
  double usq = 0.0;
  for (int i = 1; i <= 3; ++i)
    for (int j = 1; j <= 3; ++j) usq += G.gam[i][j] * P[i] * P[j];
  const double W = std::sqrt(1.0 + usq);
  if (W > p.w_max) {
    double s = std::sqrt((p.w_max * p.w_max - 1.0) / usq);
    for (int i = 1; i <= 3; ++i) P[i] *= s;
    st |= ST_W_CAP;
  }
  return st;
}

// ---------------------------------------------------------------- grid helpers
struct Grid {
  const orc_params& p;
  int nx, ny, nz, ng, gx, gy, gz;
  explicit Grid(const orc_params& pp) : p(pp) {
    nx = p.nx; ny = p.ny; nz = p.nz; ng = p.ng;
    gx = nx + 2 * ng; gy = ny + 2 * ng; gz = nz + 2 * ng;
  }
  // ghosted index of interior-relative (i, j, k), each in [-ng, n + ng)
  long gi(int i, int j, int k) const { return ((long)(k + ng) * gy + (j + ng)) * gx + (i + ng); }
  long gsize() const { return (long)gx * gy * gz; }
  long ii(int i, int j, int k) const { return ((long)k * ny + j) * nx + i; }
  long isize() const { return (long)nx * ny * nz; }
  double xc(int d, int i) const { return p.x0[d] + (i + 0.5) * p.dx[d]; }
  double xf(int d, int i) const { return p.x0[d] + i * p.dx[d]; }
};

static int wrap(int i, int n) { return ((i % n) + n) % n; }

// Spherical blocks (metric 2) covering theta in [0, pi] and phi in [0, 2 pi) with nz even (bc = 2): phi is
// periodic, and a ghost beyond a pole is the cell mirrored across it and turned by pi in phi. The coordinate
// map (r, theta, phi) -> point continues analytically through the pole, where (r, -theta, phi) and
// (r, theta, phi + pi) are one point and d/dtheta reverses: the theta components of W v and of B change sign
// (primitives 2 and 6), everything else is copied. The radial ghosts are left as loaded (fixed). nvar = 1
// fills a scalar field (no sign change).
static void ghost_fill_spherical(const Grid& g, double* P, int nvar = 8) {
  const long n = g.gsize();
  for (int k = -g.ng; k < g.nz + g.ng; ++k)
    for (int j = -g.ng; j < g.ny + g.ng; ++j)
      for (int i = 0; i < g.nx; ++i) {
        const bool jin = j >= 0 && j < g.ny, kin = k >= 0 && k < g.nz;
        if (jin && kin) continue;
        int sj = j, sk = wrap(k, g.nz);
        double sign = 1.0;
        if (j < 0 || j >= g.ny) {
          sj = j < 0 ? -j - 1 : 2 * g.ny - j - 1;
          sk = wrap(sk + g.nz / 2, g.nz);
          sign = -1.0;
        }
        const long dst = g.gi(i, j, k), src = g.gi(i, sj, sk);
        for (int v = 0; v < nvar; ++v) {
          const double f = (nvar == 8 && (v == 2 || v == 6)) ? sign : 1.0;
          P[v * n + dst] = f * P[v * n + src];
        }
      }
}

static void ghost_fill_periodic(const Grid& g, double* P, int nvar = 8) {
  const long n = g.gsize();
  for (int k = -g.ng; k < g.nz + g.ng; ++k)
    for (int j = -g.ng; j < g.ny + g.ng; ++j)
      for (int i = -g.ng; i < g.nx + g.ng; ++i) {
        bool interior = i >= 0 && i < g.nx && j >= 0 && j < g.ny && k >= 0 && k < g.nz;
        if (interior) continue;
        long dst = g.gi(i, j, k), src = g.gi(wrap(i, g.nx), wrap(j, g.ny), wrap(k, g.nz));
        for (int v = 0; v < nvar; ++v) P[v * n + dst] = P[v * n + src];
      }
}

// Periodic fill of the face arrays: every face outside [0, N_d) along its normal d or outside the
// interior along the other two directions copies its wrapped face (face N_d wraps to face 0, which the
// CT update leaves equal to it anyway).
static void ghost_fill_faces_periodic(const Grid& g, double* Bf) {
  const long n = g.gsize();
  const int N[3] = {g.nx, g.ny, g.nz};
  for (int d = 0; d < 3; ++d)
    for (int k = -g.ng; k < g.nz + g.ng; ++k)
      for (int j = -g.ng; j < g.ny + g.ng; ++j)
        for (int i = -g.ng; i < g.nx + g.ng; ++i) {
          const int c[3] = {i, j, k};
          bool canonical = true;
          for (int e = 0; e < 3; ++e)
            if (c[e] < 0 || c[e] >= N[e]) canonical = false;
          if (canonical) continue;
          Bf[d * n + g.gi(i, j, k)] = Bf[d * n + g.gi(wrap(i, g.nx), wrap(j, g.ny), wrap(k, g.nz))];
        }
}

}  // namespace

// ======================================================================= C ABI
extern "C" {

// Geometry at points: out[101] per point =
//   alpha, beta^1..3, gamma_11,12,13,22,23,33, gamma^11,12,13,22,23,33, sqrtgam, sqrtmg,
//   dlnalpha_1..3, g_{ab}[16], g^{ab}[16], d_k g_{ab} [3][16]
int orc_geom_points(const orc_params* p, long n, const double* xyz, double* out) {
  for (long q = 0; q < n; ++q) {
    Geom G;
    metric_eval(*p, xyz[3 * q], xyz[3 * q + 1], xyz[3 * q + 2], G);
    double* o = out + 101 * q;
    int c = 0;
    o[c++] = G.alpha;
    for (int i = 1; i <= 3; ++i) o[c++] = G.beta[i];
    const int pr[6][2] = {{1, 1}, {1, 2}, {1, 3}, {2, 2}, {2, 3}, {3, 3}};
    for (int t = 0; t < 6; ++t) o[c++] = G.gam[pr[t][0]][pr[t][1]];
    for (int t = 0; t < 6; ++t) o[c++] = G.gamu[pr[t][0]][pr[t][1]];
    o[c++] = G.sqrtgam;
    o[c++] = G.sqrtmg;
    for (int i = 1; i <= 3; ++i) o[c++] = G.dlnalpha[i];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) o[c++] = G.g[a][b];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) o[c++] = G.gu[a][b];
    for (int k = 1; k <= 3; ++k)
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) o[c++] = G.dg[k][a][b];
  }
  return 0;
}

// Pointwise prim -> (densitized U, densitized F^1..3, speeds lm/lp per direction, T^{mu nu}, S).
// Any output pointer may be NULL.
//   U[n][8], F[n][3][8], lam[n][3][2], T[n][16], S[n][8] (sqrt(-g) S)
int orc_prim2con_points(const orc_params* p, long n, const double* xyz, const double* P, double* U, double* F,
                        double* lam, double* T, double* S) {
  for (long q = 0; q < n; ++q) {
    Geom G;
    metric_eval(*p, xyz[3 * q], xyz[3 * q + 1], xyz[3 * q + 2], G);
    Fluid Fl;
    fluid_from_prims(*p, G, P + 8 * q, Fl);
    double Uc[8];
    cons_from_fluid(G, Fl, Uc);
    if (U)
      for (int v = 0; v < 8; ++v) U[8 * q + v] = G.sqrtgam * Uc[v];
    for (int d = 1; d <= 3; ++d) {
      if (F) {
        double Fd[8];
        flux_from_fluid(G, Fl, Uc, d, Fd);
        for (int v = 0; v < 8; ++v) F[24 * q + 8 * (d - 1) + v] = G.sqrtmg * Fd[v];
      }
      if (lam) speeds_from_fluid(*p, G, Fl, d, lam[6 * q + 2 * (d - 1)], lam[6 * q + 2 * (d - 1) + 1]);
    }
    if (T) {
      double TT[4][4];
      tmunu(G, Fl, TT);
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) T[16 * q + 4 * a + b] = TT[a][b];
    }
    if (S) {
      double Sv[8];
      sources(G, Fl, Sv);
      for (int v = 0; v < 8; ++v) S[8 * q + v] = G.sqrtmg * Sv[v];
    }
  }
  return 0;
}

// Pointwise con2prim of densitized U at points; floors applied when apply_floors != 0.
int orc_c2p_points(const orc_params* p, long n, const double* xyz, const double* U, double* P, uint8_t* status,
                   int* iters, int do_floors) {
  for (long q = 0; q < n; ++q) {
    Geom G;
    metric_eval(*p, xyz[3 * q], xyz[3 * q + 1], xyz[3 * q + 2], G);
    double Uc[8];
    for (int v = 0; v < 8; ++v) Uc[v] = U[8 * q + v] / G.sqrtgam;
    C2PResult R;
    con2prim_point(*p, G, Uc, R);
    int st = R.status;
    if (do_floors) st |= apply_floors(*p, G, R.P);
    for (int v = 0; v < 8; ++v) P[8 * q + v] = R.P[v];
    if (status) status[q] = (uint8_t)st;
    if (iters) iters[q] = R.iters;
  }
  return 0;
}

// Root mu = 1/(h W) of the master function and the bracket end mu_+ for densitized U at points
// (the targets of the learned con2prim guess); aux [n][2] (may be NULL) receives eps and W of the
// master-function intermediates at mu_+ (two of its features).
int orc_c2p_mu_points(const orc_params* p, long n, const double* xyz, const double* U, double* mu, double* mup,
                      double* aux) {
  for (long q = 0; q < n; ++q) {
    Geom G;
    metric_eval(*p, xyz[3 * q], xyz[3 * q + 1], xyz[3 * q + 2], G);
    double Uc[8];
    for (int v = 0; v < 8; ++v) Uc[v] = U[8 * q + v] / G.sqrtgam;
    C2PResult R;
    con2prim_point(*p, G, Uc, R);
    mu[q] = R.mu;
    mup[q] = R.mup;
    if (aux) {
      aux[2 * q] = R.eps_p;
      aux[2 * q + 1] = R.W_p;
    }
  }
  return 0;
}

// Reconstruction of both faces of each cell from its 5-point stencil f[n][5] = f_{j-2..j+2}.
int orc_recon_points(int method, long n, const double* f, double weno_eps, double* qm, double* qp) {
  for (long q = 0; q < n; ++q) recon_cell(method, f + 5 * q, weno_eps, qm[q], qp[q]);
  return 0;
}

// WENO5-Z building blocks for tests: face value and weights of the right face.
int orc_weno5z_points(long n, const double* f, double eps, double* val, double* w, double* sigma_side) {
  for (long q = 0; q < n; ++q) {
    double ww[3];
    val[q] = weno5z_face(f + 5 * q, eps, ww);
    for (int k = 0; k < 3; ++k) w[3 * q + k] = ww[k];
    sigma_side[q] = weno_sigma_side(ww);
  }
  return 0;
}

// Riemann flux at points in direction d (1..3) from left/right primitives.
int orc_riemann_points(const orc_params* p, long n, const double* xyz, const double* PL, const double* PR, int d,
                       double* Fhat, double* cmax) {
  for (long q = 0; q < n; ++q) {
    Geom G;
    metric_eval(*p, xyz[3 * q], xyz[3 * q + 1], xyz[3 * q + 2], G);
    FaceSide L, R;
    face_side(*p, G, PL + 8 * q, d, L);
    face_side(*p, G, PR + 8 * q, d, R);
    double c = riemann(*p, L, R, Fhat + 8 * q);
    if (cmax) cmax[q] = c;
  }
  return 0;
}

// Densitized conserved state of the interior from primitives.
int orc_prim2con_grid(const orc_params* p, const double* P, double* U) {
  Grid g(*p);
  const long gn = g.gsize(), in = g.isize();
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        Geom G;
        metric_eval(*p, g.xc(0, i), g.xc(1, j), g.xc(2, k), G);
        double Pc[8], Uc[8];
        for (int v = 0; v < 8; ++v) Pc[v] = P[v * gn + g.gi(i, j, k)];
        Fluid Fl;
        fluid_from_prims(*p, G, Pc, Fl);
        cons_from_fluid(G, Fl, Uc);
        for (int v = 0; v < 8; ++v) U[v * in + g.ii(i, j, k)] = G.sqrtgam * Uc[v];
      }
  return 0;
}

int orc_ghost_fill(const orc_params* p, double* P) {
  Grid g(*p);
  if (p->bc == 0) ghost_fill_periodic(g, P);
  if (p->bc == 2) ghost_fill_spherical(g, P);
  return 0;
}

}  // extern "C"

namespace {

// One RK stage (both constrained-transport flavours):
//   Unew = g0 U0 + g1 Ucur + beta dt L(P),  L = -sum_d dF^d/dx^d + sqrt(-g) S with CT for B,
// followed by con2prim + floors writing the interior of P (ghosts are filled first when periodic).
// dt <= 0 selects dt = cfl / max_d(max |lambda| / dx_d) over the interior faces of this stage.
//
// Bfcur == NULL: Toth flux-CT on the cell-centred field (Sec. 3.1), B evolved in U.
// Bfcur != NULL: face-centred upwind CT (Sec. 5 names face-centred CT as planned work and gives no
// scheme; this is the reading taken). The face arrays carry the state of B:
//   * the normal component of both Riemann states of a d-face is Bf_d / sqrt(gamma) at the face centre
//     (it is continuous across the face), the tangential ones are reconstructed as before;
//   * edge EMFs follow the upwind "contact" CT of Gardiner & Stone (2005, J. Comput. Phys. 205, 509):
//     the mean of the four face EMFs around the edge plus, on each of the four half-faces, the
//     difference between face and cell-centred EMF taken in the cell the face's mass flux comes from
//     (the mean of both cells when the mass flux is zero);
//   * faces advance by the discrete Stokes theorem, Bfnew = g0 Bf0 + g1 Bfcur + beta dt (curl), so that
//     the face divergence sum_d (Bf_d(+) - Bf_d(-)) / dx_d does not change;
//   * the cell-centred densitized field in Unew is the mean of the cell's two new faces of each direction.
// With Omega_c = sqrt(gamma) (B^a v~^b - B^b v~^a) for (c, a, b) cyclic, Omega_c = F^b_{B^a} = -F^a_{B^b}.
// CT fluxes of B through the lower d-face of ghosted cell (i, j, k) (Toth flux-CT, Sec. 3.1): each is the
// mean of the two edge EMFs bounding the face along the transverse direction, with the sign of E = -v x B
// (F^x_{B^y} = -Omega_z, F^x_{B^z} = +Omega_y, F^y_{B^x} = +Omega_z, F^y_{B^z} = -Omega_x,
// F^z_{B^x} = -Omega_y, F^z_{B^y} = +Omega_x); the normal component is zero. E holds Omega_x, Omega_y,
// Omega_z, each [gsize], on the edges stored at the ghosted cell index.
static void ct_face_flux_b(const Grid& g, const double* E, int d, int i, int j, int k, double Fb[3]) {
  const long gn = g.gsize();
  auto Ev = [&](int c, int ii, int jj, int kk) { return E[c * gn + g.gi(ii, jj, kk)]; };
  if (d == 0) {
    Fb[0] = 0.0;
    Fb[1] = -0.5 * (Ev(2, i, j, k) + Ev(2, i, j + 1, k));
    Fb[2] = 0.5 * (Ev(1, i, j, k) + Ev(1, i, j, k + 1));
  } else if (d == 1) {
    Fb[0] = 0.5 * (Ev(2, i, j, k) + Ev(2, i + 1, j, k));
    Fb[1] = 0.0;
    Fb[2] = -0.5 * (Ev(0, i, j, k) + Ev(0, i, j, k + 1));
  } else {
    Fb[0] = -0.5 * (Ev(1, i, j, k) + Ev(1, i + 1, j, k));
    Fb[1] = 0.5 * (Ev(0, i, j, k) + Ev(0, i, j + 1, k));
    Fb[2] = 0.0;
  }
}

// a6 for one cell: con2prim of the densitized conserved state Un (Sec. 3.1), floors and the W ceiling
// (Sec. 3.2); when any status bit is set the hydro part of Un is re-derived from the floored primitives
// (B is kept as evolved). Returns the status; Pout gets the primitives.
static int finish_cell(const orc_params& p, const Geom& G, double* Un, double* Pout, int* iters) {
  double Uc[8];
  for (int v = 0; v < 8; ++v) Uc[v] = Un[v] / G.sqrtgam;
  C2PResult R;
  con2prim_point(p, G, Uc, R);
  if (iters) *iters += R.iters;
  const int st = R.status | apply_floors(p, G, R.P);
  if (st) {
    Fluid Ff;
    fluid_from_prims(p, G, R.P, Ff);
    double Uf[8];
    cons_from_fluid(G, Ff, Uf);
    for (int v = 0; v < 5; ++v) Un[v] = G.sqrtgam * Uf[v];
  }
  for (int v = 0; v < 8; ++v) Pout[v] = R.P[v];
  return st;
}

static int stage_impl(const orc_params* p, double* P, const double* U0, const double* Ucur, double* Unew,
                      uint8_t* status, double g0, double g1, double beta, double dt, double* dt_used,
                      double* maxspeed, int* iters_total, double* Fdbg, double* Edbg, const double* Bf0,
                      double* Bfcur, double* Bfnew) {
  Grid g(*p);
  const long gn = g.gsize(), in = g.isize();
  const int N[3] = {g.nx, g.ny, g.nz};
  const bool face_ct = Bfcur != nullptr;
  if (p->bc == 0) {
    ghost_fill_periodic(g, P);
    if (face_ct) ghost_fill_faces_periodic(g, Bfcur);
  } else if (p->bc == 2) {
    ghost_fill_spherical(g, P);
  }

  // a2 + a3: face fluxes. Direction d face index fd in [0, N_d]; transverse cells in [-1, N].
  std::vector<double> F(3 * 8 * gn, 0.0);
  double ms[3] = {0.0, 0.0, 0.0};
  for (int d = 0; d < 3; ++d) {
    int lo[3] = {-1, -1, -1}, hi[3] = {N[0] + 1, N[1] + 1, N[2] + 1};  // exclusive hi
    lo[d] = 0; hi[d] = N[d] + 1;
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) {
          const int c[3] = {i, j, k};
          // Left state from cell c - e_d (its + face), right state from cell c (its - face).
          double PL[8], PR[8];
          // spherical coordinates: the phi components of W v and B grow like 1 / sin(theta) towards the axis;
          // sin(theta) times them is regular there (and continues through it with the sign of sin(theta)),
          // so that product is reconstructed and divided by the face's sin(theta)
          const bool sph = p->metric == 2;
          const double sfc = sph ? std::sin(d == 1 ? g.xf(1, c[1]) : g.xc(1, j)) : 1.0;
          for (int v = 0; v < 8; ++v) {
            const bool reg = sph && (v == 3 || v == 7) && std::fabs(sfc) > 1e-12;
            double sL[5], sR[5];
            for (int s = 0; s < 5; ++s) {
              int cl[3] = {i, j, k}, cr[3] = {i, j, k};
              cl[d] += s - 3;  // stencil of cell c-1: c-3 .. c+1
              cr[d] += s - 2;  // stencil of cell c:   c-2 .. c+2
              sL[s] = P[v * gn + g.gi(cl[0], cl[1], cl[2])] * (reg ? std::sin(g.xc(1, cl[1])) : 1.0);
              sR[s] = P[v * gn + g.gi(cr[0], cr[1], cr[2])] * (reg ? std::sin(g.xc(1, cr[1])) : 1.0);
            }
            double qm, qp;
            recon_cell(p->recon, sL, p->weno_eps, qm, qp);
            PL[v] = reg ? qp / sfc : qp;
            recon_cell(p->recon, sR, p->weno_eps, qm, qp);
            PR[v] = reg ? qm / sfc : qm;
          }
          double xf[3] = {g.xc(0, i), g.xc(1, j), g.xc(2, k)};
          xf[d] = g.xf(d, c[d]);
          if (p->metric == 2 && d == 1 && std::fabs(std::sin(xf[1])) < 1e-12) {
            // Reading (spherical coordinates): a theta face on the polar axis has zero area (sqrt(-g) = 0,
            // where the metric itself is singular), so it carries no flux.
            for (int v = 0; v < 8; ++v) F[(d * 8 + v) * gn + g.gi(i, j, k)] = 0.0;
            continue;
          }
          Geom G;
          metric_eval(*p, xf[0], xf[1], xf[2], G);
          // Reading (Sec. 3.2, atmosphere treatment: the density must stay above its floor and the
          // specific internal energy is floored likewise): the reconstructed states of a face take the
          // floors at the face, rho >= rho_flr and rho eps >= rho eps_flr. The paper does not say where
          // the floors act; on the face states they keep the states the fluxes are built from physical
          // without a switch, so the face fluxes depend continuously on the cell values.
          {
            const double fr = p->metric >= 1 ? std::pow(G.r, -p->floor_r_exp) : 1.0;
            const double rho_flr = p->rho_floor0 * fr, eps_flr = p->eps_floor0 * fr;
            for (double* S : {PL, PR}) {
              if (!(S[0] >= rho_flr)) S[0] = rho_flr;
              if (!(S[4] >= S[0] * eps_flr)) S[4] = S[0] * eps_flr;
            }
          }
          if (face_ct) {
            const double bn = Bfcur[d * gn + g.gi(i, j, k)] / G.sqrtgam;
            PL[5 + d] = bn;
            PR[5 + d] = bn;
          }
          FaceSide L, R;
          face_side(*p, G, PL, d + 1, L);
          face_side(*p, G, PR, d + 1, R);
          double Fh[8];
          double cm = riemann(*p, L, R, Fh);
          bool interior = true;
          for (int e = 0; e < 3; ++e)
            if (e != d && (c[e] < 0 || c[e] >= N[e])) interior = false;
          if (interior && cm > ms[d]) ms[d] = cm;
          for (int v = 0; v < 8; ++v) F[(d * 8 + v) * gn + g.gi(i, j, k)] = Fh[v];
        }
  }
  for (int d = 0; d < 3; ++d) maxspeed[d] = ms[d];
  // a7: time step from this stage's speeds when not given.
  if (!(dt > 0.0)) {
    double m = 0.0;
    for (int d = 0; d < 3; ++d) m = std::max(m, ms[d] / p->dx[d]);
    dt = p->cfl / m;
  }
  *dt_used = dt;

  auto Fv = [&](int d, int v, int i, int j, int k) { return F[(d * 8 + v) * gn + g.gi(i, j, k)]; };
  std::vector<double> E(3 * gn, 0.0);
  if (!face_ct) {
    // a4: Toth flux-CT edge EMFs. Omega_k on edges along k, for (i, j, k) cyclic:
    //   Omega_k = 1/4 (sum of the 4 F^j_{B^i} around the edge - sum of the 4 F^i_{B^j})
    // stored at the index of the cell whose lower faces meet at the edge.
    // Omega_z(fi, fj, k): fi in [0, nx], fj in [0, ny], k in [0, nz)
    for (int k = 0; k < g.nz; ++k)
      for (int fj = 0; fj <= g.ny; ++fj)
        for (int fi = 0; fi <= g.nx; ++fi) {
          // spherical coordinates: an edge along phi on the axis has zero length, and so a zero EMF
          // (Omega_phi is the covariant phi component of E, which carries a factor sin(theta))
          if (p->metric == 2 && std::fabs(std::sin(g.xf(1, fj))) < 1e-12) {
            E[2 * gn + g.gi(fi, fj, k)] = 0.0;
            continue;
          }
          E[2 * gn + g.gi(fi, fj, k)] = 0.25 * (Fv(1, 5, fi - 1, fj, k) + Fv(1, 5, fi, fj, k) -
                                                Fv(0, 6, fi, fj - 1, k) - Fv(0, 6, fi, fj, k));
        }
    // Omega_x(i, fj, fk)
    for (int fk = 0; fk <= g.nz; ++fk)
      for (int fj = 0; fj <= g.ny; ++fj)
        for (int i = 0; i < g.nx; ++i)
          E[0 * gn + g.gi(i, fj, fk)] = 0.25 * (Fv(2, 6, i, fj - 1, fk) + Fv(2, 6, i, fj, fk) -
                                                Fv(1, 7, i, fj, fk - 1) - Fv(1, 7, i, fj, fk));
    // spherical coordinates: the edges along r on the axis (theta face 0 or ny) are one line for every phi,
    // where E_r is single-valued: their EMF is the mean over phi of the values computed there
    if (p->metric == 2)
      for (int fj = 0; fj <= g.ny; fj += g.ny) {
        if (std::fabs(std::sin(g.xf(1, fj))) >= 1e-12) continue;
        for (int i = 0; i < g.nx; ++i) {
          double m = 0.0;
          for (int fk = 0; fk < g.nz; ++fk) m += E[0 * gn + g.gi(i, fj, fk)];
          m /= g.nz;
          for (int fk = 0; fk <= g.nz; ++fk) E[0 * gn + g.gi(i, fj, fk)] = m;
        }
      }
    // Omega_y(fi, j, fk)
    for (int fk = 0; fk <= g.nz; ++fk)
      for (int j = 0; j < g.ny; ++j)
        for (int fi = 0; fi <= g.nx; ++fi)
          E[1 * gn + g.gi(fi, j, fk)] = 0.25 * (Fv(0, 7, fi, j, fk - 1) + Fv(0, 7, fi, j, fk) -
                                                Fv(2, 5, fi - 1, j, fk) - Fv(2, 5, fi, j, fk));
  } else {
    // a4 (face-centred): cell-centred EMFs Omega_c = sqrt(gamma) (B^a v~^b - B^b v~^a), (c, a, b) cyclic,
    // from the cell primitives, on cells [-1, N] of every direction.
    std::vector<double> Ecc(3 * gn, 0.0);
    for (int k = -1; k <= g.nz; ++k)
      for (int j = -1; j <= g.ny; ++j)
        for (int i = -1; i <= g.nx; ++i) {
          Geom G;
          metric_eval(*p, g.xc(0, i), g.xc(1, j), g.xc(2, k), G);
          double Pc[8];
          for (int v = 0; v < 8; ++v) Pc[v] = P[v * gn + g.gi(i, j, k)];
          Fluid Fl;
          fluid_from_prims(*p, G, Pc, Fl);
          for (int c = 0; c < 3; ++c) {
            const int a = (c + 1) % 3 + 1, b = (c + 2) % 3 + 1;  // 1-based components
            Ecc[c * gn + g.gi(i, j, k)] = G.sqrtgam * (Fl.Bcon[a] * Fl.vt[b] - Fl.Bcon[b] * Fl.vt[a]);
          }
        }
    // Edge EMF of component c at the edge between face indices (fa, fb) of its transverse directions
    // a = c+1, b = c+2 (cyclic); (ia, ib) below are cell indices in the a-b plane, the c index is fixed.
    for (int c = 0; c < 3; ++c) {
      const int a = (c + 1) % 3, b = (c + 2) % 3;
      int lo[3] = {0, 0, 0}, hi[3] = {N[0] + 1, N[1] + 1, N[2] + 1};
      hi[c] = N[c];  // cells along c, faces along a and b
      for (int k = lo[2]; k < hi[2]; ++k)
        for (int j = lo[1]; j < hi[1]; ++j)
          for (int i = lo[0]; i < hi[0]; ++i) {
            const int e[3] = {i, j, k};
            // index of the point with a-index ia, b-index ib and the edge's c-index
            auto at = [&](int ia, int ib) {
              int q[3];
              q[c] = e[c];
              q[a] = ia;
              q[b] = ib;
              return g.gi(q[0], q[1], q[2]);
            };
            const int fa = e[a], fb = e[b];
            // face EMFs: a-faces (normal a) at (fa, ib) give -F^a_{B^b}; b-faces at (ia, fb) give +F^b_{B^a}
            auto OA = [&](int ib) { return -F[(a * 8 + 5 + b) * gn + at(fa, ib)]; };
            auto OB = [&](int ia) { return F[(b * 8 + 5 + a) * gn + at(ia, fb)]; };
            auto Oc = [&](int ia, int ib) { return Ecc[c * gn + at(ia, ib)]; };
            auto DA = [&](int ib) { return F[(a * 8 + 0) * gn + at(fa, ib)]; };  // mass flux through a-face
            auto DB = [&](int ia) { return F[(b * 8 + 0) * gn + at(ia, fb)]; };
            // each half-face term chooses its cell by the sign of that face's mass flux
            auto pick = [](double m, double lo_cell, double hi_cell) {
              return m > 0.0 ? lo_cell : (m < 0.0 ? hi_cell : 0.5 * (lo_cell + hi_cell));
            };
            // b-direction half-faces of the a-faces below (fb - 1) and above (fb) the edge
            const double xb_lo = pick(DA(fb - 1), OB(fa - 1) - Oc(fa - 1, fb - 1), OB(fa) - Oc(fa, fb - 1));
            const double xb_hi = pick(DA(fb), Oc(fa - 1, fb) - OB(fa - 1), Oc(fa, fb) - OB(fa));
            // a-direction half-faces of the b-faces left (fa - 1) and right (fa) of the edge
            const double xa_lo = pick(DB(fa - 1), OA(fb - 1) - Oc(fa - 1, fb - 1), OA(fb) - Oc(fa - 1, fb));
            const double xa_hi = pick(DB(fa), Oc(fa, fb - 1) - OA(fb - 1), Oc(fa, fb) - OA(fb));
            E[c * gn + g.gi(i, j, k)] = 0.25 * (OA(fb - 1) + OA(fb) + OB(fa - 1) + OB(fa)) +
                                        0.25 * (xb_lo - xb_hi) + 0.25 * (xa_lo - xa_hi);
          }
    }
    // Faces: discrete Stokes theorem on the edge EMFs. d/dt Bf_x = -dOmega_z/dy + dOmega_y/dz,
    // d/dt Bf_y = dOmega_z/dx - dOmega_x/dz, d/dt Bf_z = -dOmega_y/dx + dOmega_x/dy.
    std::memcpy(Bfnew, Bfcur, sizeof(double) * 3 * gn);
    auto Ev = [&](int c, int i, int j, int k) { return E[c * gn + g.gi(i, j, k)]; };
    for (int d = 0; d < 3; ++d) {
      int hi[3] = {N[0], N[1], N[2]};
      hi[d] = N[d] + 1;
      for (int k = 0; k < hi[2]; ++k)
        for (int j = 0; j < hi[1]; ++j)
          for (int i = 0; i < hi[0]; ++i) {
            double curl;
            if (d == 0)
              curl = -(Ev(2, i, j + 1, k) - Ev(2, i, j, k)) / p->dx[1] + (Ev(1, i, j, k + 1) - Ev(1, i, j, k)) / p->dx[2];
            else if (d == 1)
              curl = (Ev(2, i + 1, j, k) - Ev(2, i, j, k)) / p->dx[0] - (Ev(0, i, j, k + 1) - Ev(0, i, j, k)) / p->dx[2];
            else
              curl = -(Ev(1, i + 1, j, k) - Ev(1, i, j, k)) / p->dx[0] + (Ev(0, i, j + 1, k) - Ev(0, i, j, k)) / p->dx[1];
            const long f = d * gn + g.gi(i, j, k);
            const double b0 = Bf0 ? Bf0[f] : 0.0;
            Bfnew[f] = g0 * b0 + g1 * Bfcur[f] + beta * dt * curl;
          }
    }
  }
  if (Fdbg) std::memcpy(Fdbg, F.data(), sizeof(double) * F.size());
  if (Edbg) std::memcpy(Edbg, E.data(), sizeof(double) * E.size());

  // a5 + a6: divergence, sources, RK combination, con2prim, floors.
  if (iters_total) *iters_total = 0;
  const long sx = 1, sy = g.gx, sz = (long)g.gx * g.gy;
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        Geom G;
        metric_eval(*p, g.xc(0, i), g.xc(1, j), g.xc(2, k), G);
        double Pc[8];
        for (int v = 0; v < 8; ++v) Pc[v] = P[v * gn + g.gi(i, j, k)];
        Fluid Fl;
        fluid_from_prims(*p, G, Pc, Fl);
        double S[8];
        sources(G, Fl, S);
        double L[8];
        for (int v = 0; v < 5; ++v) {
          double div = (Fv(0, v, i + 1, j, k) - Fv(0, v, i, j, k)) / p->dx[0] +
                       (Fv(1, v, i, j + 1, k) - Fv(1, v, i, j, k)) / p->dx[1] +
                       (Fv(2, v, i, j, k + 1) - Fv(2, v, i, j, k)) / p->dx[2];
          L[v] = -div + G.sqrtmg * S[v];
        }
        // CT-corrected B fluxes through the cell's lower (m) and upper (p) faces of each direction
        double Bxm[3], Bxp[3], Bym[3], Byp[3], Bzm[3], Bzp[3];
        ct_face_flux_b(g, E.data(), 0, i, j, k, Bxm);
        ct_face_flux_b(g, E.data(), 0, i + 1, j, k, Bxp);
        ct_face_flux_b(g, E.data(), 1, i, j, k, Bym);
        ct_face_flux_b(g, E.data(), 1, i, j + 1, k, Byp);
        ct_face_flux_b(g, E.data(), 2, i, j, k, Bzm);
        ct_face_flux_b(g, E.data(), 2, i, j, k + 1, Bzp);
        L[5] = -((Byp[0] - Bym[0]) / p->dx[1] + (Bzp[0] - Bzm[0]) / p->dx[2]);
        L[6] = -((Bxp[1] - Bxm[1]) / p->dx[0] + (Bzp[1] - Bzm[1]) / p->dx[2]);
        L[7] = -((Bxp[2] - Bxm[2]) / p->dx[0] + (Byp[2] - Bym[2]) / p->dx[1]);
        const long c = g.ii(i, j, k);
        double Un[8];
        for (int v = 0; v < 8; ++v) {
          double u0 = U0 ? U0[v * in + c] : 0.0;
          Un[v] = g0 * u0 + g1 * Ucur[v * in + c] + beta * dt * L[v];
        }
        if (face_ct) {
          // the cell-centred densitized field is the mean of the cell's two new faces of each direction
          const long gc = g.gi(i, j, k);
          const long st[3] = {sx, sy, sz};
          for (int d = 0; d < 3; ++d) Un[5 + d] = 0.5 * (Bfnew[d * gn + gc] + Bfnew[d * gn + gc + st[d]]);
        }
        // a6: con2prim, floors, re-derived hydro state
        double Pn[8];
        const int st = finish_cell(*p, G, Un, Pn, iters_total);
        for (int v = 0; v < 8; ++v) Unew[v * in + c] = Un[v];
        for (int v = 0; v < 8; ++v) P[v * gn + g.gi(i, j, k)] = Pn[v];
        status[c] = (uint8_t)st;
      }
  return 0;
}

}  // namespace

// ======================================================================= C ABI (stages)
extern "C" {

// One RK stage with Toth flux-CT on the cell-centred field.
// Outputs: Unew, P (updated in place), status, *dt_used, maxspeed[3] (max |lambda| per direction).
// Optional debug outputs (may be NULL): Fx/Fy/Fz [8][gsize] face fluxes, Ex/Ey/Ez [gsize] edge EMFs.
int orc_stage(const orc_params* p, double* P, const double* U0, const double* Ucur, double* Unew, uint8_t* status,
              double g0, double g1, double beta, double dt, double* dt_used, double* maxspeed, int* iters_total,
              double* Fdbg, double* Edbg) {
  return stage_impl(p, P, U0, Ucur, Unew, status, g0, g1, beta, dt, dt_used, maxspeed, iters_total, Fdbg, Edbg,
                    nullptr, nullptr, nullptr);
}

// One flux-CT RK stage that also advances a passive scalar (Sec. 2.1: Phoebus evolves passive scalars X by
// (X rho u^mu)_{;mu} = S, the electron fraction Y_e with the radiation's lepton exchange as S; without
// radiation S = 0). Conserved: sqrt(gamma) D X (D = rho W); primitive: X, [gsize] ghosted like P (its
// ghosts filled first when periodic). Reading (the discretisation is not given): X is reconstructed like
// the primitives, and the face flux of sqrt(gamma) D X is the face mass flux of the stage (sqrt(-g) F^d_D
// after the Riemann solver) times X on the upwind side of that flux (either side when it is zero);
// DXnew = g0 DX0 + g1 DXcur - beta dt div F_X; then X = DXnew / (sqrt(gamma) D) with the stage's final
// sqrt(gamma) D (after floors: a floor that adds mass dilutes X, D X stays conserved). DX0 may be NULL
// when g0 = 0. Optional outputs (may be NULL): the stage's face fluxes Fdbg [3][8][gsize] and edge EMFs
// Edbg [3][gsize], and the scalar's face fluxes FXdbg [3][gsize]. The other arguments are those of orc_stage.
int orc_stage_scalar(const orc_params* p, double* P, const double* U0, const double* Ucur, double* Unew,
                     uint8_t* status, double g0, double g1, double beta, double dt, double* dt_used, double* maxspeed,
                     int* iters_total, double* X, const double* DX0, const double* DXcur, double* DXnew,
                     double* Fdbg, double* Edbg, double* FXdbg) {
  const Grid g(*p);
  const long gn = g.gsize(), in = g.isize();
  const int N[3] = {g.nx, g.ny, g.nz};
  std::vector<double> F(3 * 8 * gn, 0.0);
  const int rc = stage_impl(p, P, U0, Ucur, Unew, status, g0, g1, beta, dt, dt_used, maxspeed, iters_total,
                            F.data(), Edbg, nullptr, nullptr, nullptr);
  if (Fdbg) std::memcpy(Fdbg, F.data(), sizeof(double) * F.size());
  if (rc) return rc;
  dt = *dt_used;
  if (p->bc == 0) ghost_fill_periodic(g, X, 1);
  if (p->bc == 2) ghost_fill_spherical(g, X, 1);
  // face fluxes of sqrt(gamma) D X on the faces of the interior
  std::vector<double> FX(3 * gn, 0.0);
  for (int d = 0; d < 3; ++d) {
    int hi[3] = {N[0], N[1], N[2]};
    hi[d] = N[d] + 1;
    for (int k = 0; k < hi[2]; ++k)
      for (int j = 0; j < hi[1]; ++j)
        for (int i = 0; i < hi[0]; ++i) {
          double sL[5], sR[5];
          for (int q = 0; q < 5; ++q) {
            int cl[3] = {i, j, k}, cr[3] = {i, j, k};
            cl[d] += q - 3;  // stencil of the cell below the face
            cr[d] += q - 2;  // stencil of the cell above it
            sL[q] = X[g.gi(cl[0], cl[1], cl[2])];
            sR[q] = X[g.gi(cr[0], cr[1], cr[2])];
          }
          double qm, qp, XL, XR;
          recon_cell(p->recon, sL, p->weno_eps, qm, qp);
          XL = qp;
          recon_cell(p->recon, sR, p->weno_eps, qm, qp);
          XR = qm;
          const long f = g.gi(i, j, k);
          const double mdot = F[(d * 8 + 0) * gn + f];
          FX[d * gn + f] = mdot * (mdot >= 0.0 ? XL : XR);
        }
  }
  for (int k = 0; k < N[2]; ++k)
    for (int j = 0; j < N[1]; ++j)
      for (int i = 0; i < N[0]; ++i) {
        auto Fv = [&](int d, int a, int b, int c) { return FX[d * gn + g.gi(a, b, c)]; };
        const double div = (Fv(0, i + 1, j, k) - Fv(0, i, j, k)) / p->dx[0] +
                           (Fv(1, i, j + 1, k) - Fv(1, i, j, k)) / p->dx[1] +
                           (Fv(2, i, j, k + 1) - Fv(2, i, j, k)) / p->dx[2];
        const long c = g.ii(i, j, k);
        const double x0 = DX0 ? DX0[c] : 0.0;
        DXnew[c] = g0 * x0 + g1 * DXcur[c] + beta * dt * (-div);
        X[g.gi(i, j, k)] = DXnew[c] / Unew[c];  // Unew[0 * in + c]: the densitized D
      }
  if (FXdbg) std::memcpy(FXdbg, FX.data(), sizeof(double) * FX.size());
  (void)in;
  return 0;
}

// One RK stage with face-centred upwind CT. Bfcur [3][gsize] is the face field of this stage (its ghost
// faces are filled first when periodic), Bf0 the one at the start of the step (NULL when g0 = 0), Bfnew
// receives the advanced faces (ghost faces copied from Bfcur). U0 / Ucur B components are not read.
int orc_stage_face_ct(const orc_params* p, double* P, const double* U0, const double* Ucur, double* Unew,
                      uint8_t* status, double g0, double g1, double beta, double dt, double* dt_used,
                      double* maxspeed, int* iters_total, double* Fdbg, double* Edbg, const double* Bf0,
                      double* Bfcur, double* Bfnew) {
  if (!Bfcur || !Bfnew) return 1;
  return stage_impl(p, P, U0, Ucur, Unew, status, g0, g1, beta, dt, dt_used, maxspeed, iters_total, Fdbg, Edbg,
                    Bf0, Bfcur, Bfnew);
}

// Cell-centred field from the faces: B^d of every cell whose two d-faces are both stored (all ghosted
// cells but the last layer along d) becomes (Bf_d(lower) + Bf_d(upper)) / (2 sqrt(gamma)) at the cell
// centre; the last layer keeps its value. Periodic blocks get their ghost faces filled first.
// The face fluxes a flux-CT stage's update uses, from its face fluxes F [3][8][gsize] and edge EMFs
// E [3][gsize] (the stage's debug outputs): the hydro components (0..4) are F's, the B components the CT
// fluxes; every face of the interior (index 0..n along its normal, interior across it) is written, the
// rest of Fused [3][8][gsize] is left as it was.
int orc_face_fluxes_used(const orc_params* p, const double* F, const double* E, double* Fused) {
  const Grid g(*p);
  const long gn = g.gsize();
  const int N[3] = {g.nx, g.ny, g.nz};
  for (int d = 0; d < 3; ++d) {
    int hi[3] = {N[0], N[1], N[2]};
    hi[d] = N[d] + 1;
    for (int k = 0; k < hi[2]; ++k)
      for (int j = 0; j < hi[1]; ++j)
        for (int i = 0; i < hi[0]; ++i) {
          const long f = g.gi(i, j, k);
          for (int v = 0; v < 5; ++v) Fused[(d * 8 + v) * gn + f] = F[(d * 8 + v) * gn + f];
          double Fb[3];
          ct_face_flux_b(g, E, d, i, j, k, Fb);
          for (int c = 0; c < 3; ++c) Fused[(d * 8 + 5 + c) * gn + f] = Fb[c];
        }
  }
  return 0;
}

// a6 at n points: Un [n][8] densitized conserved states (updated in place when a status bit re-derives the
// hydro part), P [n][8] and status [n] out; the metric at xyz [n][3].
int orc_finish_points(const orc_params* p, long n, const double* xyz, double* Un, double* P, uint8_t* status) {
  for (long q = 0; q < n; ++q) {
    Geom G;
    metric_eval(*p, xyz[3 * q], xyz[3 * q + 1], xyz[3 * q + 2], G);
    status[q] = (uint8_t)finish_cell(*p, G, Un + 8 * q, P + 8 * q, nullptr);
  }
  return 0;
}

int orc_face_b_to_cells(const orc_params* p, double* Bf, double* P) {
  Grid g(*p);
  const long gn = g.gsize();
  if (p->bc == 0) ghost_fill_faces_periodic(g, Bf);
  const long st[3] = {1, g.gx, (long)g.gx * g.gy};
  const int hi[3] = {g.nx + g.ng, g.ny + g.ng, g.nz + g.ng};
  for (int k = -g.ng; k < hi[2]; ++k)
    for (int j = -g.ng; j < hi[1]; ++j)
      for (int i = -g.ng; i < hi[0]; ++i) {
        Geom G;
        metric_eval(*p, g.xc(0, i), g.xc(1, j), g.xc(2, k), G);
        const int c[3] = {i, j, k};
        const long gc = g.gi(i, j, k);
        for (int d = 0; d < 3; ++d) {
          if (c[d] + 1 >= hi[d]) continue;
          P[(5 + d) * gn + gc] = 0.5 * (Bf[d * gn + gc] + Bf[d * gn + gc + st[d]]) / G.sqrtgam;
        }
      }
  return 0;
}

}  // extern "C"
