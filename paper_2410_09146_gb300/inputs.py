"""Seeded synthetic workloads for the GRMHD stage (shared by the tests, the bench and the CUDA path).

This module holds grid set-ups and random initial data only; it contains none of the
method's arithmetic (no metric, no prim->cons map, no flux, no con2prim). Random
numbers come from numpy's PCG64 generator, whose stream is the same on every platform.

Workloads (sizes and distributions follow the stage's standard test problems):
  * ``linear_wave``  uniform Minkowski state plus a small-amplitude eigenmode along x (the
    eigenvector is passed in by the caller), periodic, the setting of the paper's
    linear-wave convergence tests (Sec. 4.1.1).
  * ``kerr_schild_random``  Kerr-Schild (a = 0.9) cube [3, 23]^3 outside the horizon with
    smooth seeded random fields: rho log-uniform in [1e-6, 1], P = 0.01 rho^(5/3),
    flat-norm |W v| from a Lorentz factor log-uniform in [1, 10], and B the discrete
    corner-to-cell curl of a node-centred vector potential whose amplitude follows a
    magnetisation target log-uniform in [1e-2, 50] (so Toth's corner divergence of B is
    zero up to roundoff). Ghost zones are filled from the same fields (fixed ghosts).
    With ``faces=True`` it also returns the same potential's curl on the faces (the face-centred field
    of the face-CT form), whose mean over a cell's two faces of each direction is the cell field.
  * ``smooth_random`` every variable a smooth random perturbation of a uniform state (no normalised
    direction field), B from a random potential, with its face field.
  * ``plane_random`` a periodic state that varies along one direction only, with its face field.
  * ``boosted_wave`` a plane linear wave along the diagonal of a periodic square in flat space with a
    constant shift (the coordinate boost of the paper's 2-D linear-wave tests); mode shapes and speeds
    are passed in (tests/golden/boosted_waves.json, written from the oracle).
  * ``field_loop`` a weak magnetic field loop in a uniform flow on a periodic square (the standard
    constrained-transport advection test), with its face field.
  * ``c2p_states``  i.i.d. primitive states for the flat con2prim batch: rho, W, sigma
    log-uniform over [1e-8, 1], [1, 50], [1e-4, 1e3], P = 0.01 rho^(5/3) 10^U(-1,1),
    isotropic velocity and field directions.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Tuple

import numpy as np

GAMMA_DEFAULT = 5.0 / 3.0


@dataclasses.dataclass
class Setup:
    """Grid and physics options of one meshblock (names follow the paper's notation)."""
    n: Tuple[int, int, int]
    ng: int = 4
    x0: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    dx: Tuple[float, float, float] = (1.0, 1.0, 1.0)
    metric: str = "minkowski"          # "minkowski" | "kerr_schild"
    spin: float = 0.0
    mass: float = 1.0
    gamma_eos: float = GAMMA_DEFAULT
    recon: str = "plm_mc"              # "constant" | "plm_minmod" | "plm_mc" | "weno5z_aoah"
    riemann: str = "llf"               # "llf" | "hll"
    bc: str = "periodic"               # "periodic" | "fixed"
    rho_floor0: float = 1e-10
    eps_floor0: float = 1e-8
    floor_r_exp: float = 2.0
    w_max: float = 100.0
    c2p_tol: float = 1e-10
    c2p_max_iter: int = 30
    cfl: float = 0.4
    weno_eps: float = 1e-26
    precision: str = "fp64"            # "fp64" | "mixed"
    ct: str = "flux"                   # "flux" (Toth flux-CT, cell field) | "face" (face-centred upwind CT)
    shift: Tuple[float, float, float] = (0.0, 0.0, 0.0)  # Minkowski: constant shift (boosted coordinates)
    scalar: bool = False               # also evolve one passive scalar (the electron fraction, say)
    # a tile of a larger block (kerr_schild_tile): (parent Setup, offset of the tile's first interior cell)
    tile_of: object = dataclasses.field(default=None, repr=False, compare=False)

    @property
    def ghosted(self):
        return tuple(k + 2 * self.ng for k in self.n)

    def prim_shape(self):
        nx, ny, nz = self.n
        g = 2 * self.ng
        return (8, nz + g, ny + g, nx + g)

    def cons_shape(self):
        nx, ny, nz = self.n
        return (8, nz, ny, nx)

    def cell_centres(self, d: int, ghosts: bool = True):
        n = self.n[d]
        lo = -self.ng if ghosts else 0
        hi = n + self.ng if ghosts else n
        return self.x0[d] + (np.arange(lo, hi) + 0.5) * self.dx[d]


# ----------------------------------------------------------------------------- set-ups
def linear_wave_setup(n: int = 32, ny: int | None = None, nz: int | None = None, recon: str = "plm_mc",
                      riemann: str = "llf") -> Setup:
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    return Setup(n=(n, ny, nz), x0=(0.0, 0.0, 0.0), dx=(1.0 / n, 1.0 / n, 1.0 / n), metric="minkowski",
                 recon=recon, riemann=riemann, bc="periodic")


def kerr_schild_setup(n: int = 128, recon: str = "plm_mc", riemann: str = "hll", precision: str = "fp64",
                      lo: float = 3.0, hi: float = 23.0) -> Setup:
    h = (hi - lo) / n
    return Setup(n=(n, n, n), x0=(lo, lo, lo), dx=(h, h, h), metric="kerr_schild", spin=0.9, mass=1.0,
                 recon=recon, riemann=riemann, bc="fixed", precision=precision)


# ----------------------------------------------------------------------------- generators
def linear_wave_prims(s: Setup, background, eigvec, amplitude: float = 1e-6) -> np.ndarray:
    """Primitive array [8][nz+2g][ny+2g][nx+2g]: background + amplitude * eigvec * sin(2 pi x / L)."""
    P = np.empty(s.prim_shape())
    x = s.cell_centres(0)
    L = s.n[0] * s.dx[0]
    ph = np.sin(2.0 * math.pi * (x - s.x0[0]) / L)
    for v in range(8):
        P[v] = background[v] + amplitude * eigvec[v] * ph[None, None, :]
    return P


class _SmoothField:
    """Sum of random Fourier modes on the unit cube, normalised to unit variance."""

    def __init__(self, rng: np.random.Generator, nmodes: int = 8, kmax: int = 3):
        ks = []
        while len(ks) < nmodes:
            k = rng.integers(-kmax, kmax + 1, size=3)
            if np.any(k != 0):
                ks.append(k)
        self.k = np.array(ks, dtype=np.float64)
        self.phi = rng.uniform(0.0, 2.0 * math.pi, size=nmodes)
        self.amp = rng.normal(size=nmodes)
        self.norm = 1.0 / math.sqrt(0.5 * float(np.sum(self.amp ** 2)))

    def __call__(self, ux, uy, uz):
        """Evaluate on the tensor grid ux (x) uy (x) uz of unit-cube coordinates -> [z][y][x]."""
        out = np.zeros((len(uz), len(uy), len(ux)))
        for m in range(len(self.amp)):
            ex = np.exp(1j * (2.0 * math.pi * self.k[m, 0] * ux + self.phi[m]))
            ey = np.exp(1j * (2.0 * math.pi * self.k[m, 1] * uy))
            ez = np.exp(1j * (2.0 * math.pi * self.k[m, 2] * uz))
            yz = ez[:, None] * ey[None, :]
            out += self.amp[m] * np.imag(yz[:, :, None] * ex[None, None, :])
        return out * self.norm


def _to_uniform(g):
    """Map an approximately standard-normal field to (0, 1) through the normal CDF."""
    from scipy.special import erf
    return np.clip(0.5 * (1.0 + erf(g / math.sqrt(2.0))), 0.0, 1.0)


def _logu(field, lo, hi, grid):
    u = _to_uniform(field(*grid))
    return 10.0 ** (math.log10(lo) + (math.log10(hi) - math.log10(lo)) * u)


def _ks_fields(seed, kmax):
    rng = np.random.default_rng(seed)
    f_rho, f_w, f_sig = (_SmoothField(rng, kmax=kmax) for _ in range(3))
    f_dir = [_SmoothField(rng, kmax=kmax) for _ in range(3)]
    f_a = [_SmoothField(rng, kmax=kmax) for _ in range(3)]
    return f_rho, f_w, f_sig, f_dir, f_a


def _ks_coords(s: Setup):
    """Unit-cube coordinates of the ghosted cell centres and of the cell corners of block s."""
    ng = s.ng
    span = [s.n[d] * s.dx[d] for d in range(3)]
    xc = [(s.cell_centres(d) - s.x0[d]) / span[d] for d in range(3)]
    xn = [(s.x0[d] + np.arange(-ng, s.n[d] + ng + 1) * s.dx[d] - s.x0[d]) / span[d] for d in range(3)]
    return xc, xn


def _ks_unscaled_b(fields, xn, dx, rho_range, w_range, sigma_range):
    """Face and cell-centred curl of the node-centred potential, before the global scale."""
    f_rho, f_w, f_sig, _, f_a = fields
    rho_n = _logu(f_rho, *rho_range, xn)
    W_n = _logu(f_w, *w_range, xn)
    sig_n = _logu(f_sig, *sigma_range, xn)
    amp = W_n * np.sqrt(sig_n * rho_n)
    del rho_n, W_n, sig_n
    A = [amp * f(*xn) for f in f_a]
    del amp
    Bface = _face_curl(A, dx)
    return Bface, np.stack([_mu(Bface[c], _AX_OF[c]) for c in range(3)])


_SCALE_CACHE = {}


def _ks_b_scale(s: Setup, seed, rho_range, w_range, sigma_range, kmax, slab=16):
    """The global field scale of block s (the median of |B|^2/(rho W^2) over its ghosted cells set to the
    median target magnetisation), evaluated over z-slabs of the block so that large blocks fit in memory;
    the values equal those of the whole-block evaluation."""
    key = (s.n, s.ng, s.x0, s.dx, seed, tuple(rho_range), tuple(w_range), tuple(sigma_range), kmax)
    if key in _SCALE_CACHE:
        return _SCALE_CACHE[key]
    fields = _ks_fields(seed, kmax)
    f_rho, f_w = fields[0], fields[1]
    xc, xn = _ks_coords(s)
    nzg = len(xc[2])
    proxy = []
    for k0 in range(0, nzg, slab):
        k1 = min(k0 + slab, nzg)
        rho = _logu(f_rho, *rho_range, [xc[0], xc[1], xc[2][k0:k1]])
        W = _logu(f_w, *w_range, [xc[0], xc[1], xc[2][k0:k1]])
        _, B = _ks_unscaled_b(fields, [xn[0], xn[1], xn[2][k0:k1 + 1]], s.dx, rho_range, w_range, sigma_range)
        proxy.append((np.sum(B ** 2, axis=0) / (rho * W * W)).ravel())
    target = math.sqrt(sigma_range[0] * sigma_range[1])
    scale = math.sqrt(target / float(np.median(np.concatenate(proxy))))
    _SCALE_CACHE[key] = scale
    return scale


def kerr_schild_tile(parent: Setup, offset, n) -> Setup:
    """The set-up of an n[0] x n[1] x n[2] tile of block `parent` whose first interior cell is the parent's
    interior cell `offset` (same cell widths, ghosts and options): kerr_schild_random_prims(tile, ...,
    parent=parent) gives exactly the parent's primitives on the tile's cells, ghosts included."""
    if any(o < 0 or o + k > N for o, k, N in zip(offset, n, parent.n)):
        raise ValueError("the tile must lie inside the parent's interior")
    x0 = tuple(parent.x0[d] + offset[d] * parent.dx[d] for d in range(3))
    return dataclasses.replace(parent, n=tuple(n), x0=x0, tile_of=(parent, tuple(offset)))


def kerr_schild_random_prims(s: Setup, seed: int = 1, rho_range=(1e-6, 1.0), w_range=(1.0, 10.0),
                             sigma_range=(1e-2, 50.0), p_coef: float = 0.01, kmax: int = 3,
                             faces: bool = False):
    """Smooth seeded random primitives over the ghosted block (see module docstring).

    ``kmax`` bounds the integer wavenumbers of the Fourier modes (per unit cube); small grids
    use kmax = 1 so that the fields stay resolved. With ``faces=True`` also returns the face field
    ``Bf`` [3][gz][gy][gx] (entry (i, j, k) of component d on the lower d-face of ghosted cell (i, j, k)):
    the same potential's curl on the faces, with the same scale, so that the mean of a cell's two
    d-faces is its B^d in ``P``. Used as the face-centred field sqrt(gamma) B^d.

    For a tile made by ``kerr_schild_tile`` the fields are those of the parent block (its unit cube and
    its global field scale): the result is the parent's primitives on the tile's ghosted cells.
    """
    fields = _ks_fields(seed, kmax)
    f_rho, f_w, f_sig, f_dir, f_a = fields
    tile = s.tile_of
    if tile is None:
        xc, xn = _ks_coords(s)
    else:
        parent, off = tile
        pxc, pxn = _ks_coords(parent)
        xc = [pxc[d][off[d]:off[d] + s.n[d] + 2 * s.ng] for d in range(3)]
        xn = [pxn[d][off[d]:off[d] + s.n[d] + 2 * s.ng + 1] for d in range(3)]

    P = np.empty(s.prim_shape())
    rho = _logu(f_rho, *rho_range, xc)
    W = _logu(f_w, *w_range, xc)
    P[0] = rho
    P[4] = p_coef * rho ** (5.0 / 3.0) / (s.gamma_eos - 1.0)
    dirs = np.stack([f(*xc) for f in f_dir])
    dirs /= np.sqrt(np.sum(dirs ** 2, axis=0)) + 1e-300
    P[1:4] = np.sqrt(W * W - 1.0) * dirs
    del dirs

    # Node-centred vector potential with amplitude W sqrt(sigma_target rho) evaluated at the nodes.
    Bface, B = _ks_unscaled_b(fields, xn, s.dx, rho_range, w_range, sigma_range)
    # One global scale so the median of |B|^2 / (rho W^2) matches the median target sigma.
    if tile is None:
        proxy = np.sum(B ** 2, axis=0) / (rho * W * W)
        target = math.sqrt(sigma_range[0] * sigma_range[1])
        scale = math.sqrt(target / float(np.median(proxy)))
    else:
        scale = _ks_b_scale(tile[0], seed, rho_range, w_range, sigma_range, kmax)
    P[5:8] = B * scale
    if not faces:
        return P
    Bf = np.empty((3,) + P.shape[1:])
    for c in range(3):
        sl = [slice(None)] * 3
        sl[_AX_OF[c]] = slice(0, -1)  # drop the upper face of the last ghost layer
        Bf[c] = Bface[c][tuple(sl)] * scale
    return P, Bf


_AX_OF = {0: 2, 1: 1, 2: 0}  # array axis of the x, y, z direction ([z][y][x] order)


def _mu(a, ax):
    """Mean of neighbouring entries along array axis ax."""
    sl0 = [slice(None)] * 3; sl1 = [slice(None)] * 3
    sl0[ax] = slice(0, -1); sl1[ax] = slice(1, None)
    return 0.5 * (a[tuple(sl0)] + a[tuple(sl1)])


def _face_curl(A, dx):
    """Curl of node-centred A on the faces: component c on the c-faces is D_a mu_b A_b - D_b mu_a A_a
    for (c, a, b) cyclic, where mu_d averages the two nodes along d and D_d differences them over dx_d.

    A[c] has shape [nz+1][ny+1][nx+1] over the cell corners; component c of the result has the node
    count along c and the cell count along the other two directions. Its mean over the two c-faces of
    each cell is the cell-centred curl of the random field (zero corner divergence)."""
    def D(a, ax, h):
        sl0 = [slice(None)] * 3; sl1 = [slice(None)] * 3
        sl0[ax] = slice(0, -1); sl1[ax] = slice(1, None)
        return (a[tuple(sl1)] - a[tuple(sl0)]) / h

    out = []
    for c in range(3):
        a, b = (c + 1) % 3, (c + 2) % 3
        t1 = D(_mu(A[b], _AX_OF[b]), _AX_OF[a], dx[a])
        t2 = D(_mu(A[a], _AX_OF[a]), _AX_OF[b], dx[b])
        out.append(t1 - t2)
    return out


def boosted_wave_setup(n: int = 32, recon: str = "plm_mc", riemann: str = "hll", shift=(0.617213, 0.617213, 0.0)) -> Setup:
    """Periodic unit square of n x n cells (one cell in z), flat metric with a constant shift: the coordinate
    boost of the paper's 2-D linear-wave tests (Sec. 4.1.1)."""
    return Setup(n=(n, n, 1), x0=(0.0, 0.0, 0.0), dx=(1.0 / n, 1.0 / n, 1.0 / n), metric="minkowski",
                 recon=recon, riemann=riemann, bc="periodic", shift=tuple(shift))


def boosted_wave_prims(s: Setup, background, eigvec, speed: float, amplitude: float = 1e-6, t: float = 0.0) -> np.ndarray:
    """Plane wave along the diagonal n = (1, 1, 0)/sqrt(2) with one wavelength across the square's diagonal period:
    P = P0 + amplitude * eigvec * sin(2 pi [(x + y) - sqrt(2) speed t]) at the cell centres (the exact solution of
    the linearised equations at time t; `speed` is the mode's coordinate speed along n)."""
    xc = s.cell_centres(0)
    yc = s.cell_centres(1)
    phase = 2.0 * math.pi * ((xc[None, :] + yc[:, None]) - math.sqrt(2.0) * speed * t)  # [y][x]
    w = np.sin(phase)
    P = np.empty(s.prim_shape())
    for v in range(8):
        P[v] = background[v] + amplitude * eigvec[v] * w[None, :, :]
    return P


def smooth_random_prims(s: Setup, seed: int = 6, amp: float = 0.3, b_amp: float = 0.3, kmax: int = 1):
    """Seeded smooth state over the ghosted block, and its face field: rho = 1 + amp f, rho eps =
    1.5 (1 + amp f), W v^i = amp f_i, each f a sum of random Fourier modes over the interior (periodic
    on it), and B the curl of a node-centred random potential of amplitude b_amp (as in
    ``kerr_schild_random_prims``). Unlike that generator it has no normalised direction field, so every
    variable is smooth. Returns (P, Bf)."""
    rng = np.random.default_rng(seed)
    fs = [_SmoothField(rng, kmax=kmax) for _ in range(5)]
    fa = [_SmoothField(rng, kmax=kmax) for _ in range(3)]
    span = [s.n[d] * s.dx[d] for d in range(3)]
    xc = [(s.cell_centres(d) - s.x0[d]) / span[d] for d in range(3)]
    xn = [np.arange(-s.ng, s.n[d] + s.ng + 1) / s.n[d] for d in range(3)]
    P = np.empty(s.prim_shape())
    g = [f(*xc) for f in fs]
    P[0] = 1.0 + amp * np.tanh(g[0])
    P[4] = 1.5 * (1.0 + amp * np.tanh(g[1]))
    for c in range(3):
        P[1 + c] = amp * np.tanh(g[2 + c])
    A = [b_amp * span[0] / (2.0 * math.pi) * f(*xn) for f in fa]
    Bface = _face_curl(A, s.dx)
    Bf = np.empty((3,) + P.shape[1:])
    for c in range(3):
        sl = [slice(None)] * 3
        sl[_AX_OF[c]] = slice(0, -1)
        Bf[c] = Bface[c][tuple(sl)]
        P[5 + c] = _mu(Bface[c], _AX_OF[c])
    return P, Bf


def plane_random_prims(s: Setup, d: int, seed: int = 5, amp: float = 0.3):
    """Seeded random state that varies along direction d only (periodic Minkowski block), and its
    face field. Every variable is a constant plus a sum of three random Fourier modes of the cell
    coordinate along d; the normal field B^d is constant (a divergence-free plane field).
    Returns (P, Bf) with Bf [3][gz][gy][gx]: a d-face carries B^d, a face of another direction c
    carries the B^c of its cell."""
    rng = np.random.default_rng(seed)
    n = s.n[d]
    x = (np.arange(-s.ng, n + s.ng) + 0.5) / n  # unit coordinate of the cells along d

    def profile(base, a):
        k = rng.integers(1, 4, size=3)
        ph = rng.uniform(0.0, 2.0 * math.pi, size=3)
        c = rng.normal(size=3)
        f = np.sum(c[:, None] * np.sin(2.0 * math.pi * k[:, None] * x[None, :] + ph[:, None]), axis=0)
        return base + a * f / np.max(np.abs(f))

    prof = [profile(1.0, amp), profile(0.0, amp), profile(0.0, amp), profile(0.0, amp), profile(1.5, amp * 1.5),
            None, None, None]
    for c in range(3):
        prof[5 + c] = np.full_like(x, 0.4) if c == d else profile(0.0, 0.5)
    ax = _AX_OF[d]
    shape = [1, 1, 1]
    shape[ax] = len(x)
    P = np.empty(s.prim_shape())
    for v in range(8):
        P[v] = prof[v].reshape(shape)
    Bf = np.ascontiguousarray(P[5:8].copy())
    return P, Bf


def field_loop_setup(n: int = 32, recon: str = "plm_mc", riemann: str = "hll") -> Setup:
    """Periodic Minkowski square [0, 1]^2 of n x n cells, one cell thick in z."""
    return Setup(n=(n, n, 1), x0=(0.0, 0.0, 0.0), dx=(1.0 / n, 1.0 / n, 1.0 / n), metric="minkowski",
                 recon=recon, riemann=riemann, bc="periodic")


def field_loop_prims(s: Setup, v=(0.3, 0.15), radius: float = 0.3, a0: float = 1e-3, rho: float = 1.0,
                     press: float = 1.0):
    """Weak magnetic field loop advected by a uniform flow (the standard CT advection test): uniform
    rho, pressure and velocity v (as W v^i in P), B the curl of A_z = a0 (radius - r) inside the loop
    (r from the square's centre), zero outside. Returns (P, Bf), Bf the face curl of the node-centred
    A_z; P's cell field is the mean of its faces."""
    vx, vy = v
    W = 1.0 / math.sqrt(1.0 - vx * vx - vy * vy)
    P = np.zeros(s.prim_shape())
    P[0] = rho
    P[1] = W * vx
    P[2] = W * vy
    P[4] = press / (s.gamma_eos - 1.0)
    gz, gy, gx = P.shape[1:]
    xn = [s.x0[d] + np.arange(-s.ng, s.n[d] + s.ng + 1) * s.dx[d] for d in range(3)]
    X, Y = np.meshgrid(xn[0], xn[1], indexing="xy")  # [y][x] node grid
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2)
    az = np.where(r < radius, a0 * (radius - r), 0.0)
    Az = np.broadcast_to(az[None, :, :], (gz + 1,) + az.shape).copy()
    zero = np.zeros_like(Az)
    Bface = _face_curl([zero, zero, Az], s.dx)
    Bf = np.empty((3,) + P.shape[1:])
    for c in range(3):
        sl = [slice(None)] * 3
        sl[_AX_OF[c]] = slice(0, -1)
        Bf[c] = Bface[c][tuple(sl)]
    for c in range(3):
        P[5 + c] = _mu(Bface[c], _AX_OF[c])
    return P, Bf


def c2p_states(n: int, seed: int = 4, gamma_eos: float = GAMMA_DEFAULT, rho_range=(1e-8, 1.0), w_range=(1.0, 50.0),
               sigma_range=(1e-4, 1e3)) -> np.ndarray:
    """i.i.d. primitive states [n][8] (rho, W v^i, rho eps, B^i) in flat space.

    |B| is set from the magnetisation proxy sigma ~ B^2/(rho W^2); the caller maps them to
    conserved states with its own prim->cons routine.
    """
    rng = np.random.default_rng(seed)

    def logu(lo, hi):
        return 10.0 ** rng.uniform(math.log10(lo), math.log10(hi), size=n)

    rho = logu(*rho_range)
    W = logu(*w_range)
    sig = logu(*sigma_range)
    press = 0.01 * rho ** (5.0 / 3.0) * 10.0 ** rng.uniform(-1.0, 1.0, size=n)
    dv = rng.normal(size=(n, 3)); dv /= np.linalg.norm(dv, axis=1, keepdims=True)
    db = rng.normal(size=(n, 3)); db /= np.linalg.norm(db, axis=1, keepdims=True)
    P = np.empty((n, 8))
    P[:, 0] = rho
    P[:, 1:4] = np.sqrt(W * W - 1.0)[:, None] * dv
    P[:, 4] = press / (gamma_eos - 1.0)
    P[:, 5:8] = (W * np.sqrt(sig * rho))[:, None] * db
    return P


def c2p_states_device(n: int, seed: int, device, gamma_eos: float = GAMMA_DEFAULT, rho_range=(1e-8, 1.0),
                      w_range=(1.0, 50.0), sigma_range=(1e-4, 1e3)):
    """The distribution of c2p_states drawn on a CUDA device from a seeded torch generator:
    primitive states [8][n] (float64, structure of arrays) for workloads too large to draw on the host.
    The states differ from c2p_states' (another generator); the distribution is the same."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    f64 = dict(dtype=torch.float64, device=device)

    def logu(lo, hi):
        return 10.0 ** (math.log10(lo) + (math.log10(hi) - math.log10(lo)) * torch.rand(n, generator=g, **f64))

    rho = logu(*rho_range)
    W = logu(*w_range)
    sig = logu(*sigma_range)
    press = 0.01 * rho ** (5.0 / 3.0) * 10.0 ** (2.0 * torch.rand(n, generator=g, **f64) - 1.0)
    dv = torch.randn(3, n, generator=g, **f64)
    dv /= torch.linalg.vector_norm(dv, dim=0, keepdim=True)
    db = torch.randn(3, n, generator=g, **f64)
    db /= torch.linalg.vector_norm(db, dim=0, keepdim=True)
    P = torch.empty(8, n, **f64)
    P[0] = rho
    P[1:4] = torch.sqrt(W * W - 1.0) * dv
    P[4] = press / (gamma_eos - 1.0)
    P[5:8] = W * torch.sqrt(sig * rho) * db
    return P


# ----------------------------------------------------------------------------- two-level block meshes
def batched_setups(sizes=None, precision: str = "mixed", ids=None):
    """The 640-block batched workload: 448 x 16^3, 160 x 32^3 and 32 x 64^3 meshblocks (4 ghosts), each of
    physical size 1.6 on its own sub-cube of a 9 x 9 x 8 lattice from (3, 3, 3) in Kerr-Schild coordinates
    (a = 0.9), WENO5-Z-AOAH + HLL, fixed ghosts; block b's primitives come from kerr_schild_random_prims with
    seed 3 + b. ids selects a subset of the 640 blocks (same sizes, places and seeds as in the full batch)."""
    if sizes is None:
        sizes = [16] * 448 + [32] * 160 + [64] * 32
    setups = []
    for b in (range(len(sizes)) if ids is None else ids):
        n = sizes[b]
        ix, iy, iz = b % 9, (b // 9) % 9, b // 81
        h = 1.6 / n
        setups.append(Setup(n=(n, n, n), x0=(3.0 + 1.6 * ix, 3.0 + 1.6 * iy, 3.0 + 1.6 * iz), dx=(h, h, h),
                            metric="kerr_schild", spin=0.9, recon="weno5z_aoah", riemann="hll", bc="fixed",
                            precision=precision))
    return setups


@dataclasses.dataclass
class TwoLevelMesh:
    """Leaves of a two-level block mesh over an nb[0] x nb[1] x nb[2] grid of root blocks. ``root`` holds the
    physics options, the cell counts of every block (even), the mesh corner (x0) and the level-0 cell
    width (dx). Block b has level ``levels[b]`` (0: a root block; 1: one of the 8 children of a refined
    root block, half the cell width) and position ``pos[b]`` in its level's block lattice (level 1:
    0 <= pos < 2 nb). ``periodic``: the mesh wraps; else the ghosts outside it keep their loaded values."""
    root: Setup
    nb: Tuple[int, int, int]
    periodic: bool
    levels: list
    pos: list

    @property
    def nblocks(self):
        return len(self.levels)

    def setup(self, b: int) -> Setup:
        h = 0.5 ** self.levels[b]
        dx = tuple(self.root.dx[d] * h for d in range(3))
        x0 = tuple(self.root.x0[d] + self.pos[b][d] * self.root.n[d] * dx[d] for d in range(3))
        return dataclasses.replace(self.root, x0=x0, dx=dx, bc="fixed")

    def extent(self):
        return tuple(self.nb[d] * self.root.n[d] * self.root.dx[d] for d in range(3))


def two_level_mesh(root: Setup, nb, refined, periodic: bool) -> TwoLevelMesh:
    """The root blocks not in ``refined`` (level 0, lattice order, x fastest), then the 8 children of each
    refined root block in the order given (x fastest)."""
    refined = [tuple(r) for r in refined]
    levels, pos = [], []
    for z in range(nb[2]):
        for y in range(nb[1]):
            for x in range(nb[0]):
                if (x, y, z) not in refined:
                    levels.append(0)
                    pos.append((x, y, z))
    for r in refined:
        for c in range(8):
            levels.append(1)
            pos.append((2 * r[0] + (c & 1), 2 * r[1] + ((c >> 1) & 1), 2 * r[2] + (c >> 2)))
    return TwoLevelMesh(root=root, nb=tuple(nb), periodic=periodic, levels=levels, pos=pos)


def two_level_prims(mesh: TwoLevelMesh, seed: int = 8, amp: float = 0.3, b0=(0.3, 0.0, 0.0), b_amp: float = 0.1,
                    kmax: int = 1, rho0: float = 1.0):
    """Seeded smooth state of the whole mesh, evaluated at every block's cells (ghosts included): rho =
    rho0 (1 + amp tanh f0), rho eps = 1.5 rho0 (1 + amp tanh f1), W v^i = amp tanh f_i, B = b0 + b_amp f_B,
    each f a sum of random Fourier modes on the mesh's unit cube (periodic on it). Returns [P_b]."""
    rng = np.random.default_rng(seed)
    fs = [_SmoothField(rng, kmax=kmax) for _ in range(8)]
    span = mesh.extent()
    out = []
    for b in range(mesh.nblocks):
        s = mesh.setup(b)
        u = [(s.cell_centres(d) - mesh.root.x0[d]) / span[d] for d in range(3)]
        g = [f(*u) for f in fs]
        P = np.empty(s.prim_shape())
        P[0] = rho0 * (1.0 + amp * np.tanh(g[0]))
        P[4] = 1.5 * rho0 * (1.0 + amp * np.tanh(g[1]))
        for c in range(3):
            P[1 + c] = amp * np.tanh(g[2 + c])
            P[5 + c] = b0[c] + b_amp * g[5 + c]
        out.append(P)
    return out


def two_level_wave_prims(mesh: TwoLevelMesh, background, eigvec, amplitude: float = 1e-6):
    """Plane wave along x over the whole mesh: background + amplitude * eigvec * sin(2 pi (x - x0) / L) at
    every block's cells (ghosts included), L the mesh's x extent. Returns [P_b]."""
    L = mesh.extent()[0]
    out = []
    for b in range(mesh.nblocks):
        s = mesh.setup(b)
        ph = np.sin(2.0 * math.pi * (s.cell_centres(0) - mesh.root.x0[0]) / L)
        P = np.empty(s.prim_shape())
        for v in range(8):
            P[v] = background[v] + amplitude * eigvec[v] * ph[None, None, :]
        out.append(P)
    return out


# ----------------------------------------------------------------------------- spherical Kerr-Schild
def torus_setup(n, r_lo, r_hi, th_lo, th_hi, spin=0.9, recon="weno5z_aoah", riemann="hll", nphi=4,
                dphi=0.05) -> Setup:
    """Block of n x n x nphi cells in spherical Kerr-Schild coordinates (x^1, x^2, x^3) = (ln r, theta, phi)
    over [ln r_lo, ln r_hi] x [th_lo, th_hi] x [0, nphi dphi], fixed ghosts."""
    x0 = (math.log(r_lo), th_lo, 0.0)
    dx = ((math.log(r_hi) - math.log(r_lo)) / n, (th_hi - th_lo) / n, dphi)
    return Setup(n=(n, n, nphi), x0=x0, dx=dx, metric="kerr_schild_spherical", spin=spin, mass=1.0, recon=recon,
                 riemann=riemann, bc="fixed")


def full_sphere_setup(nr, nth, nph, r_lo=3.0, r_hi=10.0, spin=0.9, mass=1.0, recon="weno5z_aoah", riemann="hll",
                      precision="fp64") -> Setup:
    """Block over ln r in [ln r_lo, ln r_hi], theta in [0, pi], phi in [0, 2 pi) in spherical Kerr-Schild
    coordinates, with the spherical boundary (polar and azimuthal ghosts; radial ghosts fixed)."""
    return Setup(n=(nr, nth, nph), x0=(math.log(r_lo), 0.0, 0.0),
                 dx=(math.log(r_hi / r_lo) / nr, math.pi / nth, 2 * math.pi / nph), metric="kerr_schild_spherical",
                 spin=spin, mass=mass, bc="spherical", recon=recon, riemann=riemann, precision=precision)


def spherical_random_prims(s: Setup, seed: int, amp=0.2):
    """Seeded primitives on every cell (ghosts included) of a spherical Kerr-Schild block: density and
    internal energy around 1 and 0.5, a rotation about the axis (u~^phi = 0.1 / r, smooth through the axis)
    and a field with components along r, theta, phi, each perturbed by uniform noise of relative size amp.
    Contravariant components in (ln r, theta, phi): a physical component of size v along r is v / r."""
    rng = np.random.default_rng(seed)
    x1, th = s.cell_centres(0), s.cell_centres(1)
    shape = s.prim_shape()[1:]                      # [phi][theta][ln r]
    r = np.broadcast_to(np.exp(x1)[None, None, :], shape)
    noise = lambda: 1.0 + amp * rng.uniform(-1.0, 1.0, shape)
    P = np.zeros(s.prim_shape())
    P[0] = noise()
    P[4] = 0.5 * noise()
    P[1] = 0.05 * (noise() - 1.0) / r
    P[2] = 0.05 * (noise() - 1.0) / r
    P[3] = 0.1 * noise() / r
    P[5] = 0.1 * noise() / r
    P[6] = 0.05 * (noise() - 1.0) / r
    P[7] = 0.05 * noise() / r
    return P


def _bl_inverse_t_phi(r, th, a, M=1.0):
    """g^{tt}, g^{t phi}, g^{phi phi} of Kerr in Boyer-Lindquist coordinates."""
    s2 = np.sin(th) ** 2
    Sig = r * r + a * a * np.cos(th) ** 2
    gtt = -(1 - 2 * M * r / Sig)
    gtp = -2 * M * a * r * s2 / Sig
    gpp = (r * r + a * a + 2 * M * a * a * r * s2 / Sig) * s2
    det = gtt * gpp - gtp * gtp
    return gpp / det, -gtp / det, gtt / det, (gtt, gtp, gpp)


def _u_t(r, th, l, a):
    """u_t of the purely azimuthal flow with specific angular momentum l = -u_phi / u_t (u_t < 0); NaN where no
    such flow exists (near the axis, where l would need a superluminal velocity: those cells are atmosphere)."""
    itt, itp, ipp, _ = _bl_inverse_t_phi(r, th, a)
    with np.errstate(invalid="ignore"):
        return -1.0 / np.sqrt(-(itt - 2 * l * itp + l * l * ipp))


def torus_l(r_max, a, M=1.0):
    """Specific angular momentum -u_phi/u_t of the prograde circular orbit at r_max in the equatorial plane
    (Keplerian angular velocity sqrt(M) / (r^{3/2} + a sqrt(M)))."""
    Om = math.sqrt(M) / (r_max ** 1.5 + a * math.sqrt(M))
    _, _, _, (gtt, gtp, gpp) = _bl_inverse_t_phi(np.array(r_max), np.array(math.pi / 2), a, M)
    return float(-(gtp + gpp * Om) / (gtt + gtp * Om))


def torus_prims(s: Setup, r_in=6.0, r_max=12.0, K=0.01, rho_atm=1e-6, u_atm=1e-8):
    """A stationary torus around a Kerr black hole: constant specific angular momentum l = -u_phi / u_t (the
    Keplerian value at r_max), isentropic p = K rho^gamma, enthalpy from h u_t = const (h = 1 at the inner
    edge r_in on the equator), at rest in r and theta; outside it a static-density atmosphere. The 4-velocity
    has u^r = u^theta = 0 in Boyer-Lindquist coordinates, so u^t and u^phi are the same in Kerr-Schild.
    Primitives at every cell of the spherical Kerr-Schild block s (ghosts included), B = 0."""
    a, gam = s.spin * s.mass, s.gamma_eos
    l = torus_l(r_max, a)
    ut_in = _u_t(np.array(r_in), np.array(math.pi / 2), l, a)
    x1, th = s.cell_centres(0), s.cell_centres(1)
    R, TH = np.meshgrid(np.exp(x1), th, indexing="xy")          # [theta][r]
    ut = _u_t(R, TH, l, a)
    h = ut_in / ut
    inside = h > 1.0
    rho = np.where(inside, (np.maximum(h - 1.0, 0.0) * (gam - 1.0) / (K * gam)) ** (1.0 / (gam - 1.0)), rho_atm)
    u = np.where(inside, K * rho ** gam / (gam - 1.0), u_atm)
    itt, itp, ipp, _ = _bl_inverse_t_phi(R, TH, a)
    uph_l = -l * ut
    ucon_t = np.where(inside, itt * ut + itp * uph_l, 0.0)
    ucon_p = np.where(inside, itp * ut + ipp * uph_l, 0.0)
    # Kerr-Schild 3+1 split in (ln r, theta, phi): alpha = 1/sqrt(1 + q), beta^1 = q / ((1 + q) r)
    Sig = R * R + a * a * np.cos(TH) ** 2
    q = 2.0 * R / Sig
    alpha = 1.0 / np.sqrt(1.0 + q)
    beta1 = q / ((1.0 + q) * R)
    # the atmosphere is at rest with respect to the normal observers (W = 1, u~ = 0)
    P = np.zeros(s.prim_shape())
    P[0] = rho[None]
    P[4] = u[None]
    P[1] = np.where(inside, beta1 * ucon_t, 0.0)[None]          # u~^1 = u^1 + beta^1 u^t, u^1 = 0
    P[3] = np.where(inside, ucon_p, 0.0)[None]                   # u~^3 = u^3 + beta^3 u^t, beta^3 = 0
    del alpha
    return P
