"""On-device ghost exchange of a lattice batch: blocks tiling one meshblock grid, their ghosts exchanged at
the start of every stage, reproduce the single large block (every face flux, EMF and cell update sees the
same inputs), periodic (Minkowski) and with fixed outer ghosts (Kerr-Schild, cell widths and corners
exactly representable so both sides evaluate the metric at the same coordinates), bit for bit in both
forms: the cell-centric fluxes reconstruct every cell at one call site, so the mixed form's float face
values do not depend on where the runs start, which moves with the block size (and with the run length a
single-block context picks for its size). Status bits identical. The time step is passed in: the batch's
CFL reduction forms max |lambda| / dx in the flux type, the single block max |lambda| then / dx, so a CFL dt
may differ in its last bit."""
import numpy as np
import pytest

from paper_2410_09146_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_09146_gb300 import build
    build.build()
    from paper_2410_09146_gb300 import grmhd
    return grmhd


def _split(s, P, nb):
    """Block set-ups and primitives (ghosts included) of the lattice nb tiling set-up s."""
    n = [s.n[d] // nb[d] for d in range(3)]
    ng = s.ng
    setups, prims = [], []
    for bz in range(nb[2]):
        for by in range(nb[1]):
            for bx in range(nb[0]):
                b = (bx, by, bz)
                x0 = tuple(s.x0[d] + b[d] * n[d] * s.dx[d] for d in range(3))
                sb = I.Setup(n=tuple(n), ng=ng, x0=x0, dx=s.dx, metric=s.metric, spin=s.spin, mass=s.mass,
                             recon=s.recon, riemann=s.riemann, bc="fixed", precision=s.precision)
                sl = tuple(slice(b[d] * n[d], b[d] * n[d] + n[d] + 2 * ng) for d in (2, 1, 0))
                setups.append(sb)
                prims.append(np.ascontiguousarray(P[(slice(None),) + sl]))
    return setups, prims


def _assemble(G, bc, s, nb, what):
    n = [s.n[d] // nb[d] for d in range(3)]
    ng = s.ng
    shape = {G.GRMHD_GET_CONS: (8,) + tuple(s.n[::-1]), G.GRMHD_GET_PRIMS: (8,) + tuple(s.n[::-1]),
             G.GRMHD_GET_STATUS: tuple(s.n[::-1])}[what]
    out = np.zeros(shape, np.uint8 if what == G.GRMHD_GET_STATUS else np.float64)
    k = 0
    for bz in range(nb[2]):
        for by in range(nb[1]):
            for bx in range(nb[0]):
                b = (bx, by, bz)
                a = bc.get(k, what)
                if what == G.GRMHD_GET_PRIMS:
                    a = a[:, ng:-ng, ng:-ng, ng:-ng]
                sl = tuple(slice(b[d] * n[d], (b[d] + 1) * n[d]) for d in (2, 1, 0))
                out[(Ellipsis,) + sl] = a
                k += 1
    return out


def _compare(G, s, P, nb, periodic, dt, steps=2):
    single = G.Context(s)
    single.set_prims(P.copy())
    setups, prims = _split(s, P, nb)
    bc = G.BatchContext(setups)
    for b, Pb in enumerate(prims):
        bc.set_prims(b, Pb)
    bc.set_lattice(nb, periodic)
    for _ in range(steps):
        single.stage(0.0, 1.0, 1.0, dt)
        single.stage(0.5, 0.5, 0.5, dt)
        bc.stage(0.0, 1.0, 1.0, dt)
        bc.stage(0.5, 0.5, 0.5, dt)
    ng = s.ng
    inner = (slice(None),) + (slice(ng, -ng),) * 3
    U, P_, st = (_assemble(G, bc, s, nb, w) for w in (G.GRMHD_GET_CONS, G.GRMHD_GET_PRIMS, G.GRMHD_GET_STATUS))
    assert np.array_equal(st, single.status())
    assert np.array_equal(U, single.cons()), s.precision
    assert np.array_equal(P_, single.prims()[inner]), s.precision


@pytest.mark.parametrize("precision,recon", [("fp64", "weno5z_aoah"), ("mixed", "weno5z_aoah"), ("mixed", "plm_mc")])
def test_periodic_lattice_is_the_large_block(G, precision, recon):
    s = I.Setup(n=(32, 24, 16), dx=(1 / 32, 1 / 32, 1 / 32), recon=recon, riemann="hll", precision=precision)
    P = I.kerr_schild_random_prims(s, seed=9, kmax=1, rho_range=(0.1, 1.0), w_range=(1.0, 3.0))
    _compare(G, s, P, (4, 3, 2), True, dt=0.2 / 32)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_kerr_schild_lattice_with_fixed_outer_ghosts(G, precision):
    s = I.kerr_schild_setup(32, recon="weno5z_aoah", riemann="hll", precision=precision, lo=4.0, hi=12.0)
    assert s.dx == (0.25, 0.25, 0.25)
    P = I.kerr_schild_random_prims(s, seed=4)
    _compare(G, s, P, (2, 2, 2), False, dt=0.05)


def test_lattice_refusals(G):
    s = I.kerr_schild_setup(16, lo=4.0, hi=8.0)
    setups, prims = _split(s, I.kerr_schild_random_prims(s, seed=1), (2, 2, 2))
    bc = G.BatchContext(setups)
    with pytest.raises(G.GrmhdError):
        bc.set_lattice((2, 2, 1), False)   # block count
    with pytest.raises(G.GrmhdError):
        bc.set_lattice((1, 2, 4), False)   # corners off that lattice order
    bc.set_lattice((2, 2, 2), False)
    bc.set_lattice((0, 0, 0), False)       # switched off again
