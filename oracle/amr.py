"""Oracle of one RK stage on a two-level block mesh (the multi-block / AMR fill that the meshblock method
relies on: every meshblock's ghosts come from its neighbours, at the same level, a finer one or a coarser
one, and the coarse side of a coarse-fine face takes the fine fluxes). TEST INFRASTRUCTURE: only the tests,
the package's smoke check and the benchmark's CPU baseline use it; the product path never does.

The paper names the AMR fill without formulas; the readings taken here:
* ghosts are exchanged as primitives, in two passes at the start of every stage. Pass 1: a ghost whose
  point lies in a leaf of the same level copies that leaf's cell; a coarse ghost over a fine leaf takes
  the mean of the 8 fine cells it covers (restriction). Pass 2: a fine ghost over a coarse leaf is the
  coarse cell's value plus, per direction, a minmod-limited slope times the offset (+-1/4 of the coarse
  width) of the fine centre (prolongation; the mean of the 8 children is the coarse value). The slope
  stencil may read coarse ghosts, which pass 1 filled.
* every block then takes the single-block stage (flux-CT, fixed ghosts);
* refluxing (Berger and Colella): a coarse cell with a face on a fine leaf replaces, in its update, that
  face's flux (for B the flux-CT face flux formed from the edge EMFs) by the mean of the 4 fine face
  fluxes covering it, so that the mesh conserves every variable; it is applied after the stage,
  U += beta dt s (F_coarse - F_fine) / dx (s = +1 for the cell's upper face, -1 for its lower), and the
  cell then takes con2prim, floors and the re-derived hydro state again (the stage's last step).
* one time step for all levels (no subcycling);
* a passive scalar X (optional) is exchanged like a primitive (the same copy, restriction and
  prolongation) and its conserved sqrt(gamma) D X refluxed like the other variables, with the scalar's
  face fluxes, after the fluid's refluxing; the refluxed cell's X is then DX / D with its refluxed D.
Out of the mesh the coordinates wrap when periodic; otherwise those ghosts keep their loaded values.
"""
import numpy as np

from . import finish_points, face_fluxes_used, params, stage, stage_scalar

LEAF_NONE = -1


def leaf_map(mesh):
    """Block id covering each fine-block-sized unit of the mesh, [2 nbz][2 nby][2 nbx]; checks that the
    leaves tile the mesh once."""
    nb = mesh.nb
    m = np.full((2 * nb[2], 2 * nb[1], 2 * nb[0]), LEAF_NONE, dtype=np.int64)
    for b, (lev, p) in enumerate(zip(mesh.levels, mesh.pos)):
        w = 2 if lev == 0 else 1  # units per block side
        u = [p[d] * w for d in range(3)]
        sl = m[u[2]:u[2] + w, u[1]:u[1] + w, u[0]:u[0] + w]
        assert np.all(sl == LEAF_NONE), "leaves overlap"
        sl[...] = b
    assert np.all(m != LEAF_NONE), "leaves do not cover the mesh"
    return m


def _minmod(a, b):
    return np.where(a * b > 0.0, np.sign(a) * np.minimum(np.abs(a), np.abs(b)), 0.0)


def _ghost_points(mesh, b):
    """Ghost cells of block b: their local ghosted indices (k, j, i) and global indices in the block's level,
    wrapped when periodic, with a mask of those inside the mesh (or wrapped)."""
    s = mesh.root
    n, ng = s.n, s.ng
    lev, p = mesh.levels[b], mesh.pos[b]
    idx = [np.arange(-ng, n[d] + ng) for d in range(3)]
    K, J, I = np.meshgrid(idx[2], idx[1], idx[0], indexing="ij")
    loc = [I, J, K]
    ghost = np.zeros(I.shape, bool)
    for d in range(3):
        ghost |= (loc[d] < 0) | (loc[d] >= n[d])
    glob, inside = [], np.ones(I.shape, bool)
    for d in range(3):
        N = mesh.nb[d] * n[d] * (2 ** lev)
        g = p[d] * n[d] + loc[d]
        out = (g < 0) | (g >= N)
        if mesh.periodic:
            g = np.mod(g, N)
        else:
            inside &= ~out
        glob.append(g)
    sel = ghost & inside
    return [loc[d][sel] for d in range(3)], [glob[d][sel] for d in range(3)]


def fill_ghosts(mesh, Ps, lm=None):
    """The two-pass ghost exchange (module docstring) on the ghosted primitives Ps[b], in place."""
    lm = leaf_map(mesh) if lm is None else lm
    n, ng = mesh.root.n, mesh.root.ng
    for pass_ in (1, 2):
        for b in range(mesh.nblocks):
            lev = mesh.levels[b]
            loc, glob = _ghost_points(mesh, b)
            fine = [glob[d] if lev == 1 else 2 * glob[d] for d in range(3)]   # a fine cell of the point
            leaf = lm[fine[2] // n[2], fine[1] // n[1], fine[0] // n[0]]
            dst = (slice(None), loc[2] + ng, loc[1] + ng, loc[0] + ng)
            for src in np.unique(leaf):
                m = leaf == src
                ls, ps = mesh.levels[src], mesh.pos[src]
                dsel = (slice(None), dst[1][m], dst[2][m], dst[3][m])
                if pass_ == 1 and ls == lev:
                    li = [glob[d][m] - ps[d] * n[d] + ng for d in range(3)]
                    Ps[b][dsel] = Ps[src][:, li[2], li[1], li[0]]
                elif pass_ == 1 and lev == 0 and ls == 1:
                    f0 = [2 * glob[d][m] - ps[d] * n[d] + ng for d in range(3)]
                    acc = 0.0
                    for c in range(8):
                        acc = acc + Ps[src][:, f0[2] + (c >> 2), f0[1] + ((c >> 1) & 1), f0[0] + (c & 1)]
                    Ps[b][dsel] = acc / 8.0
                elif pass_ == 2 and lev == 1 and ls == 0:
                    lc = [glob[d][m] // 2 - ps[d] * n[d] + ng for d in range(3)]
                    off = [np.where(glob[d][m] % 2 == 1, 0.25, -0.25) for d in range(3)]
                    C = Ps[src]
                    pc = C[:, lc[2], lc[1], lc[0]]
                    val = pc.copy()
                    for d in range(3):
                        e = [0, 0, 0]
                        e[d] = 1
                        up = C[:, lc[2] + e[2], lc[1] + e[1], lc[0] + e[0]]
                        dn = C[:, lc[2] - e[2], lc[1] - e[1], lc[0] - e[0]]
                        val = val + off[d] * _minmod(up - pc, pc - dn)
                    Ps[b][dsel] = val


def _reflux(mesh, lm, Fu):
    """Per coarse block: {interior cell index (k, j, i): dU [8] / (beta dt)} from every coarse-fine face."""
    n = mesh.root.n
    corr = [dict() for _ in range(mesh.nblocks)]
    for b in range(mesh.nblocks):
        if mesh.levels[b] != 0:
            continue
        s = mesh.setup(b)
        p = mesh.pos[b]
        for d in range(3):
            a1, a2 = [e for e in range(3) if e != d]
            for side in (-1, 1):
                cell_d = 0 if side < 0 else n[d] - 1
                N = mesh.nb[d] * n[d]
                gnb = p[d] * n[d] + cell_d + side     # coarse index across the face
                if gnb < 0 or gnb >= N:
                    if not mesh.periodic:
                        continue
                    gnb %= N
                for t2 in range(n[a2]):
                    for t1 in range(n[a1]):
                        gc = [0, 0, 0]
                        gc[d] = gnb
                        gc[a1] = p[a1] * n[a1] + t1
                        gc[a2] = p[a2] * n[a2] + t2
                        src = lm[2 * gc[2] // n[2], 2 * gc[1] // n[1], 2 * gc[0] // n[0]]
                        if mesh.levels[src] != 1:
                            continue
                        ps = mesh.pos[src]
                        cell = [0, 0, 0]
                        cell[d], cell[a1], cell[a2] = cell_d, t1, t2
                        # the face's flux in the coarse block: lower face of cell (side -1) or of cell + 1
                        fc = list(cell)
                        if side > 0:
                            fc[d] += 1
                        ng = s.ng
                        Fc = Fu[b][d][:, fc[2] + ng, fc[1] + ng, fc[0] + ng]
                        # the 4 fine faces: on the fine block's upper boundary (index n) when it lies below
                        ff = [0, 0, 0]
                        ff[d] = 0 if side > 0 else n[d]
                        Ff = 0.0
                        for c2 in range(2):
                            for c1 in range(2):
                                ff[a1] = 2 * gc[a1] - ps[a1] * n[a1] + c1
                                ff[a2] = 2 * gc[a2] - ps[a2] * n[a2] + c2
                                Ff = Ff + Fu[src][d][:, ff[2] + ng, ff[1] + ng, ff[0] + ng]
                        dU = side * (Fc - Ff / 4.0) / s.dx[d]
                        key = (cell[2], cell[1], cell[0])
                        corr[b][key] = corr[b].get(key, 0.0) + dU
    return corr


def mesh_stage(mesh, Ps, U0s, Ucurs, g0, g1, beta, dt, Xs=None, DX0s=None, DXcurs=None):
    """One RK stage of the mesh: Unew = g0 U0 + g1 Ucur + beta dt L on every leaf, with the ghost exchange
    before and the refluxing after (module docstring). Ps (and the scalar's Xs, when given with its
    conserved DXcurs and, for g0 != 0, DX0s) are updated in place. Returns (Unew list, status list,
    per-block maxspeed / dx maxima), and the DXnew list last when a scalar is given."""
    lm = leaf_map(mesh)
    fill_ghosts(mesh, Ps, lm)
    if Xs is not None:
        fill_ghosts(mesh, [X[None] for X in Xs], lm)  # as a one-variable primitive
    outs, Fu, FX, speeds = [], [], [], []
    for b in range(mesh.nblocks):
        p = params(mesh.setup(b))
        U0 = None if U0s is None else U0s[b]
        if Xs is None:
            o = stage(p, Ps[b], U0, Ucurs[b], g0, g1, beta, dt, debug=True)
        else:
            o = stage_scalar(p, Ps[b], Xs[b], U0, Ucurs[b], None if DX0s is None else DX0s[b], DXcurs[b], g0, g1,
                             beta, dt, debug=True)
            FX.append([o["FX"][d][None] for d in range(3)])
        outs.append(o)
        Fu.append(face_fluxes_used(p, o["F"], o["E"]))
        speeds.append(max(o["maxspeed"][d] / mesh.setup(b).dx[d] for d in range(3)))
    Unew = [o["U"] for o in outs]
    status = [o["status"] for o in outs]
    corr = _reflux(mesh, lm, Fu)
    for b in range(mesh.nblocks):
        if not corr[b]:
            continue
        s = mesh.setup(b)
        keys = sorted(corr[b])
        kji = np.array(keys)
        xyz = np.stack([s.x0[d] + (kji[:, 2 - d] + 0.5) * s.dx[d] for d in range(3)], 1)
        U = np.stack([Unew[b][:, k, j, i] + beta * dt * corr[b][(k, j, i)] for (k, j, i) in keys])
        Un, P, st = finish_points(params(s), xyz, U)
        ng = s.ng
        for q, (k, j, i) in enumerate(keys):
            Unew[b][:, k, j, i] = Un[q]
            Ps[b][:, k + ng, j + ng, i + ng] = P[q]
            status[b][k, j, i] = st[q]
    if Xs is None:
        return Unew, status, speeds
    DXnew = [o["DX"] for o in outs]
    corrX = _reflux(mesh, lm, FX)
    for b in range(mesh.nblocks):
        ng = mesh.setup(b).ng
        for (k, j, i), dX in corrX[b].items():
            DXnew[b][k, j, i] = DXnew[b][k, j, i] + beta * dt * dX[0]
            Xs[b][k + ng, j + ng, i + ng] = DXnew[b][k, j, i] / Unew[b][0, k, j, i]
    return Unew, status, speeds, DXnew


def mesh_dt(mesh, speeds):
    """CFL time step of the mesh: cfl / (max over blocks and directions of |lambda| / dx)."""
    return mesh.root.cfl / max(speeds)


def mesh_prim2con(mesh, Ps):
    from . import prim2con_grid
    return [prim2con_grid(params(mesh.setup(b)), Ps[b].copy()) for b in range(mesh.nblocks)]


def mesh_totals(mesh, Us):
    """Sum over the leaves of cell volume x densitized conserved state, per variable."""
    tot = np.zeros(8)
    for b in range(mesh.nblocks):
        s = mesh.setup(b)
        tot += Us[b].reshape(8, -1).sum(1) * (s.dx[0] * s.dx[1] * s.dx[2])
    return tot
