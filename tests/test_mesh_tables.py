"""Host logic of two-level meshes (build_mesh_tables in csrc/grmhd_mesh_host.h, compiled for the host through
tests/mesh_tables_shim.cu; no GPU): the leaf map equals the two-level oracle's, the coarse-fine cell list
holds exactly the coarse cells the oracle refluxes, each with the fine block across each of its coarse-fine
faces, the ghost table lists every ghost cell of a block once, the fine list the level-1 blocks; bad meshes
are refused (overlapping or missing leaves, cell widths or corners off their level and position, odd cell
counts)."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import amr
from paper_2410_09146_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tempfile.mkdtemp(prefix="mesh_tables_")
    so = os.path.join(d, "libmt.so")
    # the library's device headers are written for sm_103a (paired FP32 instructions), so the shim is too
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O1", "-Xcompiler", "-fPIC",
                    "-shared", "-o", so,
                    os.path.join(HERE, "mesh_tables_shim.cu")], check=True, capture_output=True)
    L = ctypes.CDLL(so)
    L.mt_build.restype = ctypes.c_int
    return L


def _build(lib, m, level=None, pos=None, x0=None, dx=None, nb=None, periodic=None):
    nbk = m.nblocks
    n = np.array(m.root.n, np.int32)
    X0 = np.array([m.setup(b).x0 for b in range(nbk)], np.float64) if x0 is None else np.asarray(x0, np.float64)
    DX = np.array([m.setup(b).dx for b in range(nbk)], np.float64) if dx is None else np.asarray(dx, np.float64)
    lv = np.array(m.levels if level is None else level, np.int32)
    ps = np.array(m.pos if pos is None else pos, np.int32)
    nb = m.nb if nb is None else nb
    per = m.periodic if periodic is None else periodic
    leaf = np.zeros(8 * nb[0] * nb[1] * nb[2], np.int32)
    G = int(np.prod([k + 2 * m.root.ng for k in m.root.n]))
    cells = np.zeros((nbk * G, 8), np.int32)
    ghost = np.zeros(G, np.uint32)
    fine = np.zeros(nbk, np.int32)
    cnt = [ctypes.c_longlong(0) for _ in range(4)]
    why = ctypes.create_string_buffer(200)
    P = lambda a, t: a.ctypes.data_as(ctypes.POINTER(t))
    rc = lib.mt_build(nbk, P(n, ctypes.c_int), m.root.ng, P(X0, ctypes.c_double), P(DX, ctypes.c_double),
                      nb[0], nb[1], nb[2], int(per), P(lv, ctypes.c_int), P(ps, ctypes.c_int), P(leaf, ctypes.c_int),
                      ctypes.byref(cnt[0]), P(cells, ctypes.c_int), ctypes.byref(cnt[1]), P(ghost, ctypes.c_uint),
                      ctypes.byref(cnt[2]), P(fine, ctypes.c_int), ctypes.byref(cnt[3]), why, 200)
    if rc:
        return why.value.decode()
    return dict(leaf=leaf[:cnt[0].value], cells=cells[:cnt[1].value], ghost=ghost[:cnt[2].value],
                fine=fine[:cnt[3].value])


MESHES = [("periodic, one refined", lambda: I.two_level_mesh(I.Setup(n=(8, 8, 8), dx=(1 / 16,) * 3), (2, 2, 2), [(1, 0, 0)], True)),
          ("periodic, edge and corner", lambda: I.two_level_mesh(I.Setup(n=(8, 6, 4), dx=(0.1, 0.2, 0.25)), (3, 2, 2),
                                                                  [(0, 0, 0), (1, 1, 1)], True)),
          ("fixed outer, Kerr-Schild", lambda: I.two_level_mesh(I.Setup(n=(8, 8, 8), x0=(2.0,) * 3, dx=(0.5,) * 3), (2, 2, 2),
                                                                 [(0, 0, 0)], False)),
          ("periodic 1-root-thick", lambda: I.two_level_mesh(I.Setup(n=(8, 4, 4), dx=(1 / 32,) * 3), (4, 1, 1), [(1, 0, 0)], True))]


@pytest.mark.parametrize("name,make", MESHES, ids=[m[0] for m in MESHES])
def test_tables_match_the_oracle(lib, name, make):
    m = make()
    t = _build(lib, m)
    assert isinstance(t, dict), t
    lm = amr.leaf_map(m)
    assert np.array_equal(t["leaf"], lm.ravel())
    # coarse cells at coarse-fine faces: the cells the oracle refluxes (its reflux with zero fluxes lists them)
    zero = [[np.zeros((1,) + m.setup(b).prim_shape()[1:]) for d in range(3)] for b in range(m.nblocks)]
    want = {(b, k, j, i) for b, cb in enumerate(amr._reflux(m, lm, zero)) for (k, j, i) in cb}
    n = m.root.n
    got = {(int(c[0]), int(c[1]) // (n[0] * n[1]), (int(c[1]) // n[0]) % n[1], int(c[1]) % n[0]) for c in t["cells"]}
    assert got == want and len(got) == len(t["cells"])
    # the fine block across each flagged face is the leaf covering the cell across it
    for c in t["cells"]:
        b, cell = int(c[0]), int(c[1])
        ci = [cell % n[0], (cell // n[0]) % n[1], cell // (n[0] * n[1])]
        for d in range(3):
            for s in range(2):
                f = int(c[2 + 2 * d + s])
                g = [m.pos[b][e] * n[e] + ci[e] for e in range(3)]
                g[d] += 1 if s else -1
                N = m.nb[d] * n[d]
                if not m.periodic and not 0 <= g[d] < N:
                    assert f == -1
                    continue
                g[d] %= N
                src = lm[2 * g[2] // n[2], 2 * g[1] // n[1], 2 * g[0] // n[0]]
                assert f == (src if m.levels[src] == 1 else -1)
    # ghost table: every ghost cell of a block once; fine list: the level-1 blocks
    gx = [k + 2 * m.root.ng for k in n]
    gh = t["ghost"]
    ijk = np.stack([gh & 1023, (gh >> 10) & 1023, gh >> 20], 1).astype(int)
    assert len(np.unique(gh)) == len(gh) == np.prod(gx) - np.prod(n)
    inner = np.all((ijk >= m.root.ng) & (ijk < np.array(n) + m.root.ng), axis=1)
    assert not inner.any() and np.all(ijk < np.array(gx))
    assert list(t["fine"]) == [b for b in range(m.nblocks) if m.levels[b] == 1]


def test_bad_meshes_are_refused(lib):
    m = MESHES[0][1]()
    lv, ps = list(m.levels), [list(p) for p in m.pos]
    assert isinstance(_build(lib, m, level=lv[:-1] + [0]), str)     # a fine block declared coarse
    dx = np.array([m.setup(b).dx for b in range(m.nblocks)])
    dx[1] *= 0.5
    assert "width" in _build(lib, m, dx=dx)                          # a root block with a child's width
    bad = [list(p) for p in ps]
    bad[-1] = list(bad[-2])
    x0b = np.array([m.setup(b).x0 for b in range(m.nblocks)])
    x0b[-1] = x0b[-2]
    assert "overlap" in _build(lib, m, pos=bad, x0=x0b)              # two leaves on one spot
    assert "cover" in _build(lib, m, nb=(3, 2, 2))                   # a root grid the leaves do not fill
    x0 = np.array([m.setup(b).x0 for b in range(m.nblocks)])
    x0[3, 1] += 0.01
    assert "corner" in _build(lib, m, x0=x0)                         # a corner off its position
    assert "outside" in _build(lib, m, pos=ps[:-1] + [[4, 0, 0]])    # beyond the level's lattice
    odd = I.two_level_mesh(I.Setup(n=(6, 6, 5), dx=(0.1,) * 3), (1, 1, 1), [], True)
    assert "even" in _build(lib, odd)
