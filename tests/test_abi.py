"""The C-ABI library builds, loads and exports every entry point include/grmhd.h declares (no GPU needed).

Only host-side entry points that touch no device run here: workspace sizing and parameter
validation of grmhd_create.
"""
import ctypes

import numpy as np

import pytest

from paper_2410_09146_gb300 import build as B
from paper_2410_09146_gb300 import grmhd as G
from paper_2410_09146_gb300 import inputs as I


@pytest.fixture(scope="module")
def lib():
    B.build()
    return G.lib()


def test_exports_every_declared_symbol(lib):
    names = G.exported_names()
    assert {"grmhd_create", "grmhd_set_prims", "grmhd_stage", "grmhd_c2p", "grmhd_get",
            "grmhd_destroy", "grmhd_last_error", "grmhd_workspace_bytes"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_workspace_bytes_and_validation(lib):
    s = I.kerr_schild_setup(16)
    p = G.params(s)
    nb = G.grmhd_workspace_bytes(p)
    G_ = (16 + 8) ** 3
    assert nb >= 8 * G_ * 8 + 3 * 8 * 16 ** 3 * 8 + 3 * 8 * G_ * 8
    s.precision = "mixed"
    assert G.grmhd_workspace_bytes(G.params(s)) < nb
    bad = G.params(s)
    bad.ng = 2
    bad.recon = G.RECON["weno5z_aoah"]
    assert G.grmhd_workspace_bytes(bad) == 0
    out = ctypes.c_void_p()
    rc = lib.grmhd_create(ctypes.byref(bad), None, 0, None, ctypes.byref(out))
    assert rc == G.GRMHD_E_INVALID and out.value is None
    assert b"ng" in lib.grmhd_last_error(None)
    # too-small workspace is rejected before any device work
    p2 = G.params(I.kerr_schild_setup(8))
    rc = lib.grmhd_create(ctypes.byref(p2), ctypes.c_void_p(256), 16, None, ctypes.byref(out))
    assert rc == G.GRMHD_E_WORKSPACE


def test_scalar_and_mesh_parameter_validation(lib):
    """Host-side checks of the passive scalar's parameters (no device work)."""
    import dataclasses
    s = dataclasses.replace(I.kerr_schild_setup(16), scalar=True)
    with_x = G.grmhd_workspace_bytes(G.params(s))
    without = G.grmhd_workspace_bytes(G.params(dataclasses.replace(s, scalar=False)))
    G_, I_ = (16 + 8) ** 3, 16 ** 3
    assert with_x - without >= G_ * 8 + 3 * I_ * 8 + 3 * G_ * 8   # X, three D X slots, its face fluxes
    assert G.grmhd_workspace_bytes(G.params(dataclasses.replace(s, ng=2, recon="plm_mc"))) == 0
    assert G.grmhd_workspace_bytes(G.params(dataclasses.replace(s, ct="face"))) == 0
    bad = G.params(s)
    bad.scalar = 2
    assert G.grmhd_workspace_bytes(bad) == 0
    blocks = [G.block_of(dataclasses.replace(s, bc="fixed"))] * 3
    assert (G.grmhd_batch_workspace_bytes(G.params(s), blocks) >
            G.grmhd_batch_workspace_bytes(G.params(dataclasses.replace(s, scalar=False)), blocks))


def test_struct_layout_matches_header(tmp_path):
    """Every field offset of the ctypes mirror equals the C compiler's offsetof on include/grmhd.h."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    names = [f[0] for f in G.grmhd_params._fields_]
    body = "".join(f'printf("%zu\\n", offsetof(grmhd_params, {n}));' for n in names)
    src = tmp_path / "layout.c"
    src.write_text(f'#include "{G.HEADER}"\n#include <stdio.h>\n#include <stddef.h>\n'
                   f'int main(void){{printf("%zu\\n", sizeof(grmhd_params));{body}return 0;}}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", str(src), "-o", str(exe)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(G.grmhd_params)
    assert vals[1:] == [getattr(G.grmhd_params, n).offset for n in names]


def test_noalloc_refusals_on_the_host(lib):
    """grmhd_stage_noalloc checks its parameters as grmhd_create does, and its block size against the fixed
    scratch, before any device work (dummy pointers: nothing is dereferenced)."""
    import dataclasses
    vp = ctypes.c_void_p
    d = vp(256)

    def call(p, g0=0.0, g1=1.0, beta=1.0, dt=0.0):
        return lib.grmhd_stage_noalloc(ctypes.byref(p), d, d, d, d, d, g0, g1, beta, dt, None)

    ks = I.kerr_schild_setup(8)
    bad_mass = G.params(dataclasses.replace(ks, mass=0.0))
    assert call(bad_mass) == G.GRMHD_E_INVALID and b"mass" in lib.grmhd_last_error(None)
    flat = I.linear_wave_setup(8)
    assert call(G.params(dataclasses.replace(flat, shift=(0.8, 0.7, 0.0)))) == G.GRMHD_E_INVALID
    assert b"shift" in lib.grmhd_last_error(None)
    assert call(G.params(flat), beta=float("nan")) == G.GRMHD_E_INVALID
    assert b"NaN" in lib.grmhd_last_error(None)
    assert call(G.params(dataclasses.replace(flat, precision="mixed"))) == G.GRMHD_E_INVALID
    # 9 x 10 x 863 = 77,670 ghosted cells: one more than the 16 MiB scratch holds
    assert call(G.params(I.linear_wave_setup(1, 2, 855))) == G.GRMHD_E_INVALID
    assert b"77669" in lib.grmhd_last_error(None)


def test_spherical_kerr_schild_parameter_validation(lib):
    """Host-side checks of the spherical Kerr-Schild metric and the spherical boundary (no device work)."""
    import dataclasses
    s = I.full_sphere_setup(8, 12, 16)
    assert G.grmhd_workspace_bytes(G.params(s)) > 0
    assert G.grmhd_workspace_bytes(G.params(dataclasses.replace(s, bc="fixed"))) > 0
    assert G.grmhd_workspace_bytes(G.params(dataclasses.replace(s, mass=0.0, spin=0.0))) > 0
    assert G.grmhd_workspace_bytes(G.params(dataclasses.replace(s, precision="mixed"))) > 0
    for bad in (dict(ct="face"), dict(scalar=True), dict(bc="periodic"),
                dict(mass=-1.0), dict(spin=1.0),
                dict(n=(8, 12, 15), dx=(s.dx[0], s.dx[1], 2 * np.pi / 15)),     # odd nz
                dict(x0=(s.x0[0], 0.1, 0.0)),                                   # theta range not [0, pi]
                dict(n=(8, 2, 16), dx=(s.dx[0], np.pi / 2, s.dx[2]))):          # ng > ny
        assert G.grmhd_workspace_bytes(G.params(dataclasses.replace(s, **bad))) == 0, bad
    # the spherical boundary needs the spherical metric
    assert G.grmhd_workspace_bytes(G.params(dataclasses.replace(I.kerr_schild_setup(16), bc="spherical"))) == 0

