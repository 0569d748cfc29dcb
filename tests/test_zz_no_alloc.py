"""grmhd_stage_noalloc, the entry point for callers that cannot allocate device memory.

Such callers (code running inside a CUDA-graph capture, hosts whose framework owns every device
allocation, embedded hosts without a device allocator) get the stage's scratch from a fixed array
built into the library instead of a caller-provided workspace. Through the C ABI, two stages in a
row on caller-owned device arrays must reproduce two stages of the context entry point
(grmhd_stage), within the parity tolerance the other GPU tests use (they run the same kernels, so
in practice the results are bitwise equal). An oversized block must be refused with a clear error.

This file is collected last, so a run that stops at the first failure has run every other test.
"""
import json
import os

import numpy as np
import pytest

from paper_2410_09146_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fast_wave_minkowski.json")


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_09146_gb300 import build
    build.build()
    from paper_2410_09146_gb300 import grmhd
    return torch, grmhd


def _workloads():
    gw = json.load(open(GOLDEN))
    s1 = I.linear_wave_setup(16, recon="plm_mc", riemann="llf")
    P1 = I.linear_wave_prims(s1, gw["background_prims"], gw["eigvec_prims"], amplitude=1e-3)
    s2 = I.kerr_schild_setup(14, recon="weno5z_aoah", riemann="hll")
    P2 = I.kerr_schild_random_prims(s2, seed=3)
    return [(s1, P1), (s2, P2)]


def test_noalloc_matches_context_entry_point(env):
    from tests.parity import rel_err_cons
    torch, G = env
    stream = torch.cuda.current_stream().cuda_stream
    for s, P in _workloads():
        ref = G.Context(s)
        ref.set_prims(P.copy())
        U0 = ref.cons()
        ref.stage(0.0, 1.0, 1.0, 0.0)
        U1_ref, P1_ref, st1_ref = ref.cons(), ref.prims(), ref.status()
        ref.stage(0.5, 0.5, 0.5, 0.0)
        U2_ref, P2_ref, st2_ref = ref.cons(), ref.prims(), ref.status()

        p = G.params(s)
        Pd = torch.tensor(P, device="cuda")
        U0d = torch.tensor(U0, device="cuda")
        U1d = torch.empty_like(U0d)
        U2d = torch.empty_like(U0d)
        st = torch.empty(U0.shape[1:], dtype=torch.uint8, device="cuda")
        # first call: CFL time step from this call's face speeds
        G.grmhd_stage_noalloc(p, Pd.data_ptr(), 0, U0d.data_ptr(), U1d.data_ptr(), st.data_ptr(), 0.0, 1.0, 1.0, 0.0,
                              stream)
        torch.cuda.synchronize()
        assert rel_err_cons(U1d.cpu().numpy(), U1_ref).max() <= 1e-12
        assert np.array_equal(st.cpu().numpy(), st1_ref)
        # second call, also with dt <= 0: it reuses the time step the first call left in the scratch array,
        # as grmhd_rk2_step's second stage reuses its first stage's
        G.grmhd_stage_noalloc(p, Pd.data_ptr(), U0d.data_ptr(), U1d.data_ptr(), U2d.data_ptr(), st.data_ptr(), 0.5, 0.5,
                              0.5, 0.0, stream)
        torch.cuda.synchronize()
        assert rel_err_cons(U2d.cpu().numpy(), U2_ref).max() <= 1e-12
        assert np.array_equal(st.cpu().numpy(), st2_ref)
        ng = s.ng
        inner = (slice(None),) + (slice(ng, -ng),) * 3
        Pn = Pd.cpu().numpy()
        scale = np.maximum(np.abs(P2_ref[inner]), 1e-3 * np.abs(P2_ref[inner]).max(axis=(1, 2, 3), keepdims=True))
        assert (np.abs(Pn[inner] - P2_ref[inner]) / scale).max() <= 1e-12


def test_noalloc_block_at_the_scratch_limit(env):
    """The largest block the fixed scratch holds with 4 ghosts (13 x 29 x 206 = 77,662 ghosted cells, the limit
    being 77,669) runs and matches the context entry point; one ghosted cell more than the limit is refused."""
    from tests.parity import rel_err_cons
    torch, G = env
    gw = json.load(open(GOLDEN))
    s = I.linear_wave_setup(5, 21, 198, recon="plm_mc", riemann="llf")
    P = I.linear_wave_prims(s, gw["background_prims"], gw["eigvec_prims"], amplitude=1e-3)
    ref = G.Context(s)
    ref.set_prims(P.copy())
    U0 = ref.cons()
    ref.stage(0.0, 1.0, 1.0, 0.0)
    U1_ref = ref.cons()
    p = G.params(s)
    Pd = torch.tensor(P, device="cuda")
    U0d = torch.tensor(U0, device="cuda")
    U1d = torch.empty_like(U0d)
    st = torch.empty(U0.shape[1:], dtype=torch.uint8, device="cuda")
    G.grmhd_stage_noalloc(p, Pd.data_ptr(), 0, U0d.data_ptr(), U1d.data_ptr(), st.data_ptr(), 0.0, 1.0, 1.0, 0.0,
                          torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rel_err_cons(U1d.cpu().numpy(), U1_ref).max() <= 1e-12
    assert np.array_equal(st.cpu().numpy(), ref.status())
    over = G.params(I.linear_wave_setup(1, 2, 855))  # 9 x 10 x 863 = 77,670 ghosted cells
    with pytest.raises(G.GrmhdError, match="77669"):
        G.grmhd_stage_noalloc(over, Pd.data_ptr(), 0, U0d.data_ptr(), U1d.data_ptr(), st.data_ptr(), 0.0, 1.0, 1.0,
                              0.0, 0)


def test_noalloc_rejects_blocks_beyond_its_scratch(env):
    torch, G = env
    s = I.kerr_schild_setup(40)  # 48^3 ghosted cells: beyond the fixed scratch
    p = G.params(s)
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(G.GrmhdError, match="maximum"):
        G.grmhd_stage_noalloc(p, dummy.data_ptr(), 0, dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), 0.0, 1.0,
                              1.0, 0.0, 0)
