"""paris_divergence_noalloc: the divergence entry point for callers that cannot
allocate device memory (it needs no context and keeps its block sums in a
fixed static device array).  Checked through the C ABI against paris_divergence
(the context-based entry point) on two calls in a row, so that a call which
finds the previous call's data in the shared array is covered too.  This file
is collected last on purpose."""
import ctypes as ct

import numpy as np
import pytest

import paris_inputs as pi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_divergence_matches_context_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2012_11744_gb300 as paris
    from paper_2012_11744_gb300 import _abi
    paris.build()
    lib = _abi.load()
    grid = pi.Grid(64, 40, 48, 1.0 / 64, (pi.PERIODIC, pi.WALL, pi.PERIODIC))
    gs = _abi.Grid()
    gs.nx, gs.ny, gs.nz, gs.h = grid.nx, grid.ny, grid.nz, grid.h
    for a in range(3):
        gs.bc[a] = grid.bc[a]
    stream = torch.cuda.current_stream()
    with paris.Context(grid) as ctx:
        for seed in (1, 2):  # two calls in a row with different inputs
            pr = pi.random_problem(grid, seed=seed)
            u, v, w = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (pr.u, pr.v, pr.w))
            ref, ref_mean = ctx.divergence(u, v, w, pr.dt)
            rhs = torch.full(grid.shape, float("nan"), dtype=torch.float64, device="cuda")
            mean = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            st = lib.paris_divergence_noalloc(ct.byref(gs), ct.c_void_p(u.data_ptr()),
                                              ct.c_void_p(v.data_ptr()), ct.c_void_p(w.data_ptr()),
                                              pr.dt, ct.c_void_p(rhs.data_ptr()),
                                              ct.c_void_p(mean.data_ptr()),
                                              ct.c_void_p(stream.cuda_stream))
            assert st == _abi.PARIS_OK
            torch.cuda.synchronize()
            r, a = rhs.cpu().numpy(), ref.cpu().numpy()
            scale = np.abs(a).max()
            np.testing.assert_allclose(r, a, rtol=0, atol=1e-14 * scale)
            assert abs(mean.item() - ref_mean) <= 1e-14 * scale


def test_noalloc_divergence_rejects_grids_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_11744_gb300 import _abi
    lib = _abi.load()
    gs = _abi.Grid()
    gs.nx, gs.ny, gs.nz, gs.h = 544, 256, 256, 1.0 / 256  # 17 x 32 x 32 blocks > 16384
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = ct.c_void_p(dummy.data_ptr())
    st = lib.paris_divergence_noalloc(ct.byref(gs), p, p, p, 1e-3, p, None,
                                      ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _abi.PARIS_ERR_INVALID_ARG
