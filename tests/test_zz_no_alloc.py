"""teno_rhs_noalloc: the right-hand side for callers that cannot allocate device
memory (plugins inside another framework's memory pool, hosts that forbid
cudaMalloc on their threads, fixed-footprint deployments).  It takes only the
input and output arrays and uses a fixed device array inside the library as its
scratch.  Its results must equal teno_rhs's, call after call: the scratch array
keeps the previous call's contents, so a second call on different data checks
that everything that must start from zero is cleared.

This file is collected last on purpose (a failure here leaves every other test
already run)."""
import ctypes

import numpy as np
import pytest

from paper_2003_09145_gb300 import inputs
from parity import RHS_RTOL, flux_scale, rel_max_err

torch = pytest.importorskip("torch")

TENO_ERR_WORKSPACE = 6


def _lib():
    from paper_2003_09145_gb300 import _lib
    return _lib, _lib.load()


def _noalloc(L, lib, grid, U):
    out = torch.empty_like(U)
    st = lib.teno_rhs_noalloc(ctypes.byref(grid.c), ctypes.c_void_p(U.data_ptr()),
                              ctypes.c_void_p(out.data_ptr()),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    L.check(st, "teno_rhs_noalloc")
    return out


@pytest.mark.gpu
def test_noalloc_matches_teno_rhs_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_09145_gb300 import api
    L, lib = _lib()
    n = (48, 40)
    # call 1: fast flow (large LF speeds); call 2: slow flow on the same grid, so
    # stale wave-speed maxima from call 1 would change call 2's result
    rng = np.random.default_rng(1)
    shape = tuple(reversed(n))
    fast = inputs.prim_to_cons(rng.uniform(0.5, 2.0, shape),
                               [rng.uniform(-4.0, 4.0, shape), rng.uniform(-4.0, 4.0, shape)],
                               rng.uniform(0.5, 5.0, shape))
    slow = inputs.random_smooth_state(2, n, seed=2, amp=0.02)
    grid = api.EulerGrid(n, (0.02, 0.025), (1, 0))
    for U0 in (fast, slow, inputs.riemann_2d(n=48, ny=40).U0):
        U = torch.from_numpy(np.ascontiguousarray(U0)).cuda()
        ref = api.rhs(grid, U)
        got = _noalloc(L, lib, grid, U)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert rel_max_err(g, r, flux_scale(U0, n, grid.dx)) <= RHS_RTOL
    # a 1D grid after the 2D ones (different scratch layout)
    P = inputs.shu_osher(4096)
    g1 = api.EulerGrid(P.n, P.dx, P.bc)
    U = torch.from_numpy(P.U0).cuda()
    for _ in range(2):
        ref = api.rhs(g1, U)
        got = _noalloc(L, lib, g1, U)
        torch.cuda.synchronize()
        assert rel_max_err(got.cpu().numpy(), ref.cpu().numpy(), flux_scale(P.U0, P.n, P.dx)) <= RHS_RTOL


def test_noalloc_rejects_grids_beyond_its_scratch():
    L, lib = _lib()
    too_big = L.make_grid((200000,), (1e-5,), 1)        # 1D limit is 131,065 cells
    # aligned non-null stand-ins: the size check fails before any pointer is used
    st = lib.teno_rhs_noalloc(ctypes.byref(too_big), ctypes.c_void_p(256), ctypes.c_void_p(512), None)
    assert st == TENO_ERR_WORKSPACE
    cube = L.make_grid((43, 43, 43), (0.1,) * 3, 0)      # 3D limit is 42^3
    st = lib.teno_rhs_noalloc(ctypes.byref(cube), ctypes.c_void_p(256), ctypes.c_void_p(512), None)
    assert st == TENO_ERR_WORKSPACE
