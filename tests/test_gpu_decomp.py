"""Decomposed stepping on the GPU: the staged entry points (teno_rk3_stage_begin
/ _end) reproduce teno_rk3_step, and a grid split into slabs along its slowest
axis -- ghost planes exchanged with teno_planes_copy before every stage, the
Lax-Friedrichs speed words combined by their maximum -- advances every slab's
interior exactly as the undivided grid (eq. 4.1-4.3; Sec. 4's global LF
splitting, reading C7).  Several slabs live on the one GPU here, standing in
for ranks; tests/test_decomp_ranks.py drives the same orchestration over
gloo ranks on CPU."""
import numpy as np
import pytest

from paper_2003_09145_gb300 import decomp, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_09145_gb300 import api as A
    return A


def _problem(name):
    if name == "3d-periodic":
        P = inputs.solenoidal_turbulence(n=24)
        return P.U0, P.n, P.dx, P.bc
    if name == "2d-transmissive":
        P = inputs.riemann_2d(n=48)
        return P.U0, P.n, P.dx, P.bc
    if name == "3d-mixed":
        n = (10, 9, 16)
        return inputs.random_discontinuous_state(3, n, seed=12), n, (0.1, 0.1, 0.1), (0, 1, 1)
    P = inputs.shock_tube(200)
    return P.U0, P.n, P.dx, P.bc


def test_staged_step_equals_rk3_step(api):
    U0, n, dx, bc = _problem("3d-mixed")
    grid = api.EulerGrid(n, dx, bc)
    ref = torch.from_numpy(U0).cuda()
    solver = api.Solver(grid)
    eng = api.SlabEngine(grid)
    U = ref.clone()
    U1, U2 = torch.empty_like(U), torch.empty_like(U)
    for _ in range(4):
        solver.step(ref)
        for k, (Uin, Uout) in enumerate(((U, U1), (U1, U2), (U2, U)), start=1):
            eng.begin(Uin)
            eng.end(k, Uin, U, Uout)
    torch.cuda.synchronize()
    assert torch.equal(U, ref)
    assert eng.t.item() == solver.t.item()


@pytest.mark.parametrize("name,nslab,steps", [("3d-periodic", 2, 5), ("3d-periodic", 3, 3),
                                              ("2d-transmissive", 3, 5), ("3d-mixed", 4, 3),
                                              ("1d", 2, 6)])
def test_slabs_equal_undivided(api, name, nslab, steps):
    U0, n, dx, bc = _problem(name)
    grid = api.EulerGrid(n, dx, bc)
    ax = grid.ndim - 1
    Ug = torch.from_numpy(U0).cuda()
    ref = Ug.clone()
    solver = api.Solver(grid)
    dts = []
    for _ in range(steps):
        solver.step(ref)
        dts.append(solver.dt.item())
    plans = [decomp.SlabPlan(n[ax], nslab, r, periodic=(bc[ax] == 0)) for r in range(nslab)]
    engines = [api.SlabEngine(api.slab_grid(grid, p)) for p in plans]
    Us = [api.slab_from_global(Ug, grid, p) for p in plans]
    U1s = [torch.empty_like(u) for u in Us]
    U2s = [torch.empty_like(u) for u in Us]
    group = decomp.LocalGroup(engines, plans, lambda ws: torch.stack(ws).amax(dim=0))
    for k in range(steps):
        group.step(Us, U1s, U2s)
        assert all(e.dt.item() == dts[k] for e in engines)
    torch.cuda.synchronize()
    shape = (grid.nvar,) + tuple(reversed(n))
    R = ref.reshape(shape)
    for p, u in zip(plans, Us):
        assert torch.equal(api.slab_interior(u, grid, p), R[:, p.start:p.start + p.count])
    assert all(e.status() == 0 for e in engines)


def test_planes_copy_validation(api):
    from paper_2003_09145_gb300 import _lib
    import ctypes
    grid = api.EulerGrid((8, 6), (0.1, 0.1), (1, 1))
    U = torch.zeros(4 * 48, dtype=torch.float64, device="cuda")
    lib = grid.lib
    c = ctypes.byref(grid.c)
    p = ctypes.c_void_p(U.data_ptr())
    assert lib.teno_planes_copy(c, p, 4, 0, p, 0, 0, 3, None) == 1      # beyond the last plane
    assert lib.teno_planes_copy(c, p, 0, 0, p, 4, 0, 2, None) == 0
    host = np.zeros(4 * 48)
    assert lib.teno_planes_copy(c, ctypes.c_void_p(host.ctypes.data), 0, 0, p, 0, 0, 1, None) == 1
    bad = ctypes.c_void_p(U.data_ptr())
    assert lib.teno_rk3_stage_end(c, 4, bad, bad, bad, 0.5, 0.0, bad, 1.0, None, bad, 0, None) == 1
