"""Reflecting walls (bc 2) on the GPU: the two interacting blast waves of
Sec. 4.2 (eq. 4.11) and 2D / 3D / narrow-grid cases against the oracle, and
the mirror identity (reflecting = the doubled periodic domain at rest)."""
import numpy as np
import pytest

from paper_2003_09145_gb300 import inputs
from parity import RHS_RTOL, STEP_RTOL, compare_rhs, flux_scale, rel_l1_err, rel_max_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_09145_gb300 import api as A
    return A


def _both_paths(api, P):
    grid = api.EulerGrid(P.n, P.dx, P.bc)
    U = torch.from_numpy(np.ascontiguousarray(P.U0)).cuda()
    a, fl = api.rhs(grid, U, want_flags=True)
    b = api.rhs(grid, U, want_flags=False)
    torch.cuda.synchronize()
    return a.cpu().numpy(), fl.cpu().numpy(), b.cpu().numpy()


def _check_rhs(api, oracle, P):
    a, fl, b = _both_paths(api, P)
    err, rep = compare_rhs(P.U0, P.n, P.dx, P.bc, b, fl, oracle)
    assert not rep.unexplained
    assert err <= RHS_RTOL, err
    assert rel_max_err(b, a, flux_scale(P.U0, P.n, P.dx)) <= 1e-13


def _box_blast(n, bc):
    """2D box with a pressure disc (at rest, then moving) and reflecting walls."""
    nx, ny = n
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y, indexing="xy")
    r2 = (X - 0.3) ** 2 + (Y - 0.6) ** 2
    p = np.where(r2 < 0.04, 10.0, 0.1)
    rho = 1.0 + 0.2 * np.sin(4.0 * X) * np.cos(3.0 * Y)
    U = inputs.prim_to_cons(rho, [0.3 * np.cos(2.0 * Y), -0.2 * np.sin(5.0 * X)], p)
    return inputs.Problem("box", U, (nx, ny), (1.0 / nx, 1.0 / ny), bc, 1.0)


def test_blast_waves_one_rhs(api, oracle):
    _check_rhs(api, oracle, inputs.blast_waves(400))


def test_reflecting_equals_doubled_periodic_at_rest(api):
    """At rest the LF speeds of the data and of its mirror image agree, and
    every stencil sees the same values, so the two right-hand sides are equal."""
    P = inputs.blast_waves(120)
    n = P.n[0]
    U = P.U0 * np.array([[1.0], [1.0], [1.0]])
    U[2] *= 1.0 + 0.1 * np.sin(7.0 * (np.arange(n) + 0.5) / n)
    Ud = np.ascontiguousarray(np.concatenate([U[:, ::-1] * np.array([[1.0], [-1.0], [1.0]]), U], axis=1))
    R = api.rhs(api.EulerGrid((n,), P.dx, (2,)), torch.from_numpy(np.ascontiguousarray(U)).cuda())
    Rd = api.rhs(api.EulerGrid((2 * n,), P.dx, (0,)), torch.from_numpy(Ud).cuda())
    np.testing.assert_array_equal(R.cpu().numpy(), Rd.cpu().numpy()[:, n:])


def test_blast_waves_first_steps(api, oracle):
    """N = 400, 20 CFL steps (t = 4.9e-4): the oracle's run, step for step."""
    P = inputs.blast_waves(400)
    grid = api.EulerGrid(P.n, P.dx, P.bc)
    solver = api.Solver(grid, cfl=P.cfl)
    U = torch.from_numpy(np.ascontiguousarray(P.U0)).cuda()
    for _ in range(20):
        solver.step(U, P.t_end)
    assert solver.status() == 0
    Uo, to, k = oracle.euler_run(np.array(P.U0), P.n, P.dx, P.bc, P.t_end, sigma=P.cfl, max_steps=20)
    assert k == 20 and solver.t.item() == pytest.approx(to, rel=1e-13)
    assert rel_l1_err(U.cpu().numpy(), Uo) <= STEP_RTOL


def test_blast_waves_negative_pressure_is_reported_at_the_oracles_step(api, oracle):
    """With the readings of the eigensystem (Roe average) and of the splitting
    (global LF per characteristic field), the scheme meets a negative pressure
    ahead of the right-moving blast (p there falls to 0.01 against 1000 behind
    it) -- in the oracle as on the GPU, at any CFL, and with one LF speed for
    all fields as well; the method has no positivity limiter.  The GPU's status
    word reports it at the step where the oracle first meets it."""
    P = inputs.blast_waves(400)
    V, t, first_oracle = np.array(P.U0), 0.0, None
    for s in range(60):
        V, t, k, nbad = oracle.euler_run_ex(V, P.n, P.dx, P.bc, P.t_end, sigma=P.cfl, max_steps=1, t0=t)
        if nbad:
            first_oracle = s
            break
    assert first_oracle is not None
    grid = api.EulerGrid(P.n, P.dx, P.bc)
    solver = api.Solver(grid, cfl=P.cfl)
    U = torch.from_numpy(np.ascontiguousarray(P.U0)).cuda()
    first_gpu = None
    for s in range(first_oracle + 1):
        solver.step(U, P.t_end)
        if solver.status() == 4:      # TENO_ERR_NONPHYSICAL
            first_gpu = s
            break
    assert first_gpu == first_oracle


@pytest.mark.parametrize("bc", [(2, 2), (2, 0), (1, 2)])
def test_2d_reflecting_rhs_and_steps(api, oracle, bc):
    P = _box_blast((48, 40), bc)
    _check_rhs(api, oracle, P)
    grid = api.EulerGrid(P.n, P.dx, P.bc)
    solver = api.Solver(grid, cfl=0.5)
    U = torch.from_numpy(np.ascontiguousarray(P.U0)).cuda()
    for _ in range(15):
        solver.step(U, 1.0)
    assert solver.status() == 0
    Uo, to, k = oracle.euler_run(np.array(P.U0), P.n, P.dx, P.bc, 1.0, sigma=0.5, max_steps=15)
    assert rel_l1_err(U.cpu().numpy(), Uo) <= STEP_RTOL


@pytest.mark.parametrize("n", [(9, 7, 11), (12, 2, 5), (1, 6, 3)])
def test_3d_and_narrow_reflecting(api, oracle, n):
    """All walls reflecting in 3D, including axes narrower than the stencil
    (a point is reflected more than once)."""
    U = inputs.random_smooth_state(3, n, seed=31, amp=0.2)
    P = inputs.Problem("r3", U, n, (0.1, 0.12, 0.09), (2, 2, 2), 1.0)
    _check_rhs(api, oracle, P)
