"""The paper's other test problems on the same kernels (Sec. 4.2 and 4.3.1):
Sod's and Lax's tubes at the paper's size and time (eq. 4.8, 4.9), and
configurations 3 and 12 of the 2D Riemann family (eq. 4.14, 4.13), against
the oracle and, in 1D, the exact Riemann solution."""
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


def _gpu_to_end(api, P, max_steps=1 << 20):
    grid = api.EulerGrid(P.n, P.dx, P.bc, api.Scheme(gamma=P.gamma))
    solver = api.Solver(grid, cfl=P.cfl)
    U = torch.from_numpy(np.ascontiguousarray(P.U0)).cuda()
    steps = solver.run(U, P.t_end, max_steps=max_steps, chunk=32)
    assert solver.status() == 0
    return U.cpu().numpy(), solver.t.item(), steps


def _exact_rel_l1(oracle, P, rho):
    x = P.centers(0)
    ex = oracle.riemann_sample(P.extra["left"], P.extra["right"], (x - P.extra["x_jump"]) / P.t_end)
    mean = np.mean(np.abs(ex[0]))
    return np.mean(np.abs(rho - ex[0])) / mean, (ex[0].max() - ex[0].min()) / mean


@pytest.mark.parametrize("make", [inputs.sod_paper, inputs.lax_tube], ids=["sod_paper", "lax"])
def test_tube_to_the_paper_time(api, oracle, make):
    """N = 400 to the paper's final time: equal to the oracle's run, and within a
    few cells of smearing of the exact solution."""
    P = make(400)
    Ug, t, steps = _gpu_to_end(api, P)
    assert t == P.t_end
    Uo, to, k = oracle.euler_run(np.array(P.U0), P.n, P.dx, P.bc, P.t_end, sigma=P.cfl)
    assert to == pytest.approx(P.t_end, rel=1e-14)
    assert rel_l1_err(Ug, Uo) <= STEP_RTOL
    err, jump = _exact_rel_l1(oracle, P, Ug[0])
    assert err * P.n[0] <= 4.0 * jump, (err, jump)


@pytest.mark.parametrize("make", [inputs.sod_paper, inputs.lax_tube], ids=["sod_paper", "lax"])
def test_tube_converges_to_the_exact_solution(api, oracle, make):
    errs = []
    for n in (200, 400, 800, 1600):
        P = make(n)
        Ug, _, _ = _gpu_to_end(api, P)
        errs.append(_exact_rel_l1(oracle, P, Ug[0])[0])
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < errs[0] / 2.5, errs


@pytest.mark.parametrize("make", [inputs.riemann_2d_config3, inputs.riemann_2d_config12],
                         ids=["config3", "config12"])
def test_2d_riemann_one_rhs_at_paper_size(api, oracle, make):
    """One right-hand side on the paper's 1024^2 grid, both GPU paths, full grid."""
    P = make(1024)
    grid = api.EulerGrid(P.n, P.dx, P.bc)
    U = torch.from_numpy(np.ascontiguousarray(P.U0)).cuda()
    a, fl = api.rhs(grid, U, want_flags=True)
    b = api.rhs(grid, U, want_flags=False)
    torch.cuda.synchronize()
    a, fl, b = a.cpu().numpy(), fl.cpu().numpy(), b.cpu().numpy()
    err, rep = compare_rhs(P.U0, P.n, P.dx, P.bc, b, fl, oracle)
    assert not rep.unexplained
    assert err <= RHS_RTOL, err
    assert rel_max_err(b, a, flux_scale(P.U0, P.n, P.dx)) <= 1e-13


@pytest.mark.parametrize("make", [inputs.riemann_2d_config3, inputs.riemann_2d_config12],
                         ids=["config3", "config12"])
def test_2d_riemann_steps(api, oracle, make):
    """30 CFL steps on 192^2 against the oracle; the data are symmetric under
    (x, y, u, v) -> (y, x, v, u), and so is the GPU solution, to rounding (its
    sums over velocity components run in x, y order in both sweeps, so mirrored
    interfaces round differently)."""
    P = make(192)
    grid = api.EulerGrid(P.n, P.dx, P.bc)
    solver = api.Solver(grid, cfl=P.cfl)
    U = torch.from_numpy(np.ascontiguousarray(P.U0)).cuda()
    for _ in range(30):
        solver.step(U, P.t_end)
    assert solver.status() == 0
    Ug = U.cpu().numpy()
    Uo, to, k = oracle.euler_run(np.array(P.U0), P.n, P.dx, P.bc, P.t_end, sigma=P.cfl, max_steps=30)
    assert k == 30
    assert rel_l1_err(Ug, Uo) <= STEP_RTOL
    assert solver.t.item() == pytest.approx(to, rel=1e-13)
    # transpose symmetry: rho and E symmetric, (rho u, rho v) swapped
    for a, b in ((Ug[0], Ug[0].T), (Ug[3], Ug[3].T), (Ug[1], Ug[2].T)):
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))
