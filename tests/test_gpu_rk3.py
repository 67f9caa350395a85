"""GPU parity of teno_rk3_step (SSP-RK3, eq. 4.1-4.3, CFL step eq. dt1/dt2) with the
oracle after a fixed number of steps: 1e-10 relative L1 per field, identical
step sizes."""
import numpy as np
import pytest

from paper_2003_09145_gb300 import inputs
from parity import STEP_RTOL, rel_l1_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_09145_gb300 import api as A
    return A


def _gpu_run(api, P, steps, t_end=None, dt_fixed=0.0):
    grid = api.EulerGrid(P.n, P.dx, P.bc, api.Scheme(gamma=P.gamma))
    solver = api.Solver(grid, cfl=P.cfl)
    U = torch.from_numpy(np.ascontiguousarray(P.U0)).cuda()
    dts = []
    te = P.t_end if t_end is None else t_end
    for _ in range(steps):
        solver.step(U, te, dt_fixed)
        dts.append(solver.dt.item())
    assert solver.status() == 0
    return U.cpu().numpy(), solver.t.item(), dts


def _oracle_run(oracle, P, steps, t_end=None, dt_fixed=0.0):
    U = np.array(P.U0)
    t = 0.0
    dts = []
    te = P.t_end if t_end is None else t_end
    for _ in range(steps):
        U, t2, k = oracle.euler_run(U, P.n, P.dx, P.bc, te, sigma=P.cfl, dt_fixed=dt_fixed,
                                    max_steps=1, t0=t, params=oracle.Params(gamma=P.gamma))
        dts.append(t2 - t if k else 0.0)
        t = t2
    return U, t, dts


@pytest.mark.parametrize("case,steps", [
    ("sod", 400),          # runs to t = 0.2 and past (steps beyond t_end are no-ops)
    ("shu_osher", 100),
    ("riemann2d", 20),
    ("turb3d", 6),
    ("smooth3d_aniso", 8),  # three different spacings: the ratios dx_0/dx_d differ from 1
])
def test_fixed_steps(api, oracle, case, steps):
    P = {"sod": lambda: inputs.shock_tube(200),
         "shu_osher": lambda: inputs.shu_osher(4096),
         "riemann2d": lambda: inputs.riemann_2d(n=128, t_end=10.0),
         "turb3d": lambda: inputs.solenoidal_turbulence(n=24, t_end=10.0),
         "smooth3d_aniso": lambda: inputs.Problem(
             "s3a", inputs.random_smooth_state(3, (14, 11, 9), seed=21, amp=0.03), (14, 11, 9),
             (0.1, 0.07, 0.13), (0, 1, 0), 10.0)}[case]()
    Ug, tg, dg = _gpu_run(api, P, steps)
    Uo, to, do = _oracle_run(oracle, P, steps)
    err = rel_l1_err(Ug, Uo)
    assert err <= STEP_RTOL, err
    # the step sizes agree to rounding
    np.testing.assert_allclose(dg, do, rtol=1e-12, atol=0)
    assert tg == pytest.approx(to, rel=1e-13)
    if case == "sod":
        assert tg == P.t_end


def test_first_dt(api, oracle):
    """The CFL step of eq. dt1 / dt2 (3D: harmonic form) from the device wave speeds."""
    for P in (inputs.shock_tube(200), inputs.riemann_2d(n=64), inputs.solenoidal_turbulence(n=16)):
        _, _, dg = _gpu_run(api, P, 1, t_end=100.0)
        dt_or = oracle.euler_dt(P.U0, P.n, P.dx, P.cfl, P.gamma)
        assert dg[0] == pytest.approx(dt_or, rel=1e-14)


def test_clip_and_no_op_after_t_end(api):
    P = inputs.shock_tube(64)
    grid = api.EulerGrid(P.n, P.dx, P.bc)
    solver = api.Solver(grid, cfl=0.5)
    U = torch.from_numpy(np.ascontiguousarray(P.U0)).cuda()
    t_end = 1e-4
    solver.step(U, t_end)
    assert solver.t.item() == t_end
    before = U.clone()
    solver.step(U, t_end)
    assert solver.dt.item() == 0.0
    assert torch.equal(before, U)
    assert solver.status() == 0


def test_no_op_first_step_reports_no_error(api):
    """A first step already at t_end (dt = 0) leaves U unchanged and raises
    no status: the stages that follow a skipped stage read U^n, not the
    uninitialised stage buffers of a fresh workspace."""
    P = inputs.shock_tube(64)
    grid = api.EulerGrid(P.n, P.dx, P.bc)
    solver = api.Solver(grid, cfl=0.5)
    U = torch.from_numpy(np.ascontiguousarray(P.U0)).cuda()
    before = U.clone()
    solver.step(U, 0.0)
    assert solver.dt.item() == 0.0
    assert torch.equal(before, U)
    assert solver.status() == 0


def test_nonphysical_state_is_reported(api):
    P = inputs.shock_tube(64)
    U0 = np.array(P.U0)
    U0[2, 10] = -1.0          # negative total energy -> negative pressure
    grid = api.EulerGrid(P.n, P.dx, P.bc)
    solver = api.Solver(grid)
    U = torch.from_numpy(U0).cuda()
    solver.step(U, 1.0, dt_fixed=1e-5)
    assert solver.status() == 4      # TENO_ERR_NONPHYSICAL
    assert solver.status() == 0      # cleared by the query


def test_host_pipeline_equals_one_item_at_a_time(api):
    """api.HostPipeline (copy-in, step and copy-out of neighbouring items
    overlapped on three streams) gives, for every item, the state one step of
    that item alone gives -- including items that repeat a host buffer."""
    P = inputs.solenoidal_turbulence(n=20, t_end=10.0)
    grid = api.EulerGrid(P.n, P.dx, P.bc)
    items = []
    for k in range(5):
        Uk = np.array(P.U0)
        Uk[0] *= 1.0 + 0.01 * k
        items.append(torch.from_numpy(np.ascontiguousarray(Uk)).pin_memory())
    host_in = items + [items[1]]
    host_out = [torch.empty_like(h).pin_memory() for h in host_in]
    solver = api.Solver(grid)
    pipe = api.HostPipeline(solver, torch.from_numpy(P.U0))
    pipe.run(host_in, host_out)
    torch.cuda.synchronize()
    for hi, ho in zip(host_in, host_out):
        U = hi.cuda()
        api.Solver(grid).step(U)
        assert torch.equal(U.cpu(), ho)


def _full_grid_steps(api, oracle, P, steps):
    """`steps` CFL steps of the whole grid on the GPU (the benchmark's
    flag-free path: certified closed form plus pending pass) and in the oracle
    (one call, all host cores)."""
    Ug, tg, dg = _gpu_run(api, P, steps)
    Uo, to, k = oracle.euler_run(P.U0, P.n, P.dx, P.bc, P.t_end, sigma=P.cfl, max_steps=steps,
                                 params=oracle.Params(gamma=P.gamma))
    assert k == steps
    assert tg == pytest.approx(to, rel=1e-13)
    err = rel_l1_err(Ug, Uo)
    assert err <= STEP_RTOL, err
    return err


@pytest.mark.slow
def test_four_quadrant_2048_twenty_steps_full_grid(api, oracle):
    """The 2D four-quadrant configuration at its benchmark size, 20 RK3
    steps, every cell against the oracle (eq. 4.1-4.3, eq. dt2)."""
    _full_grid_steps(api, oracle, inputs.riemann_2d(n=2048, t_end=10.0), 20)


@pytest.mark.slow
def test_turbulence_256_two_steps_full_grid(api, oracle):
    """The 3D turbulence box at the benchmark's size and launch configuration
    (api.Solver, the flag-free two-pass flux evaluation), 2 RK3 steps, every
    cell against the oracle."""
    _full_grid_steps(api, oracle, inputs.solenoidal_turbulence(n=256, t_end=10.0), 2)
