"""The paper's comparison schemes on the GPU (teno_grid.scheme): TENO5 with a
fixed C_T = 1e-7 (Sec. 2, Sec. 4), TENO5-A (eq. 2.16-2.18) and WENO-Z
(tau_5 of eq. 2.12), through the same C-ABI entry points, against the oracle
run with the same scheme.

Tolerances as for the LAD path: 1e-12 relative max-norm on one RHS (flag
path and the benchmark's flag-free path), selections identical except
counted rounding-boundary flips, 1e-10 relative L1 after a run of steps."""
import numpy as np
import pytest

from paper_2003_09145_gb300 import inputs
from parity import RHS_RTOL, STEP_RTOL, compare_rhs, flux_scale, rel_l1_err, rel_max_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCHEMES = ["teno5", "teno5a", "wenoz"]


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_09145_gb300 import api as A
    return A


def _problems():
    return {
        "sod": inputs.shock_tube(200),
        "shu": inputs.shu_osher(4096),
        "rand2d": inputs.Problem("r2", inputs.random_discontinuous_state(2, (40, 30), seed=5), (40, 30),
                                 (0.02, 0.03), (1, 0), 0.0),
        "rand3d": inputs.Problem("r3", inputs.random_discontinuous_state(3, (12, 10, 9), seed=6), (12, 10, 9),
                                 (0.1, 0.1, 0.1), (0, 1, 0), 0.0),
        "quad128": inputs.riemann_2d(n=128),
        "turb32": inputs.solenoidal_turbulence(n=32),
    }


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("case", ["sod", "shu", "rand2d", "rand3d", "quad128", "turb32"])
def test_rhs_matches_oracle(api, oracle, scheme, case):
    P = _problems()[case]
    sch = api.Scheme(gamma=P.gamma, scheme=scheme, ct_m=7)
    params = oracle.Params(gamma=P.gamma, scheme=scheme, ct_m=7)
    grid = api.EulerGrid(P.n, P.dx, P.bc, sch)
    U = torch.from_numpy(np.ascontiguousarray(P.U0)).cuda()
    a, fl = api.rhs(grid, U, want_flags=True)
    b = api.rhs(grid, U, want_flags=False)
    torch.cuda.synchronize()
    a, fl, b = a.cpu().numpy(), fl.cpu().numpy(), b.cpu().numpy()
    fs = flux_scale(P.U0, P.n, P.dx, P.gamma)
    for R in (a, b):
        err, rep = compare_rhs(P.U0, P.n, P.dx, P.bc, R, fl, oracle, params)
        assert not rep.unexplained, rep.unexplained[:3]
        assert rep.mismatched <= rep.total * 1e-4
        assert err <= RHS_RTOL, err
    assert rel_max_err(b, a, fs) <= 1e-13
    m = fl >> 3
    if scheme == "teno5":
        assert np.all(m == 7)
    elif scheme == "teno5a":
        assert np.all((m >= 7) & (m <= 10))
    else:
        assert np.all(fl == 7)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_sod_run_matches_oracle(api, oracle, scheme):
    P = inputs.shock_tube(200)
    grid = api.EulerGrid(P.n, P.dx, P.bc, api.Scheme(scheme=scheme))
    U = torch.from_numpy(P.U0.copy()).cuda()
    solver = api.Solver(grid, cfl=P.cfl)
    solver.run(U, P.t_end)
    torch.cuda.synchronize()
    Uo, to, ko = oracle.euler_run(P.U0, P.n, P.dx, P.bc, P.t_end, sigma=P.cfl,
                                  params=oracle.Params(scheme=scheme))
    assert abs(solver.t.item() - P.t_end) <= 1e-14
    assert rel_l1_err(U.cpu().numpy(), Uo) <= STEP_RTOL


@pytest.mark.parametrize("scheme", SCHEMES)
def test_scalar_mode_matches_oracle(api, oracle, scheme):
    n = 200
    dx = 2.0 / n
    for u0 in (inputs.scalar_smooth(n), inputs.scalar_composite(n)):
        adv = api.ScalarAdvection(n, dx, mode="lad", scheme=api.Scheme(scheme=scheme))
        r = adv.rhs(torch.from_numpy(u0).cuda()).cpu().numpy()
        ro = oracle.scalar_rhs(u0, dx, "lad", oracle.Params(scheme=scheme))
        assert np.max(np.abs(r - ro)) <= RHS_RTOL * np.max(np.abs(u0)) / dx


@pytest.mark.parametrize("scheme", ["teno5", "teno5a"])
def test_adjoint_of_teno_variants(api, oracle, scheme):
    """The TENO cutoffs are piecewise constant, so the adjoint (selections
    frozen) applies to every TENO variant."""
    from oracle import grad
    U = inputs.random_discontinuous_state(2, (19, 13), seed=3)
    n, dx, bc = (19, 13), (0.1, 0.08), (0, 1)
    rng = np.random.default_rng(7)
    Rbar = rng.standard_normal(U.shape)
    ref, _ = grad.rhs_vjp(U, n, dx, bc, Rbar, oracle.Params(scheme=scheme))
    grid = api.EulerGrid(n, dx, bc, api.Scheme(scheme=scheme))
    got = api.rhs_adjoint(grid, torch.from_numpy(U).cuda(), torch.from_numpy(Rbar).cuda()).cpu().numpy()
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-10


def test_wenoz_adjoint_unsupported(api):
    from paper_2003_09145_gb300 import _lib
    grid = api.EulerGrid((16,), (0.1,), (1,), api.Scheme(scheme="wenoz"))
    U = torch.from_numpy(inputs.shock_tube(16).U0).cuda()
    with pytest.raises(RuntimeError, match="UNSUPPORTED"):
        api.rhs_adjoint(grid, U, torch.ones_like(U))


def test_teno5_fixed_equals_lad_with_one_magnitude(api):
    """TENO5 at C_T = 1e-7 and LAD with B_l = 7, B_u = 8 keep the same
    stencils everywhere (m differs only where tau_5 = 0, where both keep all),
    so the flag paths (binary64 selections everywhere) agree bit for bit."""
    P = inputs.riemann_2d(n=96)
    U = torch.from_numpy(P.U0).cuda()
    a, fa = api.rhs(api.EulerGrid(P.n, P.dx, P.bc, api.Scheme(scheme="teno5", ct_m=7)), U, want_flags=True)
    b, fb = api.rhs(api.EulerGrid(P.n, P.dx, P.bc, api.Scheme(b_l=7, b_u=8)), U, want_flags=True)
    assert torch.equal(a, b)
    assert torch.equal(fa & 7, fb & 7)
