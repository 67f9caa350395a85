"""Sec. 4.3.2's Rayleigh-Taylor problem on the GPU: fixed-state top and bottom
faces (TENO_BC_DIRICHLET), reflecting side walls and the body-force source
(0, rho g, rho u.g) with g = (0, 1), through teno_rhs / teno_rk3_step, against
the oracle at 1e-12 (one RHS, flag path and the benchmark's flag-free path)
and 1e-10 relative L1 after 20 steps; hydrostatic balance on the GPU."""
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


def _params(oracle, P, scheme="lad"):
    st = np.zeros((3, 2, 5))
    for k, faces in enumerate(P.extra["bc_state"]):
        if faces is not None:
            for side in range(2):
                st[k, side, :len(faces[side])] = faces[side]
    return oracle.Params(gamma=P.gamma, grav=tuple(P.extra["grav"]) + (0.0,), bc_state=st, scheme=scheme)


def _grid(api, P, scheme="lad"):
    return api.EulerGrid(P.n, P.dx, P.bc, api.Scheme(gamma=P.gamma, scheme=scheme), grav=P.extra["grav"],
                         bc_state=P.extra["bc_state"])


@pytest.mark.parametrize("n", [(16, 64), (64, 256), (13, 47)])
@pytest.mark.parametrize("scheme", ["lad", "teno5a"])
def test_rt_rhs_matches_oracle(api, oracle, n, scheme):
    P = inputs.rayleigh_taylor(*n)
    grid = _grid(api, P, scheme)
    U = torch.from_numpy(np.ascontiguousarray(P.U0)).cuda()
    a, fl = api.rhs(grid, U, want_flags=True)
    b = api.rhs(grid, U, want_flags=False)
    torch.cuda.synchronize()
    a, fl, b = a.cpu().numpy(), fl.cpu().numpy(), b.cpu().numpy()
    prm = _params(oracle, P, scheme)
    for R in (a, b):
        err, rep = compare_rhs(P.U0, P.n, P.dx, P.bc, R, fl, oracle, prm)
        assert not rep.unexplained, rep.unexplained[:3]
        assert err <= RHS_RTOL, err
    assert rel_max_err(b, a, flux_scale(P.U0, P.n, P.dx, P.gamma)) <= 1e-13


def test_rt_steps_match_oracle(api, oracle):
    P = inputs.rayleigh_taylor(32, 128)
    grid = _grid(api, P)
    solver = api.Solver(grid, cfl=P.cfl)
    U = torch.from_numpy(P.U0.copy()).cuda()
    for _ in range(20):
        solver.step(U)
    torch.cuda.synchronize()
    assert solver.status() == 0
    Uo, to, k = oracle.euler_run(P.U0, P.n, P.dx, P.bc, float("inf"), sigma=P.cfl, max_steps=20,
                                 params=_params(oracle, P))
    assert k == 20 and solver.t.item() == pytest.approx(to, rel=1e-13)
    assert rel_l1_err(U.cpu().numpy(), Uo) <= STEP_RTOL


def test_rt_hydrostatic_balance(api):
    P = inputs.rayleigh_taylor(8, 64, perturb=False)
    R = api.rhs(_grid(api, P), torch.from_numpy(P.U0).cuda()).cpu().numpy().reshape(4, 64, 8)
    rows = [j for j in range(64) if 3 <= j < 29 or 35 <= j < 61]
    assert np.max(np.abs(R[:, rows])) <= 1e-12 * 3.0 / P.dx[1]


def test_fixed_state_validation(api):
    from paper_2003_09145_gb300 import _lib
    P = inputs.rayleigh_taylor(8, 32)
    st = [None, [[2.0, 0.0, 0.0, -1.0], [1.0, 0.0, 0.0, 3.75]]]     # negative energy: no pressure
    grid = api.EulerGrid(P.n, P.dx, P.bc, api.Scheme(gamma=P.gamma), grav=(0.0, 1.0), bc_state=st)
    with pytest.raises(ValueError):
        grid.workspace_bytes(_lib.OP_RHS)
    ok = _grid(api, P)
    U = torch.from_numpy(P.U0).cuda()
    with pytest.raises(RuntimeError, match="UNSUPPORTED"):
        api.rhs_adjoint(ok, U, torch.ones_like(U))
