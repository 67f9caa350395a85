"""GPU adjoint (teno_rhs_adjoint, teno_rk3_step_adjoint, TenoRK3Rollout) against
the reverse-mode gradient oracle (oracle/grad.py) and central differences."""
import math

import numpy as np
import pytest

from paper_2003_09145_gb300 import inputs
from parity import rel_l1_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ADJ_RTOL = 1e-10


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_09145_gb300 import api as A
    return A


def _jit(U, s):
    rng = np.random.default_rng(s)
    return np.ascontiguousarray(U * (1.0 + 1e-3 * rng.standard_normal(U.shape)))


def _cases():
    return [
        ("1d-trans", inputs.random_discontinuous_state(1, (57,), seed=1), (57,), (0.02,), (1,)),
        ("1d-per", _jit(inputs.random_smooth_state(1, (40,), seed=2), 1), (40,), (0.05,), (0,)),
        ("1d-tiny", inputs.random_discontinuous_state(1, (3,), seed=9), (3,), (0.3,), (1,)),
        ("2d-mixed", inputs.random_discontinuous_state(2, (19, 13), seed=3), (19, 13), (0.1, 0.08), (0, 1)),
        ("3d-per", _jit(inputs.random_smooth_state(3, (9, 7, 6), seed=4), 2), (9, 7, 6), (0.2, 0.2, 0.25), (0, 0, 0)),
        ("3d-trans", inputs.random_discontinuous_state(3, (8, 6, 7), seed=5), (8, 6, 7), (0.1, 0.1, 0.1), (1, 1, 1)),
        ("turb16", inputs.solenoidal_turbulence(n=16).U0, (16, 16, 16), (2 * math.pi / 16,) * 3, (0, 0, 0)),
        # periodic lines shorter than the six-point stencil (the gather's slot-by-slot path)
        ("1d-per-2", inputs.random_discontinuous_state(1, (2,), seed=13), (2,), (0.1,), (0,)),
        ("2d-short-per", inputs.random_discontinuous_state(2, (5, 4), seed=10), (5, 4), (0.1, 0.1), (0, 0)),
        ("3d-short-mixed", inputs.random_discontinuous_state(3, (7, 4, 5), seed=11), (7, 4, 5), (0.1, 0.1, 0.1),
         (0, 1, 0)),
    ]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_rhs_adjoint_matches_oracle_gradient(api, oracle, case):
    from oracle import grad
    _, U, n, dx, bc = case
    rng = np.random.default_rng(7)
    Rbar = rng.standard_normal(U.shape)
    ref, _ = grad.rhs_vjp(U, n, dx, bc, Rbar)
    grid = api.EulerGrid(n, dx, bc)
    Ut = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    got = api.rhs_adjoint(grid, Ut, torch.from_numpy(Rbar).cuda()).cpu().numpy()
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err <= ADJ_RTOL, err


def test_rhs_adjoint_accumulates_and_is_deterministic(api):
    U = inputs.random_discontinuous_state(2, (21, 17), seed=8)
    grid = api.EulerGrid((21, 17), (0.1, 0.1), (1, 0))
    Ut = torch.from_numpy(U).cuda()
    Rb = torch.randn(Ut.shape, dtype=torch.float64, device="cuda")
    a = api.rhs_adjoint(grid, Ut, Rb)
    b = api.rhs_adjoint(grid, Ut, Rb)
    assert torch.equal(a, b)
    base = torch.full_like(Ut, 0.5)
    c = api.rhs_adjoint(grid, Ut, Rb, U_bar=base.clone())
    assert torch.allclose(c, a + 0.5, rtol=0, atol=1e-12 * a.abs().max().item())


def test_dot_product_identity_with_central_differences(api):
    """<J^T v, w> = <v, J w>, J w by central differences of the GPU RHS; the state is
    the first of a few seeded smooth states whose selections do not change under
    the +-h perturbation (a selector flip makes the difference quotient meaningless)."""
    n, dx, bc = (12, 10, 8), (0.1, 0.1, 0.1), (0, 0, 0)
    grid = api.EulerGrid(n, dx, bc)
    h = 1e-6
    for seed in range(6):
        U = _jit(inputs.random_smooth_state(3, n, seed=seed, amp=0.03), seed + 10)
        rng = np.random.default_rng(seed)
        v = torch.from_numpy(rng.standard_normal(U.shape)).cuda()
        w = torch.from_numpy(rng.standard_normal(U.shape) * np.abs(U)).cuda()
        Ut = torch.from_numpy(U).cuda()
        Rp, fp = api.rhs(grid, Ut + h * w, want_flags=True)
        Rm, fm = api.rhs(grid, Ut - h * w, want_flags=True)
        _, f0 = api.rhs(grid, Ut, want_flags=True)
        if torch.equal(fp & 7, f0 & 7) and torch.equal(fm & 7, f0 & 7):
            break
    else:
        pytest.fail("no seeded state with stable selections")
    lhs = float((api.rhs_adjoint(grid, Ut, v) * w).sum())
    rhs_ = float((v * (Rp - Rm)).sum()) / (2 * h)
    assert lhs == pytest.approx(rhs_, rel=1e-6)


def test_rk3_step_adjoint_matches_oracle(api, oracle):
    from oracle import grad
    U = _jit(inputs.random_smooth_state(2, (12, 10), seed=5), 3)
    n, dx, bc = (12, 10), (0.1, 0.12), (0, 1)
    dt = 0.01
    rng = np.random.default_rng(4)
    Bnext = rng.standard_normal(U.shape)
    Ut = torch.from_numpy(U).requires_grad_(True)
    out = grad.rk3_rollout(Ut, n, dx, bc, dt, 1)
    (ref,) = torch.autograd.grad(out, Ut, torch.from_numpy(Bnext).reshape(out.shape))
    grid = api.EulerGrid(n, dx, bc)
    adj = api.AdjointStepper(grid)
    got = adj.step(torch.from_numpy(U).cuda(), dt, torch.from_numpy(Bnext).cuda()).cpu().numpy()
    err = np.max(np.abs(got - ref.numpy())) / np.max(np.abs(ref.numpy()))
    assert err <= ADJ_RTOL, err


def test_turbulence_16_rollout_gradient(api, oracle):
    """The adjoint workload at 16^3: loss = 1/2 |rho_40 - rho_target|^2 after 40
    fixed-dt RK3 steps (dt from U0 at CFL 0.5); gradient w.r.t. U0 from the GPU
    rollout adjoint against the oracle's reverse mode."""
    from oracle import grad
    P = inputs.solenoidal_turbulence(n=16)
    dt = oracle.euler_dt(P.U0, P.n, P.dx, 0.5)
    grid = api.EulerGrid(P.n, P.dx, P.bc)
    U0 = torch.from_numpy(P.U0).cuda().requires_grad_(True)
    out = api.rollout(U0, grid, 40, dt, checkpoint_every=6)
    target = torch.from_numpy(inputs.perturbed_target(P.U0[0], seed=2)).cuda()
    loss = 0.5 * ((out[0] - target) ** 2).sum()
    loss.backward()
    g_gpu = U0.grad.cpu().numpy()
    Ut = torch.from_numpy(P.U0).requires_grad_(True)
    o = grad.rk3_rollout(Ut, P.n, P.dx, P.bc, dt, 40)
    lo = 0.5 * ((o[0] - torch.from_numpy(inputs.perturbed_target(P.U0[0], seed=2))) ** 2).sum()
    (g_or,) = torch.autograd.grad(lo, Ut)
    g_or = g_or.numpy()
    assert float(loss.detach()) == pytest.approx(float(lo.detach()), rel=1e-10)
    rel_l2 = np.linalg.norm(g_gpu - g_or) / np.linalg.norm(g_or)
    assert rel_l2 <= ADJ_RTOL, rel_l2


@pytest.mark.parametrize("name", ["2d-mixed", "3d-per", "turb16"])
def test_staged_step_adjoint_equals_recomputed(api, name):
    """teno_rk3_step_adjoint_staged with the stages the staged forward entry
    points wrote (fixed dt) gives teno_rk3_step_adjoint's result bit for bit:
    the stages are the ones the latter recomputes."""
    _, U, n, dx, bc = next(c for c in _cases() if c[0] == name)
    grid = api.EulerGrid(n, dx, bc)
    Ut = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    Rb = torch.from_numpy(np.random.default_rng(21).standard_normal(U.shape)).cuda()
    dt = 0.1 * min(dx)
    adj = api.AdjointStepper(grid)
    eng = api.SlabEngine(grid)
    U1, U2, Un1 = api.rk3_step_stages(eng, Ut, dt)
    ref = Ut.clone()
    api.Solver(grid).step(ref, float("inf"), dt_fixed=dt)
    assert torch.equal(Un1, ref)
    a = adj.step(Ut, dt, Rb)
    b = adj.step(Ut, dt, Rb, stages=(U1, U2))
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert adj.status() == 0


def test_rollout_gradient_same_with_kept_stages(api, oracle):
    """The rollout's backward with kept stages and with recomputed ones gives
    the same gradient bit for bit (16^3 turbulence box, 12 steps at CFL 0.5,
    segments of 5)."""
    P = inputs.solenoidal_turbulence(n=16)
    grid = api.EulerGrid(P.n, P.dx, P.bc)
    dt = oracle.euler_dt(P.U0, P.n, P.dx, 0.5)
    grads = []
    for keep in (True, False):
        U0 = torch.from_numpy(P.U0).cuda().requires_grad_(True)
        out = api.rollout(U0, grid, 12, dt, checkpoint_every=5, keep_stages=keep)
        (0.5 * (out ** 2).sum()).backward()
        grads.append(U0.grad.clone())
    assert torch.equal(grads[0], grads[1])


def test_staged_step_adjoint_argument_checks(api):
    from paper_2003_09145_gb300 import _lib
    import ctypes
    grid = api.EulerGrid((12, 10), (0.1, 0.1), (0, 1))
    U = torch.ones(4 * 120, dtype=torch.float64, device="cuda")
    B = torch.zeros_like(U)
    adj = api.AdjointStepper(grid)
    c = ctypes.byref(grid.c)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    ws, nb = p(adj.ws), adj.ws.numel()
    # Ubar_n may not alias a stage input; dt must be finite and >= 0
    assert grid.lib.teno_rk3_step_adjoint_staged(c, p(U), p(U), p(U), 0.01, p(B), p(U), ws, nb, None) == 1
    assert grid.lib.teno_rk3_step_adjoint_staged(c, p(U), p(U), p(U), float("nan"), p(B), p(B), ws, nb, None) == 1
    assert grid.lib.teno_rk3_step_adjoint_staged(c, p(U), None, p(U), 0.01, p(B), p(B), ws, nb, None) == 1
    assert grid.lib.teno_rk3_step_adjoint_staged(c, p(U), p(U), p(U), 0.01, p(B), p(B), ws, 16, None) == 6


@pytest.mark.parametrize("name", ["2d-mixed", "3d-per"])
def test_rhs_adjoint_every_interface_pending(api, oracle, name):
    """A scheme without a keep-all magnitude (B_l = 1, B_u = 2, H = 1e16)
    leaves every interface to the pending passes: the list holds all of
    them, the partition splits it into the all-kept and the cut ones, and
    the gradient still matches the oracle's."""
    from oracle import grad
    sch = dict(H=1e16, b_l=1, b_u=2)
    _, U, n, dx, bc = next(c for c in _cases() if c[0] == name)
    Rbar = np.random.default_rng(23).standard_normal(U.shape)
    ref, _ = grad.rhs_vjp(U, n, dx, bc, Rbar, oracle.Params(**sch))
    grid = api.EulerGrid(n, dx, bc, api.Scheme(**sch))
    Ut = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    got = api.rhs_adjoint(grid, Ut, torch.from_numpy(Rbar).cuda()).cpu().numpy()
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err <= ADJ_RTOL, err
