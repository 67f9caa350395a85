"""Pins of the reverse-mode gradient oracle (oracle/grad.py, PyTorch CPU float64):
its forward value equals the C oracle's right-hand side (an independent second
restatement of eq. 2.2), and its gradient matches central finite differences of
the same frozen-selection function (no GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2003_09145_gb300 import inputs


def _jitter(U, seed):
    """Break the symmetries of the smooth test states (ties in max |lambda| make the
    global LF speed non-differentiable)."""
    rng = np.random.default_rng(seed)
    V = U * (1.0 + 1e-3 * rng.standard_normal(U.shape))
    return np.ascontiguousarray(V)


def _cases():
    return [
        ("1d-trans", inputs.random_discontinuous_state(1, (23,), seed=1), (23,), (0.04,), (1,)),
        ("1d-per", _jitter(inputs.random_smooth_state(1, (17,), seed=2), 1), (17,), (0.05,), (0,)),
        ("2d-mixed", inputs.random_discontinuous_state(2, (9, 7), seed=3), (9, 7), (0.1, 0.08), (0, 1)),
        ("3d-per", _jitter(inputs.random_smooth_state(3, (6, 5, 4), seed=4), 2), (6, 5, 4), (0.2, 0.2, 0.25), (0, 0, 0)),
        ("3d-trans", inputs.random_discontinuous_state(3, (5, 6, 7), seed=5), (5, 6, 7), (0.1, 0.1, 0.1), (1, 1, 1)),
    ]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_forward_matches_c_oracle(oracle, case):
    from oracle import grad
    _, U, n, dx, bc = case
    R_c, flags = oracle.euler_rhs(U, n, dx, bc, want_flags=True)
    R_t = grad.rhs(torch.from_numpy(U), n, dx, bc, flags).numpy()
    scale = np.max(np.abs(R_c))
    assert np.max(np.abs(R_t - R_c)) <= 1e-12 * scale


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_gradient_matches_central_differences(oracle, case):
    """<J^T v, w> against (v . (R(U + h w) - R(U - h w)) / 2h) with the selections
    frozen at U (the perturbation is small enough that alpha's arg-max cell is
    unchanged)."""
    from oracle import grad
    _, U, n, dx, bc = case
    rng = np.random.default_rng(11)
    _, flags = oracle.euler_rhs(U, n, dx, bc, want_flags=True)
    v = rng.standard_normal(U.shape)
    w = rng.standard_normal(U.shape) * np.abs(U)
    Ut = torch.from_numpy(U).requires_grad_(True)
    R = grad.rhs(Ut, n, dx, bc, flags)
    (g,) = torch.autograd.grad(R, Ut, torch.from_numpy(v).reshape(R.shape))
    lhs = float(np.sum(g.numpy() * w))
    h = 1e-6
    Rp = grad.rhs(torch.from_numpy(U + h * w), n, dx, bc, flags).numpy()
    Rm = grad.rhs(torch.from_numpy(U - h * w), n, dx, bc, flags).numpy()
    rhs_ = float(np.sum(v * (Rp - Rm))) / (2 * h)
    assert lhs == pytest.approx(rhs_, rel=1e-6, abs=1e-8 * np.sum(np.abs(v * Rp)))


def test_rollout_gradient_matches_differences(oracle):
    """Three frozen-selection RK3 steps on a small periodic 2D box."""
    from oracle import grad
    n, dx, bc = (8, 6), (0.1, 0.1), (0, 0)
    U = _jitter(inputs.random_smooth_state(2, n, seed=7), 3)
    rng = np.random.default_rng(3)
    wdir = rng.standard_normal(U.shape) * np.abs(U)
    Ut = torch.from_numpy(U).requires_grad_(True)
    out = grad.rk3_rollout(Ut, n, dx, bc, 0.01, 3)
    loss = 0.5 * (out[0] ** 2).sum()
    (g,) = torch.autograd.grad(loss, Ut)
    h = 1e-6
    lp = 0.5 * (grad.rk3_rollout(torch.from_numpy(U + h * wdir), n, dx, bc, 0.01, 3)[0] ** 2).sum().item()
    lm = 0.5 * (grad.rk3_rollout(torch.from_numpy(U - h * wdir), n, dx, bc, 0.01, 3)[0] ** 2).sum().item()
    assert float(np.sum(g.numpy() * wdir)) == pytest.approx((lp - lm) / (2 * h), rel=1e-6)
