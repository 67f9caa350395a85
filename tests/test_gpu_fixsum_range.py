"""The closed-form pass's fixed-point sums at the ends of their range, on the
GPU, through the flag-free path that the benchmark times.

* A smooth 2D state whose y momentum is a field of order 1e-290: its sums'
  largest exponent lies below the fixed point's range (values below
  2^-959), so every interface the FP32 test keeps is sent to the pending
  list instead, and the characteristic path evaluates it in binary64.
* A smooth 3D state whose z momentum is exactly zero: its U~ sums and the
  z sweep's mass-flux sums have no nonzero term (largest exponent 0) and
  are taken as exactly 0 in the fixed point.
In both cases the flag-free result must match the flag path (binary64
chains throughout) and the oracle at the usual tolerances."""
import numpy as np
import pytest

from paper_2003_09145_gb300 import inputs
from parity import RHS_RTOL, compare_rhs, flux_scale, rel_max_err

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


def test_tiny_component_goes_to_the_pending_list(api, oracle):
    n = (48, 40)
    U = inputs.random_smooth_state(2, n, seed=21, amp=0.03)
    U = U.reshape(4, n[1], n[0]).copy()
    y = (np.arange(n[1]) + 0.5) / n[1]
    x = (np.arange(n[0]) + 0.5) / n[0]
    U[2] = 1e-290 * (1.0 + 0.5 * np.sin(2 * np.pi * (x[None, :] + 2 * y[:, None])))
    P = inputs.Problem("tiny_my", np.ascontiguousarray(U.reshape(4, -1)), n, (0.02, 0.025), (0, 1), 0.0)
    a, fl, b = _both_paths(api, P)
    fs = flux_scale(P.U0, P.n, P.dx)
    assert rel_max_err(b, a, fs) <= 1e-13
    err, rep = compare_rhs(P.U0, P.n, P.dx, P.bc, b, fl, oracle)
    assert not rep.unexplained
    assert err <= RHS_RTOL, err


def test_zero_component_sums_to_zero(api, oracle):
    n = (20, 16, 12)
    U = inputs.random_smooth_state(3, n, seed=22, amp=0.03).reshape(5, -1).copy()
    rho, mx, my, mz, E = U
    E -= 0.5 * mz * mz / rho         # remove the z kinetic energy, keep p
    U[3] = 0.0
    P = inputs.Problem("zero_mz", np.ascontiguousarray(U), n, (0.1, 0.1, 0.1), (0, 0, 0), 0.0)
    a, fl, b = _both_paths(api, P)
    assert rel_max_err(b, a, flux_scale(P.U0, P.n, P.dx)) <= 1e-13
    err, rep = compare_rhs(P.U0, P.n, P.dx, P.bc, b, fl, oracle)
    assert not rep.unexplained
    assert err <= RHS_RTOL, err
