"""The largest grids one GPU holds: a 3D state of 768 x 768 x 736 cells
(434 M cells; a state is 2.17e9 doubles, so element offsets pass 2^31)
that is uniform along z with no z momentum.  Along z every interface sees
six equal states, so the z sweep adds exactly nothing, and every z slice of
the 3D right-hand side (eq. 2.2) and of one fixed-dt SSP-RK3 step (eq.
4.1-4.3) must equal the 2D result of the slice (the z-momentum field
carries zeros through the projection and the reconstruction).  The 2D
slice is the four-quadrant problem (Sec. 4.3.1) after 20 steps, and its
right-hand side is checked against the oracle at sampled cells."""
import numpy as np
import pytest

from paper_2003_09145_gb300 import inputs
from parity import flux_scale, rel_max_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NX, NY, NZ = 768, 768, 736
SLICE_RTOL = 1e-13


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_09145_gb300 import api as A
    return A


def _slice_state(api):
    P = inputs.riemann_2d(n=NX)
    grid2 = api.EulerGrid(P.n, P.dx, P.bc)
    U2 = torch.from_numpy(np.ascontiguousarray(P.U0)).cuda()
    s = api.Solver(grid2)
    for _ in range(20):
        s.step(U2, float("inf"))
    torch.cuda.synchronize()
    return P, grid2, U2


def _extrude(U2):
    """[4][ny][nx] -> [5][nz][ny][nx]: (rho, m_x, m_y, 0, E), the same on every slice."""
    U3 = torch.empty((5, NZ, NY, NX), dtype=torch.float64, device="cuda")
    for v3, v2 in ((0, 0), (1, 1), (2, 2), (4, 3)):
        U3[v3].copy_(U2.view(4, NY, NX)[v2].unsqueeze(0).expand(NZ, NY, NX))
    U3[3].zero_()
    return U3.view(-1)


def _need(nbytes):
    free, _ = torch.cuda.mem_get_info()
    if free < nbytes:
        pytest.skip(f"needs {nbytes / 2**30:.0f} GiB of free device memory, {free / 2**30:.0f} GiB free")


def _compare_slices(A3, A2, scale):
    """Every z slice of A3 against A2 (relative to `scale`); field 3 must be zero."""
    a3 = A3.view(5, NZ, NY, NX)
    a2 = A2.view(4, NY, NX)
    assert torch.count_nonzero(a3[3]).item() == 0
    worst = 0.0
    for v3, v2 in ((0, 0), (1, 1), (2, 2), (4, 3)):
        d = (a3[v3] - a2[v2].unsqueeze(0)).abs().amax().item()
        worst = max(worst, d / scale[v2])
    return worst


def test_max_size_rhs_and_step_equal_2d_slices(api, oracle):
    P, grid2, U2 = _slice_state(api)
    dx = P.dx[0]
    grid3 = api.EulerGrid((NX, NY, NZ), (P.dx[0], P.dx[1], 0.7 * dx), (P.bc[0], P.bc[1], 0))
    state = 5 * grid3.ncell * 8
    _need(3 * state + grid3.workspace_bytes(1))

    # the 2D slice's right-hand side (the flag-free path), anchored to the
    # oracle at sampled cells under the flag path's selections
    R2 = api.rhs(grid2, U2)
    _, fl2 = api.rhs(grid2, U2, want_flags=True)
    U2h = U2.cpu().numpy()
    cells = np.sort(np.random.default_rng(5).choice(grid2.ncell, 400, replace=False))
    ref = oracle.euler_rhs_sample(U2h, P.n, P.dx, P.bc, cells, flags_in=fl2.cpu().numpy())
    got = R2.cpu().numpy().reshape(4, -1)[:, cells]
    assert rel_max_err(got, np.ascontiguousarray(ref.T), flux_scale(U2h, P.n, P.dx)) <= 1e-12

    # one 3D right-hand side on the extruded state
    U3 = _extrude(U2)
    R3 = api.rhs(grid3, U3)
    torch.cuda.synchronize()
    scale = [float(R2.view(4, -1)[v].abs().max()) + 1e-300 for v in range(4)]
    assert _compare_slices(R3, R2, scale) <= SLICE_RTOL
    del R3
    torch.cuda.empty_cache()

    # one fixed-dt SSP-RK3 step of both
    dt = 0.2 * dx
    api.Solver(grid2).step(U2, float("inf"), dt_fixed=dt)
    s3 = api.Solver(grid3)
    s3.step(U3, float("inf"), dt_fixed=dt)
    torch.cuda.synchronize()
    assert s3.status() == 0
    scale = [float(U2.view(4, -1)[v].abs().max()) for v in range(4)]
    assert _compare_slices(U3, U2, scale) <= SLICE_RTOL
