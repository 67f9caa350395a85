"""Scalar mode (teno_scalar_rhs, teno_scalar_rk3_step): linear advection
u_t + a u_x = 0 on a periodic grid (Sec. 4.1) with the same TENO5-LAD device
code, against the oracle's scalar restatement; Tab. 1 reproduced on the GPU;
the composite waves of eq. 4.6 run to the paper's t = 6."""
import math
import os

import numpy as np
import pytest

from paper_2003_09145_gb300 import inputs
from parity import RHS_RTOL, STEP_RTOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_09145_gb300 import api as A
    return A


def _rel_max(a, b, scale):
    return float(np.max(np.abs(a - b))) / scale


@pytest.mark.parametrize("mode", ["lad", "upwind5"])
@pytest.mark.parametrize("case,n", [("smooth", 20), ("smooth", 80), ("smooth", 320), ("composite", 200),
                                    ("composite", 37)])
def test_scalar_rhs_matches_oracle(api, oracle, mode, case, n):
    u0 = inputs.scalar_smooth(n) if case == "smooth" else inputs.scalar_composite(n)
    dx = 2.0 / n
    adv = api.ScalarAdvection(n, dx, mode=mode)
    r = adv.rhs(torch.from_numpy(u0).cuda()).cpu().numpy()
    ro = oracle.scalar_rhs(u0, dx, "lad" if mode == "lad" else "upwind")
    # measured against the size of the fluxes the difference cancels, max|u|/dx
    assert _rel_max(r, ro, np.max(np.abs(u0)) / dx) <= RHS_RTOL


@pytest.mark.parametrize("mode", ["lad", "upwind5"])
def test_scalar_steps_match_oracle(api, oracle, mode):
    n = 80
    dx = 2.0 / n
    u0 = inputs.scalar_smooth(n)
    adv = api.ScalarAdvection(n, dx, mode=mode)
    u = torch.from_numpy(u0.copy()).cuda()
    k = adv.run(u, 2.0, dx ** (5.0 / 3.0))
    uo, ko = oracle.scalar_run(u0, dx, 2.0, dx ** (5.0 / 3.0), "lad" if mode == "lad" else "upwind")
    assert k == ko
    ug = u.cpu().numpy()
    assert np.sum(np.abs(ug - uo)) / np.sum(np.abs(uo)) <= STEP_RTOL


def test_tab1_on_the_gpu(api):
    """Tab. 1 (eq. 4.5 to t = 2, dt = dx^(5/3)/8 so that the spatial error
    shows): the L2 errors of the GPU's LAD and Upwind5 runs match the printed
    Upwind5 column within 2 % and its orders within 0.03."""
    rows = []
    with open(os.path.join(GOLDEN, "tab1_upwind5_l2.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                n, l2, order = line.split()
                rows.append((int(n), float(l2), None if order == "-" else float(order)))
    for mode in ("lad", "upwind5"):
        errs = []
        for n, l2, _ in rows:
            dx = 2.0 / n
            u0 = inputs.scalar_smooth(n)
            adv = api.ScalarAdvection(n, dx, mode=mode)
            u = torch.from_numpy(u0.copy()).cuda()
            adv.run(u, 2.0, dx ** (5.0 / 3.0) / 8.0)
            e = math.sqrt(float(np.mean((u.cpu().numpy() - u0) ** 2)))   # exact: u0(x - 2) = u0
            assert abs(e / l2 - 1.0) < 0.02, (mode, n, e, l2)
            errs.append(e)
        for (n, _, order), o in zip(rows[1:], [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]):
            assert abs(o - order) <= 0.03 + 1e-12, (mode, n, o, order)


def test_composite_waves_to_t6(api, oracle):
    """Fig. 2's run (eq. 4.6, N = 200, t = 6, here dt = dx/2): GPU equals the
    oracle over 1200 steps; the square and triangle stay within [0, 1] to 1 %."""
    n = 200
    dx = 2.0 / n
    u0 = inputs.scalar_composite(n)
    adv = api.ScalarAdvection(n, dx, mode="lad")
    u = torch.from_numpy(u0.copy()).cuda()
    k = adv.run(u, 6.0, 0.5 * dx)
    uo, ko = oracle.scalar_run(u0, dx, 6.0, 0.5 * dx, "lad")
    assert k == ko and k >= 1200        # the last, clipped step may be tiny
    ug = u.cpu().numpy()
    assert np.sum(np.abs(ug - uo)) / np.sum(np.abs(uo)) <= STEP_RTOL
    assert ug.max() <= 1.01 and ug.min() >= -0.01


def test_negative_speed_is_the_mirror_image(api):
    """u_t - u_x = 0 on mirrored data is the mirror image of u_t + u_x = 0:
    f^- takes the role of f^+ (x -> -x maps point i to (n - i) mod n)."""
    n = 64
    dx = 2.0 / n
    u0 = inputs.scalar_composite(n) + 0.3 * inputs.scalar_smooth(n)
    mirror = (-np.arange(n)) % n
    fwd = api.ScalarAdvection(n, dx, a=1.0).rhs(torch.from_numpy(u0).cuda()).cpu().numpy()
    bwd = api.ScalarAdvection(n, dx, a=-1.0).rhs(torch.from_numpy(np.ascontiguousarray(u0[mirror])).cuda())
    bwd = bwd.cpu().numpy()
    assert np.max(np.abs(bwd[mirror] - fwd)) <= 1e-14 * np.max(np.abs(fwd))
