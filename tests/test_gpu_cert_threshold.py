"""The certified FP32 keep-all pre-tests at their threshold, on the GPU.

The flag-free paths (scalar mode, the pending pass, the one-pass kernel, the
batched mode) first ask FP32 whether binary64 would keep every stencil
(eq. 2.14 with C_T of eq. 3.1-3.4).  Here the inputs sit where that decision
is closest: five-point windows whose exact tau/dmin is thr (1 +- 1e-3 ...
1e-7) at magnitudes up to 1e8, windows that vary by less than the FP32
truncation of large values, and Euler states at pressures of 1e5 (SI units)
with small fluctuations.  Whatever the pre-tests certify must be what
binary64 decides: the GPU's flag-free result must equal the oracle (under
the flag path's selections, flips counted) at 1e-12, and the flag path to
rounding."""
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


THR = 10.0      # H (K/3 - 1): below it every stencil is kept (m >= 7)
EPS = 1e-6


def _ratio(v):
    e = np.diff(v)
    a = e[1:] - e[:-1]
    c = np.array([3 * e[1] - e[0], e[1] + e[2], e[3] - 3 * e[2]])
    b = 13.0 / 3.0 * a * a + c * c
    return abs(b[2] - b[0]) / (b.min() + 4 * EPS)


def _window(rng, target, offset):
    shape = rng.standard_normal(5)
    lo, hi = 1e-12, 1e12
    for _ in range(90):
        mid = np.sqrt(lo * hi)
        lo, hi = (mid, hi) if _ratio(offset + mid * shape) < target else (lo, mid)
    return offset + np.sqrt(lo * hi) * shape


def _threshold_line(seed, nwin):
    """Blocks of five values: block k is the stencil of interface 5k+2+1/2
    (f^+ of a > 0).  Each block sits at the keep-all threshold at a magnitude
    of 1e-8 ... 1e8, or varies by less than the truncation of a large value."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(nwin):
        mag = 10.0 ** rng.uniform(-8, 8) * rng.choice([-1.0, 1.0])
        if k % 5 == 4:
            out.append(mag * 1e4 * (1.0 + 2.0**-20 * rng.uniform(-2, 2, 5)))
        else:
            rel = 10.0 ** -rng.uniform(3, 7) * rng.choice([-1.0, 1.0])
            out.append(_window(rng, THR * (1 + rel), mag if k % 2 else 0.0))
    return np.concatenate(out)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_scalar_mode_at_threshold(api, oracle, seed):
    u0 = _threshold_line(seed, 400)
    n = u0.size
    dx = 2.0 / n
    adv = api.ScalarAdvection(n, dx, mode="lad")
    r = adv.rhs(torch.from_numpy(u0).cuda()).cpu().numpy()
    ro = oracle.scalar_rhs(u0, dx, "lad")
    # per block: errors against that block's own magnitude (the blocks span
    # sixteen decades, so one global scale would hide the small ones)
    for k in range(2, n // 5 - 2):
        sl = slice(5 * k, 5 * k + 5)
        scale = max(np.max(np.abs(u0[5 * k - 5:5 * k + 10])), 1e-300) / dx
        assert np.max(np.abs(r[sl] - ro[sl])) <= RHS_RTOL * scale, (k, u0[sl])


def _large_pressure_state(seed, n, ndim):
    """Air at rest-ish, rho ~ 1.2 kg/m^3, p ~ 1e5 Pa, u ~ 10 m/s, with smooth
    fluctuations whose amplitude runs over many decades along y (or from line
    to line), so that some windows sit at the keep-all threshold."""
    rng = np.random.default_rng(seed)
    shp = tuple(reversed(n))
    x = [np.arange(m) / m for m in n]
    grids = np.meshgrid(*reversed(x), indexing="ij")
    amp = 10.0 ** np.linspace(-9, -2, shp[0]).reshape((-1,) + (1,) * (ndim - 1))
    wave = sum(np.sin(2 * np.pi * (k + 1) * g + rng.uniform(0, 6.3)) for k, g in enumerate(grids))
    wave = wave + 0.3 * rng.standard_normal(shp)
    rho = 1.2 * (1 + amp * wave)
    p = 1.0e5 * (1 + amp * np.roll(wave, 1, axis=-1))
    vel = [10.0 * (1 + amp * np.roll(wave, 2 + k, axis=-1)) for k in range(ndim)]
    return inputs.prim_to_cons(rho, vel, p)


@pytest.mark.parametrize("ndim,n,bc", [(1, (600,), (1,)), (2, (96, 40), (0, 1)), (3, (24, 16, 12), (0, 1, 0))])
def test_euler_large_pressure_paths_agree(api, oracle, ndim, n, bc):
    if ndim == 1:
        U = np.concatenate([_large_pressure_state(s, (60,), 1) for s in range(10)], axis=1)
    else:
        U = _large_pressure_state(11 + ndim, n, ndim)
    dx = tuple(1.0 / m for m in n)
    grid = api.EulerGrid(n, dx, bc)
    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    a, fl = api.rhs(grid, Ud, want_flags=True)
    b = api.rhs(grid, Ud, want_flags=False)
    torch.cuda.synchronize()
    a, fl, b = a.cpu().numpy(), fl.cpu().numpy(), b.cpu().numpy()
    fs = flux_scale(U, n, dx)
    assert rel_max_err(b, a, fs) <= 1e-13
    err, rep = compare_rhs(U, n, dx, bc, b, fl, oracle)
    assert not rep.unexplained, rep.unexplained[:3]
    assert err <= RHS_RTOL, err
    # the state exercises both outcomes of the decision
    sel = fl & 7
    assert np.any(sel == 7) and np.any(sel != 7)
