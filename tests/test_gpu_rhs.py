"""GPU parity of teno_rhs (through the C-ABI) with the FP64 oracle.

Tolerance: 1e-12 relative max-norm per field on one RHS evaluation; selection
flags identical except counted rounding-boundary flips (tests/parity.py)."""
import numpy as np
import pytest

from paper_2003_09145_gb300 import inputs
from parity import RHS_RTOL, classify_flags, compare_rhs, flux_scale, rel_max_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_09145_gb300 import api as A
    return A


def _gpu_rhs(api, P, want_flags=True):
    grid = api.EulerGrid(P.n, P.dx, P.bc, api.Scheme(gamma=P.gamma))
    U = torch.from_numpy(np.ascontiguousarray(P.U0)).cuda()
    out = api.rhs(grid, U, want_flags=want_flags)
    torch.cuda.synchronize()
    if want_flags:
        return out[0].cpu().numpy(), out[1].cpu().numpy()
    return out.cpu().numpy(), None


def _check(api, oracle, P, max_flips=0):
    R, fl = _gpu_rhs(api, P)
    err, rep = compare_rhs(P.U0, P.n, P.dx, P.bc, R, fl, oracle, oracle.Params(gamma=P.gamma))
    assert not rep.unexplained, rep.unexplained[:3]
    assert rep.mismatched <= max(max_flips, rep.total * 1e-4), rep
    assert err <= RHS_RTOL, err
    return err, rep


def test_sod_200(api, oracle):
    _check(api, oracle, inputs.shock_tube(200))


def test_shu_osher_4096(api, oracle):
    _check(api, oracle, inputs.shu_osher(4096))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 33, 129, 1000])
@pytest.mark.parametrize("bc", [0, 1])
def test_1d_ragged_sizes(api, oracle, n, bc):
    U = inputs.random_discontinuous_state(1, (n,), seed=n)
    P = inputs.Problem("rand1d", U, (n,), (1.0 / n,), (bc,), 0.0)
    _check(api, oracle, P)


@pytest.mark.parametrize("n", [(17, 9), (64, 64), (5, 130)])
@pytest.mark.parametrize("bc", [0, 1])
def test_2d_random(api, oracle, n, bc):
    U = inputs.random_discontinuous_state(2, n, seed=sum(n))
    P = inputs.Problem("rand2d", U, n, (0.01, 0.013), (bc, bc), 0.0)
    _check(api, oracle, P)


def test_2d_four_quadrant_128(api, oracle):
    _check(api, oracle, inputs.riemann_2d(n=128))


@pytest.mark.parametrize("n", [(8, 8, 8), (13, 6, 9), (24, 24, 24)])
@pytest.mark.parametrize("bc", [0, 1])
def test_3d_random(api, oracle, n, bc):
    U = inputs.random_discontinuous_state(3, n, seed=sum(n) + bc)
    P = inputs.Problem("rand3d", U, n, (0.1, 0.07, 0.05), (bc,) * 3, 0.0)
    _check(api, oracle, P)


def test_3d_turbulence_32(api, oracle):
    _check(api, oracle, inputs.solenoidal_turbulence(n=32))


def test_smooth_periodic_3d(api, oracle):
    U = inputs.random_smooth_state(3, (16, 12, 10), seed=3)
    P = inputs.Problem("smooth3d", U, (16, 12, 10), (0.1, 0.1, 0.1), (0, 0, 0), 0.0)
    _check(api, oracle, P)


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_constant_state_exact_zero(api, ndim):
    n = (9, 7, 5)[:ndim]
    prim = [1.3] + [0.4, -0.7, 0.2][:ndim] + [2.1]
    rho = np.full(tuple(reversed(n)), prim[0])
    U = inputs.prim_to_cons(rho, [np.full_like(rho, v) for v in prim[1:-1]], np.full_like(rho, prim[-1]))
    for bc in (0, 1):
        P = inputs.Problem("const", U, n, (0.1,) * ndim, (bc,) * ndim, 0.0)
        R, fl = _gpu_rhs(api, P)
        assert np.all(R == 0.0)
        assert np.all(fl & 7 == 7)


def _sampled(api, oracle, P, m, seed):
    """Full-size launch; the oracle evaluates m sampled cells one by one."""
    grid = api.EulerGrid(P.n, P.dx, P.bc)
    U = torch.from_numpy(np.ascontiguousarray(P.U0)).cuda()
    R, fl = api.rhs(grid, U, want_flags=True)
    torch.cuda.synchronize()
    R = R.cpu().numpy().reshape(P.U0.shape[0], -1)
    fl = fl.cpu().numpy()
    rng = np.random.default_rng(seed)
    cells = np.unique(np.concatenate([rng.integers(0, P.ncell, size=m), [0, P.ncell - 1]]))
    fo = np.zeros_like(fl)
    S = oracle.euler_rhs_sample(P.U0, P.n, P.dx, P.bc, cells, flags_out=fo)
    touched = np.nonzero(fo)[0]
    ref = fl.copy()
    ref[touched] = fo[touched]          # oracle's own selections on the sampled faces
    rep = classify_flags(P.U0, P.n, P.dx, P.bc, fl, ref, oracle)
    assert not rep.unexplained, rep.unexplained[:3]
    Sf = oracle.euler_rhs_sample(P.U0, P.n, P.dx, P.bc, cells, flags_in=fl)
    G = R[:, cells]
    # relative max-norm of the sampled vector, and per field against the flux scale
    err = rel_max_err(G, np.ascontiguousarray(Sf.T), flux_scale(P.U0, P.n, P.dx))
    assert err <= RHS_RTOL, err
    return rep


def _sampled_flag_free(api, oracle, P, m, seed):
    """The benchmark's path (no flag output: certified fast paths) at full size,
    against the oracle on m sampled cells, with the selections the flag path
    reports for the same state."""
    grid = api.EulerGrid(P.n, P.dx, P.bc)
    U = torch.from_numpy(np.ascontiguousarray(P.U0)).cuda()
    R_fast = api.rhs(grid, U, want_flags=False)
    R_flag, fl = api.rhs(grid, U, want_flags=True)
    torch.cuda.synchronize()
    R_fast = R_fast.cpu().numpy().reshape(P.U0.shape[0], -1)
    fl = fl.cpu().numpy()
    rng = np.random.default_rng(seed)
    cells = np.unique(np.concatenate([rng.integers(0, P.ncell, size=m), [0, P.ncell - 1]]))
    Sf = oracle.euler_rhs_sample(P.U0, P.n, P.dx, P.bc, cells, flags_in=fl)
    err = rel_max_err(R_fast[:, cells], np.ascontiguousarray(Sf.T), flux_scale(P.U0, P.n, P.dx))
    assert err <= RHS_RTOL, err
    # and the two GPU paths agree to rounding on the whole grid
    assert rel_max_err(R_fast, R_flag.cpu().numpy().reshape(R_fast.shape),
                       flux_scale(P.U0, P.n, P.dx)) <= 1e-13


@pytest.mark.slow
def test_turbulence_256_flag_free_sampled(api, oracle):
    _sampled_flag_free(api, oracle, inputs.solenoidal_turbulence(n=256), 2000, 3)


@pytest.mark.slow
def test_four_quadrant_2048_flag_free_sampled(api, oracle):
    _sampled_flag_free(api, oracle, inputs.riemann_2d(n=2048), 3000, 4)


@pytest.mark.slow
def test_four_quadrant_2048_sampled(api, oracle):
    _sampled(api, oracle, inputs.riemann_2d(n=2048), 4000, 1)


@pytest.mark.slow
def test_turbulence_256_sampled(api, oracle):
    _sampled(api, oracle, inputs.solenoidal_turbulence(n=256), 2000, 2)


@pytest.mark.parametrize("case", ["sod", "shu", "rand2d", "rand3d", "turb", "smooth3d"])
def test_flag_free_path(api, oracle, case):
    """Without a flag output the kernel takes the certified fast paths (FP32
    pre-tests, and the closed form when every stencil is kept).  Its right-hand
    side must match the oracle (under the selections the flag path reports) to
    the same 1e-12, and the flag path to rounding."""
    P = {"sod": lambda: inputs.shock_tube(300),
         "shu": lambda: inputs.shu_osher(4096),
         "rand2d": lambda: inputs.Problem("r2", inputs.random_discontinuous_state(2, (40, 30), seed=5),
                                          (40, 30), (0.02, 0.03), (1, 0), 0.0),
         "rand3d": lambda: inputs.Problem("r3", inputs.random_discontinuous_state(3, (12, 10, 9), seed=6),
                                          (12, 10, 9), (0.1, 0.1, 0.1), (0, 1, 0), 0.0),
         "turb": lambda: inputs.solenoidal_turbulence(n=32),
         "smooth3d": lambda: inputs.Problem("s3", inputs.random_smooth_state(3, (20, 16, 12), seed=7, amp=0.03),
                                            (20, 16, 12), (0.1, 0.1, 0.1), (0, 0, 0), 0.0)}[case]()
    a, fl = _gpu_rhs(api, P, want_flags=True)
    b, _ = _gpu_rhs(api, P, want_flags=False)
    assert rel_max_err(b, a, flux_scale(P.U0, P.n, P.dx)) <= 1e-13
    err, rep = compare_rhs(P.U0, P.n, P.dx, P.bc, b, fl, oracle)
    assert not rep.unexplained
    assert err <= RHS_RTOL, err


@pytest.mark.parametrize("case", ["rand2d", "smooth3d"])
def test_every_interface_pending(api, oracle, case):
    """A scheme without a keep-all magnitude (B_l = 1, B_u = 2, H = 1e16:
    3 (1 + max chi~)^6 C_T >= 1 at m = 2) sends every interface of the
    flag-free path through the pending list: the list fills completely and the
    result still matches the flag path and the oracle."""
    sch = dict(H=1e16, b_l=1, b_u=2)
    P = {"rand2d": lambda: inputs.Problem("r2", inputs.random_discontinuous_state(2, (33, 20), seed=15),
                                          (33, 20), (0.02, 0.03), (1, 0), 0.0),
         "smooth3d": lambda: inputs.Problem("s3", inputs.random_smooth_state(3, (17, 12, 9), seed=17, amp=0.03),
                                            (17, 12, 9), (0.1, 0.1, 0.1), (0, 1, 0), 0.0)}[case]()
    grid = api.EulerGrid(P.n, P.dx, P.bc, api.Scheme(**sch))
    U = torch.from_numpy(np.ascontiguousarray(P.U0)).cuda()
    a, fl = api.rhs(grid, U, want_flags=True)
    b = api.rhs(grid, U, want_flags=False)
    torch.cuda.synchronize()
    a, fl, b = a.cpu().numpy(), fl.cpu().numpy(), b.cpu().numpy()
    assert rel_max_err(b, a, flux_scale(P.U0, P.n, P.dx)) <= 1e-13
    err, rep = compare_rhs(P.U0, P.n, P.dx, P.bc, b, fl, oracle, oracle.Params(**sch))
    assert not rep.unexplained
    assert err <= RHS_RTOL, err


def test_cuda_graph_replay_matches_eager(api):
    """Steps captured in a CUDA graph give the same state as eager steps."""
    P = inputs.shu_osher(1024)
    grid = api.EulerGrid(P.n, P.dx, P.bc)
    U1 = torch.from_numpy(P.U0).cuda()
    U2 = U1.clone()
    s1 = api.Solver(grid)
    for _ in range(11):
        s1.step(U1, P.t_end)
    s2 = api.Solver(grid)
    s2.capture(U2, 5, P.t_end)        # one eager warm-up step + graph of 5
    s2.graph.replay()
    s2.graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(U1, U2)
    assert s1.t.item() == s2.t.item()
