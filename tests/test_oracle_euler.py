"""Pins of the oracle's Euler right-hand side, time step and exact Riemann solver
(no GPU).  Each check is fixed by the paper or by the mathematics, not by the
oracle itself:

* the characteristic eigensystem: L R = I, and the Roe property
  R diag(lambda) L (U_b - U_a) = F(U_b) - F(U_a) (the reading of the paper's
  "characteristic space" paragraph in Sec. 4);
* a constant state has an exactly zero right-hand side (eq. 2.2);
* telescoping conservation on periodic grids (eq. 2.2);
* dimensional consistency: a 2D/3D state without variation across reproduces 1D;
* transpose symmetry of the 2D four-quadrant problem;
* 5th-order convergence on a smooth entropy wave (Sec. 4.1's order study on Euler);
* the exact Riemann solver: textbook star state, jump conditions, Riemann
  invariants; the scheme's Sod solution converges to it (eq. 4.8);
* the CFL step formulas eq. dt1 / dt2.
"""
import math
import os

import numpy as np
import pytest

from paper_2003_09145_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cons(ndim, rho, vel, p, g=1.4):
    return np.array([rho] + [rho * v for v in vel] + [p / (g - 1) + 0.5 * rho * sum(v * v for v in vel)])


def _flux(ndim, d, U, g=1.4):
    rho = U[0]
    vel = U[1:1 + ndim] / rho
    E = U[-1]
    p = (g - 1) * (E - 0.5 * rho * np.sum(vel * vel))
    F = np.zeros(ndim + 2)
    F[0] = rho * vel[d]
    F[1:1 + ndim] = rho * vel * vel[d]
    F[1 + d] += p
    F[-1] = vel[d] * (E + p)
    return F


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_eigensystem_inverse_and_roe_property(oracle, ndim):
    rng = np.random.default_rng(ndim)
    for _ in range(50):
        a = _cons(ndim, rng.uniform(0.1, 3), rng.uniform(-2, 2, ndim), rng.uniform(0.1, 5))
        b = _cons(ndim, rng.uniform(0.1, 3), rng.uniform(-2, 2, ndim), rng.uniform(0.1, 5))
        for d in range(ndim):
            L, R = oracle.roe_eigensystem(ndim, d, a, b)
            np.testing.assert_allclose(L @ R, np.eye(ndim + 2), atol=1e-12)
            # eigenvalues of the Roe matrix: u_d - c, u_d (x ndim), u_d + c
            sa, sb = math.sqrt(a[0]), math.sqrt(b[0])
            u = (a[1:1 + ndim] / sa + b[1:1 + ndim] / sb) / (sa + sb)
            Ha = (a[-1] + (1.4 - 1) * (a[-1] - 0.5 * np.sum(a[1:1 + ndim] ** 2) / a[0])) / a[0]
            Hb = (b[-1] + (1.4 - 1) * (b[-1] - 0.5 * np.sum(b[1:1 + ndim] ** 2) / b[0])) / b[0]
            H = (sa * Ha + sb * Hb) / (sa + sb)
            c = math.sqrt(0.4 * (H - 0.5 * np.sum(u * u)))
            lam = np.array([u[d] - c] + [u[d]] * ndim + [u[d] + c])
            A = R @ np.diag(lam) @ L
            dF = _flux(ndim, d, b) - _flux(ndim, d, a)
            np.testing.assert_allclose(A @ (b - a), dF, rtol=1e-10, atol=1e-10 * np.max(np.abs(dF)))


@pytest.mark.parametrize("ndim,bc", [(1, 0), (1, 1), (2, 0), (2, 1), (3, 0), (3, 1)])
def test_constant_state_rhs_is_exactly_zero(oracle, ndim, bc):
    n = (7, 6, 5)[:ndim]
    U0 = _cons(ndim, 1.3, [0.4, -0.7, 0.2][:ndim], 2.1)
    U = np.ascontiguousarray(np.broadcast_to(U0.reshape((-1,) + (1,) * ndim), (ndim + 2,) + tuple(reversed(n))))
    R, flags = oracle.euler_rhs(U, n, [0.1] * ndim, [bc] * ndim, want_flags=True)
    assert np.all(R == 0.0)
    assert np.all(flags & 7 == 7)


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_periodic_telescoping_conservation(oracle, ndim):
    n = (24, 10, 8)[:ndim]
    U = inputs.random_discontinuous_state(ndim, n, seed=11)
    dx = [0.05, 0.07, 0.09][:ndim]
    R = oracle.euler_rhs(U, n, dx, [0] * ndim)
    cell_vol = np.prod(dx)
    for v in range(ndim + 2):
        s = np.sum(R[v]) * cell_vol
        scale = np.sum(np.abs(R[v])) * cell_vol
        assert abs(s) <= 64 * np.finfo(float).eps * scale, (v, s, scale)


def test_multid_reduces_to_1d(oracle):
    """A state that varies only along one axis gives, on that axis, the 1D RHS in
    every row; the transverse momentum is passively carried (zero here)."""
    n1 = 40
    U1 = inputs.random_discontinuous_state(1, (n1,), seed=4)
    R1 = oracle.euler_rhs(U1, (n1,), [0.025], [1])
    for ndim, axis in ((2, 0), (2, 1), (3, 0), (3, 2)):
        n = [5] * ndim
        n[axis] = n1
        shape = tuple(reversed(n))
        U = np.zeros((ndim + 2,) + shape)
        bshape = [1] * ndim
        bshape[ndim - 1 - axis] = n1
        U[0] = U1[0].reshape(bshape)
        U[1 + axis] = U1[1].reshape(bshape)
        U[-1] = U1[2].reshape(bshape)
        dx = [0.3] * ndim
        dx[axis] = 0.025
        R = oracle.euler_rhs(U, tuple(n), dx, [1] * ndim)
        for comp_nd, comp_1d in ((0, 0), (1 + axis, 1), (ndim + 1, 2)):
            np.testing.assert_allclose(R[comp_nd], np.broadcast_to(R1[comp_1d].reshape(bshape), shape),
                                       rtol=0, atol=1e-12 * np.max(np.abs(R1[comp_1d])))
        for t in range(ndim):
            if t != axis:
                assert np.all(R[1 + t] == 0.0)


def test_four_quadrant_transpose_symmetry(oracle):
    """(x, y, u, v) -> (y, x, v, u) maps the four-quadrant data onto itself; the
    dimension-by-dimension RHS must be transpose-symmetric."""
    P = inputs.riemann_2d(n=48, split=(0.5, 0.5))
    U = P.U0
    R = oracle.euler_rhs(U, P.n, P.dx, P.bc)
    np.testing.assert_array_equal(U[0], U[0].T)
    for a, b in ((0, 0), (1, 2), (3, 3)):
        np.testing.assert_allclose(R[a], R[b].T, rtol=0, atol=1e-13 * np.max(np.abs(R[a])))


def test_entropy_wave_fifth_order(oracle):
    """rho = 1 + 0.2 sin(pi x), u = p = 1 on [-1,1] periodic is advected exactly;
    with dt = dx^(5/3) (Sec. 4.1's choice) the L1 error falls at 5th order."""
    errs = []
    ns = (16, 32, 64)
    for n in ns:
        P = inputs.entropy_wave(n, t_end=0.5)
        dx = P.dx[0]
        dt = min(0.5 * dx / 2.2, dx ** (5.0 / 3.0))
        nsteps = math.ceil(P.t_end / dt)
        dt = P.t_end / nsteps
        U, t, k = oracle.euler_run(P.U0, P.n, P.dx, P.bc, P.t_end, dt_fixed=dt)
        x = P.centers(0)
        exact = 1.0 + 0.2 * np.sin(np.pi * (x - t))
        errs.append(np.mean(np.abs(U[0] - exact)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert orders[-1] >= 4.7, orders


def _riemann_golden():
    vals = {}
    with open(os.path.join(GOLDEN, "sod_exact_star_state.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_exact_riemann_sod_star_state(oracle):
    g = _riemann_golden()
    st = oracle.riemann_star((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert st["p"] == pytest.approx(g["p_star"], abs=6e-6)
    assert st["u"] == pytest.approx(g["u_star"], abs=6e-6)
    assert st["rho_l"] == pytest.approx(g["rho_star_left"], abs=6e-6)
    assert st["rho_r"] == pytest.approx(g["rho_star_right"], abs=6e-6)


def _rh_residual(rho0, u0, p0, rho1, u1, p1, s, g=1.4):
    """Rankine-Hugoniot residuals of mass, momentum and energy across speed s."""
    E0 = p0 / (g - 1) + 0.5 * rho0 * u0 * u0
    E1 = p1 / (g - 1) + 0.5 * rho1 * u1 * u1
    r = [rho1 * (u1 - s) - rho0 * (u0 - s),
         rho1 * u1 * (u1 - s) + p1 - (rho0 * u0 * (u0 - s) + p0),
         E1 * (u1 - s) + p1 * u1 - (E0 * (u0 - s) + p0 * u0)]
    return max(abs(x) for x in r)


def test_exact_riemann_jump_conditions_and_invariants(oracle):
    rng = np.random.default_rng(5)
    g = 1.4
    for _ in range(200):
        left = (rng.uniform(0.1, 2), rng.uniform(-1, 1), rng.uniform(0.1, 10))
        right = (rng.uniform(0.1, 2), rng.uniform(-1, 1), rng.uniform(0.1, 10))
        st = oracle.riemann_star(left, right)
        p, u = st["p"], st["u"]
        scale = max(left[2], right[2], 1.0)
        if st["left_shock"] > 0.5:
            assert _rh_residual(*left, st["rho_l"], u, p, st["s_l_head"]) <= 1e-11 * scale
        else:  # isentropic fan: p/rho^g and u + 2c/(g-1) constant
            cl = math.sqrt(g * left[2] / left[0])
            cs = math.sqrt(g * p / st["rho_l"])
            assert p / st["rho_l"] ** g == pytest.approx(left[2] / left[0] ** g, rel=1e-12)
            assert u + 2 * cs / (g - 1) == pytest.approx(left[1] + 2 * cl / (g - 1), rel=1e-12, abs=1e-12)
        if st["right_shock"] > 0.5:
            assert _rh_residual(*right, st["rho_r"], u, p, st["s_r_head"]) <= 1e-11 * scale
        else:
            cr = math.sqrt(g * right[2] / right[0])
            cs = math.sqrt(g * p / st["rho_r"])
            assert p / st["rho_r"] ** g == pytest.approx(right[2] / right[0] ** g, rel=1e-12)
            assert u - 2 * cs / (g - 1) == pytest.approx(right[1] - 2 * cr / (g - 1), rel=1e-12, abs=1e-12)
        # sampled profile: continuous pressure and velocity across the contact
        xi = np.array([u - 1e-9, u + 1e-9])
        s = oracle.riemann_sample(left, right, xi)
        assert s[1, 0] == pytest.approx(s[1, 1], abs=1e-12)
        assert s[2, 0] == pytest.approx(s[2, 1], rel=1e-12)


def test_sod_converges_to_exact_solution(oracle):
    """Eq. 4.8 data (the standard Sod layout: [0,1], jump at 0.5, t = 0.2): the L1 density
    error against the exact solution decreases with N and is small at N = 200."""
    errs = []
    for n in (50, 100, 200):
        P = inputs.shock_tube(n)
        U, t, k = oracle.euler_run(P.U0, P.n, P.dx, P.bc, P.t_end, sigma=P.cfl)
        assert t == P.t_end
        xi = (P.centers(0) - 0.5) / t
        ex = oracle.riemann_sample(P.extra["left"], P.extra["right"], xi)
        errs.append(np.mean(np.abs(U[0] - ex[0])))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 4e-3


def test_cfl_formulas(oracle):
    """eq. dt1: sigma dx / max(|u| + c); eq. dt2: sigma dtx dty / (dtx + dty)."""
    P = inputs.shock_tube(64)
    rho, m, E = P.U0
    u = m / rho
    p = 0.4 * (E - 0.5 * rho * u * u)
    c = np.sqrt(1.4 * p / rho)
    assert oracle.euler_dt(P.U0, P.n, P.dx, 0.5) == pytest.approx(0.5 * P.dx[0] / np.max(np.abs(u) + c), rel=1e-15)
    Q = inputs.riemann_2d(n=32)
    rho, mu, mv, E = Q.U0
    u, v = mu / rho, mv / rho
    p = 0.4 * (E - 0.5 * rho * (u * u + v * v))
    c = np.sqrt(1.4 * p / rho)
    dtx = Q.dx[0] / np.max(np.abs(u) + c)
    dty = Q.dx[1] / np.max(np.abs(v) + c)
    assert oracle.euler_dt(Q.U0, Q.n, Q.dx, 0.5) == pytest.approx(0.5 * dtx * dty / (dtx + dty), rel=1e-14)


def test_flags_layout_and_forced_replay(oracle):
    """Flags from one RHS evaluation, fed back as forced selections, reproduce the
    same RHS bit for bit; every flag byte holds m in 4..10 and a non-empty delta."""
    P = inputs.riemann_2d(n=20, split=(0.45, 0.55))
    R, flags, alpha = oracle.euler_rhs(P.U0, P.n, P.dx, P.bc, want_flags=True, want_alpha=True)
    m = flags >> 3
    assert np.all((m >= 4) & (m <= 10))
    assert np.all(flags & 7 != 0)
    assert flags.size == oracle.flag_count(2, P.n) == 4 * 2 * (21 * 20) * 2
    R2 = oracle.euler_rhs(P.U0, P.n, P.dx, P.bc, flags_in=flags)
    np.testing.assert_array_equal(R, R2)
    # alpha: acoustic speeds bound the convective one
    assert np.all(alpha[:, 0] >= 0) and np.all(alpha[:, -1] >= alpha[:, 1])


# ---------------------------------------------------------------------------
# Reflecting walls (bc 2; the two-blast-wave test of Sec. 4.2, eq. 4.11)
# ---------------------------------------------------------------------------
def _blast_prims(x):
    """eq. 4.11 (middle range read as 0.1 <= x < 0.9): at rest, p = 1000 / 0.01 / 100."""
    p = np.where(x < 0.1, 1000.0, np.where(x < 0.9, 0.01, 100.0))
    return np.ones_like(x), np.zeros_like(x), p


def test_reflecting_constant_state_at_rest_is_steady(oracle):
    n = 23
    U = inputs.prim_to_cons(np.full(n, 1.3), [np.zeros(n)], np.full(n, 0.7))
    R = oracle.euler_rhs(U, (n,), (1.0 / n,), (2,))
    assert np.all(R == 0.0)


@pytest.mark.parametrize("n", [5, 40])
def test_reflecting_equals_mirrored_periodic(oracle, n):
    """Data at rest on [0, 1] with reflecting walls, and the doubled periodic
    domain [-1, 1] holding the data and its mirror image (velocity reversed):
    every stencil sees the same values, and at rest the LF speeds agree, so the
    right-hand sides on [0, 1] are equal bit for bit."""
    x = (np.arange(n) + 0.5) / n
    rho, u, p = _blast_prims(x)
    p = p * (1.0 + 0.1 * np.sin(7.0 * x))            # break the piecewise constancy
    U = inputs.prim_to_cons(rho, [u], p)
    Ud = np.concatenate([U[:, ::-1] * np.array([[1.0], [-1.0], [1.0]]), U], axis=1)
    R = oracle.euler_rhs(U, (n,), (1.0 / n,), (2,))
    Rd = oracle.euler_rhs(np.ascontiguousarray(Ud), (2 * n,), (1.0 / n,), (0,))
    np.testing.assert_array_equal(R, Rd[:, n:])


def test_reflecting_in_x_periodic_in_y_equals_1d(oracle):
    """A 2D grid varying along x only, reflecting in x and periodic in y, gives
    the 1D reflecting right-hand side in every row (and zero y-momentum)."""
    n, m = 30, 4
    x = (np.arange(n) + 0.5) / n
    rho, u, p = _blast_prims(x)
    rho = rho + 0.2 * np.cos(3.0 * x)
    u = 0.3 * np.sin(5.0 * x)
    U1 = inputs.prim_to_cons(rho, [u], p)
    U2 = inputs.prim_to_cons(np.tile(rho, (m, 1)), [np.tile(u, (m, 1)), np.zeros((m, n))], np.tile(p, (m, 1)))
    R1 = oracle.euler_rhs(U1, (n,), (1.0 / n,), (2,))
    R2 = oracle.euler_rhs(U2, (n, m), (1.0 / n, 0.25), (2, 0))
    for j in range(m):
        np.testing.assert_array_equal(R2[0][j], R1[0])
        np.testing.assert_array_equal(R2[1][j], R1[1])
        np.testing.assert_array_equal(R2[3][j], R1[2])
    assert np.all(R2[2] == 0.0)
