"""The adjoint core's two interface VJPs on the host (no GPU): the all-kept
closed form (interface_vjp_kept, the one the adjoint kernels use where every
stencil is kept) against the general frozen-selection VJP (interface_vjp)
with every stencil selected -- two independent derivations of the same
derivative -- and the closed form against central differences of the
flux restated here from the paper's linear weights (eq. 2.3) and Roe
eigensystem; and the per-cell flux Jacobian transpose against central
differences of eq. 4.7."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2003_09145_gb300", "csrc")
GAMMA = 1.4


@pytest.fixture(scope="module")
def lib():
    out = os.path.join(tempfile.mkdtemp(prefix="teno_adj_host_"), "libadj.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-ffp-contract=off", f"-I{CSRC}",
                           "-o", out, os.path.join(HERE, "adjoint_core_host.cpp")])
    L = ctypes.CDLL(out)
    P = ctypes.POINTER(ctypes.c_double)
    L.adj_interface_vjp3.argtypes = [ctypes.c_int, ctypes.c_int, P, P, ctypes.c_double, P, P, P]
    L.adj_interface_vjp3.restype = None
    L.adj_flux_vjp3.argtypes = [ctypes.c_int, P, ctypes.c_double, P, P]
    L.adj_flux_vjp3.restype = None
    L.adj_flux_vjp_acc3.argtypes = [ctypes.c_int, P, ctypes.c_double, P, P]
    L.adj_flux_vjp_acc3.restype = None
    L.adj_interface_vjp3_sel.argtypes = [ctypes.c_int, ctypes.c_int, P, P, ctypes.POINTER(ctypes.c_uint),
                                         ctypes.c_double, P, P, P]
    L.adj_interface_vjp3_sel.restype = None
    L.adj_kept_scaled3.argtypes = [ctypes.c_int, P, P, ctypes.c_double, P, ctypes.c_double, ctypes.c_double, P, P]
    L.adj_kept_scaled3.restype = None
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vjp(lib, d, kept, Up, alpha, Fb):
    Up = np.ascontiguousarray(Up, dtype=np.float64)
    ub = np.zeros((6, 5))
    ab = np.zeros(5)
    lib.adj_interface_vjp3(d, kept, _p(Up), _p(np.ascontiguousarray(alpha)), GAMMA, _p(np.ascontiguousarray(Fb)),
                           _p(ub), _p(ab))
    return ub, ab


def _state(rng):
    rho = rng.uniform(0.5, 2.0, 6)
    u = rng.uniform(-0.8, 0.8, (6, 3))
    p = rng.uniform(0.5, 2.0, 6)
    U = np.zeros((6, 5))
    U[:, 0] = rho
    U[:, 1:4] = rho[:, None] * u
    U[:, 4] = p / (GAMMA - 1) + 0.5 * rho * (u * u).sum(1)
    return U


def _closed_flux(Up, alpha, d):
    """F^ of one interface with every stencil kept (eq. 2.3 linear weights):
    R [ L sum_j P_j F_j + diag(alpha) L sum_j M_j U_j ] with the Roe
    eigensystem of points 2 and 3; written with explicit L and R matrices."""
    P = np.array([1, -8, 37, 37, -8, 1]) / 60.0
    M = np.array([1, -5, 10, -10, 5, -1]) / 60.0

    def flux(U):
        rho, m, E = U[0], U[1:4], U[4]
        u = m / rho
        p = (GAMMA - 1) * (E - 0.5 * rho * u @ u)
        F = u[d] * U
        F[1 + d] += p
        F[4] += p * u[d]
        return F

    def prim(U):
        rho, m, E = U[0], U[1:4], U[4]
        u = m / rho
        p = (GAMMA - 1) * (E - 0.5 * rho * u @ u)
        return rho, u, (E + p) / rho

    ra, ua, Ha = prim(Up[2])
    rb, ub, Hb = prim(Up[3])
    sa, sb = np.sqrt(ra), np.sqrt(rb)
    u = (sa * ua + sb * ub) / (sa + sb)
    H = (sa * Ha + sb * Hb) / (sa + sb)
    q = u @ u
    c = np.sqrt((GAMMA - 1) * (H - 0.5 * q))
    t = [k for k in range(3) if k != d]
    Rm = np.zeros((5, 5))
    Rm[:, 0] = [1, *(u - c * np.eye(3)[d]), H - u[d] * c]
    Rm[:, 1] = [1, *u, 0.5 * q]
    for f, k in enumerate(t):
        Rm[:, 2 + f] = [0, *np.eye(3)[k], u[k]]
    Rm[:, 4] = [1, *(u + c * np.eye(3)[d]), H + u[d] * c]
    Lm = np.linalg.inv(Rm)
    Ft = sum(P[j] * flux(Up[j]) for j in range(6))
    Ut = sum(M[j] * Up[j] for j in range(6))
    return Rm @ (Lm @ Ft + alpha * (Lm @ Ut))


@pytest.mark.parametrize("d", [0, 1, 2])
def test_kept_closed_form_equals_general_vjp(lib, d):
    rng = np.random.default_rng(100 + d)
    for _ in range(20):
        Up = _state(rng)
        a0, am, aE = rng.uniform(0.5, 3.0, 3)
        alpha = np.array([a0, am, am, am, aE])
        Fb = rng.standard_normal(5)
        ub_k, ab_k = _vjp(lib, d, 1, Up, alpha, Fb)
        ub_g, ab_g = _vjp(lib, d, 0, Up, alpha, Fb)
        scale = np.abs(ub_g).max()
        assert np.abs(ub_k - ub_g).max() <= 1e-12 * scale
        # the kept form lumps the middle speeds' derivative into entry 1
        lumped = ab_g.copy()
        lumped[1] = ab_g[1:4].sum()
        lumped[2:4] = 0.0
        assert np.abs(ab_k - lumped).max() <= 1e-12 * np.abs(ab_g).max()


@pytest.mark.parametrize("d", [0, 1, 2])
def test_split_kept_form_equals_general_vjp(lib, d):
    """The all-kept VJP as the kernels assemble it -- the kept pass's
    interface part with the adjoints of the two Roe cells' parameters, then
    per point the gather's maps (A(U_j)^T P_j Fbar, M_j U~bar, the Roe
    parameters' map at points 2 and 3) -- against the general VJP."""
    rng = np.random.default_rng(400 + d)
    for _ in range(20):
        Up = _state(rng)
        a0, am, aE = rng.uniform(0.5, 3.0, 3)
        alpha = np.array([a0, am, am, am, aE])
        Fb = rng.standard_normal(5)
        ub_s, ab_s = _vjp(lib, d, 2, Up, alpha, Fb)
        ub_k, ab_k = _vjp(lib, d, 1, Up, alpha, Fb)
        ub_g, _ = _vjp(lib, d, 0, Up, alpha, Fb)
        assert np.abs(ub_s - ub_g).max() <= 1e-12 * np.abs(ub_g).max()
        assert np.array_equal(ab_s, ab_k)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_general_vjp_without_flux_term(lib, d):
    """The pending interfaces' contributions leave out P_j A(U_j)^T Fbar (the
    gather adds it for every interface through one stencil): with any
    selections, the reduced VJP plus that term (A^T from flux_vjp) is the
    whole VJP."""
    rng = np.random.default_rng(500 + d)
    P = np.array([1, -8, 37, 37, -8, 1]) / 60.0
    for _ in range(20):
        Up = np.ascontiguousarray(_state(rng))
        alpha = np.ascontiguousarray(rng.uniform(0.5, 3.0, 5))
        Fb = np.ascontiguousarray(rng.standard_normal(5))
        sel = np.ascontiguousarray(rng.integers(1, 8, (5, 2)).astype(np.uint32))
        out = {}
        for excl in (0, 1):
            ub, ab = np.zeros((6, 5)), np.zeros(5)
            lib.adj_interface_vjp3_sel(d, excl, _p(Up), _p(alpha), sel.ctypes.data_as(ctypes.POINTER(ctypes.c_uint)),
                                       GAMMA, _p(Fb), _p(ub), _p(ab))
            out[excl] = (ub, ab)
        back = out[1][0].copy()
        for j in range(6):
            AF = np.zeros(5)
            lib.adj_flux_vjp3(d, _p(np.ascontiguousarray(Up[j])), GAMMA, _p(np.ascontiguousarray(P[j] * Fb)), _p(AF))
            back[j] += AF
        assert np.abs(back - out[0][0]).max() <= 1e-12 * np.abs(out[0][0]).max()
        assert np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("d", [0, 1, 2])
def test_kept_scaled_form(lib, d):
    """The kept pass feeds the interface VJP 60 U~ (integer weights) and Fbar
    without its factor scale / dx, carried by the speeds instead: U~bar and
    the Roe-parameter adjoints come out unchanged, d/dalpha times s / f."""
    rng = np.random.default_rng(600 + d)
    for _ in range(20):
        Up = np.ascontiguousarray(_state(rng))
        a0, am, aE = rng.uniform(0.5, 3.0, 3)
        alpha = np.array([a0, am, am, am, aE])
        Fb = np.ascontiguousarray(rng.standard_normal(5))
        s, f = 60.0, float(rng.uniform(0.01, 100.0))
        plain, scaled = np.zeros((4, 5)), np.zeros((4, 5))
        lib.adj_kept_scaled3(d, _p(Up), _p(alpha), GAMMA, _p(Fb), s, f, _p(plain), _p(scaled))
        for r in range(3):
            assert np.abs(scaled[r] - plain[r]).max() <= 1e-12 * np.abs(plain[r]).max(), r
        assert np.abs(scaled[3] * f / s - plain[3]).max() <= 1e-12 * np.abs(plain[3]).max()


@pytest.mark.parametrize("d", [0, 1, 2])
def test_kept_vjp_matches_central_differences(lib, d):
    rng = np.random.default_rng(200 + d)
    Up = _state(rng)
    alpha = np.array([2.1, 0.7, 0.7, 0.7, 2.4])
    Fb = rng.standard_normal(5)
    ub, _ = _vjp(lib, d, 1, Up, alpha, Fb)
    h = 1e-6
    for j in range(6):
        for v in range(5):
            Pp, Pm = Up.copy(), Up.copy()
            Pp[j, v] += h
            Pm[j, v] -= h
            fd = Fb @ (_closed_flux(Pp, alpha, d) - _closed_flux(Pm, alpha, d)) / (2 * h)
            assert abs(ub[j, v] - fd) <= 1e-7 * max(1.0, abs(fd)), (j, v)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_flux_jacobian_transpose_matches_central_differences(lib, d):
    """flux_vjp = A(U)^T G with A = dF_d/dU (eq. 4.7), the per-cell product
    the adjoint gather applies once per cell."""
    rng = np.random.default_rng(300 + d)

    def flux(U):
        rho, m, E = U[0], U[1:4], U[4]
        u = m / rho
        p = (GAMMA - 1) * (E - 0.5 * rho * u @ u)
        F = u[d] * U
        F[1 + d] += p
        F[4] += p * u[d]
        return F

    for _ in range(5):
        U = _state(rng)[0]
        G = rng.standard_normal(5)
        out = np.zeros(5)
        lib.adj_flux_vjp3(d, _p(np.ascontiguousarray(U)), GAMMA, _p(np.ascontiguousarray(G)), _p(out))
        h = 1e-6
        for v in range(5):
            Up, Um = U.copy(), U.copy()
            Up[v] += h
            Um[v] -= h
            fd = G @ (flux(Up) - flux(Um)) / (2 * h)
            assert abs(out[v] - fd) <= 1e-7 * max(1.0, abs(fd)), v
        # the gather's form: acc += A(U)^T G through the cell's shared primitives
        acc0 = rng.standard_normal(5)
        acc = acc0.copy()
        lib.adj_flux_vjp_acc3(d, _p(np.ascontiguousarray(U)), GAMMA, _p(np.ascontiguousarray(G)), _p(acc))
        assert np.abs((acc - acc0) - out).max() <= 1e-13 * max(1.0, np.abs(out).max())
