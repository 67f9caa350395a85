"""The closed form's fixed-point six-point sums (teno_fixsum.cuh) on the host,
against exact rational arithmetic (fractions.Fraction).

For every sum of six binary64 values x_j with the closed form's integer
weights (c = 1,-8,37,37,-8,1 and m = 1,-5,10,-10,5,-1, the fifth-order
upwind and downwind reconstructions of eq. 2.3 added and subtracted), the
device routine must return exactly the correctly rounded value of
sum_j w_j sign(x_j) trunc(|x_j| 2^(1075+3-E)) 2^(E-1075-3), E the largest
biased exponent, and so lie within sum_j |w_j| / 8 ulps of the largest
value (plus half an ulp of the result) of the exact sum; outside its stated
exponent range it must decline."""
import ctypes
import os
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2003_09145_gb300", "csrc")
C_W = (1, -8, 37, 37, -8, 1)
M_W = (1, -5, 10, -10, 5, -1)
GUARD = 3


@pytest.fixture(scope="module")
def lib():
    out = os.path.join(tempfile.mkdtemp(prefix="teno_fix_host_"), "libfix.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-ffp-contract=off", f"-I{CSRC}",
                           "-o", out, os.path.join(HERE, "fixsum_host.cpp")])
    L = ctypes.CDLL(out)
    L.fix_sum6_batch.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p]
    L.fix_sum6_batch.restype = None
    L.fix_sum7_batch.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.fix_sum7_batch.restype = None
    return L


def _run(lib, x, w):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 6)
    n = x.shape[0]
    wa = np.ascontiguousarray(w, dtype=np.int32)
    out = np.zeros(n)
    ok = np.zeros(n, dtype=np.int32)
    E = np.zeros(n, dtype=np.uint32)
    lib.fix_sum6_batch(n, x.ctypes.data, wa.ctypes.data, out.ctypes.data, ok.ctypes.data, E.ctypes.data)
    return out, ok.astype(bool), E.astype(np.int64)


def _biased_exponent(v):
    return (int(np.float64(v).view(np.uint64)) >> 52) & 0x7FF


def _spec(xs, w):
    """The stated result: each term truncated to the grid 2^(E-1075-G), the
    exact sum of the truncated terms rounded once (Python's int / int true
    division rounds correctly)."""
    E = max(_biased_exponent(v) for v in xs)
    if E == 0:
        return 0.0, E
    scale = 1075 + GUARD - E
    A = 0
    for wj, v in zip(w, xs):
        A += wj * int(Fraction(float(v)) * (Fraction(2) ** scale))   # int() truncates toward zero
    if scale >= 0:
        return A / (1 << scale) if A else 0.0, E
    return float(A * (1 << -scale)), E


def _ulp(v):
    return float(np.spacing(np.float64(abs(v))))


def _check(lib, x, w):
    out, ok, E = _run(lib, x, w)
    x = np.asarray(x, dtype=np.float64).reshape(-1, 6)
    for i in range(x.shape[0]):
        assert ok[i]
        want, e = _spec(x[i], w)
        assert E[i] == e
        assert out[i] == want or (out[i] == 0.0 and want == 0.0), (x[i], out[i], want)
        exact = sum(Fraction(wj) * Fraction(float(v)) for wj, v in zip(w, x[i]))
        mx = float(np.max(np.abs(x[i])))
        bound = Fraction(sum(abs(wj) for wj in w), 8) * Fraction(_ulp(mx)) + Fraction(_ulp(out[i])) / 2
        assert abs(Fraction(float(out[i])) - exact) <= bound
    return out


@pytest.mark.parametrize("w", [C_W, M_W])
def test_random_magnitudes_against_exact(lib, w):
    rng = np.random.default_rng(11)
    n = 3000
    mant = rng.uniform(-1.0, 1.0, (n, 6))
    # per sum a common scale, per value a spread of up to 2^+-40 around it
    scale = np.exp2(rng.integers(-300, 300, (n, 1)).astype(np.float64))
    spread = np.exp2(rng.integers(-40, 41, (n, 6)).astype(np.float64))
    x = mant * scale * spread
    x[rng.random((n, 6)) < 0.05] = 0.0
    _check(lib, x, w)


@pytest.mark.parametrize("w", [C_W, M_W])
def test_smooth_stencils_cancel_like_the_flux(lib, w):
    """Six samples of a smooth field: the m-sum is a fifth difference, far
    below the values (the regime where a binary64 chain loses most)."""
    rng = np.random.default_rng(12)
    n = 2000
    x0 = rng.uniform(0.5, 2.0, (n, 1)) * np.exp2(rng.integers(-20, 20, (n, 1)))
    h = rng.uniform(1e-4, 1e-1, (n, 1))
    k = np.arange(6)[None, :]
    x = x0 * (1.0 + 0.3 * np.sin(h * k + rng.uniform(0, 6.3, (n, 1))))
    _check(lib, x, w)


def test_integer_data_is_exact(lib):
    """Integers of up to 50 bits lie on the grid (G = 3 guard bits below the
    largest value's ulp), so the sum is the correctly rounded exact sum."""
    rng = np.random.default_rng(13)
    x = rng.integers(-(2 ** 50), 2 ** 50, (500, 6)).astype(np.float64)
    out, ok, _ = _run(lib, x, C_W)
    assert ok.all()
    for i in range(x.shape[0]):
        exact = sum(int(wj) * int(v) for wj, v in zip(C_W, x[i]))
        assert out[i] == float(exact)


def test_ties_round_to_even(lib):
    """Sums that land exactly halfway between two binary64 values round to the
    even one: 2^53 + 1 and 2^53 + 3 (exact integers on the grid)."""
    big = float(2 ** 52)
    # 2 (2^52) + 1 = 2^53 + 1 -> 2^53 (even); 2 (2^52) + 3 = 2^53 + 3 -> 2^53 + 4
    x = np.array([[big, 0.0, 0.0, big, 0.0, 1.0], [big, 0.0, 0.0, big, 0.0, 3.0]])
    w = (1, 0, 0, 1, 0, 1)
    out, ok, _ = _run(lib, x, w)
    assert ok.all()
    assert out[0] == float(2 ** 53) and out[1] == float(2 ** 53 + 4)


def test_signs_zeros_and_mirrors(lib):
    """Negating every value negates the sum; mirrored stencils with the
    mirrored weights give the same sum (the result is order-independent);
    all-zero stencils (either sign) give +0."""
    rng = np.random.default_rng(14)
    x = rng.standard_normal((400, 6)) * np.exp2(rng.integers(-60, 60, (400, 1)))
    a, _, _ = _run(lib, x, C_W)
    b, _, _ = _run(lib, -x, C_W)
    assert np.array_equal(a, -b)
    c, _, _ = _run(lib, x[:, ::-1], C_W[::-1])
    assert np.array_equal(a, c)
    z, ok, E = _run(lib, np.array([[0.0, -0.0, 0.0, 0.0, -0.0, 0.0]]), C_W)
    assert ok[0] and E[0] == 0 and z[0] == 0.0


def test_declines_outside_its_range(lib):
    """Largest exponents 1..63 (values below 2^-959), above 2030 (values from
    2^1008), infinities and NaN are left to the binary64 chain; a stencil of
    subnormals alone has E = 0 and sums to 0."""
    tiny = 2.0 ** -1000
    x = np.array([
        [tiny, 0, 0, 0, 0, 0],
        [2.0 ** 1010, 1, 0, 0, 0, 0],
        [np.inf, 1, 0, 0, 0, 0],
        [np.nan, 1, 0, 0, 0, 0],
        [2.0 ** -959, 1e-300, 0, 0, 0, 0],
        [5e-324, -5e-324, 0, 0, 0, 0],
        [2.0 ** 1007 * 1.9, 2.0 ** -900, 0, 0, 0, 0],
    ], dtype=np.float64)
    out, ok, E = _run(lib, x, C_W)
    assert list(ok) == [False, False, False, False, True, True, True]
    assert E[5] == 0 and out[5] == 0.0
    # at the ends of the range the spec still holds
    _check(lib, x[[4, 6]], C_W)


def test_matches_binary64_chain_on_flux_like_data(lib):
    """On values shaped like the Euler fluxes of a smooth flow the fixed-point
    sum and a binary64 chain of fused multiply-adds agree to the chain's
    rounding (a few tens of ulps of the largest value)."""
    rng = np.random.default_rng(15)
    n = 2000
    x = rng.uniform(0.8, 1.2, (n, 6)) * np.exp2(rng.integers(-5, 20, (n, 1)))
    out, ok, _ = _run(lib, x, C_W)
    assert ok.all()
    chain = x[:, 0].copy()
    for j in range(1, 5):
        chain = chain + C_W[j] * x[:, j]
    chain = chain + x[:, 5]
    mx = np.max(np.abs(x), axis=1)
    assert np.all(np.abs(out - chain) <= 256 * np.spacing(mx))


# the adjoint gather's sums: the antisymmetric stencil on Rbar (weights
# 1, -1, -9, 9, 45, -45: sum |w| = 110) and the M-weighted slot sum with the
# periodic face's second copy as a seventh term
@pytest.mark.parametrize("w", [(1, -1, -9, 9, 45, -45, 0), (1, -5, 10, -10, 5, -1, 10), (1, -5, 10, -10, 5, -1, 0)])
def test_seven_term_sums_against_exact(lib, w):
    rng = np.random.default_rng(16)
    n = 2000
    x = rng.standard_normal((n, 7)) * np.exp2(rng.integers(-200, 200, (n, 1)).astype(np.float64))
    x *= np.exp2(rng.integers(-30, 31, (n, 7)).astype(np.float64))
    x[rng.random((n, 7)) < 0.05] = 0.0
    out = np.zeros(n)
    ok = np.zeros(n, dtype=np.int32)
    wa = np.ascontiguousarray(w, dtype=np.int32)
    lib.fix_sum7_batch(n, np.ascontiguousarray(x).ctypes.data, wa.ctypes.data, out.ctypes.data, ok.ctypes.data)
    assert ok.all()
    for i in range(n):
        want, _ = _spec(x[i], w)
        assert out[i] == want, (x[i], out[i], want)
        exact = sum(Fraction(wj) * Fraction(float(v)) for wj, v in zip(w, x[i]))
        mx = float(np.max(np.abs(x[i])))
        bound = Fraction(sum(abs(wj) for wj in w), 8) * Fraction(_ulp(mx)) + Fraction(_ulp(out[i])) / 2
        assert abs(Fraction(float(out[i])) - exact) <= bound
    # declines on NaN and on values out of range
    bad = np.zeros((2, 7))
    bad[0, 3] = np.nan
    bad[1, 0] = 2.0 ** 1010
    lib.fix_sum7_batch(2, np.ascontiguousarray(bad).ctypes.data, wa.ctypes.data, out.ctypes.data, ok.ctypes.data)
    assert not ok[:2].any()

