"""The certified FP32 keep-all tests (teno_cert.cuh) on the host, against
exact rational arithmetic.

The flux passes ask FP32 whether the binary64 evaluation of the cutoff
(eq. 2.9-2.14 with C_T from eq. 3.1-3.4) keeps every stencil; a pass must
imply, for the exact values the FP32 inputs approximate, that
tau_5 <= thr * (min_k beta_k + eps) with the 1e-5 margin the binary64
evaluations need (thr: the threshold below which every chi_k >= C_T).
The device code is compiled here for the host with -ffp-contract=off, so it
rounds as on the GPU (every FP32 operation is written with explicit
rounding).  Inputs are chosen to sit at the threshold: five-point lines and
six-cell Euler interface stencils scaled so that the exact tau/dmin is
thr (1 +- 1e-3 ... 1e-7), at magnitudes 1e-8 ... 1e8, with mantissas the
20-bit truncation treats worst and sub-truncation perturbations of large
values.  Every certified case is checked exactly (fractions.Fraction)."""
import ctypes
import os
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2003_09145_gb300", "csrc")
GAMMA = 1.4
MARGIN = 1 - Fraction(9, 10**6)


@pytest.fixture(scope="module")
def lib():
    out = os.path.join(tempfile.mkdtemp(prefix="teno_cert_host_"), "libcert.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-ffp-contract=off", f"-I{CSRC}",
                           "-o", out, os.path.join(HERE, "cert_host.cpp")])
    L = ctypes.CDLL(out)
    P = ctypes.POINTER(ctypes.c_double)
    L.cert_values_batch.argtypes = [ctypes.c_int64, P, ctypes.c_float, ctypes.c_float,
                                    ctypes.POINTER(ctypes.c_int)]
    L.cert_floats.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.c_float, ctypes.c_float, ctypes.c_float]
    L.cert_floats.restype = ctypes.c_int
    L.cert_hi_float.argtypes = [ctypes.c_double]
    L.cert_hi_float.restype = ctypes.c_float
    L.cert_interface_batch.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, P, P, P, P, P, P, P, P,
                                       ctypes.c_float, ctypes.c_float, ctypes.POINTER(ctypes.c_int)]
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _down(x):
    """binary32 value below x, as the library rounds the test's constants."""
    f = np.float32(x)
    while float(f) > x:
        f = np.nextafter(f, np.float32(0))
    return np.nextafter(f, np.float32(0))


def scheme_thresholds(H=10.0, eps=1e-6, b_l=4, b_u=10):
    """(thr_keep as binary64, its FP32 rounding, 4 eps rounded down): the
    largest m-threshold whose m range keeps every stencil by the bound
    chi_k >= 1/(3 (1 + max chi~)^6) > C_T (eq. 2.13-2.14, 3.1-3.2)."""
    K = b_u - b_l
    thr = [H * (K / j - 1.0) for j in range(1, K)] + [H * 2.0**-53]
    keep = []
    for c in range(1, K + 1):
        x = 1.0 + thr[c - 1]
        keep.append(3.0 * x**6 * 10.0 ** -(b_l + c) <= 1.0 - 1e-9)
    idx = next(c for c in range(K) if all(keep[c:]) and keep[c])
    return thr[idx], _down(thr[idx]), _down(4.0 * eps)


def exact_keep(v, thr_f, eps):
    """tau_5 <= thr (min beta_k + eps) (1 - 9e-6) in exact arithmetic, the
    indicators of eq. 2.9-2.12 scaled by 4 (eps by 4 alike)."""
    x = [Fraction(a) for a in v]
    e = [x[k + 1] - x[k] for k in range(4)]
    a = [e[1] - e[0], e[2] - e[1], e[3] - e[2]]
    c = [3 * e[1] - e[0], e[1] + e[2], e[3] - 3 * e[2]]
    b = [Fraction(13, 3) * a[k] ** 2 + c[k] ** 2 for k in range(3)]
    tau = abs(b[2] - b[0])
    return tau <= Fraction(float(thr_f)) * (min(b) + 4 * Fraction(eps)) * MARGIN


def _ratio(v, eps):
    v = np.asarray(v, dtype=np.float64)
    e = np.diff(v, axis=-1)
    a = e[..., 1:] - e[..., :-1]
    c = np.stack([3 * e[..., 1] - e[..., 0], e[..., 1] + e[..., 2], e[..., 3] - 3 * e[..., 2]], -1)
    b = 13.0 / 3.0 * a * a + c * c
    return np.abs(b[..., 2] - b[..., 0]) / (b.min(-1) + 4 * eps)


def _scale_to(shape, offset, target, eps, lo=1e-12, hi=1e12):
    """lambda with ratio(offset + lambda shape) ~ target (bisection in log)."""
    for _ in range(90):
        mid = np.sqrt(lo * hi)
        if _ratio(offset + mid * shape, eps) < target:
            lo = mid
        else:
            hi = mid
    return np.sqrt(lo * hi)


def _value_cases(rng, thr, eps, n):
    cases = []
    rel = [1e-3, 1e-4, 1e-5, 1e-6, 1e-7]
    for i in range(n):
        kind = i % 4
        shape = rng.standard_normal(5)
        if kind == 1:   # smooth line plus a small kink
            t = np.arange(5.0)
            shape = rng.standard_normal() * t + 0.1 * rng.standard_normal() * t * t + 1e-3 * rng.standard_normal(5)
        mag = 10.0 ** rng.uniform(-8, 8)
        if kind == 2:   # a mantissa that the 20-bit truncation cuts the most
            e = np.floor(np.log2(mag))
            offset = 2.0**e * (2.0 - 2.0**-20 + 2.0**-30 * rng.uniform())
        elif kind == 3:
            offset = 0.0
        else:
            offset = mag * rng.choice([-1.0, 1.0])
        target = thr * (1.0 + rng.choice([-1.0, 1.0]) * rng.choice(rel)) if i % 3 else thr * rng.uniform(0.2, 1.5)
        lam = _scale_to(shape, offset, target, eps)
        cases.append(offset + lam * shape)
    # sub-truncation perturbations of large values: all five fall in one or
    # two 2^-20 buckets
    for i in range(n // 4):
        M = 10.0 ** rng.uniform(2, 9) * rng.choice([-1.0, 1.0])
        cases.append(M * (1.0 + 2.0**-20 * rng.uniform(-2, 2, 5)))
        cases.append(np.array([M, M + 0.05, M + 0.05, M + 0.05, M + 0.05]) * (abs(M) / 1e5))
    return np.array(cases)


@pytest.mark.parametrize("params", [dict(), dict(H=1.0), dict(H=100.0, eps=1e-8), dict(b_l=3, b_u=12)])
def test_values_certificate_sound(lib, params):
    eps = params.get("eps", 1e-6)
    thr, thr_f, eps4_f = scheme_thresholds(**params)
    rng = np.random.default_rng(7)
    V = np.ascontiguousarray(_value_cases(rng, thr, eps, 2400))
    out = np.zeros(len(V), dtype=np.int32)
    lib.cert_values_batch(len(V), _p(V), thr_f, eps4_f, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    cert = np.flatnonzero(out)
    bad = [i for i in cert if not exact_keep(V[i], thr_f, eps)]
    assert not bad, f"certified but not kept exactly: {V[bad[0]].tolist()}"
    # not vacuous: the test certifies cases a little below the threshold
    r = _ratio(V, eps)
    near = (r < thr * (1 - 1e-3)) & (r > thr * 0.5)
    assert np.count_nonzero(out[near]) > 0.3 * np.count_nonzero(near)


def test_values_large_magnitude_regression(lib):
    # five values inside one 2^-20 truncation bucket of 1e5: the exact
    # tau/dmin is in the thousands (stencil 0 is cut); no keep-all certificate
    thr, thr_f, eps4_f = scheme_thresholds()
    v = np.array([[1e5, 1e5 + 0.05, 1e5 + 0.05, 1e5 + 0.05, 1e5 + 0.05]])
    assert not exact_keep(v[0], thr_f, 1e-6)
    out = np.zeros(1, dtype=np.int32)
    lib.cert_values_batch(1, _p(v), thr_f, eps4_f, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    assert out[0] == 0


def test_hi_float_truncation(lib):
    rng = np.random.default_rng(3)
    x = np.concatenate([10.0 ** rng.uniform(-37, 38, 2000) * rng.choice([-1, 1], 2000),
                        [1.0, -1.0, 2.0**-126, 3.0e38, 2.0 - 2.0**-40]])
    for v in x:
        f = float(lib.cert_hi_float(float(v)))
        assert abs(f) <= abs(v) and abs(f - v) <= 2.0**-20 * abs(v), (v, f)
    for v in (0.0, 1e-300, -1e-45):
        assert abs(float(lib.cert_hi_float(v))) == 2.0**-126
    for v in (float("inf"), float("nan"), 1e300):
        f = float(lib.cert_hi_float(v))
        assert np.isfinite(f) and abs(f) > 3.4e38


# --------------------------------------------------------------------------
# Euler interfaces: cert_begin / cert_point / cert_keep
# --------------------------------------------------------------------------

def _roe(U2, U3, ndim, d):
    """A binary64 Roe state of two cells (the certificate's claim is about
    exact arithmetic on whatever binary64 state it is given)."""
    def prim(U):
        rho = U[0]
        u = U[1:1 + ndim] / rho
        p = (GAMMA - 1) * (U[-1] - 0.5 * rho * u @ u)
        return rho, u, p
    ra, ua, pa = prim(U2)
    rb, ub, pb = prim(U3)
    sa, sb = np.sqrt(ra), np.sqrt(rb)
    u = (sa * ua + sb * ub) / (sa + sb)
    H = ((U2[-1] + pa) / sa + (U3[-1] + pb) / sb) / (sa + sb)
    q2 = u @ u
    c2 = (GAMMA - 1) * (H - 0.5 * q2)
    c = np.sqrt(c2)
    hb1 = 0.5 * (GAMMA - 1) / c2
    return u, hb1, 0.5 * hb1 * q2, 0.5 / c


def _split_values_exact(Up, un, pn, u, hb1, hb2, hic, alpha, ndim, d):
    """The binary64 path's split characteristic values v+ (points 0..4) and
    v- (points 5..1) per field, in exact arithmetic: w = L U_j (Roe left
    eigenvectors), t = (p/2) z, v+ = (u_d/2 + alpha) w + t, v- = v+ - 2 alpha w."""
    F = Fraction
    nv = ndim + 2
    uu = [F(x) for x in u]
    hb1, hb2, hic = F(hb1), F(hb2), F(hic)
    b1 = 2 * hb1
    hud = uu[d] / 2
    al = [F(a) for a in alpha]
    vp = [[None] * nv for _ in range(6)]
    vm = [[None] * nv for _ in range(6)]
    for j in range(6):
        X = [F(x) for x in Up[j]]
        S = -X[nv - 1] + sum(uu[k] * X[1 + k] for k in range(ndim))
        A = hb2 * X[0] - hb1 * S
        B = (uu[d] * X[0] - X[1 + d]) * hic
        w = [A + B, X[0] - 2 * A] + [X[1 + t] - uu[t] * X[0] for t in range(ndim) if t != d] + [A - B]
        hu, hp = F(un[j]), F(pn[j])
        az = hp * (b1 * (hu - hud))
        bz = hp * hic
        t = [az - bz, -2 * az] + [F(0)] * (ndim - 1) + [az + bz]
        for f in range(nv):
            vp[j][f] = (hu + al[f]) * w[f] + t[f]
            vm[j][f] = vp[j][f] - 2 * al[f] * w[f]
    recs = []
    for f in range(nv):
        recs.append([vp[j][f] for j in range(5)])
        recs.append([vm[j][f] for j in (5, 4, 3, 2, 1)])
    return recs


def _interface_case(rng, ndim, d, lam, base, pert, scale):
    nv = ndim + 2
    rho = base[0] * (1 + lam * pert[:, 0])
    vel = base[1] + lam * pert[:, 1:1 + ndim]
    p = base[2] * (1 + lam * pert[:, -1])
    rho, p = rho * scale[0], p * scale[1]
    vel = vel * np.sqrt(scale[1] / scale[0])
    U = np.zeros((6, nv))
    U[:, 0] = rho
    U[:, 1:1 + ndim] = rho[:, None] * vel
    U[:, -1] = p / (GAMMA - 1) + 0.5 * rho * (vel * vel).sum(1)
    un = 0.5 * (U[:, 1 + d] / U[:, 0])
    pn = 0.5 * ((GAMMA - 1) * (U[:, -1] - 0.5 * (U[:, 1:1 + ndim] ** 2).sum(1) / U[:, 0]))
    u, hb1, hb2, hic = _roe(U[2], U[3], ndim, d)
    cs = np.sqrt(GAMMA * 2 * pn / U[:, 0])
    a_ac = 0.5 * np.max(np.abs(2 * un) + cs) * (1 + 0.1 * rng.uniform())
    a_mid = 0.5 * np.max(np.abs(2 * un)) * (1 + 0.1 * rng.uniform())
    alpha = np.array([a_ac] + [a_mid] * ndim + [a_ac])
    return U, un, pn, u, hb1, hb2, hic, alpha


def _max_ratio_float(case, ndim, d, eps):
    U, un, pn, u, hb1, hb2, hic, alpha = case
    recs = _split_values_exact(U, un, pn, u, hb1, hb2, hic, alpha, ndim, d)
    return max(_ratio(np.array([float(x) for x in r]), eps) for r in recs)


@pytest.mark.parametrize("ndim,d", [(1, 0), (3, 0), (3, 1), (3, 2), (2, 1)])
def test_interface_certificate_sound(lib, ndim, d):
    eps = 1e-6
    thr, thr_f, eps4_f = scheme_thresholds()
    rng = np.random.default_rng(100 + 10 * ndim + d)
    cases = []
    for i in range(60):
        # a third of the cases ride on a hypersonic mean flow (Mach up to
        # 20): the projections then cancel heavily, so the truncation and
        # rounding bounds of cert_point decide the outcome
        vmax = 20.0 if i % 3 == 2 else 0.8
        base = (rng.uniform(0.5, 2.0), rng.uniform(-vmax, vmax, ndim), rng.uniform(0.5, 2.0))
        pert = rng.standard_normal((6, ndim + 2))
        if i % 2:
            t = np.arange(6.0)[:, None]
            pert = rng.standard_normal((1, ndim + 2)) * t + 0.2 * rng.standard_normal((1, ndim + 2)) * t * t
        pert = pert / np.abs(pert).max()   # states stay physical for lambda < 1/2
        scale = (10.0 ** rng.uniform(-4, 4), 10.0 ** rng.uniform(-4, 6))
        target = thr * (1 + rng.choice([-1.0, 1.0]) * 10.0 ** -rng.uniform(3, 7)) if i % 4 else thr * rng.uniform(0.3, 1.2)
        lo, hi = 1e-9, 0.45
        for _ in range(40):
            mid = np.sqrt(lo * hi)
            r = _max_ratio_float(_interface_case(np.random.default_rng(i), ndim, d, mid, base, pert, scale), ndim, d, eps)
            lo, hi = (mid, hi) if r < target else (lo, mid)
        cases.append(_interface_case(np.random.default_rng(i), ndim, d, lo, base, pert, scale))
    n = len(cases)
    nv = ndim + 2
    arr = [np.ascontiguousarray(np.array([c[k] for c in cases], dtype=np.float64)) for k in range(8)]
    out = np.zeros(n, dtype=np.int32)
    lib.cert_interface_batch(ndim, d, n, *[_p(a) for a in arr], thr_f, eps4_f,
                             out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    assert np.all(out >= 0)
    for i in np.flatnonzero(out):
        U, un, pn, u, hb1, hb2, hic, alpha = cases[i]
        for rec in _split_values_exact(U, un, pn, u, hb1, hb2, hic, alpha, ndim, d):
            x = rec
            e = [x[k + 1] - x[k] for k in range(4)]
            a = [e[1] - e[0], e[2] - e[1], e[3] - e[2]]
            c = [3 * e[1] - e[0], e[1] + e[2], e[3] - 3 * e[2]]
            b = [Fraction(13, 3) * a[k] ** 2 + c[k] ** 2 for k in range(3)]
            assert abs(b[2] - b[0]) <= Fraction(float(thr_f)) * (min(b) + 4 * Fraction(eps)) * MARGIN, (ndim, d, i)
    assert np.count_nonzero(out) >= 5, "the certificate passed too few cases to test anything"
    assert nv == arr[0].shape[2]
