"""Pins of the oracle's comparison schemes: TENO5 with a fixed C_T (Sec. 2;
Sec. 4 uses 1e-7), TENO5-A (eq. 2.16-2.18) and WENO-Z (tau_5 of eq. 2.12).

* TENO5 with C_T = 10^-7 is the LAD reconstruction with B_l = 7, B_u = 8: m
  is then 7 except where theta == 1 exactly, where tau_5 = 0 and every
  stencil is kept under both (eq. 3.1-3.2), so f^ and delta agree bit for bit.
* TENO5-A: hand-derived worked examples (tests/golden); C_T stays inside
  [1e-10, 1e-7] (Sec. 2); smooth data give C_T = 1e-10, a step 1e-7.
* WENO-Z: with tau_5 = 0 the weights are the linear ones exactly (eq. 2.3);
  at a step the smooth candidate takes the weight (ENO property); fifth
  order on the smooth advection test of Sec. 4.1.
* All three keep every stencil (or, WENO-Z, converge) on Tab. 1's smooth
  profile: the TENO columns equal Upwind5 there (reading C1)."""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_teno5_fixed_equals_lad_with_one_magnitude(oracle):
    rng = np.random.default_rng(11)
    fixed = oracle.Params(scheme="teno5", ct_m=7)
    lad = oracle.Params(b_l=7, b_u=8)
    n_cut = 0
    for i in range(3000):
        v = rng.standard_normal(5) * 10.0 ** rng.uniform(-4, 1)
        if i % 3 == 0:
            v[rng.integers(0, 5):] += rng.uniform(0.1, 3.0)       # a jump
        f1, fl1, d1 = oracle.teno5_lad(v, fixed)
        f2, fl2, _ = oracle.teno5_lad(v, lad)
        assert f1 == f2 and (fl1 & 7) == (fl2 & 7)
        assert fl1 >> 3 == 7 and d1["CT"] == 1e-7
        n_cut += (fl1 & 7) != 7
    assert n_cut > 300


@pytest.mark.parametrize("ct_m", [5, 6, 7, 9])
def test_teno5_fixed_cutoff_definition(oracle, ct_m):
    """delta_k = [chi_k >= 10^-ct_m] with chi of eq. 2.8 / 2.13, recomputed
    here from the diagnostic indicators."""
    rng = np.random.default_rng(ct_m)
    P = oracle.Params(scheme="teno5", ct_m=ct_m)
    for _ in range(500):
        v = rng.standard_normal(5) * 10.0 ** rng.uniform(-3, 1)
        _, fl, dg = oracle.teno5_lad(v, P)
        b = [dg[f"beta{k}"] for k in range(3)]
        tau = abs(b[2] - b[0])
        g = [(1 + tau / (bk + P.eps)) ** 6 for bk in b]
        chi = [gk / sum(g) for gk in g]
        for k in range(3):
            if abs(chi[k] - 10.0 ** -ct_m) > 1e-9 * 10.0 ** -ct_m:
                assert ((fl >> k) & 1) == (chi[k] >= 10.0 ** -ct_m)


def _golden_teno5a():
    rows = []
    with open(os.path.join(GOLDEN, "teno5a_worked_examples.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            cols = [c.split() for c in line.split("|")]
            rows.append(([float(x) for x in cols[0]],) + tuple(float(c[0]) for c in cols[1:]))
    return rows


@pytest.mark.parametrize("row", _golden_teno5a())
def test_teno5a_worked_examples(oracle, row):
    v, eta, mA, g, betaA, m = row
    _, fl, dg = oracle.teno5_lad(v, oracle.Params(scheme="teno5a"))
    assert dg["eta"] == pytest.approx(eta, rel=1e-9)
    assert dg["mA"] == pytest.approx(mA, rel=1e-9, abs=1e-15)
    assert dg["gA"] == pytest.approx(g, rel=1e-9, abs=1e-15)
    assert dg["betaA"] == pytest.approx(betaA, rel=1e-12)
    assert fl >> 3 == int(m) == dg["m"]
    assert dg["CT"] == 10.0 ** -int(m)


def test_teno5a_cutoff_range_and_limits(oracle):
    """C_T = 10^-floor(beta) stays in [1e-10, 1e-7] (Sec. 2): g(0) = 1 gives
    beta = alpha_1 = 10.5, g(1) = 0 gives alpha_1 - alpha_2 = 7."""
    rng = np.random.default_rng(5)
    P = oracle.Params(scheme="teno5a")
    seen = set()
    for i in range(4000):
        v = rng.standard_normal(5) * 10.0 ** rng.uniform(-6, 2)
        if i % 4 == 0:
            v = np.sin(0.3 * np.arange(5) + rng.uniform(0, 6)) * rng.uniform(0.1, 10)
        _, fl, dg = oracle.teno5_lad(v, P)
        m = fl >> 3
        assert 7 <= m <= 10 and 1e-10 <= dg["CT"] <= 1e-7
        assert 0.0 <= dg["mA"] <= 1.0 and 0.0 <= dg["gA"] <= 1.0
        seen.add(m)
    assert seen == {7, 8, 9, 10}


def test_wenoz_linear_weights_when_tau_vanishes(oracle):
    P = oracle.Params(scheme="wenoz")
    for v in ([0.0, 1.0, 2.0, 3.0, 4.0], [2.0, 2.0, 2.0, 2.0, 2.0], [-3.0, -1.0, 1.0, 3.0, 5.0]):
        f, fl, dg = oracle.teno5_lad(v, P)
        assert dg["tau"] == 0.0
        assert (dg["omega0"], dg["omega1"], dg["omega2"]) == (0.1, 0.6, 0.3)
        assert f == pytest.approx(oracle.upwind5(v), rel=0, abs=4e-16 * max(1.0, max(abs(x) for x in v)))
        assert fl == 7


def test_wenoz_step_takes_the_smooth_candidate(oracle):
    P = oracle.Params(scheme="wenoz")
    f, _, dg = oracle.teno5_lad([0.0, 0.0, 0.0, 1.0, 1.0], P)
    # beta = (0, 1/3, 5/6) unscaled, tau = 5/6: alpha_0 = 0.1 (1 + tau/eps) dominates
    assert dg["omega0"] > 1 - 1e-5 and abs(f) < 1e-5
    f, _, dg = oracle.teno5_lad([0.0, 0.0, 1.0, 1.0, 1.0], P)
    assert dg["omega2"] > 1 - 1e-5 and abs(f - 1.0) < 1e-5


def _scalar_l2(oracle, n, scheme):
    dx = 2.0 / n
    x = -1.0 + dx * np.arange(n)
    u0 = np.sin(np.pi * x)
    dt = dx ** (5.0 / 3.0) / 8
    if scheme == "upwind":
        u, _ = oracle.scalar_run(u0, dx, 2.0, dt, "upwind")
    else:
        u, _ = oracle.scalar_run(u0, dx, 2.0, dt, "lad", oracle.Params(scheme=scheme))
    return math.sqrt(np.mean((u - u0) ** 2))


@pytest.mark.slow
def test_smooth_advection_orders(oracle):
    """Sec. 4.1 (eq. 4.5, t = 2): the TENO variants keep every stencil and
    reproduce Upwind5 (Tab. 1, reading C1); WENO-Z converges at fifth order
    (its critical points on sin are first order, where it keeps fifth)."""
    ns = [40, 80, 160]
    up = [_scalar_l2(oracle, n, "upwind") for n in ns]
    for sch in ("teno5", "teno5a"):
        e = [_scalar_l2(oracle, n, sch) for n in ns]
        np.testing.assert_allclose(e, up, rtol=1e-9, atol=1e-14)   # rounding of the two sums
    wz = [_scalar_l2(oracle, n, "wenoz") for n in ns]
    orders = [math.log2(wz[i] / wz[i + 1]) for i in range(len(ns) - 1)]
    assert min(orders) >= 4.7, orders
    assert all(w >= u * (1 - 1e-9) for w, u in zip(wz, up))
