"""Pins of three oracle functions that the other CPU tests leave loose.

* or_lf_alpha (the global Lax-Friedrichs speeds of Sec. 4, reading C7):
  against max |u_d - c|, max |u_d|, max |u_d + c| computed here from the
  primitive variables (eq. 4.7, c = sqrt(gamma p / rho)), on states where the
  three maxima are different numbers, per field and direction.
* or_euler_rhs_sample (the checker of the full-size GPU tests): equal bit
  for bit to or_euler_rhs at the sampled cells, for every boundary type and
  dimension, with flags_out, flags_in and alpha_in.
* or_euler_interface_diag (used to classify selector flips): its m and
  delta equal the flags of or_euler_rhs at the same interface, and its f^
  equals the scalar TENO5-LAD reconstruction of the split characteristic
  values formed here from the Roe eigenvectors (eq. 2.2 splitting, Sec. 4).
"""
import numpy as np
import pytest

from paper_2003_09145_gb300 import inputs

GAMMA = 1.4


def _prims(U, ndim):
    rho = U[0]
    vel = [U[1 + k] / rho for k in range(ndim)]
    p = (GAMMA - 1) * (U[-1] - 0.5 * rho * sum(v * v for v in vel))
    return rho, vel, p


def _skewed_state(ndim, n, seed):
    """Flow along +x, -y, +z at different Mach numbers, so that for every
    direction max|u-c|, max|u| and max|u+c| differ."""
    rng = np.random.default_rng(seed)
    shp = tuple(reversed(n))
    rho = rng.uniform(0.5, 2.0, shp)
    p = rng.uniform(0.3, 3.0, shp)
    base = [0.9, -1.7, 0.4]
    vel = [base[k] + 0.3 * rng.standard_normal(shp) for k in range(ndim)]
    return inputs.prim_to_cons(rho, vel, p)


@pytest.mark.parametrize("ndim,n", [(1, (37,)), (2, (11, 9)), (3, (7, 6, 5))])
def test_lf_alpha_definition(oracle, ndim, n):
    U = _skewed_state(ndim, n, seed=ndim)
    rho, vel, p = _prims(U, ndim)
    c = np.sqrt(GAMMA * p / rho)
    for d in range(ndim):
        lam = [np.max(np.abs(vel[d] - c)), np.max(np.abs(vel[d])), np.max(np.abs(vel[d] + c))]
        assert len({round(x, 6) for x in lam}) == 3, "the state must separate the three speeds"
        want = np.array([lam[0]] + [lam[1]] * ndim + [lam[2]])
        got = oracle.lf_alpha(ndim, n, d, U)
        np.testing.assert_allclose(got, want, rtol=1e-15, atol=0)


@pytest.mark.parametrize("ndim,n,bc", [(1, (23,), (0,)), (1, (23,), (1,)), (1, (23,), (2,)),
                                       (2, (9, 8), (0, 1)), (2, (9, 8), (2, 0)),
                                       (3, (6, 5, 7), (1, 0, 2)), (3, (4, 5, 3), (0, 0, 0))])
def test_rhs_sample_equals_full_rhs(oracle, ndim, n, bc):
    U = inputs.random_discontinuous_state(ndim, n, seed=sum(n) + sum(bc))
    dx = tuple(0.1 + 0.01 * k for k in range(ndim))
    R, fl, alpha = oracle.euler_rhs(U, n, dx, bc, want_flags=True, want_alpha=True)
    ncell = int(np.prod(n))
    cells = np.arange(ncell)[::2] if ncell > 40 else np.arange(ncell)
    Rv = R.reshape(ndim + 2, -1)
    # plain, and with the flag output
    fo = np.zeros_like(fl)
    S = oracle.euler_rhs_sample(U, n, dx, bc, cells, flags_out=fo)
    np.testing.assert_array_equal(S, Rv[:, cells].T)
    touched = np.nonzero(fo)[0]
    assert touched.size > 0
    np.testing.assert_array_equal(fo[touched], fl[touched])
    # forced selections: flip every flag to "keep all" and compare with the
    # full forced evaluation
    forced = (fl & ~np.uint8(7)) | np.uint8(7)
    Rf = oracle.euler_rhs(U, n, dx, bc, flags_in=forced).reshape(ndim + 2, -1)
    Sf = oracle.euler_rhs_sample(U, n, dx, bc, cells, flags_in=forced)
    np.testing.assert_array_equal(Sf, Rf[:, cells].T)
    assert not np.array_equal(Sf, S)
    # given LF speeds
    Sa = oracle.euler_rhs_sample(U, n, dx, bc, cells, alpha=alpha)
    np.testing.assert_array_equal(Sa, Rv[:, cells].T)
    Sb = oracle.euler_rhs_sample(U, n, dx, bc, cells, alpha=alpha * 1.5)
    assert not np.array_equal(Sb, S)


def _split_values(oracle, U, n, bc, d, ifc, ndim):
    """The eight (six-point) split characteristic values of one interface,
    formed here: Roe eigenvectors of cells i, i+1 (oracle.roe_eigensystem),
    w = L U_j, g = L F(U_j) with F of eq. 4.7, v+- = (g +- alpha w)/2."""
    nv = ndim + 2
    Ug = U.reshape(nv, *reversed(n))
    i = ifc[d] - 1

    def cell(j):
        idx = list(ifc)
        k = i - 2 + j
        m = n[d]
        flip = False
        if bc[d] == 0:
            k %= m
        elif bc[d] == 1:
            k = min(max(k, 0), m - 1)
        else:
            while k < 0 or k >= m:
                k = -1 - k if k < 0 else 2 * m - 1 - k
                flip = not flip
        idx[d] = k
        v = Ug[(slice(None),) + tuple(reversed(idx))].copy()
        if flip:
            v[1 + d] = -v[1 + d]
        return v

    pts = [cell(j) for j in range(6)]
    L, _ = oracle.roe_eigensystem(ndim, d, pts[2], pts[3])
    alpha = oracle.lf_alpha(ndim, n, d, U)
    vp, vm = [], []
    for Uj in pts:
        rho = Uj[0]
        vel = Uj[1:1 + ndim] / rho
        p = (GAMMA - 1) * (Uj[-1] - 0.5 * rho * vel @ vel)
        F = vel[d] * Uj
        F[1 + d] += p
        F[-1] += vel[d] * p
        w, g = L @ Uj, L @ F
        vp.append(0.5 * (g + alpha * w))
        vm.append(0.5 * (g - alpha * w))
    return np.array(vp), np.array(vm)


@pytest.mark.parametrize("ndim,n,bc", [(1, (30,), (1,)), (2, (10, 9), (0, 2)), (3, (6, 5, 4), (2, 1, 0))])
def test_interface_diag_matches_rhs_flags_and_reconstruction(oracle, ndim, n, bc):
    U = inputs.random_discontinuous_state(ndim, n, seed=40 + ndim)
    dx = (0.1,) * ndim
    _, fl = oracle.euler_rhs(U, n, dx, bc, want_flags=True)
    nv = ndim + 2
    rng = np.random.default_rng(ndim)
    checked = 0
    for d in range(ndim):
        nifc = oracle.num_interfaces(ndim, n, d)
        off = oracle.flag_offset(ndim, n, d)
        m0 = n[0] + (d == 0)
        m1 = (n[1] if ndim > 1 else 1) + (d == 1)
        for ilin in rng.choice(nifc, size=min(nifc, 12), replace=False):
            ifc = [ilin % m0, (ilin // m0) % m1, ilin // (m0 * m1)][:ndim]
            vp, vm = _split_values(oracle, U, n, bc, d, ifc, ndim)
            for f in range(nv):
                for side in range(2):
                    dg = oracle.euler_interface_diag(U, n, dx, bc, d, ifc, f, side)
                    flag = int(fl[off + (f * 2 + side) * nifc + ilin])
                    assert int(dg["m"]) == flag >> 3
                    delta = sum(1 << k for k in range(3) if dg[f"chi{k}"] >= dg["CT"])
                    assert delta == flag & 7
                    v = vp[0:5, f] if side == 0 else vm[[5, 4, 3, 2, 1], f]
                    fh, fl1, _ = oracle.teno5_lad(v)
                    if fl1 != flag:
                        continue   # a selector on a rounding boundary of this restatement
                    scale = np.max(np.abs(v)) + 1e-300
                    assert abs(dg["fhat"] - fh) <= 1e-12 * scale
                    checked += 1
    assert checked > 50
