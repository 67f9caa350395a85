"""Pins of the oracle's fixed-state faces and body-force source (Sec. 4.3.2's
Rayleigh-Taylor problem, eq. 4.12).

* Hydrostatic balance: at rest with rho constant and p linear in y, every
  reconstruction sees linear data (all stencils kept, eq. 2.3 exact for
  it), so the discrete pressure gradient is exact and balances the source:
  away from the density jump and the fixed-state faces L(U) vanishes to
  rounding.  A sign slip or a missing factor in the source breaks this.
* The source is additive: L with gravity minus L without equals
  (0, rho g, rho u.g) to rounding.
* A fixed-state face whose state equals the boundary cells' (uniform along
  the face) gives the transmissive result bit for bit; a uniform state equal
  to both face states gives L = 0 exactly."""
import numpy as np
import pytest

from paper_2003_09145_gb300 import inputs


def rt_params(oracle, P, grav=True):
    st = np.zeros((3, 2, 5))
    for k, faces in enumerate(P.extra["bc_state"]):
        if faces is not None:
            for side in range(2):
                st[k, side, :len(faces[side])] = faces[side]
    g = tuple(P.extra["grav"]) + (0.0,) if grav else (0.0, 0.0, 0.0)
    return oracle.Params(gamma=P.gamma, grav=g, bc_state=st)


def test_hydrostatic_balance(oracle):
    P = inputs.rayleigh_taylor(8, 64, perturb=False)
    R = oracle.euler_rhs(P.U0, P.n, P.dx, P.bc, rt_params(oracle, P)).reshape(4, 64, 8)
    rows = [j for j in range(64) if 3 <= j < 29 or 35 <= j < 61]
    scale = 3.0 / P.dx[1]            # the pressure fluxes the difference cancels
    assert np.max(np.abs(R[:, rows])) <= 1e-12 * scale
    # without the source the same rows carry -dp/dy = -rho
    R0 = oracle.euler_rhs(P.U0, P.n, P.dx, P.bc, rt_params(oracle, P, grav=False)).reshape(4, 64, 8)
    np.testing.assert_allclose(R0[2, rows], -np.where(np.array(rows) < 32, 2.0, 1.0)[:, None] * np.ones(8),
                               rtol=1e-10)


def test_source_is_additive(oracle):
    P = inputs.rayleigh_taylor(12, 40)
    Rg = oracle.euler_rhs(P.U0, P.n, P.dx, P.bc, rt_params(oracle, P))
    R0 = oracle.euler_rhs(P.U0, P.n, P.dx, P.bc, rt_params(oracle, P, grav=False))
    S = np.zeros_like(P.U0)
    S[2] = P.U0[0]                # rho g_y, g = (0, 1)
    S[3] = P.U0[2]                # (rho v) g_y
    np.testing.assert_allclose(Rg - R0, S, rtol=1e-12, atol=1e-12 * np.max(np.abs(R0)))
    # the sampled RHS adds it alike
    cells = np.arange(0, 480, 7)
    Ss = oracle.euler_rhs_sample(P.U0, P.n, P.dx, P.bc, cells, rt_params(oracle, P))
    np.testing.assert_array_equal(Ss, Rg.reshape(4, -1)[:, cells].T)


def test_fixed_state_faces(oracle):
    rng = np.random.default_rng(3)
    nx, ny = 9, 14
    rho = 1.0 + 0.2 * rng.random((ny, nx))
    u = 0.3 * rng.standard_normal((ny, nx))
    v = 0.3 * rng.standard_normal((ny, nx))
    p = 1.0 + 0.2 * rng.random((ny, nx))
    # boundary rows uniform along the face, so a fixed state can equal them
    for j in (0, ny - 1):
        rho[j], u[j], v[j], p[j] = rho[j, 0], u[j, 0], v[j, 0], p[j, 0]
    U = inputs.prim_to_cons(rho, [u, v], p)
    st = np.zeros((3, 2, 5))
    st[1, 0, :4] = U[:, 0, 0]
    st[1, 1, :4] = U[:, ny - 1, 0]
    fixed = oracle.euler_rhs(U, (nx, ny), (0.1, 0.1), (0, 3), oracle.Params(bc_state=st))
    trans = oracle.euler_rhs(U, (nx, ny), (0.1, 0.1), (0, 1))
    np.testing.assert_array_equal(fixed, trans)
    # a different fixed state changes only the rows within three cells of it
    st2 = st.copy()
    st2[1, 0, 0] *= 1.5
    st2[1, 0, 3] *= 1.5
    R2 = oracle.euler_rhs(U, (nx, ny), (0.1, 0.1), (0, 3), oracle.Params(bc_state=st2)).reshape(4, ny, nx)
    diff = np.any(R2 != trans.reshape(4, ny, nx), axis=(0, 2))
    assert diff[:3].all() and not diff[3:].any()
    # a uniform state equal to both faces' states: L = 0 exactly
    Uc = np.broadcast_to(U[:, :1, :1], U.shape).copy()
    st3 = np.zeros((3, 2, 5))
    st3[1, :, :4] = Uc[:, 0, 0]
    assert np.all(oracle.euler_rhs(Uc, (nx, ny), (0.1, 0.1), (0, 3), oracle.Params(bc_state=st3)) == 0.0)
