"""Reverse-mode gradient oracle of the TENO5-LAD Euler right-hand side.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).  A second, independent plain
restatement of the right-hand side of eq. 2.2 in PyTorch CPU float64 ops, so
that autograd supplies J(U)^T v.  The stencil selections are frozen: the
delta bits of every reconstruction come from the C oracle's flag output for
the same state (the cutoff is a piecewise-constant selector), and the global
Lax-Friedrichs speed of each field is the value of |lambda| at its arg-max
cell (lowest linear index on ties), so its derivative flows to that cell.

Every step follows the same readings as ``teno_oracle.c``: Roe-averaged
eigensystem with the eigenvector normalisation written there, global LF
splitting per field and direction, f^- on the mirrored stencil, transmissive
ghost cells copying the boundary cell, periodic ones wrapping.
"""
from __future__ import annotations

import numpy as np
import torch

from . import euler_rhs, flag_count, flag_offset, num_interfaces, Params

_C = (0.1, 0.6, 0.3)   # linear weights (Sec. 2)


def _ghost(i: np.ndarray, n: int, bc: int) -> np.ndarray:
    if bc == 0:
        return np.mod(i, n)
    return np.clip(i, 0, n - 1)


def _primitive(U, ndim, gamma):
    rho = U[0]
    vel = [U[1 + k] / rho for k in range(ndim)]
    q2 = sum(v * v for v in vel)
    p = (gamma - 1.0) * (U[-1] - 0.5 * rho * q2)
    return rho, vel, p


def _flux(U, ndim, d, gamma):
    """Eq. 4.7 along direction d (stacked on dim 0)."""
    rho, vel, p = _primitive(U, ndim, gamma)
    F = [rho * vel[d]]
    for k in range(ndim):
        F.append(U[1 + k] * vel[d] + (p if k == d else 0.0))
    F.append(vel[d] * (U[-1] + p))
    return torch.stack(F)


def _roe_eigensystem(Ua, Ub, ndim, d, gamma):
    """Left (rows) and right (columns) eigenvectors of the Roe state, [..., nvar, nvar]."""
    nvar = ndim + 2
    ra, va, pa = _primitive(Ua, ndim, gamma)
    rb, vb, pb = _primitive(Ub, ndim, gamma)
    sa, sb = torch.sqrt(ra), torch.sqrt(rb)
    Ha = (Ua[-1] + pa) / ra
    Hb = (Ub[-1] + pb) / rb
    u = [(sa * va[k] + sb * vb[k]) / (sa + sb) for k in range(ndim)]
    q2 = sum(x * x for x in u)
    H = (sa * Ha + sb * Hb) / (sa + sb)
    c2 = (gamma - 1.0) * (H - 0.5 * q2)
    c = torch.sqrt(c2)
    b1 = (gamma - 1.0) / c2
    b2 = 0.5 * b1 * q2
    zero = torch.zeros_like(c)
    one = torch.ones_like(c)
    Rc = [[zero] * nvar for _ in range(nvar)]     # Rc[row][col]
    Lr = [[zero] * nvar for _ in range(nvar)]     # Lr[row][col]
    # acoustic u_d - c
    Rc[0][0] = one
    for k in range(ndim):
        Rc[1 + k][0] = u[k] - (c if k == d else 0.0)
    Rc[nvar - 1][0] = H - u[d] * c
    Lr[0][0] = 0.5 * (b2 + u[d] / c)
    for k in range(ndim):
        Lr[0][1 + k] = 0.5 * (-b1 * u[k] - (1.0 / c if k == d else 0.0))
    Lr[0][nvar - 1] = 0.5 * b1
    # entropy
    Rc[0][1] = one
    for k in range(ndim):
        Rc[1 + k][1] = u[k]
    Rc[nvar - 1][1] = 0.5 * q2
    Lr[1][0] = 1.0 - b2
    for k in range(ndim):
        Lr[1][1 + k] = b1 * u[k]
    Lr[1][nvar - 1] = -b1
    # shear fields
    f = 2
    for t in range(ndim):
        if t == d:
            continue
        Rc[1 + t][f] = one
        Rc[nvar - 1][f] = u[t]
        Lr[f][0] = -u[t]
        Lr[f][1 + t] = one
        f += 1
    # acoustic u_d + c
    Rc[0][nvar - 1] = one
    for k in range(ndim):
        Rc[1 + k][nvar - 1] = u[k] + (c if k == d else 0.0)
    Rc[nvar - 1][nvar - 1] = H + u[d] * c
    Lr[nvar - 1][0] = 0.5 * (b2 - u[d] / c)
    for k in range(ndim):
        Lr[nvar - 1][1 + k] = 0.5 * (-b1 * u[k] + (1.0 / c if k == d else 0.0))
    Lr[nvar - 1][nvar - 1] = 0.5 * b1
    L = torch.stack([torch.stack(row, dim=-1) for row in Lr], dim=-2)
    R = torch.stack([torch.stack(row, dim=-1) for row in Rc], dim=-2)
    return L, R


def _weights(bits: np.ndarray):
    """TENO weights of eq. 2.15 from the delta bits (eq. 2.14), [..., 3]."""
    delta = np.stack([(bits >> k) & 1 for k in range(3)], axis=-1).astype(np.float64)
    dc = delta * np.asarray(_C)
    return torch.from_numpy(dc / dc.sum(axis=-1, keepdims=True))


def _teno_frozen(v, omega):
    """Eq. 2.4-2.7 with frozen weights; v [..., 5] = (f_{i-2}, ..., f_{i+2})."""
    f0 = 1.0 / 3.0 * v[..., 0] - 7.0 / 6.0 * v[..., 1] + 11.0 / 6.0 * v[..., 2]
    f1 = -1.0 / 6.0 * v[..., 1] + 5.0 / 6.0 * v[..., 2] + 1.0 / 3.0 * v[..., 3]
    f2 = 1.0 / 3.0 * v[..., 2] + 5.0 / 6.0 * v[..., 3] - 1.0 / 6.0 * v[..., 4]
    return omega[..., 0] * f0 + omega[..., 1] * f1 + omega[..., 2] * f2


def _lf_alpha(U, ndim, d, gamma):
    """alpha_s = |lambda_s| at the arg-max cell (first maximal linear index)."""
    rho, vel, p = _primitive(U, ndim, gamma)
    c = torch.sqrt(gamma * p / rho)
    lam = [torch.abs(vel[d] - c), torch.abs(vel[d]), torch.abs(vel[d] + c)]
    out = []
    for l in lam:
        flat = l.reshape(-1)
        out.append(flat[int(np.argmax(flat.detach().numpy()))])
    return out


def rhs(U: torch.Tensor, n, dx, bc, flags: np.ndarray, params: Params | None = None) -> torch.Tensor:
    """L(U) (eq. 2.2) with the selections of ``flags`` (layout of the C oracle).

    U: torch float64 [nvar][n_z][n_y][n_x] (squeezed like the inputs)."""
    P = params or Params()
    gamma = P.gamma
    ndim = len(n)
    nvar = ndim + 2
    shape = tuple(reversed(n))
    U = U.reshape((nvar,) + shape)
    total = torch.zeros_like(U)
    for d in range(ndim):
        axis = ndim - d                        # tensor axis of direction d (dim 0 = variable)
        nd = n[d]
        a_m, a_0, a_p = _lf_alpha(U, ndim, d, gamma)
        alpha = [a_m] + [a_0] * (nvar - 2) + [a_p]
        Ut = torch.movedim(U, axis, -1)        # [nvar, ..., n_d]
        ifc = np.arange(nd + 1)
        idx = np.stack([_ghost(ifc - 3 + j, nd, bc[d]) for j in range(6)], axis=-1)  # [n_d+1, 6]
        Pts = Ut[..., torch.from_numpy(idx)]   # [nvar, ..., n_d+1, 6]
        Fp = _flux(Pts, ndim, d, gamma)
        L, R = _roe_eigensystem(Pts[..., 2], Pts[..., 3], ndim, d, gamma)   # [..., n_d+1, nvar, nvar]
        w = torch.einsum("...rk,k...j->...jr", L, Pts)     # [..., n_d+1, 6, nvar]
        g = torch.einsum("...rk,k...j->...jr", L, Fp)
        # flags of this direction as [..., n_d+1, nvar, 2] (interface grid with n_d+1 along d)
        off = flag_offset(ndim, n, d)
        nifc = num_interfaces(ndim, n, d)
        fl = flags[off:off + nvar * 2 * nifc].reshape((nvar, 2) + tuple(
            (m + 1 if (ndim - 1 - a) == d else m) for a, m in enumerate(shape)))
        fl = np.moveaxis(fl, 2 + (ndim - 1 - d), -1)       # [nvar, 2, ..., n_d+1]
        fl = np.moveaxis(np.moveaxis(fl, 0, -1), 0, -1)    # [..., n_d+1, nvar, 2]
        om_p = _weights(fl[..., 0])
        om_m = _weights(fl[..., 1])
        fchar = []
        for s in range(nvar):
            vp = 0.5 * (g[..., :5, s] + alpha[s] * w[..., :5, s])
            vm = 0.5 * (g[..., :, s] - alpha[s] * w[..., :, s]).flip(-1)[..., :5]
            fchar.append(_teno_frozen(vp, om_p[..., s, :]) + _teno_frozen(vm, om_m[..., s, :]))
        fchar = torch.stack(fchar, dim=-1)                 # [..., n_d+1, nvar]
        Fhat = torch.einsum("...rk,...k->...r", R, fchar)  # [..., n_d+1, nvar]
        Rd = -(Fhat[..., 1:, :] - Fhat[..., :-1, :]) / dx[d]   # [..., n_d, nvar]
        Rd = torch.movedim(torch.movedim(Rd, -1, 0), -1, axis)
        total = total + Rd
    return total


def rhs_with_oracle_flags(U: torch.Tensor, n, dx, bc, params: Params | None = None):
    """rhs() with the selections the C oracle makes for the (detached) state."""
    Un = np.ascontiguousarray(U.detach().numpy())
    _, flags = euler_rhs(Un, n, dx, bc, params, want_flags=True)
    return rhs(U, n, dx, bc, flags, params), flags


def rk3_rollout(U0: torch.Tensor, n, dx, bc, dt: float, steps: int, params: Params | None = None):
    """`steps` SSP-RK3 steps (eq. 4.1-4.3) of fixed dt with frozen selections per
    stage (taken from the C oracle on each stage's state)."""
    U = U0
    for _ in range(steps):
        L0, _ = rhs_with_oracle_flags(U, n, dx, bc, params)
        U1 = U + dt * L0
        L1, _ = rhs_with_oracle_flags(U1, n, dx, bc, params)
        U2 = 3.0 / 4.0 * U + 1.0 / 4.0 * U1 + 1.0 / 4.0 * dt * L1
        L2, _ = rhs_with_oracle_flags(U2, n, dx, bc, params)
        U = 1.0 / 3.0 * U + 2.0 / 3.0 * U2 + 2.0 / 3.0 * dt * L2
    return U


def rhs_vjp(U: np.ndarray, n, dx, bc, Rbar: np.ndarray, params: Params | None = None):
    """J(U)^T Rbar with frozen selections; returns (vjp, flags)."""
    Ut = torch.from_numpy(np.ascontiguousarray(U)).requires_grad_(True)
    R, flags = rhs_with_oracle_flags(Ut, n, dx, bc, params)
    (gr,) = torch.autograd.grad(R, Ut, torch.from_numpy(np.ascontiguousarray(Rbar)).reshape(R.shape))
    return gr.numpy(), flags
