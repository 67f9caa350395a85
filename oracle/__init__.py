"""Plain FP64 CPU oracle for the TENO5-LAD Euler right-hand side (arXiv 2003.09145).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library: the arithmetic lives in ``teno_oracle.c`` (compiled with gcc,
no FMA contraction) and the reverse-mode gradient in ``grad.py`` (plain PyTorch
CPU ops in float64).  This module only marshals numpy arrays into the C calls.

Array conventions (same as the problem statement, eq. 2.2 and eq. 4.7):
``U`` is ``[nvar][n_z][n_y][n_x]`` float64 with x fastest, ``nvar = ndim + 2``
and components ``(rho, rho*u, [rho*v, [rho*w]], E)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "teno_oracle.c")
_LIB = os.path.join(_HERE, "libteno_oracle.so")
_lock = threading.Lock()
_lib = None

BC_PERIODIC = 0
BC_TRANSMISSIVE = 1
BC_REFLECTIVE = 2
BC_DIRICHLET = 3


def build(force: bool = False) -> str:
    """Compile ``teno_oracle.c`` with gcc (``-O2 -ffp-contract=off -fopenmp``)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("H", ctypes.c_double), ("eps", ctypes.c_double),
                ("b_l", ctypes.c_int), ("b_u", ctypes.c_int), ("scheme", ctypes.c_int), ("ct_m", ctypes.c_int),
                ("grav", ctypes.c_double * 3), ("bc_state", ctypes.c_double * 30)]


# The reconstruction's cutoff or weights (see or_teno5_lad): the paper's
# adaptive LAD cutoff (eq. 3.1-3.4), a fixed C_T = 10^-ct_m (TENO5, Sec. 2;
# Sec. 4 uses 1e-7), TENO5-A (eq. 2.16-2.18) and WENO-Z (tau_5 of eq. 2.12).
SCHEMES = {"lad": 0, "teno5": 1, "teno5a": 2, "wenoz": 3}


@dataclass
class Params:
    """Scheme parameters: gamma (eq. 4.7), H, B_l, B_u (eq. 3.1-3.2), eps
    (eq. 2.8), the reconstruction ``scheme`` and TENO5's fixed magnitude."""
    gamma: float = 1.4
    H: float = 10.0
    eps: float = 1e-6
    b_l: int = 4
    b_u: int = 10
    scheme: str = "lad"
    ct_m: int = 7
    grav: tuple = (0.0, 0.0, 0.0)      # body acceleration of Sec. 4.3.2's source
    bc_state: object = None            # bc 3: conservative ghost states [3][2][5]

    def c(self) -> _Params:
        g = (ctypes.c_double * 3)(*[float(x) for x in (list(self.grav) + [0.0] * 3)[:3]])
        st = np.zeros(30) if self.bc_state is None else np.asarray(self.bc_state, dtype=np.float64).reshape(30)
        return _Params(self.gamma, self.H, self.eps, self.b_l, self.b_u, SCHEMES[self.scheme], self.ct_m, g,
                       (ctypes.c_double * 30)(*st.tolist()))


_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int)
_PP = ctypes.POINTER(_Params)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.or_diag_count.restype = ctypes.c_int
            L.or_ladder.argtypes = [ctypes.c_int]
            L.or_ladder.restype = ctypes.c_double
            L.or_upwind5.argtypes = [_D]
            L.or_upwind5.restype = ctypes.c_double
            L.or_teno5_lad.argtypes = [_D, _PP, ctypes.c_int, _U8, _D]
            L.or_teno5_lad.restype = ctypes.c_double
            L.or_roe_eigensystem.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_double, _D, _D]
            L.or_roe_eigensystem.restype = ctypes.c_int
            L.or_num_interfaces.argtypes = [ctypes.c_int, _I64, ctypes.c_int]
            L.or_num_interfaces.restype = ctypes.c_int64
            L.or_flag_offset.argtypes = [ctypes.c_int, _I64, ctypes.c_int]
            L.or_flag_offset.restype = ctypes.c_int64
            L.or_lf_alpha.argtypes = [ctypes.c_int, _I64, ctypes.c_int, ctypes.c_double, _D, _D]
            L.or_lf_alpha.restype = ctypes.c_int
            L.or_euler_rhs.argtypes = [ctypes.c_int, _I64, _D, _I32, _PP, _D, _D, _U8, _U8, _D]
            L.or_euler_rhs.restype = ctypes.c_int
            L.or_euler_rhs_sample.argtypes = [ctypes.c_int, _I64, _D, _I32, _PP, _D, ctypes.c_int64,
                                              _I64, _D, _U8, _U8, _D]
            L.or_euler_rhs_sample.restype = ctypes.c_int
            L.or_euler_interface_diag.argtypes = [ctypes.c_int, _I64, _D, _I32, _PP, _D, ctypes.c_int,
                                                  _I64, ctypes.c_int, ctypes.c_int, _D]
            L.or_euler_interface_diag.restype = ctypes.c_int
            L.or_euler_dt.argtypes = [ctypes.c_int, _I64, _D, ctypes.c_double, ctypes.c_double, _D]
            L.or_euler_dt.restype = ctypes.c_double
            L.or_euler_rk3_step.argtypes = [ctypes.c_int, _I64, _D, _I32, _PP, _D, ctypes.c_double]
            L.or_euler_rk3_step.restype = ctypes.c_int
            L.or_euler_run.argtypes = [ctypes.c_int, _I64, _D, _I32, _PP, _D, _D, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int64, ctypes.c_int, _I64]
            L.or_euler_run.restype = ctypes.c_int64
            L.or_scalar_rhs.argtypes = [ctypes.c_int64, ctypes.c_double, _PP, ctypes.c_int, _D, _D]
            L.or_scalar_rhs.restype = None
            L.or_scalar_run.argtypes = [ctypes.c_int64, ctypes.c_double, _PP, ctypes.c_int, _D,
                                        ctypes.c_double, ctypes.c_double]
            L.or_scalar_run.restype = ctypes.c_int64
            L.or_riemann_star.argtypes = [ctypes.c_double] * 7 + [_D]
            L.or_riemann_star.restype = ctypes.c_int
            L.or_riemann_sample.argtypes = [ctypes.c_double] * 7 + [_D, ctypes.c_int64, _D]
            L.or_riemann_sample.restype = ctypes.c_int
            L.or_num_threads.restype = ctypes.c_int
            L.or_set_num_threads.argtypes = [ctypes.c_int]
            L.or_set_num_threads.restype = None
            _lib = L
    return _lib


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------

def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _u8p(a):
    if a is None:
        return None
    assert a.dtype == np.uint8 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_U8)


def _shape3(n):
    n = list(n) + [1] * (3 - len(n))
    return (ctypes.c_int64 * 3)(*n)


def _dx3(dx):
    dx = list(dx) + [1.0] * (3 - len(dx))
    return (ctypes.c_double * 3)(*dx)


def _bc3(bc):
    bc = list(bc) + [0] * (3 - len(bc))
    return (ctypes.c_int * 3)(*bc)


DIAG_NAMES = ["beta0", "beta1", "beta2", "tau", "chit0", "chit1", "chit2", "theta", "m", "CT",
              "gamma0", "gamma1", "gamma2", "chi0", "chi1", "chi2", "f0", "f1", "f2",
              "omega0", "omega1", "omega2", "fhat", "eta", "mA", "gA", "betaA"]


def num_threads() -> int:
    return lib().or_num_threads()


def set_num_threads(k: int) -> None:
    lib().or_set_num_threads(int(k))


def ladder(m: int) -> float:
    """Lad(m) = 10^-m (eq. 3.3-3.4)."""
    return lib().or_ladder(int(m))


def upwind5(v) -> float:
    """Eq. 2.3 on v = (f_{i-2}, ..., f_{i+2})."""
    a = np.ascontiguousarray(v, dtype=np.float64)
    return lib().or_upwind5(_dp(a))


def teno5_lad(v, params: Params | None = None, forced: int = -1):
    """One TENO5-LAD reconstruction (eq. 2.4-2.15, 3.1-3.4).

    Returns ``(fhat, flag, diag)``: ``flag`` bits 0..2 = delta_k, bits 3..6 = m;
    ``diag`` maps the paper's symbols to their values."""
    p = params or Params()
    a = np.ascontiguousarray(v, dtype=np.float64)
    flag = ctypes.c_uint8(0)
    diag = np.zeros(lib().or_diag_count(), dtype=np.float64)
    pc = p.c()
    f = lib().or_teno5_lad(_dp(a), ctypes.byref(pc), int(forced), ctypes.byref(flag), _dp(diag))
    return f, flag.value, dict(zip(DIAG_NAMES, diag.tolist()))


def roe_eigensystem(ndim: int, d: int, Ua, Ub, gamma: float = 1.4):
    """Left/right eigenvector matrices (L, R) of the Roe state of Ua, Ub along d."""
    nvar = ndim + 2
    a = np.ascontiguousarray(Ua, dtype=np.float64)
    b = np.ascontiguousarray(Ub, dtype=np.float64)
    L = np.zeros((nvar, nvar))
    R = np.zeros((nvar, nvar))
    st = lib().or_roe_eigensystem(ndim, d, _dp(a), _dp(b), gamma, _dp(L), _dp(R))
    if st != 0:
        raise ValueError("Roe state has no real sound speed")
    return L, R


def num_interfaces(ndim: int, n, d: int) -> int:
    return lib().or_num_interfaces(ndim, _shape3(n), d)


def flag_offset(ndim: int, n, d: int) -> int:
    return lib().or_flag_offset(ndim, _shape3(n), d)


def flag_count(ndim: int, n) -> int:
    return flag_offset(ndim, n, ndim)


def lf_alpha(ndim: int, n, d: int, U: np.ndarray, gamma: float = 1.4) -> np.ndarray:
    nvar = ndim + 2
    out = np.zeros(nvar)
    lib().or_lf_alpha(ndim, _shape3(n), d, gamma, _dp(np.ascontiguousarray(U)), _dp(out))
    return out


def euler_rhs(U: np.ndarray, n, dx, bc, params: Params | None = None,
              want_flags: bool = False, flags_in: np.ndarray | None = None,
              want_alpha: bool = False):
    """L(U) of eq. 2.2 for the Euler equations (eq. 4.7), dimension by dimension.

    Returns ``rhs`` or a tuple ``(rhs, flags?, alpha?)`` as requested."""
    p = params or Params()
    ndim = len(n)
    U = np.ascontiguousarray(U, dtype=np.float64)
    R = np.zeros_like(U)
    flags = np.zeros(flag_count(ndim, n), dtype=np.uint8) if want_flags else None
    fin = None if flags_in is None else np.ascontiguousarray(flags_in, dtype=np.uint8)
    alpha = np.zeros((ndim, ndim + 2)) if want_alpha else None
    pc = p.c()
    st = lib().or_euler_rhs(ndim, _shape3(n), _dx3(dx), _bc3(bc), ctypes.byref(pc), _dp(U), _dp(R),
                            _u8p(flags), _u8p(fin), None if alpha is None else _dp(alpha))
    if st != 0:
        raise FloatingPointError("non-physical state in the oracle RHS")
    if not want_flags and not want_alpha:
        return R
    out = [R]
    if want_flags:
        out.append(flags)
    if want_alpha:
        out.append(alpha)
    return tuple(out)


def euler_rhs_sample(U: np.ndarray, n, dx, bc, cells, params: Params | None = None,
                     flags_out: np.ndarray | None = None, flags_in: np.ndarray | None = None,
                     alpha: np.ndarray | None = None) -> np.ndarray:
    """L(U) at the given linear cell indices; returns [m][nvar].  ``flags_out`` /
    ``flags_in`` are full-size flag arrays (only the sampled faces are touched)."""
    p = params or Params()
    ndim = len(n)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.zeros((cells.size, ndim + 2))
    pc = p.c()
    a = None if alpha is None else np.ascontiguousarray(alpha, dtype=np.float64)
    st = lib().or_euler_rhs_sample(ndim, _shape3(n), _dx3(dx), _bc3(bc), ctypes.byref(pc),
                                   _dp(np.ascontiguousarray(U)), cells.size,
                                   cells.ctypes.data_as(_I64), _dp(out), _u8p(flags_out), _u8p(flags_in),
                                   None if a is None else _dp(a))
    if st != 0:
        raise FloatingPointError("non-physical state in the oracle RHS")
    return out


def euler_interface_diag(U, n, dx, bc, d: int, ifc, field: int, side: int,
                         params: Params | None = None) -> dict:
    """Diagnostic record of the reconstruction at one interface (see teno5_lad)."""
    p = params or Params()
    ndim = len(n)
    diag = np.zeros(lib().or_diag_count())
    pc = p.c()
    ifc3 = (ctypes.c_int64 * 3)(*(list(ifc) + [0] * (3 - len(ifc))))
    lib().or_euler_interface_diag(ndim, _shape3(n), _dx3(dx), _bc3(bc), ctypes.byref(pc),
                                  _dp(np.ascontiguousarray(U)), d, ifc3, field, side, _dp(diag))
    return dict(zip(DIAG_NAMES, diag.tolist()))


def euler_dt(U, n, dx, sigma: float, gamma: float = 1.4) -> float:
    """CFL step, eq. dt1 (1D), eq. dt2 (2D), harmonic 3D extension."""
    return lib().or_euler_dt(len(n), _shape3(n), _dx3(dx), gamma, sigma,
                             _dp(np.ascontiguousarray(U)))


def euler_rk3_step(U: np.ndarray, n, dx, bc, dt: float, params: Params | None = None) -> np.ndarray:
    """One SSP-RK3 step (eq. 4.1-4.3); returns a new array."""
    p = params or Params()
    V = np.array(U, dtype=np.float64, copy=True, order="C")
    pc = p.c()
    st = lib().or_euler_rk3_step(len(n), _shape3(n), _dx3(dx), _bc3(bc), ctypes.byref(pc), _dp(V), dt)
    if st != 0:
        raise FloatingPointError("non-physical state in the oracle RK3 step")
    return V


def euler_run(U: np.ndarray, n, dx, bc, t_end: float, sigma: float = 0.5,
              dt_fixed: float = 0.0, max_steps: int = 1 << 40, t0: float = 0.0,
              params: Params | None = None, strict: bool = True):
    """Advance by CFL-limited SSP-RK3 steps to ``t_end`` (or ``max_steps``).

    Returns ``(U_new, t, steps)``.  ``strict``: raise at the first step whose
    stages meet a non-physical state; otherwise continue (see ``euler_run_ex``)."""
    V, t, k, _ = euler_run_ex(U, n, dx, bc, t_end, sigma, dt_fixed, max_steps, t0, params, strict)
    return V, t, k


def euler_run_ex(U, n, dx, bc, t_end, sigma=0.5, dt_fixed=0.0, max_steps=1 << 40, t0=0.0,
                 params=None, strict=False):
    """As euler_run, also returning the number of steps that met a non-physical
    intermediate state: ``(U_new, t, steps, bad_steps)``."""
    p = params or Params()
    V = np.array(U, dtype=np.float64, copy=True, order="C")
    t = ctypes.c_double(t0)
    nbad = ctypes.c_int64(0)
    pc = p.c()
    k = lib().or_euler_run(len(n), _shape3(n), _dx3(dx), _bc3(bc), ctypes.byref(pc), _dp(V),
                           ctypes.byref(t), t_end, sigma, dt_fixed, int(max_steps), 1 if strict else 0,
                           ctypes.byref(nbad))
    if k < 0:
        raise FloatingPointError("non-physical state in the oracle run")
    return V, t.value, k, nbad.value


def scalar_rhs(u: np.ndarray, dx: float, mode: str = "lad", params: Params | None = None):
    p = params or Params()
    u = np.ascontiguousarray(u, dtype=np.float64)
    r = np.zeros_like(u)
    pc = p.c()
    lib().or_scalar_rhs(u.size, dx, ctypes.byref(pc), 0 if mode == "lad" else 1, _dp(u), _dp(r))
    return r


def scalar_run(u: np.ndarray, dx: float, t_end: float, dt: float, mode: str = "lad",
               params: Params | None = None):
    p = params or Params()
    v = np.array(u, dtype=np.float64, copy=True)
    pc = p.c()
    k = lib().or_scalar_run(v.size, dx, ctypes.byref(pc), 0 if mode == "lad" else 1, _dp(v), t_end, dt)
    return v, k


def riemann_star(left, right, gamma: float = 1.4) -> dict:
    """Exact star state of the Riemann problem (rho, u, p)_L | (rho, u, p)_R."""
    out = np.zeros(11)
    st = lib().or_riemann_star(*map(float, left), *map(float, right), gamma, _dp(out))
    if st != 0:
        raise ValueError("Riemann problem generates vacuum or did not converge")
    keys = ["p", "u", "rho_l", "rho_r", "left_shock", "right_shock", "s_l_head", "s_l_tail",
            "s_r_tail", "s_r_head", "iterations"]
    return dict(zip(keys, out.tolist()))


def riemann_sample(left, right, xi, gamma: float = 1.4) -> np.ndarray:
    """Exact self-similar solution at xi = (x - x0)/t; returns [3][m] (rho, u, p)."""
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    out = np.zeros((3, xi.size))
    st = lib().or_riemann_sample(*map(float, left), *map(float, right), gamma, _dp(xi), xi.size, _dp(out))
    if st != 0:
        raise ValueError("Riemann problem generates vacuum")
    return out
