"""ctypes binding of the C-ABI in ``include/teno.h`` (argument marshalling only).

The shared library ``libteno_gb300.so`` is built in-tree by ``build.py``.  If it
is missing, loading raises: there is no CPU fallback for any entry point.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libteno_gb300.so")

TENO_OK = 0
STATUS_NAMES = {
    0: "TENO_OK", 1: "TENO_ERR_INVALID_ARG", 2: "TENO_ERR_UNSUPPORTED", 3: "TENO_ERR_CUDA",
    4: "TENO_ERR_NONPHYSICAL", 5: "TENO_ERR_TIMEOUT", 6: "TENO_ERR_WORKSPACE",
    7: "TENO_ERR_UNIMPLEMENTED",
}
OP_RHS, OP_RK3, OP_RHS_ADJOINT, OP_RK3_ADJOINT = 0, 1, 2, 3
BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTIVE, BC_DIRICHLET = 0, 1, 2, 3
KERNEL_KINDS = ("cell", "flux", "diff", "dt")


class TenoGrid(ctypes.Structure):
    """Mirror of ``teno_grid``."""
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("n", ctypes.c_int64 * 3),
        ("dx", ctypes.c_double * 3),
        ("bc", ctypes.c_int * 3),
        ("gamma", ctypes.c_double),
        ("H", ctypes.c_double),
        ("b_l", ctypes.c_int),
        ("b_u", ctypes.c_int),
        ("eps", ctypes.c_double),
        ("scheme", ctypes.c_int),
        ("ct_m", ctypes.c_int),
        ("grav", ctypes.c_double * 3),
        ("bc_state", ctypes.c_double * 30),
    ]


# teno_scheme: the paper's LAD cutoff and the schemes it is compared with
SCHEMES = {"lad": 0, "teno5": 1, "teno5a": 2, "wenoz": 3}


class TenoBatch(ctypes.Structure):
    """Mirror of ``teno_batch``."""
    _fields_ = [
        ("nprob", ctypes.c_int64),
        ("ncell", ctypes.c_int64),
        ("bc", ctypes.c_int),
        ("gamma", ctypes.c_double),
        ("H", ctypes.c_double),
        ("b_l", ctypes.c_int),
        ("b_u", ctypes.c_int),
        ("eps", ctypes.c_double),
    ]


class TenoBatchTuning(ctypes.Structure):
    """Mirror of ``teno_batch_tuning``."""
    _fields_ = [("block", ctypes.c_int), ("ctas_per_sm", ctypes.c_int)]


class TenoError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")


# (name, restype, argtypes) of every exported entry point
_VP = ctypes.c_void_p
_GP = ctypes.POINTER(TenoGrid)
SIGNATURES = [
    ("teno_grid_default", None, [_GP, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                 ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    ("teno_workspace_bytes", ctypes.c_size_t, [_GP, ctypes.c_int]),
    ("teno_flag_count", ctypes.c_int64, [_GP]),
    ("teno_rhs", ctypes.c_int, [_GP, _VP, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    ("teno_rk3_step", ctypes.c_int, [_GP, _VP, ctypes.c_double, ctypes.c_double, _VP,
                                     ctypes.c_double, _VP, _VP, ctypes.c_size_t, _VP]),
    ("teno_rk3_stage_begin", ctypes.c_int, [_GP, _VP, _VP, ctypes.c_size_t, _VP]),
    ("teno_rk3_stage_end", ctypes.c_int, [_GP, ctypes.c_int, _VP, _VP, _VP, ctypes.c_double, ctypes.c_double, _VP,
                                          ctypes.c_double, _VP, _VP, ctypes.c_size_t, _VP]),
    ("teno_alpha_offset", ctypes.c_size_t, []),
    ("teno_planes_copy", ctypes.c_int, [_GP, _VP, ctypes.c_int64, ctypes.c_int, _VP, ctypes.c_int64, ctypes.c_int,
                                        ctypes.c_int64, _VP]),
    ("teno_get_device_status", ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_int)]),
    ("teno_adjoint_workspace_bytes", ctypes.c_size_t, [_GP, ctypes.c_int]),
    ("teno_rhs_adjoint", ctypes.c_int, [_GP, _VP, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    ("teno_rk3_step_adjoint", ctypes.c_int, [_GP, _VP, ctypes.c_double, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    ("teno_rk3_step_adjoint_staged", ctypes.c_int,
     [_GP, _VP, _VP, _VP, ctypes.c_double, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    ("teno_batch_workspace_bytes", ctypes.c_size_t, [ctypes.POINTER(TenoBatch)]),
    ("teno_batch_prepare", ctypes.c_int, [ctypes.POINTER(TenoBatch), ctypes.POINTER(ctypes.c_int64), _VP,
                                          ctypes.c_size_t, _VP]),
    ("teno_rk3_step_batched", ctypes.c_int, [ctypes.POINTER(TenoBatch), _VP, _VP, _VP, _VP, _VP,
                                             ctypes.c_double, ctypes.c_double,
                                             ctypes.POINTER(TenoBatchTuning), _VP, ctypes.c_size_t, _VP]),
    ("teno_rhs_noalloc", ctypes.c_int, [_GP, _VP, _VP, _VP]),
    ("teno_scalar_workspace_bytes", ctypes.c_size_t, [_GP]),
    ("teno_scalar_rhs", ctypes.c_int, [_GP, ctypes.c_double, ctypes.c_int, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    ("teno_scalar_rk3_step", ctypes.c_int, [_GP, ctypes.c_double, ctypes.c_int, _VP, ctypes.c_double, _VP,
                                            ctypes.c_size_t, _VP]),
    ("teno_timer_begin", ctypes.c_int, []),
    ("teno_timer_end", ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
    ("teno_probe_fp64", ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int64, _VP]),
    ("teno_probe_recip", ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP]),
    ("teno_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("teno_abi_version", ctypes.c_int, []),
]

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load the library (building it first if sources are newer)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if path is None:
            from . import build as _build
            try:
                _build.build()
            except RuntimeError:
                if not os.path.exists(p):
                    raise
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with paper_2003_09145_gb300.build.build()")
        L = ctypes.CDLL(p)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def check(status: int, where: str) -> None:
    if status != TENO_OK:
        raise TenoError(status, where)


def make_grid(n, dx, bc, gamma=1.4, H=10.0, b_l=4, b_u=10, eps=1e-6, scheme="lad", ct_m=7, grav=None,
              bc_state=None) -> TenoGrid:
    """teno_grid for an ndim = len(n) grid; bc may be one value or one per axis."""
    ndim = len(n)
    g = TenoGrid()
    g.ndim = ndim
    bcs = list(bc) if isinstance(bc, (list, tuple)) else [bc] * ndim
    for k in range(3):
        g.n[k] = int(n[k]) if k < ndim else 1
        g.dx[k] = float(dx[k]) if k < ndim else 1.0
        g.bc[k] = int(bcs[k]) if k < ndim else 0
    g.gamma, g.H, g.b_l, g.b_u, g.eps = float(gamma), float(H), int(b_l), int(b_u), float(eps)
    g.scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    g.ct_m = int(ct_m)
    for k, v in enumerate(list(grav or [])[:3]):
        g.grav[k] = float(v)
    if bc_state is not None:
        # [3][2][5] conservative ghost states of fixed-state faces
        flat = [float(x) for row in bc_state for side in row for x in side]
        for i, v in enumerate(flat[:30]):
            g.bc_state[i] = v
    return g
