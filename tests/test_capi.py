"""The C-ABI library loads and exports every entry point include/teno.h declares;
host-side validation rejects bad arguments before any launch (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(teno_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2003_09145_gb300 import _lib
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 8
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_2003_09145_gb300 import _lib
    bound = {name for name, _, _ in _lib.SIGNATURES}
    assert set(_declared()) <= bound


def test_grid_validation(lib):
    from paper_2003_09145_gb300 import _lib
    good = _lib.make_grid((32, 16), (0.1, 0.1), 1)
    assert lib.teno_workspace_bytes(ctypes.byref(good), _lib.OP_RHS) > 0
    assert lib.teno_flag_count(ctypes.byref(good)) == 4 * 2 * (33 * 16 + 32 * 17)
    bad = []
    g = _lib.make_grid((32, 16), (0.1, 0.1), 1); g.ndim = 4; bad.append(g)
    g = _lib.make_grid((32, 16), (0.1, 0.1), 1); g.dx[1] = 0.0; bad.append(g)
    g = _lib.make_grid((32, 16), (0.1, 0.1), 1); g.bc[0] = 7; bad.append(g)
    g = _lib.make_grid((32, 16), (0.1, 0.1), 1); g.b_u = g.b_l; bad.append(g)
    g = _lib.make_grid((32, 16), (0.1, 0.1), 1); g.n[2] = 3; bad.append(g)
    g = _lib.make_grid((32, 16), (0.1, 0.1), 1); g.n[0] = 0; bad.append(g)     # empty grid
    g = _lib.make_grid((32, 16), (0.1, 0.1), 1); g.n[1] = -4; bad.append(g)
    g = _lib.make_grid((32, 16), (0.1, 0.1), 1); g.gamma = 1.0; bad.append(g)
    g = _lib.make_grid((32, 16), (0.1, 0.1), 1); g.eps = -1.0; bad.append(g)
    g = _lib.make_grid((32, 16), (0.1, 0.1), 1); g.scheme = 4; bad.append(g)
    g = _lib.make_grid((32, 16), (0.1, 0.1), 1, scheme="teno5", ct_m=0); bad.append(g)
    g = _lib.make_grid((32, 16), (0.1, 0.1), 1, scheme="teno5", ct_m=16); bad.append(g)
    # 2049 x 2048 x 1024 > 2^32 interfaces along x (32-bit interface indices)
    bad.append(_lib.make_grid((2048, 2048, 1024), (0.1, 0.1, 0.1), 0))
    assert lib.teno_workspace_bytes(ctypes.byref(_lib.make_grid((2048, 2047, 1023), (0.1, 0.1, 0.1), 0)),
                                    _lib.OP_RHS) > 0
    for g in bad:
        assert lib.teno_workspace_bytes(ctypes.byref(g), _lib.OP_RHS) == 0
        st = lib.teno_rhs(ctypes.byref(g), None, None, None, None, 0, None)
        assert st == 1  # TENO_ERR_INVALID_ARG


def test_null_and_host_pointers_rejected(lib):
    from paper_2003_09145_gb300 import _lib
    import numpy as np
    g = _lib.make_grid((16,), (0.1,), 1)
    U = np.ones(3 * 16)
    R = np.zeros(3 * 16)
    ws = np.zeros(1 << 16, dtype=np.uint8)
    # host memory is never accepted as a device array
    st = lib.teno_rhs(ctypes.byref(g), U.ctypes.data, R.ctypes.data, None, ws.ctypes.data, ws.size, None)
    assert st == 1
    st = lib.teno_rk3_step(ctypes.byref(g), None, 0.5, 0.0, None, 1.0, None, None, 0, None)
    assert st == 1


def test_status_strings(lib):
    lib.teno_status_string.restype = ctypes.c_char_p
    assert lib.teno_status_string(0) == b"TENO_OK"
    assert lib.teno_status_string(4) == b"TENO_ERR_NONPHYSICAL"
    assert lib.teno_status_string(99) == b"TENO_UNKNOWN_STATUS"
    assert lib.teno_abi_version() == 2


def test_scalar_mode_validation(lib):
    """Scalar mode: periodic 1D grids only; bad arguments are rejected on the host."""
    from paper_2003_09145_gb300 import _lib
    import numpy as np
    good = _lib.make_grid((40,), (0.05,), 0)
    nb = lib.teno_scalar_workspace_bytes(ctypes.byref(good))
    assert nb >= 8 * (41 + 2 * 40)
    assert lib.teno_scalar_workspace_bytes(ctypes.byref(_lib.make_grid((40,), (0.05,), 1))) == 0
    assert lib.teno_scalar_workspace_bytes(ctypes.byref(_lib.make_grid((8, 8), (0.1, 0.1), 0))) == 0
    u = np.ones(40)
    ws = np.zeros(nb, dtype=np.uint8)
    # transmissive: unsupported; bad mode, non-finite speed, host memory: invalid
    assert lib.teno_scalar_rhs(ctypes.byref(_lib.make_grid((40,), (0.05,), 1)), 1.0, 0, None, None, None, 0,
                               None) == 2   # TENO_ERR_UNSUPPORTED
    assert lib.teno_scalar_rhs(ctypes.byref(good), 1.0, 7, u.ctypes.data, u.ctypes.data, ws.ctypes.data, nb,
                               None) == 1
    assert lib.teno_scalar_rhs(ctypes.byref(good), float("nan"), 0, u.ctypes.data, None, ws.ctypes.data, nb,
                               None) == 1
    assert lib.teno_scalar_rhs(ctypes.byref(good), 1.0, 0, u.ctypes.data, None, ws.ctypes.data, nb, None) == 1
    assert lib.teno_scalar_rk3_step(ctypes.byref(good), 1.0, 0, u.ctypes.data, 0.01, ws.ctypes.data, nb,
                                    None) == 1


def test_reflecting_walls_accepted_by_the_forward_path_only(lib):
    """bc 2 (reflecting): the forward entry points size and accept it; the
    adjoint and batched entry points answer TENO_ERR_UNSUPPORTED."""
    from paper_2003_09145_gb300 import _lib
    g = _lib.make_grid((32, 16), (0.1, 0.1), (2, 0))
    assert lib.teno_workspace_bytes(ctypes.byref(g), _lib.OP_RK3) > 0
    assert lib.teno_rhs_adjoint(ctypes.byref(g), None, None, None, None, 0, None) == 2
    assert lib.teno_rk3_step_adjoint(ctypes.byref(g), None, 0.1, None, None, None, 0, None) == 2
    assert lib.teno_rk3_step_adjoint_staged(ctypes.byref(g), None, None, None, 0.1, None, None, None, 0, None) == 2
    b = _lib.TenoBatch(2, 10, 2, 1.4, 10.0, 4, 10, 1e-6)
    off = (ctypes.c_int64 * 3)(0, 5, 10)
    assert lib.teno_batch_prepare(ctypes.byref(b), off, None, 0, None) == 2


def test_empty_batch_rejected(lib):
    """A batch of no problems, or of a problem with no cells, is an invalid
    request (no work is launched for it)."""
    from paper_2003_09145_gb300 import _lib
    b = _lib.TenoBatch(0, 0, 1, 1.4, 10.0, 4, 10, 1e-6)
    assert lib.teno_batch_workspace_bytes(ctypes.byref(b)) == 0
    b = _lib.TenoBatch(2, 1, 1, 1.4, 10.0, 4, 10, 1e-6)     # fewer cells than problems
    assert lib.teno_batch_workspace_bytes(ctypes.byref(b)) == 0
