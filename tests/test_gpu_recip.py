"""The seeded reciprocal (binary32 seed, one third-order Householder step)
that the Roe average uses: within one ulp of the exact value and of CUDA's
correctly rounded 1.0 / x across the seeded range and at its edges; outside
it CUDA's result itself."""
import ctypes
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_09145_gb300 import _lib
    return _lib.load()


def _probe(lib, x: np.ndarray) -> np.ndarray:
    xd = torch.from_numpy(x).cuda()
    out = torch.empty(2 * x.size, dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.teno_probe_recip(ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                x.size, st) == 0
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(2, x.size)


def _ulps(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    return np.abs(a.view(np.int64) - b.view(np.int64))


def _inputs():
    rng = np.random.default_rng(20030914)
    wide = np.exp2(rng.uniform(-119.5, 119.5, 200_000))
    unit = rng.uniform(0.5, 2.0, 200_000)
    edges = []
    for e in (-120, -1, 0, 1, 119):
        p = math.ldexp(1.0, e)
        edges += [p, math.nextafter(p, 0.0), math.nextafter(p, math.inf)]
    edges = [v for v in edges if math.ldexp(1.0, -120) <= v < math.ldexp(1.0, 120)]
    return np.concatenate([wide, unit, np.array(edges)])


def test_within_one_ulp_of_cuda(lib):
    x = _inputs()
    rec, rec_lib = _probe(lib, x)
    assert np.array_equal(rec_lib, 1.0 / x)          # CUDA's division is correctly rounded
    assert _ulps(rec, rec_lib).max() <= 1
    # most results are the correctly rounded ones
    assert np.mean(rec == rec_lib) > 0.99


def test_within_one_ulp_of_exact(lib):
    getcontext().prec = 60
    x = _inputs()[::97]
    rec, _ = _probe(lib, x)
    for xi, ri in zip(x.tolist(), rec.tolist()):
        assert abs(Decimal(ri) - 1 / Decimal(xi)) <= Decimal(math.ulp(ri)), xi


def test_outside_the_seeded_range_uses_the_library(lib):
    x = np.array([math.ldexp(1.0, -121), math.ldexp(1.0, 120), 1e-300, 1e300, 5e-324,
                  0.0, -1.0, math.inf, math.nan, math.nextafter(math.ldexp(1.0, -120), 0.0)])
    rec, rec_lib = _probe(lib, x)
    np.testing.assert_array_equal(rec, rec_lib)
