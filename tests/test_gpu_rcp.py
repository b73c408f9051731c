"""The device reciprocal of the banded attitude solve (rcp_pos: Newton's iteration from an FP32
seed) against the correctly rounded division, over random values in its range and at its
edges.  Algorithm C.1 divides by every pivot; the band solve takes that reciprocal once per row.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def rcp(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path_factory.mktemp("rcp") / "librcp_probe.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                    "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1112_4139_gb300", "csrc"),
                    os.path.join(HERE, "gpu_unit", "rcp_pos_probe.cu"), "-o", out], check=True)
    lib = C.CDLL(out)
    lib.rcp_pos_eval.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]
    lib.rcp_pos_eval.restype = C.c_int

    def run(d):
        d = np.ascontiguousarray(d, dtype=np.float64)
        y = np.empty_like(d)
        q = np.empty_like(d)
        assert lib.rcp_pos_eval(d.ctypes.data, y.ctypes.data, q.ctypes.data, d.size) == 0
        return y, q
    return run


def _ulps(a, b):
    """|a - b| in units of the last place of b (both positive doubles)."""
    return np.abs(a - b) / np.spacing(b)


def test_rcp_pos_within_one_ulp_of_division(rcp):
    rng = np.random.default_rng(7)
    d = np.concatenate([
        2.0 ** rng.uniform(-100, 101, 2_000_000),                 # log-uniform over the Newton range
        rng.uniform(1.0, 2.0, 500_000),                            # every mantissa pattern at one exponent
        np.nextafter(2.0 ** np.arange(-100, 101), 0) * 1.0,        # just below each power of two
        2.0 ** np.arange(-100, 101),                               # powers of two (exact reciprocals)
        np.nextafter(2.0 ** np.arange(-100, 101), np.inf),         # just above
        [2.0 ** -100, np.nextafter(2.0 ** 101, 0), 3.0, 7.0, 1.0 / 3.0],
    ])
    y, q = rcp(d)
    # the compiler's division is the correctly rounded reciprocal: check that against exact
    # rational arithmetic on a sample first
    from fractions import Fraction
    for x, r in zip(d[::50_000], q[::50_000]):
        exact = 1 / Fraction(float(x))
        assert abs(Fraction(float(r)) - exact) <= Fraction(float(np.spacing(r))) / 2
    u = _ulps(y, q)
    assert np.all(np.isfinite(y))
    assert u.max() <= 1.0, f"largest difference {u.max()} ulp at d = {d[np.argmax(u)]!r}"


def test_rcp_pos_outside_the_newton_range_is_the_division(rcp):
    d = np.concatenate([2.0 ** np.arange(-1022, -100, 7.0), 2.0 ** np.arange(101, 1023, 7.0),
                        [5e-324, 1e-310, 1.7e308]])
    y, q = rcp(d)
    assert np.array_equal(y, q)
