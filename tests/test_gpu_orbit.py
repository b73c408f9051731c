"""The tabulated orbital longitude of the observation model (the circular ephemeris of the
synthetic data: L = L0 + 2 pi t / year) against sincospi of the linear longitude, the form it
replaces, over random times across a five-year table, at the table points and the ends of its
steps, and outside the table (where it takes sincospi itself)."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
STEP = 1 << 42          # the table step in ns (kOrbShift)
YEAR_S = 365.25 * 86400.0


@pytest.fixture(scope="module")
def orbit(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path_factory.mktemp("orbit") / "liborbit_probe.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                    "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1112_4139_gb300", "csrc"),
                    os.path.join(HERE, "gpu_unit", "orbit_probe.cu"), "-o", out], check=True)
    lib = C.CDLL(out)
    lib.orbit_eval.argtypes = [C.c_double, C.c_double, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_int64]
    lib.orbit_eval.restype = C.c_int

    def run(t, t0, n_tab, L0=1.234):
        t = np.ascontiguousarray(t, dtype=np.int64)
        out = np.empty((t.size, 4))
        assert lib.orbit_eval(L0, YEAR_S, int(t0), int(n_tab), t.ctypes.data, out.ctypes.data, t.size) == 0
        return out
    return run


def test_table_agrees_with_sincospi(orbit):
    t0 = -STEP
    n_tab = int((5 * YEAR_S * 1e9 + 2 * STEP) // STEP) + 1
    rng = np.random.default_rng(11)
    j = np.arange(n_tab)
    t = np.concatenate([
        rng.integers(t0, t0 + n_tab * STEP, 1_000_000),           # anywhere in the table
        t0 + j * STEP, t0 + (j + 1) * STEP - 1,                     # table points, ends of the steps
        [t0 - 1, t0 - 10**15, t0 + n_tab * STEP, t0 + n_tab * STEP + 10**15],   # outside
    ])
    out = orbit(t, t0, n_tab)
    s, c, s0, c0 = out.T
    # the longitude in extended precision on a sample (pi in extended precision too)
    pi_x = 4 * np.arctan(np.longdouble(1))
    ts = t[::50].astype(np.longdouble)
    L = np.longdouble(1.234) + 2 * pi_x * (ts * np.longdouble(1e-9)) / np.longdouble(YEAR_S)
    sx, cx = np.sin(L).astype(np.float64), np.cos(L).astype(np.float64)
    err_tab = max(np.abs(s[::50] - sx).max(), np.abs(c[::50] - cx).max())
    err_lin = max(np.abs(s0[::50] - sx).max(), np.abs(c0[::50] - cx).max())
    print(f"largest error: table {err_tab:.3g}, sincospi of the FP64 longitude {err_lin:.3g}")
    # Both forms round the longitude in FP64 (the table at its points, the linear form at every
    # t): five years out L / pi is about 10.5, an ulp of it 1.8e-15, so each is within a few
    # 1e-15 of the exact value, and the table is no worse than sincospi.  An error of 2e-14 in
    # the unit vector of the ephemeris moves the residuals by below 1e-17 rad (aberration 1e-4
    # of it, parallax 5e-9 of it, the Roemer delay 1e-11 s).
    assert err_tab < 2e-14 and err_lin < 2e-14, (err_tab, err_lin)
    assert np.max(np.abs(s - s0)) < 3e-14 and np.max(np.abs(c - c0)) < 3e-14
    assert np.max(np.abs(s * s + c * c - 1.0)) < 1e-15
    # outside the table the two are the same computation
    assert np.array_equal(out[-4:, 0], out[-4:, 2]) and np.array_equal(out[-4:, 1], out[-4:, 3])
