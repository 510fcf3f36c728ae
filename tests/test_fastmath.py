"""The library's table-driven FP64 exp and log (used for every rate constant and
ln T) against high-precision references: exp within 1 ulp everywhere in
[-707, 707]; log within 1.5 ulp on the temperature range [50, 20000] K and in
absolute terms near 1; special values and the shifted out-of-range paths."""
import ctypes as C

import numpy as np
import pytest

from paper_2508_16105_gb300 import build, rde_chem, synth

mpmath = pytest.importorskip("mpmath")


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    lib = rde_chem.load_library()
    lib.rde_selftest_math.argtypes = [C.c_int, C.c_int64, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
    return lib


def host_eval(lib, fn, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    assert lib.rde_selftest_math(fn, x.size, x.ctypes.data, y.ctypes.data, 0, None) == 0
    return y


def ulps(got, ref_mp):
    mpmath.mp.prec = 200
    out = np.empty(len(got))
    for i, (g, r) in enumerate(zip(got, ref_mp)):
        rf = float(r)
        u = np.spacing(abs(rf))
        out[i] = float(abs(mpmath.mpf(g) - r) / mpmath.mpf(u))
    return out


def test_exp_accuracy(lib):
    x = np.concatenate([synth.uniform_range(3, "exp", 4000, -707.0, 707.0),
                        synth.uniform_range(4, "exp-small", 1000, -1e-3, 1e-3),
                        np.array([0.0, 1.0, -1.0, 700.0, -700.0])])
    y = host_eval(lib, 0, x)
    mpmath.mp.prec = 200
    err = ulps(y, [mpmath.exp(mpmath.mpf(v)) for v in x])
    assert err.max() <= 1.0, err.max()
    assert y[-5] == 1.0


def test_log_accuracy(lib):
    T = synth.uniform_range(5, "logT", 4000, 50.0, 20000.0)
    y = host_eval(lib, 1, T)
    mpmath.mp.prec = 200
    err = ulps(y, [mpmath.log(mpmath.mpf(v)) for v in T])
    assert err.max() <= 1.5, err.max()
    near1 = 1.0 + synth.uniform_range(6, "log1", 1000, -0.01, 0.01)
    z = host_eval(lib, 1, near1)
    ref = np.array([float(mpmath.log(mpmath.mpf(v))) for v in near1])
    assert np.abs(z - ref).max() < 5e-17
    assert host_eval(lib, 1, np.array([1.0]))[0] == 0.0


def test_special_values(lib):
    x = np.array([np.nan, np.inf, -np.inf, 710.0, -746.0, -720.0])
    y = host_eval(lib, 0, x)
    assert np.isnan(y[0]) and y[1] == np.inf and y[2] == 0.0 and y[3] == np.inf and y[4] == 0.0
    assert 0 < y[5] < 1e-310          # subnormal result through the shifted path
    # the shifted paths against the mathematics: e^x near the overflow and subnormal
    # thresholds (subnormal results keep fewer bits: relative 2 ulp of their spacing)
    mpmath.mp.prec = 200
    xo = synth.uniform_range(7, "exp-out", 400, 707.0, 709.7)
    yo = host_eval(lib, 0, xo)
    ro = np.array([float(mpmath.exp(mpmath.mpf(v))) for v in xo])
    assert (np.abs(yo - ro) <= 2 * np.spacing(ro)).all()
    xu = synth.uniform_range(8, "exp-under", 400, -744.0, -707.0)
    yu = host_eval(lib, 0, xu)
    ru = np.array([float(mpmath.exp(mpmath.mpf(v))) for v in xu])
    assert (np.abs(yu - ru) <= np.maximum(2 * np.spacing(ru), 1e-12 * ru)).all()
    z = host_eval(lib, 1, np.array([0.0, -1.0, np.inf, 5e-324]))
    assert z[0] == -np.inf and np.isnan(z[1]) and z[2] == np.inf and abs(z[3] + 744.44007192138122) < 1e-12
