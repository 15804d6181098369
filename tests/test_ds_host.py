"""CPU checks of the double-single to FP64 conversion that the combination
kernels run on the device (the same routine, compiled for the host): for
renormalised float pairs (h, l) the result equals h + l, computed exactly in
FP64 from the two floats, to within one unit in its last place, including the
cases where h is a power of two and l points into the binade below; non-finite
pairs give NaN."""
import ctypes as C

import numpy as np
import pytest


@pytest.fixture(scope="module")
def conv():
    from paper_2606_09688_gb300 import build
    L = C.CDLL(build.build(force=False))
    f = L.st_host_ds_to_double
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]
    f.restype = C.c_int

    def run(h, l):
        h = np.ascontiguousarray(h, dtype=np.float32)
        l = np.ascontiguousarray(l, dtype=np.float32)
        out = np.empty(len(h))
        assert f(h.ctypes.data, l.ctypes.data, len(h), out.ctypes.data) == 0
        return out
    return run


def _pairs(v):
    """Renormalised pairs of FP64 values: h = fl32(v), l = fl32(v - h)."""
    h = v.astype(np.float32)
    l = (v - h.astype(np.float64)).astype(np.float32)
    return h, l


def _ulps(got, ref):
    return np.abs(got - ref) / np.spacing(np.abs(ref))


def test_random_pairs_within_one_ulp(conv):
    rng = np.random.default_rng(0)
    v = rng.standard_normal(200000) * 10.0 ** rng.uniform(-30, 30, 200000)
    h, l = _pairs(v)
    exact = h.astype(np.float64) + l.astype(np.float64)   # exact: 48 bits at most
    assert np.max(_ulps(conv(h, l), exact)) <= 1.0


def test_powers_of_two_with_low_part_below(conv):
    e = np.arange(-60, 61, dtype=np.float64)
    h = np.concatenate([2.0 ** e, -(2.0 ** e)]).astype(np.float32)
    rng = np.random.default_rng(1)
    frac = rng.uniform(0.0, 0.5, len(h))                  # l towards zero, up to half an ulp of the binade below
    l = (-np.sign(h) * frac * np.spacing(np.abs(h)) / 2).astype(np.float32)
    exact = h.astype(np.float64) + l.astype(np.float64)
    assert np.max(_ulps(conv(h, l), exact)) <= 1.0
    l_up = (np.sign(h) * frac * np.spacing(np.abs(h))).astype(np.float32)
    exact = h.astype(np.float64) + l_up.astype(np.float64)
    assert np.max(_ulps(conv(h, l_up), exact)) <= 1.0


def test_zero_tiny_and_large_magnitudes(conv):
    h = np.array([0.0, -0.0, 1e-37, 3e38, 1.5e-20, -7.25], dtype=np.float32)
    l = np.array([0.0, 0.0, 0.0, 1e31, 1e-28, 2e-7], dtype=np.float32)
    got = conv(h, l)
    assert got[0] == 0.0 and got[1] == 0.0
    exact = h.astype(np.float64) + l.astype(np.float64)
    assert np.all(_ulps(got[2:], exact[2:]) <= 1.0)
    assert np.isnan(conv(np.array([np.nan]), np.array([0.0]))[0])
    assert np.isnan(conv(np.array([np.inf]), np.array([0.0]))[0])   # non-finite values come out as NaN
