"""CPU checks of the exact fixed-point <-> FP64 conversions used by the FP64
apply path (the same host/device functions the kernels call), against
exact rational arithmetic."""
import ctypes
import os
import random
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def conv():
    import importlib.util

    spec = importlib.util.spec_from_file_location("_ed_build", os.path.join(ROOT, "paper_2605_07621_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    lib = ctypes.CDLL(mod.build())
    to_f = getattr(lib, "_ZN3edk13host_to_fixedEdi")
    to_f.restype = ctypes.c_longlong
    to_f.argtypes = [ctypes.c_double, ctypes.c_int]
    fr_f = getattr(lib, "_ZN3edk15host_from_fixedExi")
    fr_f.restype = ctypes.c_double
    fr_f.argtypes = [ctypes.c_longlong, ctypes.c_int]
    return to_f, fr_f


def _round_half_away(q: Fraction) -> int:
    n = abs(q)
    f = int(n)
    r = n - f
    k = f + (1 if r >= Fraction(1, 2) else 0)
    return k if q >= 0 else -k


def test_to_fixed_exact(conv):
    to_f, _ = conv
    rng = random.Random(5)
    vals = [0.0, -0.0, 1.0, -1.0, 0.5, 2.0 ** -1074, -(2.0 ** -1060), 0.999999999999, 1e-300, 3.25, -0.1]
    vals += [rng.uniform(-1, 1) * 2.0 ** rng.randint(-60, 0) for _ in range(3000)]
    P, E = 52, 1  # |v| < 2
    for v in vals:
        want = _round_half_away(Fraction(v) * Fraction(2) ** (P - E))
        assert to_f(v, P - E) == want, v


def test_from_fixed_round_to_nearest_even(conv):
    _, fr_f = conv
    rng = random.Random(9)
    cases = [0, 1, -1, (1 << 53) - 1, 1 << 53, (1 << 53) + 1, (1 << 54) + 2, (1 << 54) + 6, (1 << 62) - 1,
             -(1 << 62) + 1, 12345678901234567]
    cases += [rng.randint(-(1 << 62), 1 << 62) for _ in range(5000)]
    for Y in cases:
        for e2 in (-60, -52, 0, 7):
            got = fr_f(Y, e2)
            exact = Fraction(Y) * Fraction(2) ** e2
            # float(Fraction) is correctly rounded (nearest, ties to even)
            assert got == float(exact), (Y, e2)


def test_roundtrip_relative_error(conv):
    to_f, fr_f = conv
    x = np.random.default_rng(1).uniform(-1, 1, 2000)
    P, E = 52, 0
    back = np.array([fr_f(to_f(v, P - E), E - P) for v in x])
    assert np.max(np.abs(back - x)) <= 2.0 ** (E - P - 1)


@pytest.fixture(scope="module")
def wide():
    import importlib.util

    spec = importlib.util.spec_from_file_location("_ed_build", os.path.join(ROOT, "paper_2605_07621_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    lib = ctypes.CDLL(mod.build())
    fr = getattr(lib, "_ZN3edk18host_from_fixed128Exyi")
    fr.restype = ctypes.c_double
    fr.argtypes = [ctypes.c_longlong, ctypes.c_ulonglong, ctypes.c_int]
    mw = getattr(lib, "_ZN3edk13host_mul_wideExxPxPy")
    mw.restype = None
    mw.argtypes = [ctypes.c_longlong, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong),
                   ctypes.POINTER(ctypes.c_ulonglong)]
    return fr, mw


def _split128(v: int):
    u = v & ((1 << 128) - 1)
    hi = u >> 64
    if hi >= 1 << 63:
        hi -= 1 << 64
    return hi, u & ((1 << 64) - 1)


def test_mul_wide_exact(wide):
    """64 x 64 -> 128-bit signed products of the wide-weight path, against
    Python integers (two's complement halves)."""
    _, mw = wide
    rng = random.Random(3)
    cases = [(0, 0), (1, -1), (-(1 << 63), -(1 << 63)), ((1 << 63) - 1, (1 << 63) - 1), (-(1 << 63), 1),
             (-1, -1), (123456789, -987654321)]
    cases += [(rng.randint(-(1 << 63), (1 << 63) - 1), rng.randint(-(1 << 63), (1 << 63) - 1)) for _ in range(5000)]
    hi, lo = ctypes.c_longlong(), ctypes.c_ulonglong()
    for a, b in cases:
        mw(a, b, ctypes.byref(hi), ctypes.byref(lo))
        assert (hi.value, lo.value) == _split128(a * b), (a, b)


def test_from_fixed128_round_to_nearest_even(wide):
    """128-bit integer * 2^e2 -> FP64, correctly rounded (ties to even),
    including values whose leading bit is in either half and halfway cases."""
    fr, _ = wide
    rng = random.Random(11)
    cases = [0, 1, -1, (1 << 53) - 1, 1 << 53, (1 << 53) + 1, (1 << 64) - 1, 1 << 64, (1 << 64) + 1,
             (1 << 117) + (1 << 64), (1 << 117) + (1 << 64) + 1, (1 << 118) + (3 << 65), -(1 << 126),
             (1 << 126) - 1, -((1 << 126) - 1), (1 << 63), -(1 << 63)]
    for k in (64, 70, 100, 126):  # exact halfway points at several positions
        m = (1 << 52) + rng.randrange(1 << 52)
        sh = k - 52
        cases += [(m << sh) + (1 << (sh - 1)), ((m | 1) << sh) + (1 << (sh - 1)), -((m << sh) + (1 << (sh - 1)))]
    cases += [rng.randint(-(1 << 126), 1 << 126) for _ in range(5000)]
    cases += [rng.randint(-(1 << 70), 1 << 70) for _ in range(2000)]
    for v in cases:
        hi, lo = _split128(v)
        for e2 in (-170, -120, -60, 0, 5):
            want = float(Fraction(v) * Fraction(2) ** e2)
            assert fr(hi, lo, e2) == want, (v, e2)
