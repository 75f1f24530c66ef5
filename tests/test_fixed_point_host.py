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
