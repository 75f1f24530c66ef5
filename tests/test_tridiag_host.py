"""Host eigenvalues of symmetric tridiagonal matrices (``ed_tridiag_eigenvalues``,
the last stage of the entanglement spectrum: the root-free implicit QL
iteration), pinned without a GPU:

* the discrete Laplacian tridiag(-1, 2, -1), whose eigenvalues are
  2 - 2 cos(k pi / (n + 1)) in closed form;
* the 2 x 2 case, (a + c) / 2 +- sqrt(((a - c) / 2)^2 + b^2);
* Wilkinson's W21+ (its two largest eigenvalues agree to about 1e-13; both
  must be resolved) and random matrices against scipy's eigvalsh_tridiagonal;
* a matrix that splits at exact zeros (the union of the parts' spectra) and a
  graded, rank-deficient one (eigenvalues resolved to eps of its norm);
* the argument checks.
"""
import ctypes

import numpy as np
import pytest

from paper_2605_07621_gb300 import _lib

ED_OK, ED_EINVAL = 0, 1


def _eig(d, e):
    d = np.ascontiguousarray(d, dtype=np.float64)
    e = np.ascontiguousarray(e, dtype=np.float64)
    out = np.empty(len(d))
    st = _lib.load().ed_tridiag_eigenvalues(d.ctypes.data if len(d) else None,
                                              e.ctypes.data if len(e) else None, len(d),
                                              out.ctypes.data if len(d) else None)
    assert st == ED_OK, _lib.load().ed_last_error()
    return out


def test_laplacian_closed_form():
    n = 400
    lam = _eig(np.full(n, 2.0), np.full(n - 1, -1.0))
    ref = np.sort(2.0 - 2.0 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1)))
    assert np.abs(lam - ref).max() <= 1e-13


@pytest.mark.parametrize("a,b,c", [(1.0, 0.5, -2.0), (3.0, 1e-9, 3.0), (0.0, 1.0, 0.0), (1e-20, 1e-30, 2e-20)])
def test_two_by_two_closed_form(a, b, c):
    lam = _eig([a, c], [b])
    r = np.hypot((a - c) / 2, b)
    ref = np.array([(a + c) / 2 - r, (a + c) / 2 + r])
    assert np.abs(lam - ref).max() <= 4e-16 * max(abs(a), abs(b), abs(c))


def test_trivial_sizes():
    assert _eig([], []).size == 0
    assert _eig([3.5], []).tolist() == [3.5]


def test_wilkinson_w21_plus():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    d = np.abs(np.arange(-10, 11, dtype=np.float64))
    e = np.ones(20)
    lam = _eig(d, e)
    ref = np.sort(scipy_linalg.eigvalsh_tridiagonal(d, e))
    assert np.abs(lam - ref).max() <= 1e-13
    assert lam[-1] - lam[-2] > 0.0  # the close top pair is two eigenvalues


@pytest.mark.parametrize("n,seed", [(1000, 1), (257, 2)])
def test_random_against_scipy(n, seed):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(seed)
    d, e = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n - 1)
    lam = _eig(d, e)
    ref = np.sort(scipy_linalg.eigvalsh_tridiagonal(d, e))
    assert np.abs(lam - ref).max() <= 1e-12


def test_split_at_exact_zeros():
    rng = np.random.default_rng(3)
    d = rng.uniform(-1, 1, 30)
    e = rng.uniform(-1, 1, 29)
    e[9] = e[19] = 0.0
    lam = _eig(d, e)
    parts = []
    for a, b in [(0, 10), (10, 20), (20, 30)]:
        T = np.diag(d[a:b]) + np.diag(e[a:b - 1], 1) + np.diag(e[a:b - 1], -1)
        parts.append(np.linalg.eigvalsh(T))
    ref = np.sort(np.concatenate(parts))
    assert np.abs(lam - ref).max() <= 1e-14


def test_graded_rank_deficient():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(4)
    n = 300
    scale = 1e-4 * np.exp(-np.arange(n) / 20.0)
    d = scale * rng.uniform(0, 1, n)
    e = scale[:-1] * rng.uniform(-0.5, 0.5, n - 1)
    d[200:] = 0.0
    e[199:] = 0.0
    lam = _eig(d, e)
    ref = np.sort(scipy_linalg.eigvalsh_tridiagonal(d, e))
    norm = np.abs(ref).max()
    assert np.abs(lam - ref).max() <= 1e-14 * norm
    assert (lam == 0.0).sum() >= 100  # the decoupled zero block (rows 200..299) stays exactly zero


def test_argument_checks():
    lib = _lib.load()
    out = np.empty(2)
    d = np.ones(2)
    assert lib.ed_tridiag_eigenvalues(d.ctypes.data, None, -1, out.ctypes.data) == ED_EINVAL
    assert lib.ed_tridiag_eigenvalues(None, None, 2, out.ctypes.data) == ED_EINVAL
    assert lib.ed_tridiag_eigenvalues(d.ctypes.data, None, 2, out.ctypes.data) == ED_EINVAL
