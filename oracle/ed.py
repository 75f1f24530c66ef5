"""Plain CPU oracle for H|psi>, Lanczos and the Green's function (TEST INFRASTRUCTURE).

Only tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg may
use this module.  It never touches the CUDA path.

* Basis and H|psi>: ``ed_oracle.c`` (full, unsplit symmetry sector of the
  K-local model of Eq. (1); H applied term by term to bit strings).
* Lanczos: the three-term recurrence in FP64 with optional full
  re-orthogonalisation (classical Gram-Schmidt applied twice); the
  tridiagonal eigenproblem is solved by ``scipy.linalg.eigh_tridiagonal``.
  The paper uses H|psi> as the kernel of any Krylov method (its discussion
  of the Hamiltonian application) but prints no solver, so this is the
  textbook algorithm (Lanczos 1950; Golub and Van Loan, Sec. 10.1).
* Green's function: G_{ii,sigma}(w) = <c (z - (H - E0))^-1 c^dag>
  + <c^dag (z + (H - E0))^-1 c>, z = w + i eta, each term a continued
  fraction of the Lanczos coefficients started from c^dag|psi0> and
  c|psi0> (the paper only names dynamical correlations; this definition is
  the standard zero-temperature one).  ``lehmann_green_function`` gives the
  same quantity as a sum over dense eigenpairs.
* Entanglement spectrum: the eigenvalues of rho_A = Tr_B |psi><psi| per
  charge of side A, as squared singular values of the blocks Psi_s[a, b]
  built from the full-sector keys (``entanglement_spectrum``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np
import scipy.linalg

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ed_oracle.c")
_LIB = os.path.join(_HERE, "libedoracle.so")
_lock = threading.Lock()
_lib = None

OR_SPIN, OR_HUBBARD = 0, 1


class _OrModel(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("n_sites", ctypes.c_int),
        ("n_bonds", ctypes.c_int),
        ("bi", ctypes.POINTER(ctypes.c_int)),
        ("bj", ctypes.POINTER(ctypes.c_int)),
        ("jxy", ctypes.POINTER(ctypes.c_double)),
        ("jz", ctypes.POINTER(ctypes.c_double)),
        ("t", ctypes.POINTER(ctypes.c_double)),
        ("U", ctypes.POINTER(ctypes.c_double)),
        ("eps", ctypes.POINTER(ctypes.c_double)),
    ]


def lib_path() -> str:
    return _LIB


def build_oracle(force: bool = False) -> str:
    """Compile ed_oracle.c (gcc, OpenMP) into oracle/libedoracle.so."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    if _lib is None:
        build_oracle()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        lib.or_sector_dim.restype = ctypes.c_int64
        lib.or_sector_dim.argtypes = [P(_OrModel), ctypes.c_int, ctypes.c_int]
        lib.or_sector_keys.restype = ctypes.c_int64
        lib.or_sector_keys.argtypes = [P(_OrModel), ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64]
        lib.or_apply.restype = ctypes.c_int
        lib.or_apply.argtypes = [P(_OrModel), ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_int]
        lib.or_apply_range.restype = ctypes.c_int
        lib.or_apply_range.argtypes = [P(_OrModel), ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_int64, ctypes.c_void_p, ctypes.c_int]
        lib.or_dense.restype = ctypes.c_int
        lib.or_dense.argtypes = [P(_OrModel), ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        lib.or_rows.restype = ctypes.c_int64
        lib.or_rows.argtypes = [P(_OrModel), ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
        lib.or_find.restype = ctypes.c_int
        lib.or_find.argtypes = [P(_OrModel), ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                ctypes.c_void_p]
        lib.or_fermion_op.restype = ctypes.c_int
        lib.or_fermion_op.argtypes = [P(_OrModel), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                      ctypes.c_void_p]
        lib.or_num_threads.restype = ctypes.c_int
        lib.or_index_new.restype = ctypes.c_void_p
        lib.or_index_new.argtypes = [P(_OrModel), ctypes.c_void_p, ctypes.c_int64]
        lib.or_index_delete.restype = None
        lib.or_index_delete.argtypes = [ctypes.c_void_p]
        lib.or_apply_rows_ix.restype = ctypes.c_int
        lib.or_apply_rows_ix.argtypes = [P(_OrModel), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_void_p, ctypes.c_int]
        _lib = lib
    return _lib


class _ModelRef:
    """Keeps the numpy arrays behind an or_model alive."""

    def __init__(self, model):
        self.bi = np.ascontiguousarray(model.bonds[:, 0], dtype=np.int32)
        self.bj = np.ascontiguousarray(model.bonds[:, 1], dtype=np.int32)
        self.jxy = np.ascontiguousarray(model.jxy, dtype=np.float64)
        self.jz = np.ascontiguousarray(model.jz, dtype=np.float64)
        self.t = np.ascontiguousarray(model.t, dtype=np.float64)
        self.U = np.ascontiguousarray(model.U, dtype=np.float64)
        self.eps = np.ascontiguousarray(model.eps, dtype=np.float64)
        P = ctypes.POINTER
        self.s = _OrModel(
            OR_SPIN if model.kind == "spin" else OR_HUBBARD, model.n_sites, len(self.bi),
            self.bi.ctypes.data_as(P(ctypes.c_int)), self.bj.ctypes.data_as(P(ctypes.c_int)),
            self.jxy.ctypes.data_as(P(ctypes.c_double)), self.jz.ctypes.data_as(P(ctypes.c_double)),
            self.t.ctypes.data_as(P(ctypes.c_double)), self.U.ctypes.data_as(P(ctypes.c_double)),
            self.eps.ctypes.data_as(P(ctypes.c_double)))

    @property
    def ptr(self):
        return ctypes.byref(self.s)


def _sector(model, n_up, n_dw):
    return (model.n_up if n_up is None else n_up), (model.n_dw if n_dw is None else n_dw)


def num_threads() -> int:
    return int(_get().or_num_threads())


def sector_dim(model, n_up=None, n_dw=None) -> int:
    n_up, n_dw = _sector(model, n_up, n_dw)
    return int(_get().or_sector_dim(_ModelRef(model).ptr, n_up, n_dw))


def sector_keys(model, n_up=None, n_dw=None) -> np.ndarray:
    """Ascending bit-string keys of the sector (spin: popcount n_up;
    Hubbard: key = up | dw << S with popcounts n_up, n_dw)."""
    n_up, n_dw = _sector(model, n_up, n_dw)
    ref = _ModelRef(model)
    D = int(_get().or_sector_dim(ref.ptr, n_up, n_dw))
    keys = np.empty(max(D, 1), dtype=np.uint64)
    got = _get().or_sector_keys(ref.ptr, n_up, n_dw, keys.ctypes.data, D)
    if got != D:
        raise RuntimeError("oracle: sector enumeration failed")
    return keys[:D]


def apply_H(model, keys: np.ndarray, x: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """y = H x in the full sector basis ``keys`` (FP64)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    ref = _ModelRef(model)
    if _get().or_apply(ref.ptr, keys.ctypes.data, len(keys), x.ctypes.data, y.ctypes.data, int(nthreads)) != 0:
        raise RuntimeError("oracle: H connects a state outside the sector basis")
    return y


def apply_H_rows(model, keys: np.ndarray, x: np.ndarray, r0: int, r1: int, nthreads: int = 0) -> np.ndarray:
    """Rows [r0, r1) of y = H x (same arithmetic as ``apply_H``)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(max(r1 - r0, 1), dtype=np.float64)
    ref = _ModelRef(model)
    if _get().or_apply_range(ref.ptr, keys.ctypes.data, len(keys), x.ctypes.data, int(r0), int(r1), y.ctypes.data,
                             int(nthreads)) != 0:
        raise RuntimeError("oracle: H connects a state outside the sector basis")
    return y[: r1 - r0]


class RowIndex:
    """The lookup index of one sector's sorted keys, built once, for repeated
    evaluations of listed rows of y = H x (same arithmetic per row as
    ``apply_H``).  Keeps references to the keys and the model."""

    def __init__(self, model, keys: np.ndarray):
        self.keys = np.ascontiguousarray(keys, dtype=np.uint64)
        self.ref = _ModelRef(model)
        self.h = _get().or_index_new(self.ref.ptr, self.keys.ctypes.data, len(self.keys))
        if not self.h:
            raise MemoryError("oracle: index allocation failed")

    def apply_rows(self, x: np.ndarray, rows: np.ndarray, nthreads: int = 0) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        y = np.empty(max(len(rows), 1), dtype=np.float64)
        if _get().or_apply_rows_ix(self.ref.ptr, self.h, x.ctypes.data, rows.ctypes.data, len(rows), y.ctypes.data,
                                   int(nthreads)) != 0:
            raise RuntimeError("oracle: H connects a state outside the sector basis (or a row is out of range)")
        return y[: len(rows)]

    def close(self):
        if self.h:
            _get().or_index_delete(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dense_H(model, keys: np.ndarray) -> np.ndarray:
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    D = len(keys)
    H = np.empty((D, D), dtype=np.float64)
    ref = _ModelRef(model)
    if _get().or_dense(ref.ptr, keys.ctypes.data, D, H.ctypes.data) != 0:
        raise RuntimeError("oracle: H connects a state outside the sector basis")
    return H


def row_terms(model, qkeys: np.ndarray, cap_per_row: int = 512):
    """Matrix elements of the rows ``qkeys``: (diag, offsets, neighbour keys, values)."""
    q = np.ascontiguousarray(qkeys, dtype=np.uint64)
    nq = len(q)
    cap = max(1, nq * cap_per_row)
    diag = np.empty(nq, dtype=np.float64)
    off = np.empty(nq + 1, dtype=np.int64)
    nk = np.empty(cap, dtype=np.uint64)
    nv = np.empty(cap, dtype=np.float64)
    ref = _ModelRef(model)
    tot = _get().or_rows(ref.ptr, q.ctypes.data, nq, diag.ctypes.data, off.ctypes.data, nk.ctypes.data,
                         nv.ctypes.data, cap)
    if tot < 0:
        raise RuntimeError("oracle: row capacity exceeded")
    return diag, off, nk[:tot].copy(), nv[:tot].copy()


def find_keys(model, keys: np.ndarray, q: np.ndarray) -> np.ndarray:
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    q = np.ascontiguousarray(q, dtype=np.uint64)
    pos = np.empty(len(q), dtype=np.int64)
    _get().or_find(_ModelRef(model).ptr, keys.ctypes.data, len(keys), q.ctypes.data, len(q), pos.ctypes.data)
    return pos


def fermion_op(model, site: int, spin: int, create: bool, src_keys, psi, dst_keys) -> np.ndarray:
    """phi = c^dag_{site,spin} psi (create) or c_{site,spin} psi, between Hubbard sectors."""
    src = np.ascontiguousarray(src_keys, dtype=np.uint64)
    dst = np.ascontiguousarray(dst_keys, dtype=np.uint64)
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    phi = np.empty(len(dst), dtype=np.float64)
    r = _get().or_fermion_op(_ModelRef(model).ptr, site, spin, 1 if create else 0, src.ctypes.data, len(src),
                             psi.ctypes.data, dst.ctypes.data, len(dst), phi.ctypes.data)
    if r != 0:
        raise RuntimeError("oracle: fermion operator left the basis")
    return phi


# ----------------------------------------------------------------------------- Krylov


def lanczos(matvec, v0: np.ndarray, n_iter: int, reorth: bool = True, keep_basis: bool = False,
            breakdown: float = 1e-13):
    """Lanczos recurrence from v0 (normalised here).

    Returns (alpha[0..m-1], beta[1..m], V or None) where beta[k-1] is the
    norm beta_k produced after step k-1, so T_m has diagonal alpha and
    off-diagonal beta[:m-1]; beta[m-1] is the residual coupling.
    """
    v = np.array(v0, dtype=np.float64)
    nrm = np.linalg.norm(v)
    v /= nrm
    alphas, betas = [], []
    # the Krylov vectors, row k = v_k (rows 0..k-1 are the basis so far)
    basis = np.empty((n_iter + 1, len(v))) if (reorth or keep_basis) else None
    nb = 0
    if basis is not None:
        basis[0] = v
        nb = 1
    v_prev = np.zeros_like(v)
    beta = 0.0
    for j in range(n_iter):
        w = matvec(v)
        a = float(np.dot(v, w))
        w -= a * v
        if j > 0:
            w -= beta * v_prev
        if reorth:
            B = basis[:nb]
            for _ in range(2):
                w -= B.T @ (B @ w)
        b = float(np.linalg.norm(w))
        alphas.append(a)
        betas.append(b)
        if b < breakdown * max(1.0, abs(a)):
            break
        v_prev, v = v, w / b
        beta = b
        if basis is not None:
            basis[nb] = v
            v = basis[nb]
            nb += 1
    V = None
    if keep_basis:
        V = basis[: len(alphas)].copy()
    return np.array(alphas), np.array(betas), V


def tridiag_lowest(alphas: np.ndarray, betas_off: np.ndarray):
    """Lowest eigenpair of the symmetric tridiagonal matrix (alphas, betas_off)."""
    if len(alphas) == 1:
        return float(alphas[0]), np.ones(1)
    w, s = scipy.linalg.eigh_tridiagonal(alphas, betas_off, select="i", select_range=(0, 0))
    return float(w[0]), s[:, 0]


def ground_state(model, keys=None, n_iter: int = 300, v0=None, seed: int | None = None, reorth: bool = True,
                 tol: float = 1e-13, nthreads: int = 0):
    """Lanczos ground state in the model's sector: (E0, psi0, keys).

    The start vector is ``v0`` or, by default, the seeded key-indexed values
    from ``workloads.start_values``.  Iterates until the lowest Ritz value
    changes by less than ``tol`` (relative) over 5 steps or n_iter is hit.
    """
    from workloads import start_values, DEFAULT_SEED

    if keys is None:
        keys = sector_keys(model)
    if v0 is None:
        v0 = start_values(keys, DEFAULT_SEED if seed is None else seed)
    mv = lambda x: apply_H(model, keys, x, nthreads)
    D = len(keys)
    if D == 1:
        e = float(mv(np.ones(1))[0])
        return e, np.ones(1), keys
    alphas, betas, V = lanczos(mv, v0, min(n_iter, D), reorth=reorth, keep_basis=True)
    e0, s = tridiag_lowest(alphas, betas[: len(alphas) - 1])
    psi = V.T @ s
    psi /= np.linalg.norm(psi)
    return e0, psi, keys


def continued_fraction(z, w0: float, alphas, betas_off):
    """w0 / (z - a0 - b1^2/(z - a1 - b2^2/(...))) evaluated backwards, vectorised over z."""
    z = np.asarray(z, dtype=np.complex128)
    g = np.zeros_like(z)
    m = len(alphas)
    for n in range(m - 1, 0, -1):
        g = betas_off[n - 1] ** 2 / (z - alphas[n] - g)
    return w0 / (z - alphas[0] - g)


def green_function(model, psi0, e0: float, omega, eta: float, site: int = 0, spin: int = 0, n_iter: int = 300,
                   keys=None, reorth: bool = True, return_coeffs: bool = False, nthreads: int = 0):
    """G_{site,site,spin}(omega + i eta) of a Hubbard model by two Lanczos continued fractions."""
    if model.kind != "hubbard":
        raise ValueError("green_function needs a Hubbard model")
    if keys is None:
        keys = sector_keys(model)
    omega = np.asarray(omega, dtype=np.float64)
    z = omega + 1j * eta
    G = np.zeros_like(z)
    coeffs = {}
    for create in (True, False):
        d = 1 if create else -1
        nu = model.n_up + (d if spin == 0 else 0)
        nd = model.n_dw + (d if spin == 1 else 0)
        if nu < 0 or nd < 0 or nu > model.n_sites or nd > model.n_sites:
            continue
        m2 = model.with_sector(nu, nd)
        k2 = sector_keys(m2)
        phi = fermion_op(model, site, spin, create, keys, psi0, k2)
        w0 = float(np.dot(phi, phi))
        if w0 == 0.0:
            continue
        a, b, _ = lanczos(lambda x: apply_H(m2, k2, x, nthreads), phi, min(n_iter, len(k2)), reorth=reorth)
        boff = b[: len(a) - 1]
        if create:
            G += continued_fraction(z + e0, w0, a, boff)
        else:
            G -= continued_fraction(e0 - z, w0, a, boff)
        coeffs["particle" if create else "hole"] = (w0, a, boff)
    if return_coeffs:
        return G, coeffs
    return G


def lehmann_green_function(model, omega, eta: float, site: int = 0, spin: int = 0):
    """Same G as ``green_function`` from dense eigenpairs of the N, N+1, N-1 sectors."""
    keys = sector_keys(model)
    E, U = np.linalg.eigh(dense_H(model, keys))
    e0, psi0 = E[0], U[:, 0]
    z = np.asarray(omega, dtype=np.float64) + 1j * eta
    G = np.zeros_like(z)
    for create in (True, False):
        d = 1 if create else -1
        nu = model.n_up + (d if spin == 0 else 0)
        nd = model.n_dw + (d if spin == 1 else 0)
        if nu < 0 or nd < 0 or nu > model.n_sites or nd > model.n_sites:
            continue
        m2 = model.with_sector(nu, nd)
        k2 = sector_keys(m2)
        phi = fermion_op(model, site, spin, create, keys, psi0, k2)
        E2, U2 = np.linalg.eigh(dense_H(m2, k2))
        wts = (U2.T @ phi) ** 2
        if create:
            G += np.sum(wts[None, :] / (z[:, None] - (E2[None, :] - e0)), axis=1)
        else:
            G += np.sum(wts[None, :] / (z[:, None] + (E2[None, :] - e0)), axis=1)
    return G, e0


def _popcount64(v: np.ndarray) -> np.ndarray:
    """Number of set bits of every uint64 in v (bit by bit)."""
    v = np.asarray(v, dtype=np.uint64)
    c = np.zeros(v.shape, dtype=np.int64)
    for i in range(64):
        c += ((v >> np.uint64(i)) & np.uint64(1)).astype(np.int64)
    return c


def entanglement_spectrum(model, keys: np.ndarray, psi: np.ndarray):
    """Entanglement spectrum of psi across the model's cut.

    The paper's entanglement Hamiltonian is H_E = -log rho_L with
    rho_L = Tr_R |psi><psi| (its discussion of the figure on the distributed
    entanglement spectrum), with spectrum xi_{q,i} per charge q of the left
    side and sector weights W_q = sum_i exp(-xi_{q,i}) / sum_{q,i} exp(-xi_{q,i}).
    Written out: rho_A is block diagonal in the charge s of side A, and the
    eigenvalues of rho_A(s) = Psi_s Psi_s^T are the squared singular values
    of the matrix Psi_s[a, b] = psi(a, b), a over the side-A configurations
    of charge s (rows) and b over the side-B configurations.

    Spin models: side A = the sites of cut_mask, s = its number of up spins.
    Hubbard models (spin cut): side A = the up electrons, side B = the down
    electrons (one block; with all up operators ordered before the down ones
    psi(up, dw) is the Schmidt matrix itself).

    Returns (s ascending, per block the eigenvalues in descending order,
    per block ||Psi_s||^2, the entropy -sum p ln p of the spectrum divided by
    sum ||Psi_s||^2).
    """
    keys = np.asarray(keys, dtype=np.uint64)
    psi = np.asarray(psi, dtype=np.float64)
    if model.kind == "hubbard":
        n = model.n_sites
        a = keys & np.uint64((1 << n) - 1)
        b = keys >> np.uint64(n)
    else:
        amask = np.uint64(model.cut_mask)
        a = keys & amask
        b = keys & ~amask
    s_of = _popcount64(a)
    charges = np.unique(s_of)
    lams, wts = [], []
    for s in charges:
        sel = s_of == s
        ua, ra = np.unique(a[sel], return_inverse=True)
        ub, rb = np.unique(b[sel], return_inverse=True)
        Psi = np.zeros((len(ua), len(ub)))
        Psi[ra, rb] = psi[sel]
        lams.append(np.linalg.svd(Psi, compute_uv=False) ** 2)  # descending
        wts.append(float(np.sum(Psi * Psi)))
    wts = np.array(wts)
    p = np.concatenate(lams) / wts.sum()
    p = p[p > 0]
    return charges, lams, wts, float(-np.sum(p * np.log(p)))
