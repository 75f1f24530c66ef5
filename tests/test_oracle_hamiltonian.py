"""Pins of the oracle's Hamiltonian (Eq. (1) models) against closed forms and invariants.

Each pin is chosen so that a plausible slip fails it:
* wrong off-diagonal spin element or sign        -> 2-site/4-ring energies, SU(2), XX free fermions
* wrong S^z S^z normalisation                      -> 2-site singlet, 4-site ring, SU(2)
* wrong periodic wrap / JW sign for fermions       -> U=0 free-fermion energies (rings with t', PBC)
* wrong U term                                     -> Hubbard dimer closed form
* a term leaving the sector                        -> [H, S^z] = 0 / [H, N_sigma] = 0 in the full space
"""
from itertools import product
from math import comb

import numpy as np
import pytest

import workloads as W


def _dense_e0(o, m):
    keys = o.sector_keys(m)
    H = o.dense_H(m, keys)
    return np.linalg.eigvalsh(H)[0], H


def test_two_site_singlet(oracle_mod):
    for J in (1.0, 0.37):
        m = W.xxz_chain(2, J, J, n_up=1, pbc=True)  # de-duplicated: a single bond
        assert m.n_bonds == 1
        e0, _ = _dense_e0(oracle_mod, m)
        assert abs(e0 - (-0.75 * J)) < 1e-14


def test_four_site_ring(oracle_mod):
    m = W.heisenberg_chain(4, 1.3, n_up=2)
    e0, _ = _dense_e0(oracle_mod, m)
    assert abs(e0 - (-2.0 * 1.3)) < 1e-13


@pytest.mark.parametrize("L", [9, 10])
def test_xx_ring_free_fermions(oracle_mod, L):
    """XX ring (jz = 0): Jordan-Wigner free fermions with eps_k = J cos k,
    k = 2 pi (m + phi)/L, phi = 0 for odd and 1/2 for even particle number."""
    J = 0.8
    for n_up in range(1, L):
        m = W.xxz_chain(L, jxy=J, jz=0.0, n_up=n_up)
        e0, _ = _dense_e0(oracle_mod, m)
        phi = 0.0 if n_up % 2 == 1 else 0.5
        eps = np.sort(J * np.cos(2 * np.pi * (np.arange(L) + phi) / L))
        assert abs(e0 - eps[:n_up].sum()) < 1e-12, (L, n_up)


def test_spin_full_space_conserves_sz(oracle_mod):
    """[H, S^z_tot] = 0: in the full 2^N space every term keeps the popcount (integer-exact)."""
    m = W.j1j2_torus(4, 3, 1.0, 0.5)
    n = m.n_sites
    keys = np.arange(1 << n, dtype=np.uint64)
    _, off, nk, nv = oracle_mod.row_terms(m, keys)
    pop_src = np.repeat(np.array([bin(int(k)).count("1") for k in keys]), np.diff(off))
    pop_dst = np.array([bin(int(k)).count("1") for k in nk])
    assert np.array_equal(pop_src, pop_dst)


def test_hubbard_full_space_conserves_n(oracle_mod):
    m = W.hubbard_chain(5, 1.0, 3.0, pbc=True, tp=0.2)
    n = m.n_sites
    keys = np.arange(1 << (2 * n), dtype=np.uint64)
    _, off, nk, nv = oracle_mod.row_terms(m, keys)
    src = np.repeat(keys, np.diff(off))
    mask = np.uint64((1 << n) - 1)
    pc = lambda a: np.array([bin(int(v)).count("1") for v in a])
    assert np.array_equal(pc(src & mask), pc(nk & mask))
    assert np.array_equal(pc(src >> np.uint64(n)), pc(nk >> np.uint64(n)))


def test_su2_commutator(oracle_mod):
    """Isotropic Heisenberg models commute with S^+_tot: H_{n+1} S^+ = S^+ H_n."""
    o = oracle_mod
    m = W.j1j2_torus(4, 2, 1.0, 0.45)  # 8 sites
    n = m.n_sites
    for k in range(0, n):
        ka = o.sector_keys(m, k)
        kb = o.sector_keys(m, k + 1)
        Ha = o.dense_H(m.with_sector(k), ka)
        Hb = o.dense_H(m.with_sector(k + 1), kb)
        pos = {int(v): i for i, v in enumerate(kb)}
        Sp = np.zeros((len(kb), len(ka)))
        for j, key in enumerate(ka):
            for s in range(n):
                if not (int(key) >> s) & 1:
                    Sp[pos[int(key) | (1 << s)], j] += 1.0
        assert np.abs(Hb @ Sp - Sp @ Ha).max() < 1e-12


def test_hermiticity_large(oracle_mod):
    o = oracle_mod
    rng = np.random.default_rng(7)
    for m in (W.config_heis16(), W.j1j2_torus(4, 4), W.config_hub12()):
        keys = o.sector_keys(m)
        a = rng.standard_normal(len(keys))
        b = rng.standard_normal(len(keys))
        lhs = np.dot(a, o.apply_H(m, keys, b))
        rhs = np.dot(o.apply_H(m, keys, a), b)
        assert abs(lhs - rhs) <= 1e-14 * (abs(lhs) + np.linalg.norm(a) * np.linalg.norm(b))


def test_dense_symmetric_and_apply_consistent(oracle_mod):
    o = oracle_mod
    for m in (W.heisenberg_chain(10), W.hubbard_chain(6, 1.0, 4.0, 3, 2, tp=0.3, eps=np.linspace(-1, 1, 6))):
        keys = o.sector_keys(m)
        H = o.dense_H(m, keys)
        assert np.array_equal(H, H.T)
        x = np.random.default_rng(3).standard_normal(len(keys))
        assert np.abs(H @ x - o.apply_H(m, keys, x)).max() < 1e-13


@pytest.mark.parametrize("U,t", [(4.0, 1.0), (8.0, 1.0), (0.0, 0.7), (2.5, 1.3)])
def test_hubbard_dimer(oracle_mod, U, t):
    m = W.hubbard_dimer(t, U)
    e0, _ = _dense_e0(oracle_mod, m)
    assert abs(e0 - (U - np.sqrt(U * U + 16 * t * t)) / 2) < 1e-13


def _one_body(m):
    h = np.diag(np.asarray(m.eps, float)).copy()
    for (i, j), t in zip(m.bonds, m.t):
        h[i, j] -= t
        h[j, i] -= t
    return np.linalg.eigvalsh(h)


@pytest.mark.parametrize("case", range(4))
def test_hubbard_free_fermions(oracle_mod, case):
    """U = 0: E0 = sum of the lowest N_up plus lowest N_dw one-body levels.
    Periodic rings with t' and disorder exercise the Jordan-Wigner sign of
    wrap-around and next-nearest-neighbour hops."""
    rng = np.random.default_rng(100 + case)
    if case == 0:
        m = W.hubbard_chain(8, 1.0, 0.0, 3, 4, pbc=True, tp=0.25, eps=rng.uniform(-1, 1, 8))
    elif case == 1:
        m = W.hubbard_chain(7, 1.0, 0.0, 2, 5, pbc=True, tp=-0.3)
    elif case == 2:
        m = W.hubbard_open_cluster(2, 4, 1.0, 0.0, tp=0.2, eps=rng.uniform(-1, 1, 8), n_up=4, n_dw=3)
    else:
        m = W.hubbard_torus(2, 3, 1.0, 0.0, 2, 4)
    eps = _one_body(m)
    e0, _ = _dense_e0(oracle_mod, m)
    assert abs(e0 - (eps[: m.n_up].sum() + eps[: m.n_dw].sum())) < 1e-12


def test_hubbard_spin_su2(oracle_mod):
    """Hubbard with uniform U commutes with S^+ = sum_i c^dag_{i up} c_{i dw} (built from
    the oracle's own fermion operators, so the relative up/down sign convention is pinned)."""
    o = oracle_mod
    m = W.hubbard_chain(5, 1.0, 3.0, 2, 3, pbc=True, tp=0.15)
    src = m  # (2, 3) -> (3, 2)
    dst = m.with_sector(3, 2)
    ks, kd = o.sector_keys(src), o.sector_keys(dst)
    Hs, Hd = o.dense_H(src, ks), o.dense_H(dst, kd)
    mid = m.with_sector(2, 2)
    km = o.sector_keys(mid)
    Sp = np.zeros((len(kd), len(ks)))
    for j in range(len(ks)):
        e = np.zeros(len(ks))
        e[j] = 1.0
        for i in range(m.n_sites):
            tmp = o.fermion_op(src, i, 1, False, ks, e, km)      # c_{i dw}
            Sp[:, j] += o.fermion_op(mid, i, 0, True, km, tmp, kd)  # c^dag_{i up}
    assert np.abs(Hd @ Sp - Sp @ Hs).max() < 1e-12


# ---------------------------------------------------------------- Anderson impurity (star geometry)

@pytest.mark.parametrize("n_up,n_dw", [(3, 3), (4, 2), (1, 5)])
def test_impurity_atomic_limit(oracle_mod, n_up, n_dw):
    """V = 0: impurity and bath decouple.  E0 = min over the impurity
    occupations (nu, nd) of eps_d (nu + nd) + U nu nd plus the lowest
    n_up - nu and n_dw - nd bath levels."""
    eb = W.impurity_bath(5, seed=3)
    U, ed_ = 3.0, -1.2
    m = W.anderson_impurity(5, U, ed_, 0.0, eb, n_up, n_dw)
    e0, _ = _dense_e0(oracle_mod, m)
    best = min(ed_ * (nu + nd) + U * nu * nd + eb[: n_up - nu].sum() + eb[: n_dw - nd].sum()
               for nu in (0, 1) for nd in (0, 1) if n_up - nu <= 5 and n_dw - nd <= 5)
    assert abs(e0 - best) < 1e-12


def test_impurity_free_fermions(oracle_mod):
    """U = 0: Slater determinants of the star's one-body levels (distinct V_k)."""
    rng = np.random.default_rng(7)
    m = W.anderson_impurity(6, 0.0, 0.3, rng.uniform(0.2, 0.8, 6), W.impurity_bath(6, seed=5), 3, 4)
    eps = _one_body(m)
    e0, _ = _dense_e0(oracle_mod, m)
    assert abs(e0 - (eps[:3].sum() + eps[:4].sum())) < 1e-12


def test_impurity_single_bath_site_closed_form(oracle_mod):
    """One bath orbital at energy 0, one electron of each spin, eps_d = -U/2.
    The configurations with one electron on each site have energy -U/2; the
    doubly occupied and the empty impurity have energy 0.  V couples the
    spin-singlet combination of the former to the symmetric combination of
    the latter with matrix element 2V (the triplet stays at -U/2), so
    E0 = (-U/2 - sqrt(U^2/4 + 16 V^2)) / 2."""
    for U, V in ((2.0, 0.7), (6.0, 0.3), (0.0, 1.1)):
        m = W.anderson_impurity(1, U, -U / 2, V, [0.0], 1, 1)
        e0, _ = _dense_e0(oracle_mod, m)
        assert abs(e0 - (-U / 2 - np.sqrt(U * U / 4 + 16 * V * V)) / 2) < 1e-13
