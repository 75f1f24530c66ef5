"""Pins of the oracle's entanglement spectrum (CPU only).

The oracle reads the spectrum from the singular values of every sector block
Psi_s.  These tests fix it by routes that do not use that construction:
closed forms (a singlet, a product state, the free-fermion Slater product
across the spin cut), the reduced density matrix formed by an explicit
partial trace over side B in the full 2^N space, the A <-> B mirror
symmetry of the Schmidt decomposition, and the normalisation.
"""
import math

import numpy as np
import pytest

import workloads as W


def _flat(lams):
    return np.sort(np.concatenate(lams))[::-1]


def test_singlet_dimer(oracle_mod):
    # two sites, one Heisenberg bond, cut between them: the ground state is the
    # singlet (|up dw> - |dw up>)/sqrt(2), Schmidt weights 1/2, 1/2, entropy ln 2
    m = W.Model("spin", 2, np.array([[0, 1]]), jxy=np.ones(1), jz=np.ones(1), n_up=1, cut_mask=0b01)
    keys = oracle_mod.sector_keys(m)
    e0, psi, _ = oracle_mod.ground_state(m, keys)
    assert abs(e0 + 0.75) < 1e-14
    s, lams, wts, S = oracle_mod.entanglement_spectrum(m, keys, psi)
    assert list(s) == [0, 1]
    for lam in lams:
        np.testing.assert_allclose(lam, [0.5], atol=1e-14)
    assert abs(S - math.log(2.0)) < 1e-13
    np.testing.assert_allclose(wts, [0.5, 0.5], atol=1e-14)


def test_product_state(oracle_mod):
    # a single basis state has one Schmidt value 1 and zero entropy
    m = W.xxz_chain(8, 1.0, 0.5, cut_mask=0b10110010)
    keys = oracle_mod.sector_keys(m)
    psi = np.zeros(len(keys))
    psi[17] = 1.0
    s, lams, wts, S = oracle_mod.entanglement_spectrum(m, keys, psi)
    flat = _flat(lams)
    assert flat[0] == 1.0 and np.all(flat[1:] == 0.0)
    assert S == 0.0
    assert wts.sum() == 1.0


def _partial_trace_spectrum(m, keys, psi):
    """rho_A[a, a'] = sum_b psi(a, b) psi(a', b) by explicit loops over the full
    2^N space (side A = cut_mask), then its eigenvalues."""
    n = m.n_sites
    amask = m.cut_mask
    a_sites = [i for i in range(n) if (amask >> i) & 1]
    full = np.zeros(1 << n)
    full[np.asarray(keys, dtype=np.int64)] = psi

    def a_index(k):
        return sum(((k >> i) & 1) << p for p, i in enumerate(a_sites))

    dim_a = 1 << len(a_sites)
    rho = np.zeros((dim_a, dim_a))
    for k in range(1 << n):
        if full[k] == 0.0:
            continue
        for k2 in range(1 << n):
            if full[k2] != 0.0 and (k & ~amask) == (k2 & ~amask):
                rho[a_index(k), a_index(k2)] += full[k] * full[k2]
    return np.sort(np.linalg.eigvalsh(rho))[::-1]


@pytest.mark.parametrize("cut", [0b10110010, 0b00001111, 0b01010101])
def test_partial_trace_brute_force(oracle_mod, cut):
    m = W.xxz_chain(8, 1.0, 0.7, cut_mask=cut)
    keys = oracle_mod.sector_keys(m)
    psi = W.start_values(keys, 4242)
    psi /= np.linalg.norm(psi)
    _, lams, _, S = oracle_mod.entanglement_spectrum(m, keys, psi)
    ref = _partial_trace_spectrum(m, keys, psi)
    flat = _flat(lams)
    assert len(flat) == len(ref) == 16  # sum_s min(C(4,s), C(4,4-s)) = 2^4
    np.testing.assert_allclose(flat, ref, atol=1e-14)
    p = ref[ref > 1e-300]
    assert abs(S + np.sum(p * np.log(p))) < 1e-12


def test_free_fermion_spin_cut_is_a_product(oracle_mod):
    # at U = 0 a non-degenerate ground state is the Slater determinant of the
    # up electrons times that of the down electrons: one Schmidt value 1
    m = W.hubbard_chain(6, 1.0, 0.0, 2, 3, pbc=False)
    keys = oracle_mod.sector_keys(m)
    _, psi, _ = oracle_mod.ground_state(m, keys, tol=1e-15)
    s, lams, _, S = oracle_mod.entanglement_spectrum(m, keys, psi)
    assert list(s) == [2] and len(lams[0]) == 15  # C(6,2) up rows, C(6,3) = 20 down columns
    assert abs(lams[0][0] - 1.0) < 1e-10 and np.all(np.abs(lams[0][1:]) < 1e-10)
    assert S < 1e-8


def test_interacting_spin_cut_is_entangled(oracle_mod):
    # U > 0 mixes up and down configurations: several Schmidt values, S > 0
    m = W.hubbard_chain(6, 1.0, 4.0, 3, 3)
    keys = oracle_mod.sector_keys(m)
    _, psi, _ = oracle_mod.ground_state(m, keys)
    _, lams, wts, S = oracle_mod.entanglement_spectrum(m, keys, psi)
    assert lams[0][1] > 1e-4 and S > 0.1
    assert abs(lams[0].sum() - 1.0) < 1e-12 and abs(wts[0] - 1.0) < 1e-12


def test_mirror_cut_and_normalisation(oracle_mod):
    # Psi_s and its transpose have the same singular values: swapping the
    # sides gives the same spectrum; the eigenvalues sum to ||psi||^2
    m = W.j1j2_torus(4, 2, cut_mask=0b00001111)
    mc = W.j1j2_torus(4, 2, cut_mask=0b11110000)
    keys = oracle_mod.sector_keys(m)
    psi = W.start_values(keys, 99)
    _, lams, wts, S = oracle_mod.entanglement_spectrum(m, keys, psi)
    _, lamc, wtc, Sc = oracle_mod.entanglement_spectrum(mc, keys, psi)
    np.testing.assert_allclose(_flat(lams), _flat(lamc), atol=1e-13)
    assert abs(S - Sc) < 1e-12
    nrm2 = float(psi @ psi)
    assert abs(_flat(lams).sum() - nrm2) < 1e-12 * nrm2 and abs(wts.sum() - nrm2) < 1e-12 * nrm2
    assert abs(wtc.sum() - nrm2) < 1e-12 * nrm2
