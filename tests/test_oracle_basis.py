"""Pins of the oracle's sector enumeration: closed-form dimensions and brute force."""
from math import comb

import numpy as np
import pytest

import workloads as W


def test_sector_dims_closed_form(oracle_mod):
    o = oracle_mod
    assert o.sector_dim(W.config_heis16()) == comb(16, 8) == 12870
    assert o.sector_dim(W.config_hub12()) == comb(12, 6) ** 2 == 853776
    assert o.sector_dim(W.config_hub4x4()) == comb(16, 8) ** 2 == 165636900
    assert o.sector_dim(W.config_j1j2_4x8()) == comb(32, 16) == 601080390


@pytest.mark.parametrize("n,k", [(1, 0), (1, 1), (6, 3), (10, 0), (10, 10), (12, 5), (16, 8)])
def test_spin_keys_brute_force(oracle_mod, n, k):
    m = W.xxz_chain(n, n_up=k) if n > 1 else W.Model("spin", 1, np.zeros((0, 2)), n_up=k)
    keys = oracle_mod.sector_keys(m)
    brute = np.array([x for x in range(1 << n) if bin(x).count("1") == k], dtype=np.uint64)
    np.testing.assert_array_equal(keys, brute)


@pytest.mark.parametrize("n,nu,nd", [(4, 2, 2), (5, 1, 3), (6, 3, 3), (6, 0, 6)])
def test_hubbard_keys_brute_force(oracle_mod, n, nu, nd):
    m = W.hubbard_chain(n, n_up=nu, n_dw=nd)
    keys = oracle_mod.sector_keys(m)
    mask = (1 << n) - 1
    brute = np.array([x for x in range(1 << (2 * n))
                      if bin(x & mask).count("1") == nu and bin(x >> n).count("1") == nd], dtype=np.uint64)
    np.testing.assert_array_equal(keys, brute)


def test_find_keys_roundtrip(oracle_mod):
    m = W.config_hub12()
    keys = oracle_mod.sector_keys(m)
    rng = np.random.default_rng(1)
    idx = rng.integers(0, len(keys), 1000)
    pos = oracle_mod.find_keys(m, keys, keys[idx])
    np.testing.assert_array_equal(pos, idx)
    assert oracle_mod.find_keys(m, keys, np.array([0], dtype=np.uint64))[0] == -1
