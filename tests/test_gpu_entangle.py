"""GPU entanglement spectrum (``ed_entanglement_spectrum``) against the oracle.

Inputs come from the oracle (ground states) or from the seeded key-indexed
generator, never from the CUDA path.  Per block, the eigenvalues of
rho_A(s) = Psi_s Psi_s^T (descending) must agree with the oracle's squared
singular values to 1e-12 absolute for a normalised state (FP64 Gram matrix
and eigensolver: errors of a few ulps of the largest eigenvalue); the block
weights ||Psi_s||^2 to 1e-13 relative and the entropy to 1e-10.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL_LAM = 1e-12


@pytest.fixture(scope="module")
def ed():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_07621_gb300 as ed

    return ed


def _check(ed, oracle_mod, m, psi_of_keys=None, seed=None):
    """psi_of_keys: oracle-ordered vector (with the oracle's keys) or None for
    the seeded start values (normalised)."""
    import torch

    ctx = ed.build_sectors(m)
    okeys = oracle_mod.sector_keys(m)
    if psi_of_keys is None:
        psi_of_keys = W.start_values(okeys, seed)
        psi_of_keys = psi_of_keys / np.linalg.norm(psi_of_keys)
    keys = ctx.state_keys()
    pos = oracle_mod.find_keys(m, okeys, keys)
    assert (pos >= 0).all()
    x = torch.tensor(psi_of_keys[pos], dtype=torch.float64, device="cuda")
    es = ed.entanglement_spectrum(ctx, x)
    s_ref, lam_ref, w_ref, S_ref = oracle_mod.entanglement_spectrum(m, okeys, psi_of_keys)
    assert list(es.s) == list(s_ref)
    for lg, lr in zip(es.lam, lam_ref):
        assert lg.shape == lr.shape
        assert np.max(np.abs(lg - lr)) <= TOL_LAM
    np.testing.assert_allclose(es.weight, w_ref, rtol=1e-13, atol=1e-15)
    assert abs(es.entropy - S_ref) <= 1e-10
    return es


def test_heis16_ground_state(ed, oracle_mod):
    m = W.config_heis16()
    keys = oracle_mod.sector_keys(m)
    _, psi, _ = oracle_mod.ground_state(m, keys)
    es = _check(ed, oracle_mod, m, psi)
    # the singlet ground state of the ring is symmetric under up <-> down:
    # blocks s and 8 - s carry the same spectrum
    for i in range(len(es.s)):
        np.testing.assert_allclose(es.lam[i], es.lam[len(es.s) - 1 - i], atol=1e-12)


@pytest.mark.parametrize("mask", [0xFF, 0x0F0F])
def test_j1j2_4x4_ground_state(ed, oracle_mod, mask):
    m = W.j1j2_torus(4, 4, cut_mask=mask)
    keys = oracle_mod.sector_keys(m)
    _, psi, _ = oracle_mod.ground_state(m, keys)
    _check(ed, oracle_mod, m, psi)


@pytest.mark.parametrize("name", ["hub12", "j1j2_4x6", "xxz_odd_cut", "all_on_A", "all_on_B", "hub_empty_dw",
                                  "qim9"])
def test_random_states(ed, oracle_mod, name):
    # ragged Gram tiles (924 = 14 x 64 + 28), both Gram orientations
    # (d_A < d_B and d_A > d_B), one-column and one-row blocks
    m = {"hub12": W.config_hub12(),
         "j1j2_4x6": W.j1j2_torus(6, 4, cut_mask=0xFFF),
         "xxz_odd_cut": W.xxz_chain(11, 1.0, 0.5, n_up=4, cut_mask=0b10110100101),
         "all_on_A": W.heisenberg_chain(10, cut_mask=0x3FF),
         "all_on_B": W.heisenberg_chain(10, cut_mask=0),
         "hub_empty_dw": W.hubbard_chain(7, 1.0, 2.0, 3, 0),
         "qim9": W.anderson_impurity(8, 4.0, -2.0, 0.5, W.impurity_bath(8), 4, 5)}[name]
    _check(ed, oracle_mod, m, seed=777)


def test_unnormalised_input_and_errors(ed, oracle_mod):
    import ctypes

    import torch

    from paper_2605_07621_gb300 import _lib as L

    m = W.xxz_chain(11, 1.0, 0.5, n_up=4, cut_mask=0b10110100101)
    ctx = ed.build_sectors(m)
    x = torch.tensor(3.0 * W.start_values(ctx.state_keys(), 5), device="cuda")
    es = ed.entanglement_spectrum(ctx, x)
    nrm2 = float((x * x).sum())
    assert abs(sum(l.sum() for l in es.lam) - nrm2) <= 1e-12 * nrm2
    assert abs(es.weight.sum() - nrm2) <= 1e-13 * nrm2
    # size query, too-small capacity
    lib = L.load()
    n = ctypes.c_int64()
    assert lib.ed_entanglement_spectrum(ctx.handle, ctypes.c_void_p(x.data_ptr()), None, 0, ctypes.byref(n), None,
                                        None, None, None) == 0
    s, dA, dB, _ = ctx.blocks()
    assert n.value == int(np.minimum(dA, dB).sum())
    buf = np.zeros(n.value)
    st = lib.ed_entanglement_spectrum(ctx.handle, ctypes.c_void_p(x.data_ptr()), buf.ctypes.data, n.value - 1,
                                      ctypes.byref(n), None, None, None, None)
    assert st == L.ED_EINVAL
