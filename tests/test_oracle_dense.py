"""Pins of the oracle's dense-block H|psi> (CPU only).

The block formula (``dense_apply``) is checked against the operator
assembled from Kronecker products (``dense_matrix``), against the closed-form
spectrum of a single block without cross terms (eigenvalues e_i(H_L) +
e_j(H_R)), and for symmetry (adjoint pairs of cross terms).
"""
import numpy as np

import workloads.dense as WD


def test_block_formula_equals_kron_matrix():
    from oracle.dense import dense_apply, dense_matrix

    m = WD.dense_block_operator([3, 5, 4, 2, 1], n_pairs=2, seed=7)
    H = dense_matrix(m)
    rng = np.random.default_rng(1)
    for _ in range(3):
        x = rng.standard_normal(m.dim)
        np.testing.assert_allclose(dense_apply(m, x), H @ x, rtol=0, atol=1e-13)


def test_single_block_spectrum_is_sum_of_side_spectra():
    from oracle.dense import dense_matrix

    m = WD.dense_block_operator([6], n_pairs=0, seed=3)
    ev = np.sort(np.linalg.eigvalsh(dense_matrix(m)))
    el, er = np.linalg.eigvalsh(m.HL[0]), np.linalg.eigvalsh(m.HR[0])
    ref = np.sort((el[:, None] + er[None, :]).reshape(-1))
    np.testing.assert_allclose(ev, ref, atol=1e-13)


def test_operator_is_symmetric():
    from oracle.dense import dense_apply

    m = WD.dense_block_operator([4, 7, 5, 3], n_pairs=3, seed=11)
    rng = np.random.default_rng(2)
    x, z = rng.standard_normal(m.dim), rng.standard_normal(m.dim)
    assert abs(z @ dense_apply(m, x) - x @ dense_apply(m, z)) < 1e-12 * np.linalg.norm(x) * np.linalg.norm(z)


def test_block_dims_follow_the_exponential_law():
    chi = WD.block_dims(4000, 0.95, 21)
    assert abs(int(chi.sum()) - 4000) < 25 and chi.argmax() == 10
    r = chi[10] / chi[11]
    assert abs(np.log(r) - 0.95) < 0.05
