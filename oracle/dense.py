"""Plain CPU dense-block H|psi> (TEST INFRASTRUCTURE ONLY).

Only the tests and the bench's CPU-baseline leg may use this module; it never
touches the CUDA path.

The operator is the paper's bipartite form (Eq. 2) with dense side operators
on symmetry blocks (its DMRG setting): with the state stored as blocks Psi_q
(row index on the left, column index on the right),
    (H psi)_q = H_L,q Psi_q + Psi_q H_R,q^T + sum_m L_m,(q-d_m) Psi_(q-d_m) R_m,(q-d_m)^T,
which is the Vec identity [L (x) R] Vec(Psi) = Vec(L Psi R^T) applied term by
term.  ``dense_apply`` evaluates that block formula with numpy products;
``dense_matrix`` builds the same operator as one matrix from Kronecker
products (a different route, for small sizes) so the two pin each other.
"""
from __future__ import annotations

import numpy as np


def _blocks(model, x):
    off = model.offsets()
    return [np.asarray(x[off[q]:off[q + 1]], dtype=np.float64).reshape(int(c), int(c))
            for q, c in enumerate(model.chi)]


def dense_apply(model, x: np.ndarray) -> np.ndarray:
    """y = H x by the block formula (FP64)."""
    P = _blocks(model, x)
    nq = len(model.chi)
    Y = [model.HL[q] @ P[q] + P[q] @ model.HR[q].T for q in range(nq)]
    for d, Ls, Rs in zip(model.delta, model.Lm, model.Rm):
        for q in range(nq):
            if Ls[q] is None:
                continue
            Y[q + d] += Ls[q] @ P[q] @ Rs[q].T
    return np.concatenate([y.reshape(-1) for y in Y])


def dense_matrix(model) -> np.ndarray:
    """The whole operator as a matrix on the concatenated row-major blocks,
    assembled from Kronecker products: row-major Vec(A P B^T) = (A (x) B) Vec(P)."""
    off = model.offsets()
    n = int(off[-1])
    H = np.zeros((n, n))
    for q, c in enumerate(model.chi):
        c = int(c)
        s = slice(off[q], off[q + 1])
        H[s, s] += np.kron(model.HL[q], np.eye(c)) + np.kron(np.eye(c), model.HR[q])
    for d, Ls, Rs in zip(model.delta, model.Lm, model.Rm):
        for q in range(len(model.chi)):
            if Ls[q] is None:
                continue
            H[off[q + d]:off[q + d + 1], off[q]:off[q + 1]] += np.kron(Ls[q], Rs[q])
    return H
