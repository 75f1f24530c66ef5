"""Seeded synthetic dense-block operators (DMRG-style bipartite Hamiltonian).

Inputs only: the block dimensions chi_q of the symmetry sectors and random
operator matrices.  A state is a set of blocks Psi_q (chi_q x chi_q, the left
and right charges of block q are q and Q - q); the operator is
    H = sum_q H_L,q (x) 1 + 1 (x) H_R,q + sum_m L_m (x) R_m,
where H_L,q, H_R,q are symmetric chi_q x chi_q matrices and each cross term m
moves the left charge by delta_m = +1 or -1: L_m has one block
(chi_{q+delta} x chi_q) per q and R_m one block (chi_{q+delta} x chi_q) acting
on the right index.  Terms come in adjoint pairs (delta = +1 with matrices A,
B and delta = -1 with A^T, B^T), so H is symmetric.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np


@dataclass
class DenseBlocks:
    chi: np.ndarray                   # (nq,) block dimensions
    HL: List[np.ndarray]              # nq symmetric chi_q x chi_q
    HR: List[np.ndarray]
    delta: List[int]                  # per cross term: +1 or -1
    Lm: List[List[np.ndarray]]        # per term, per source block q: (chi_{q+d} x chi_q) or None
    Rm: List[List[np.ndarray]]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def dim(self) -> int:
        return int(np.sum(self.chi.astype(np.int64) ** 2))

    def offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.chi.astype(np.int64) ** 2)])


def block_dims(total: int, alpha: float, nq: int) -> np.ndarray:
    """chi_q = C exp(-alpha |q - q0|), q0 the middle sector, scaled so that
    sum_q chi_q is about `total` (each chi_q at least 1)."""
    q0 = (nq - 1) / 2.0
    w = np.exp(-alpha * np.abs(np.arange(nq) - q0))
    return np.maximum(1, np.round(total * w / w.sum())).astype(np.int64)


def dense_block_operator(chi, n_pairs: int = 2, seed: int = 20260507, name: str = "") -> DenseBlocks:
    """Random symmetric side operators (entries U[-1, 1) / sqrt(chi)) and
    n_pairs adjoint pairs of charge-moving cross terms."""
    chi = np.asarray(chi, dtype=np.int64)
    rng = np.random.default_rng(seed)
    nq = len(chi)

    def sym(n):
        a = rng.uniform(-1.0, 1.0, size=(n, n)) / np.sqrt(n)
        return 0.5 * (a + a.T)

    HL = [sym(int(c)) for c in chi]
    HR = [sym(int(c)) for c in chi]
    delta, Lm, Rm = [], [], []
    for _ in range(n_pairs):
        A = [rng.uniform(-1.0, 1.0, size=(int(chi[q + 1]), int(chi[q]))) / np.sqrt(chi[q]) if q + 1 < nq else None
             for q in range(nq)]
        B = [rng.uniform(-1.0, 1.0, size=(int(chi[q + 1]), int(chi[q]))) / np.sqrt(chi[q]) if q + 1 < nq else None
             for q in range(nq)]
        delta.append(+1)
        Lm.append(A)
        Rm.append(B)
        delta.append(-1)   # the adjoint: blocks q+1 -> q with the transposed matrices
        Lm.append([A[q - 1].T.copy() if q >= 1 else None for q in range(nq)])
        Rm.append([B[q - 1].T.copy() if q >= 1 else None for q in range(nq)])
    return DenseBlocks(chi, HL, HR, delta, Lm, Rm, name=name)


def dense_config(alpha: float, total: int = 4000, nq: int = 21, seed: int = 20260507) -> DenseBlocks:
    """The paper's block-size statistics (chi_q = C e^{-alpha q}, total bond
    dimension about 4000) with random operators."""
    return dense_block_operator(block_dims(total, alpha, nq), 2, seed, name=f"dense_a{alpha}")
