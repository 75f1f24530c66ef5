"""GPU dense-block H|psi> (``ed_dense_apply``) against the oracle's block formula.

Operators and vectors are seeded inputs from ``workloads.dense``; the oracle
(``oracle.dense.dense_apply``) is pinned on the CPU against the operator
assembled from Kronecker products.  Tolerance: relative L2 <= 1e-12 (FP64
products summed in a different order on either side).
"""
import numpy as np
import pytest

import workloads.dense as WD

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ed():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_07621_gb300 as ed

    return ed


CASES = {
    "ragged": ([1, 63, 64, 65, 130, 17, 2], 2),       # tiles with and without tails, one-element blocks
    "no_cross": ([70, 33, 129], 0),
    "many_terms": ([20, 40, 60, 40, 20], 4),
    "paper_alpha_0.95": (list(WD.block_dims(600, 0.95, 11)), 2),
    "paper_alpha_0.15": (list(WD.block_dims(600, 0.15, 11)), 2),
}


@pytest.mark.parametrize("name", list(CASES))
def test_dense_apply_parity(ed, name):
    import torch

    from oracle.dense import dense_apply

    chi, pairs = CASES[name]
    m = WD.dense_block_operator(chi, n_pairs=pairs, seed=31)
    op = ed.DenseOperator(m)
    assert op.dim == m.dim
    rng = np.random.default_rng(5)
    x = rng.standard_normal(m.dim)
    y_ref = dense_apply(m, x)
    xd = torch.tensor(x, device="cuda")
    yd = torch.full_like(xd, float("nan"))
    op.apply(xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    assert np.linalg.norm(y - y_ref) <= 1e-12 * np.linalg.norm(y_ref)


def test_dense_apply_symmetric_and_errors(ed):
    import torch

    from paper_2605_07621_gb300 import _lib as L

    m = WD.dense_block_operator([5, 90, 70, 3], n_pairs=3, seed=8)
    op = ed.DenseOperator(m)
    x = torch.randn(m.dim, dtype=torch.float64, device="cuda")
    z = torch.randn(m.dim, dtype=torch.float64, device="cuda")
    hx, hz = torch.empty_like(x), torch.empty_like(z)
    op.apply(x, hx)
    op.apply(z, hz)
    a, b = float(z @ hx), float(x @ hz)
    assert abs(a - b) <= 1e-12 * float(x.norm() * z.norm())
    st = L.load().ed_dense_apply(op._h, x.data_ptr(), x.data_ptr(), None)  # x and y overlap
    assert st == L.ED_EINVAL
