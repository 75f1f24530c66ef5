"""CPU exact-diagonalisation oracle -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_2605_07621_gb300``) and never imports it; both read their inputs
from ``workloads`` (lattices and seeded values, no method arithmetic).

Parity pins: every function here is checked by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` against closed forms, brute force and invariants.
"""
from .ed import (  # noqa: F401
    lib_path,
    build_oracle,
    sector_keys,
    sector_dim,
    apply_H,
    apply_H_rows,
    RowIndex,
    dense_H,
    row_terms,
    find_keys,
    fermion_op,
    lanczos,
    tridiag_lowest,
    ground_state,
    continued_fraction,
    green_function,
    lehmann_green_function,
    entanglement_spectrum,
    num_threads,
)
