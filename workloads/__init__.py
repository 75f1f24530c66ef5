"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This package defines *inputs only*: lattices (bond lists), couplings, target
symmetry sectors, entanglement-cut masks and seeded random vectors keyed by
basis bit strings.  It holds none of the method's arithmetic (no basis
enumeration, no Hamiltonian matrix elements, no Krylov steps), so that the
CUDA path and the CPU oracle can both consume it without sharing code.
"""
from .lattices import (  # noqa: F401
    Model,
    chain_bonds,
    torus_j1j2_bonds,
    square_torus_bonds,
    open_cluster_bonds,
    heisenberg_chain,
    xxz_chain,
    j1j2_torus,
    hubbard_chain,
    hubbard_torus,
    hubbard_open_cluster,
    hubbard_dimer,
    anderson_impurity,
    impurity_bath,
    batched_hubbard_instances,
    config_heis16,
    config_hub12,
    config_j1j2_4x8,
    config_hub4x4,
    config_j1j2_4x7,
    config_qim15,
    CONFIG_NAMES,
    config_by_name,
)
from .startvec import splitmix64, start_values, DEFAULT_SEED  # noqa: F401
