"""GB300-native bipartite (entanglement-cut) H|psi>, Lanczos and Green's-function engine.

``paper_2605_07621_gb300.ed`` is the Python binding of the C ABI in
``include/ed.h``; the compute runs only in the CUDA library built by
``paper_2605_07621_gb300.build`` (there is no CPU fallback: importing the
binding without the built library raises ImportError).
"""
from . import _lib

_lib.load()

from .ed import (  # noqa: E402,F401
    OPS_DEFAULT,
    OPS_FORCE_CSR,
    OPS_FORCE_DENSE,
    Batch,
    batch_apply,
    batch_create,
    batch_lanczos,
    Context,
    DenseOperator,
    LanczosResult,
    Server,
    apply_H,
    apply_H_noalloc,
    build_local_ops,
    build_sectors,
    EntanglementSpectrum,
    entanglement_spectrum,
    lanczos_gf,
    lanczos_ground,
    random_vector,
)
from ._lib import EDError  # noqa: E402,F401

__all__ = ["Batch", "batch_apply", "batch_create", "batch_lanczos", "Context", "DenseOperator", "LanczosResult", "Server", "apply_H", "apply_H_noalloc", "build_local_ops", "build_sectors",
           "EntanglementSpectrum", "entanglement_spectrum", "lanczos_gf",
           "lanczos_ground", "random_vector", "EDError", "OPS_DEFAULT", "OPS_FORCE_CSR", "OPS_FORCE_DENSE"]
