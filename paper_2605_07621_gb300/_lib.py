"""ctypes declarations of the C ABI in include/ed.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libed_gb300.so")

c_int, c_int64, c_uint64, c_double, c_void_p, c_char_p = (ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                                                          ctypes.c_double, ctypes.c_void_p, ctypes.c_char_p)
P = ctypes.POINTER

ED_OK, ED_EINVAL, ED_ENOMEM, ED_ECUDA, ED_ENOCONV, ED_ETIMEOUT, ED_EUNSUPPORTED, ED_ECANCELLED = range(8)
ED_F64, ED_F32 = 0, 1
ED_SPIN, ED_HUBBARD = 0, 1
ED_LZ_F64, ED_LZ_F32, ED_LZ_MIXED = 0, 1, 2
STATUS_NAMES = {0: "ED_OK", 1: "ED_EINVAL", 2: "ED_ENOMEM", 3: "ED_ECUDA", 4: "ED_ENOCONV", 5: "ED_ETIMEOUT",
                6: "ED_EUNSUPPORTED", 7: "ED_ECANCELLED"}


class ModelDesc(ctypes.Structure):
    _fields_ = [
        ("kind", c_int), ("n_sites", c_int), ("n_bonds", c_int),
        ("bi", P(c_int)), ("bj", P(c_int)),
        ("jxy", P(c_double)), ("jz", P(c_double)), ("t", P(c_double)), ("U", P(c_double)), ("eps", P(c_double)),
        ("n_up", c_int), ("n_dw", c_int), ("cut_mask", c_uint64), ("spin_cut", c_int),
    ]


class LanczosOpts(ctypes.Structure):
    _fields_ = [
        ("mode", c_int), ("max_iter", c_int), ("tol", c_double), ("check_every", c_int), ("fixed_iter", c_int),
        ("reorth", c_int), ("seed", c_uint64), ("v0", c_void_p), ("refine_block", c_int), ("stream", c_void_p),
    ]


class Report(ctypes.Structure):
    _fields_ = [
        ("iterations", c_int), ("iterations_low", c_int), ("restarts", c_int), ("converged", c_int),
        ("e_low", c_double), ("residual", c_double), ("seconds", c_double),
        ("alpha", P(c_double)), ("beta", P(c_double)), ("ab_capacity", c_int), ("n_ab", c_int),
    ]


class ServerOpts(ctypes.Structure):
    _fields_ = [("device_bytes", c_int64), ("max_slots", c_int), ("max_iter", c_int), ("check_every", c_int),
                ("tol", c_double), ("seed", c_uint64), ("inject_alloc_failures", c_int)]


class Result(ctypes.Structure):
    _fields_ = [("e0", c_double), ("iterations", c_int), ("converged", c_int), ("status", c_int),
                ("latency_s", c_double), ("queue_s", c_double), ("run_s", c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", c_int64), ("completed", c_int64), ("failed", c_int64), ("queued", c_int64),
                ("running", c_int64), ("p50_s", c_double), ("p99_s", c_double), ("mean_s", c_double),
                ("throughput_rps", c_double), ("device_bytes", c_int64), ("device_bytes_free", c_int64)]


# (name, restype, argtypes) of every function declared in include/ed.h
SIGNATURES = [
    ("ed_build_sectors", c_int, [P(ModelDesc), P(c_void_p)]),
    ("ed_build_local_ops", c_int, [c_void_p, c_int]),
    ("ed_apply_H", c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    ("ed_apply_H_noalloc", c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("ed_lanczos_default_opts", None, [P(LanczosOpts)]),
    ("ed_lanczos_ground", c_int, [c_void_p, P(LanczosOpts), P(c_double), c_void_p, P(Report)]),
    ("ed_lanczos_gf", c_int, [c_void_p, c_void_p, c_double, c_int, c_int, c_int, c_void_p, c_int, c_double,
                              c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int,
                              c_void_p]),
    ("ed_entanglement_spectrum", c_int, [c_void_p, c_void_p, c_void_p, c_int64, P(c_int64), c_void_p, c_void_p,
                                         c_void_p, c_void_p]),
    ("ed_tridiag_eigenvalues", c_int, [c_void_p, c_void_p, c_int64, c_void_p]),
    ("ed_dense_create", c_int, [c_int, c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p,
                                P(c_void_p)]),
    ("ed_dense_dim", c_int64, [c_void_p]),
    ("ed_dense_apply", c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("ed_dense_destroy", None, [c_void_p]),
    ("ed_batch_create", c_int, [c_void_p, c_int, c_int, P(c_void_p)]),
    ("ed_batch_dim", c_int64, [c_void_p]),
    ("ed_batch_offsets", c_int, [c_void_p, c_void_p]),
    ("ed_batch_info", c_int, [c_void_p, c_void_p, c_void_p]),
    ("ed_batch_apply", c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    ("ed_batch_lanczos", c_int, [c_void_p, P(LanczosOpts), c_void_p, c_void_p, P(Report)]),
    ("ed_batch_destroy", None, [c_void_p]),
    ("ed_server_default_opts", None, [P(ServerOpts)]),
    ("ed_server_create", c_int, [P(ServerOpts), P(c_void_p)]),
    ("ed_server_submit", c_int, [c_void_p, P(ModelDesc), P(c_uint64)]),
    ("ed_server_wait", c_int, [c_void_p, c_uint64, c_int, P(Result)]),
    ("ed_server_cancel", c_int, [c_void_p, c_uint64]),
    ("ed_server_get_stats", c_int, [c_void_p, P(ServerStats)]),
    ("ed_server_destroy", None, [c_void_p]),
    ("ed_profile_enable", c_int, [c_void_p, c_int]),
    ("ed_profile_read", c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    ("ed_row_pass", c_int, [c_void_p, c_int]),
    ("ed_fp64_mode", c_int, [c_void_p]),
    ("ed_dim", c_int64, [c_void_p]),
    ("ed_num_blocks", c_int, [c_void_p]),
    ("ed_blocks", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("ed_state_keys", c_int, [c_void_p, c_int64, c_int64, c_void_p]),
    ("ed_side_sites", c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    ("ed_random_vector", c_int, [c_void_p, c_uint64, c_void_p, c_int, c_void_p]),
    ("ed_device_bytes", c_int64, [c_void_p]),
    ("ed_destroy", None, [c_void_p]),
    ("ed_last_error", c_char_p, []),
]

_lib = None


class EDError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: str | None = None):
    """Load the compiled library; raises ImportError if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"CUDA extension {p} is missing: run `python -c 'import __graft_entry__ as g; g.build()'` "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(p)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def check(status: int):
    if status != ED_OK:
        raise EDError(status, (load().ed_last_error() or b"").decode(errors="replace"))
