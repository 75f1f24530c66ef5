"""Python binding of the C ABI (include/ed.h) with the same names.

Argument marshalling only: every step runs in the CUDA library.  PyTorch
provides device memory and streams; vectors are CUDA tensors laid out as the
C ABI describes (blocks Psi_s concatenated, each row-major d_A x d_B).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib as L

_MODES = {"f64": L.ED_LZ_F64, "f32": L.ED_LZ_F32, "mixed": L.ED_LZ_MIXED}

# ed_build_local_ops flags (include/ed.h)
OPS_DEFAULT = 0
OPS_FORCE_CSR = 1
OPS_FORCE_DENSE = 2


def _stream_handle(stream):
    if stream is None:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """Owns an ``ed_ctx*``; destroyed with the object."""

    def __init__(self, handle: int, model):
        self._h = ctypes.c_void_p(handle)
        self.model = model
        self._ops = False

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and self._h.value:
            L.load().ed_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def dim(self) -> int:
        return int(L.load().ed_dim(self._h))

    @property
    def num_blocks(self) -> int:
        return int(L.load().ed_num_blocks(self._h))

    def blocks(self):
        """(s, d_A, d_B, offset) arrays, one entry per block."""
        n = self.num_blocks
        s = np.zeros(n, np.int32)
        dA = np.zeros(n, np.int64)
        dB = np.zeros(n, np.int64)
        off = np.zeros(n, np.int64)
        L.check(L.load().ed_blocks(self._h, s.ctypes.data, dA.ctypes.data, dB.ctypes.data, off.ctypes.data))
        return s, dA, dB, off

    def state_keys(self, start: int = 0, count: int | None = None) -> np.ndarray:
        if count is None:
            count = self.dim - start
        keys = np.empty(max(count, 1), np.uint64)
        L.check(L.load().ed_state_keys(self._h, int(start), int(count), keys.ctypes.data))
        return keys[:count]

    def side_sites(self, side: int) -> list:
        """Lattice site of each side-local bit of side 0 (A) or 1 (B)."""
        buf = (ctypes.c_int * 64)()
        n = ctypes.c_int()
        L.check(L.load().ed_side_sites(self._h, int(side), buf, ctypes.byref(n)))
        return [buf[i] for i in range(n.value)]

    @property
    def device_bytes(self) -> int:
        return int(L.load().ed_device_bytes(self._h))

    def profile(self, enable: bool = True):
        """Per-stage CUDA-event timing of apply_H (see ed_profile_enable)."""
        L.check(L.load().ed_profile_enable(self._h, 1 if enable else 0))

    def fp64_mode(self) -> str:
        """Arithmetic of the FP64 apply (see ed_fp64_mode): "fp64", "fixed"
        (dyadic couplings), "wide" (128-bit integer weights) or "classed"
        (FP64 weights per value class)."""
        k = int(L.load().ed_fp64_mode(self._h))
        if k < 0:
            raise RuntimeError("build_local_ops has not run on this context")
        return ("fp64", "fixed", "wide", "classed")[k]

    def row_pass(self, dtype) -> str:
        """Row-pass kernel apply_H runs for ``dtype`` (see ed_row_pass)."""
        import torch

        dt = L.ED_F32 if dtype in (torch.float32, "f32") else L.ED_F64
        k = int(L.load().ed_row_pass(self._h, dt))
        return {0: "k_apply_rows", 1: "k_row5"}.get(k, "none")

    def profile_read(self, reset: bool = True):
        """(ms per stage [exp_max, to_fixed, row pass, panel pass], number of applies)."""
        ms = np.zeros(4)
        n = ctypes.c_int64()
        L.check(L.load().ed_profile_read(self._h, ms.ctypes.data, ctypes.byref(n), 1 if reset else 0))
        return ms, n.value


def model_desc(model):
    """ed_model_desc from any object with the fields of ``workloads.Model``;
    returns (desc, keepalive)."""
    kind = L.ED_SPIN if model.kind == "spin" else L.ED_HUBBARD
    bonds = np.ascontiguousarray(np.asarray(model.bonds, dtype=np.int32).reshape(-1, 2))
    keep = {
        "bi": np.ascontiguousarray(bonds[:, 0]),
        "bj": np.ascontiguousarray(bonds[:, 1]),
        "jxy": np.ascontiguousarray(model.jxy, dtype=np.float64),
        "jz": np.ascontiguousarray(model.jz, dtype=np.float64),
        "t": np.ascontiguousarray(model.t, dtype=np.float64),
        "U": np.ascontiguousarray(model.U, dtype=np.float64),
        "eps": np.ascontiguousarray(model.eps, dtype=np.float64),
    }
    P = ctypes.POINTER
    d = L.ModelDesc()
    d.kind = kind
    d.n_sites = int(model.n_sites)
    d.n_bonds = len(bonds)
    d.bi = keep["bi"].ctypes.data_as(P(ctypes.c_int))
    d.bj = keep["bj"].ctypes.data_as(P(ctypes.c_int))
    for f in ("jxy", "jz", "t", "U", "eps"):
        setattr(d, f, keep[f].ctypes.data_as(P(ctypes.c_double)))
    d.n_up = int(model.n_up)
    d.n_dw = int(model.n_dw)
    d.cut_mask = int(model.cut_mask) & 0xFFFFFFFFFFFFFFFF
    d.spin_cut = 1 if model.spin_cut else 0
    return d, keep


def build_sectors(model) -> Context:
    d, keep = model_desc(model)
    h = ctypes.c_void_p()
    L.check(L.load().ed_build_sectors(ctypes.byref(d), ctypes.byref(h)))
    return Context(h.value, model)


def build_local_ops(ctx: Context, flags: int = 0) -> Context:
    L.check(L.load().ed_build_local_ops(ctx.handle, int(flags)))
    ctx._ops = True
    return ctx


def _check_vec(ctx, t, name, dtype=None):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous() or t.numel() != ctx.dim:
        raise ValueError(f"{name} must be contiguous with {ctx.dim} elements")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")


def apply_H(ctx: Context, x, y, stream=None):
    """y = H x (both CUDA tensors, float64 or float32)."""
    import torch

    _check_vec(ctx, x, "x")
    _check_vec(ctx, y, "y", x.dtype)
    dt = {torch.float64: L.ED_F64, torch.float32: L.ED_F32}.get(x.dtype)
    if dt is None:
        raise TypeError("x must be float64 or float32")
    L.check(L.load().ed_apply_H(ctx.handle, _ptr(x), _ptr(y), dt, _stream_handle(stream)))
    return y


def apply_H_noalloc(ctx: Context, x, y, stream=None):
    """y = H x (float64 CUDA tensors) without any device allocation (see ed_apply_H_noalloc)."""
    import torch

    _check_vec(ctx, x, "x", torch.float64)
    _check_vec(ctx, y, "y", torch.float64)
    L.check(L.load().ed_apply_H_noalloc(ctx.handle, _ptr(x), _ptr(y), _stream_handle(stream)))
    return y


def random_vector(ctx: Context, x, seed: int = 20260507, stream=None):
    import torch

    _check_vec(ctx, x, "x")
    dt = {torch.float64: L.ED_F64, torch.float32: L.ED_F32}[x.dtype]
    L.check(L.load().ed_random_vector(ctx.handle, ctypes.c_uint64(seed), _ptr(x), dt, _stream_handle(stream)))
    return x


@dataclass
class LanczosResult:
    e0: float
    iterations: int
    iterations_low: int
    restarts: int
    converged: bool
    e_low: float
    residual: float
    seconds: float
    alpha: np.ndarray
    beta: np.ndarray
    status: int


def lanczos_ground(ctx: Context, mode: str = "f64", max_iter: int = 400, tol: float = 1e-12, check_every: int = 5,
                   fixed_iter: bool = False, reorth: bool = False, seed: int = 20260507, v0=None, psi0=None,
                   refine_block: int = 30, stream=None, ab_capacity: int = 1024, raise_on_noconv: bool = False):
    """Lowest eigenvalue (and optionally eigenvector into ``psi0``, a float64 CUDA tensor)."""
    o = L.LanczosOpts()
    L.load().ed_lanczos_default_opts(ctypes.byref(o))
    o.mode = _MODES[mode]
    o.max_iter = int(max_iter)
    o.tol = float(tol)
    o.check_every = int(check_every)
    o.fixed_iter = 1 if fixed_iter else 0
    o.reorth = 1 if reorth else 0
    o.seed = int(seed)
    o.refine_block = int(refine_block)
    o.stream = _stream_handle(stream)
    if v0 is not None:
        import torch

        _check_vec(ctx, v0, "v0", torch.float64)
        o.v0 = v0.data_ptr()
    if psi0 is not None:
        import torch

        _check_vec(ctx, psi0, "psi0", torch.float64)
    a = np.zeros(ab_capacity)
    b = np.zeros(ab_capacity)
    r = L.Report()
    r.alpha = a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    r.beta = b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    r.ab_capacity = ab_capacity
    e0 = ctypes.c_double()
    st = L.load().ed_lanczos_ground(ctx.handle, ctypes.byref(o), ctypes.byref(e0), _ptr(psi0), ctypes.byref(r))
    if st != L.ED_OK and (st != L.ED_ENOCONV or raise_on_noconv):
        L.check(st)
    return LanczosResult(e0.value, r.iterations, r.iterations_low, r.restarts, bool(r.converged), r.e_low,
                         r.residual, r.seconds, a[: r.n_ab].copy(), b[: r.n_ab].copy(), st)


GF_REORTH = {"auto": -1, "none": 0, "full": 1, "partial": 2}


def lanczos_gf(ctx: Context, psi0, e0: float, omega, eta: float, site: int = 0, spin: int = 0, n_iter: int = 300,
               reorth: str = "auto", stream=None):
    """G(omega + i eta) (complex numpy array) and the Lanczos coefficients.
    reorth: "auto", "none", "full" or "partial" (``ED_GF_REORTH_*``)."""
    import torch

    _check_vec(ctx, psi0, "psi0", torch.float64)
    om = np.ascontiguousarray(omega, dtype=np.float64)
    G = np.zeros(2 * len(om))
    ap, bp, ah, bh = (np.zeros(n_iter) for _ in range(4))
    wp, wh = ctypes.c_double(), ctypes.c_double()
    L.check(L.load().ed_lanczos_gf(ctx.handle, _ptr(psi0), float(e0), int(site), int(spin), int(n_iter),
                                   om.ctypes.data, len(om), float(eta), G.ctypes.data, ap.ctypes.data,
                                   bp.ctypes.data, ah.ctypes.data, bh.ctypes.data, ctypes.addressof(wp),
                                   ctypes.addressof(wh), GF_REORTH[reorth], _stream_handle(stream)))
    coeffs = {"particle": (wp.value, ap, bp), "hole": (wh.value, ah, bh)}
    return G[0::2] + 1j * G[1::2], coeffs


@dataclass
class EntanglementSpectrum:
    s: np.ndarray        # charge of side A of every block (ed_blocks order)
    lam: list            # per block: eigenvalues of rho_A(s) = Psi_s Psi_s^T, descending
    weight: np.ndarray   # per block: ||Psi_s||^2 (trace of rho_A(s))
    entropy: float       # -sum p ln p of the normalised spectrum
    stage_ms: tuple      # ms: the Gram kernels' device time; the rest of the call (device + host QL tail)


def entanglement_spectrum(ctx: Context, psi, stream=None) -> EntanglementSpectrum:
    """Entanglement spectrum of ``psi`` across the cut (``ed_entanglement_spectrum``)."""
    import torch

    _check_vec(ctx, psi, "psi", torch.float64)
    lib = L.load()
    n = ctypes.c_int64()
    L.check(lib.ed_entanglement_spectrum(ctx.handle, _ptr(psi), None, 0, ctypes.byref(n), None, None, None,
                                         _stream_handle(stream)))
    lam = np.zeros(max(n.value, 1))
    s, dA, dB, _ = ctx.blocks()
    wt = np.zeros(len(s))
    ent = ctypes.c_double()
    ms = np.zeros(2)
    L.check(lib.ed_entanglement_spectrum(ctx.handle, _ptr(psi), lam.ctypes.data, n.value, ctypes.byref(n),
                                         wt.ctypes.data, ctypes.addressof(ent), ms.ctypes.data,
                                         _stream_handle(stream)))
    cuts = np.cumsum(np.minimum(dA, dB))[:-1]
    return EntanglementSpectrum(s, np.split(lam[: n.value], cuts), wt, ent.value, (float(ms[0]), float(ms[1])))


class DenseOperator:
    """Owns an ``ed_dense*``: the bipartite operator with dense side operators
    on symmetry blocks (``ed_dense_create``), built from a
    ``workloads.dense.DenseBlocks``."""

    def __init__(self, blocks):
        nq = len(blocks.chi)
        keep = []

        def arr(a):
            a = np.ascontiguousarray(a, dtype=np.float64)
            keep.append(a)
            return a.ctypes.data

        chi = np.ascontiguousarray(blocks.chi, dtype=np.int64)
        HL = (ctypes.c_void_p * nq)(*[arr(h) for h in blocks.HL])
        HR = (ctypes.c_void_p * nq)(*[arr(h) for h in blocks.HR])
        nt = len(blocks.delta)
        delta = np.ascontiguousarray(blocks.delta, dtype=np.int32)
        Lm = (ctypes.c_void_p * max(nt * nq, 1))()
        Rm = (ctypes.c_void_p * max(nt * nq, 1))()
        for m in range(nt):
            for q in range(nq):
                if blocks.Lm[m][q] is not None:
                    Lm[m * nq + q] = arr(blocks.Lm[m][q])
                    Rm[m * nq + q] = arr(blocks.Rm[m][q])
        h = ctypes.c_void_p()
        L.check(L.load().ed_dense_create(nq, chi.ctypes.data, HL, HR, nt, delta.ctypes.data if nt else None, Lm, Rm,
                                         ctypes.byref(h)))
        self._h = h
        self.blocks = blocks

    @property
    def dim(self) -> int:
        return int(L.load().ed_dense_dim(self._h))

    def apply(self, x, y, stream=None):
        import torch

        for v, nm in ((x, "x"), (y, "y")):
            if not (isinstance(v, torch.Tensor) and v.is_cuda and v.dtype == torch.float64 and v.is_contiguous()
                    and v.numel() == self.dim):
                raise ValueError(f"{nm} must be a contiguous CUDA float64 tensor of {self.dim} elements")
        L.check(L.load().ed_dense_apply(self._h, _ptr(x), _ptr(y), _stream_handle(stream)))

    def close(self):
        if self._h is not None and self._h.value:
            L.load().ed_dense_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owns an ``ed_batch*`` (batched independent instances)."""

    def __init__(self, handle: int, models):
        self._h = ctypes.c_void_p(handle)
        self.models = models

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and self._h.value:
            L.load().ed_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def dim(self) -> int:
        return int(L.load().ed_batch_dim(self._h))

    def offsets(self) -> np.ndarray:
        off = np.zeros(len(self.models) + 1, np.int64)
        L.check(L.load().ed_batch_offsets(self._h, off.ctypes.data))
        return off

    def info(self):
        """(modes, tune_ms): each instance's H psi mode (0 CSR, 1 dense on the
        tensor cores with 64-column tiles, 2 with 128-column tiles) and the
        batched apply's device time in ms with every instance in mode 0, 1,
        2 and with the chosen modes."""
        modes = np.zeros(len(self.models), np.int32)
        ms = np.zeros(4, np.float32)
        L.check(L.load().ed_batch_info(self._h, modes.ctypes.data, ms.ctypes.data))
        return modes, ms


def batch_create(models, flags: int = 0) -> Batch:
    descs = (L.ModelDesc * len(models))()
    keep = []
    for i, m in enumerate(models):
        d, k = model_desc(m)
        descs[i] = d
        keep.append(k)
    h = ctypes.c_void_p()
    L.check(L.load().ed_batch_create(descs, len(models), int(flags), ctypes.byref(h)))
    return Batch(h.value, models)


def batch_apply(b: Batch, x, y, stream=None):
    import torch

    for t, nm in ((x, "x"), (y, "y")):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or t.numel() != b.dim:
            raise ValueError(f"{nm} must be a float32 CUDA tensor with {b.dim} elements")
    L.check(L.load().ed_batch_apply(b.handle, _ptr(x), _ptr(y), L.ED_F32, _stream_handle(stream)))
    return y


def batch_lanczos(b: Batch, max_iter: int = 400, tol: float = 1e-7, check_every: int = 5, seed: int = 20260507):
    o = L.LanczosOpts()
    L.load().ed_lanczos_default_opts(ctypes.byref(o))
    o.mode = L.ED_LZ_F32
    o.max_iter = int(max_iter)
    o.tol = float(tol)
    o.check_every = int(check_every)
    o.seed = int(seed)
    n = len(b.models)
    e0 = np.zeros(n)
    it = np.zeros(n, np.int32)
    r = L.Report()
    st = L.load().ed_batch_lanczos(b.handle, ctypes.byref(o), e0.ctypes.data, it.ctypes.data, ctypes.byref(r))
    if st not in (L.ED_OK, L.ED_ENOCONV):
        L.check(st)
    return e0, it, {"steps": r.iterations, "seconds": r.seconds, "all_converged": bool(r.converged), "status": st}


class Server:
    """Continuous-batching request loop (``ed_server*``)."""

    def __init__(self, device_bytes: int = 1 << 30, max_slots: int = 256, max_iter: int = 400, check_every: int = 5,
                 tol: float = 1e-7, seed: int = 20260507, inject_alloc_failures: int = 0):
        o = L.ServerOpts()
        L.load().ed_server_default_opts(ctypes.byref(o))
        o.device_bytes = int(device_bytes)
        o.max_slots = int(max_slots)
        o.max_iter = int(max_iter)
        o.check_every = int(check_every)
        o.tol = float(tol)
        o.seed = int(seed)
        o.inject_alloc_failures = int(inject_alloc_failures)
        h = ctypes.c_void_p()
        L.check(L.load().ed_server_create(ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    def submit(self, model) -> int:
        d, keep = model_desc(model)
        t = ctypes.c_uint64()
        L.check(L.load().ed_server_submit(self._h, ctypes.byref(d), ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int, timeout_ms: int = 60000) -> dict:
        r = L.Result()
        st = L.load().ed_server_wait(self._h, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(r))
        if st != L.ED_OK:
            L.check(st)
        return {"e0": r.e0, "iterations": r.iterations, "converged": bool(r.converged), "status": r.status,
                "latency_s": r.latency_s, "queue_s": r.queue_s, "run_s": r.run_s}

    def cancel(self, ticket: int):
        L.check(L.load().ed_server_cancel(self._h, ctypes.c_uint64(ticket)))

    def stats(self) -> dict:
        s = L.ServerStats()
        L.check(L.load().ed_server_get_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in L.ServerStats._fields_}

    def close(self):
        if self._h is not None and self._h.value:
            L.load().ed_server_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
