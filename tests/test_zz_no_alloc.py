"""ed_apply_H_noalloc: the H|psi> entry point for callers that cannot allocate
device memory (its scratch is a fixed array inside the library).  Checked
through the C ABI against ed_apply_H, within the FP64 tolerance of the other
parity tests (relative L2 <= 1e-12), on two calls in a row with different
inputs; the size limit is checked too.  Kept in its own file, collected
last, and independent of the other tests' state."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def ed():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_07621_gb300 as ed

    return ed


@pytest.mark.parametrize("name", ["hub12", "heis16", "j1j2_4x4_nondyadic"])
def test_noalloc_matches_apply_twice(ed, name):
    import torch

    if name == "hub12":
        m = W.config_hub12()
    elif name == "heis16":
        m = W.config_heis16()
    else:
        m = W.j1j2_torus(4, 4, 1.0, 0.3, cut_mask=0xFF)  # J2/2 = 0.15: not dyadic, FP64 kernels
    ctx = ed.build_local_ops(ed.build_sectors(m))
    for seed in (1, 2):
        x = torch.empty(ctx.dim, dtype=torch.float64, device="cuda")
        ed.random_vector(ctx, x, seed=seed)
        y_ref = torch.empty_like(x)
        ed.apply_H(ctx, x, y_ref)
        y = torch.full_like(x, float("nan"))
        ed.apply_H_noalloc(ctx, x, y)
        torch.cuda.synchronize()
        err = (torch.linalg.norm(y - y_ref) / torch.linalg.norm(y_ref)).item()
        assert err <= TOL64, (name, seed, err)


def test_noalloc_rejects_oversized_sector(ed):
    from paper_2605_07621_gb300 import EDError, _lib

    ctx = ed.build_local_ops(ed.build_sectors(W.config_j1j2_4x7()))  # 40,116,600 states > 4,194,272
    st = _lib.load().ed_apply_H_noalloc(ctx.handle, ctypes.c_void_p(256), ctypes.c_void_p(1 << 40), None)
    assert st == _lib.ED_EINVAL
    assert b"static scratch holds" in _lib.load().ed_last_error()
    with pytest.raises(EDError, match="ED_EINVAL"):
        _lib.check(st)
