"""ed_apply_H_noalloc: the H|psi> entry point for callers that cannot allocate
device memory (its scratch is a fixed array inside the library).  Checked
through the C ABI against ed_apply_H and against the CPU oracle (outputs
matched by bit-string key), within the FP64 tolerance of the other parity
tests (relative L2 <= 1e-12), on two calls in a row with different inputs;
the device's free memory is the same before and after those calls, and the
size limit is checked too.  Kept in its own file, collected last, and
independent of the other tests' state."""
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


def _model(name):
    if name == "hub12":
        return W.config_hub12()
    if name == "heis16":
        return W.config_heis16()
    return W.j1j2_torus(4, 4, 1.0, 0.3, cut_mask=0xFF)  # J2/2 = 0.15: not dyadic, FP64 kernels


@pytest.mark.parametrize("name", ["hub12", "heis16", "j1j2_4x4_nondyadic"])
def test_noalloc_matches_apply_and_oracle_twice(ed, oracle_mod, name):
    import torch

    m = _model(name)
    ctx = ed.build_local_ops(ed.build_sectors(m))
    okeys = oracle_mod.sector_keys(m)
    pos = oracle_mod.find_keys(m, okeys, ctx.state_keys())
    assert (pos >= 0).all()
    xs, refs, ys = [], [], []
    for seed in (1, 2):
        x = torch.empty(ctx.dim, dtype=torch.float64, device="cuda")
        ed.random_vector(ctx, x, seed=seed)
        y_ref = torch.empty_like(x)
        ed.apply_H(ctx, x, y_ref)  # the context's own scratch is allocated here, before the check below
        xs.append(x)
        refs.append(y_ref)
        ys.append(torch.full_like(x, float("nan")))
    ed.apply_H_noalloc(ctx, xs[0], ys[0])  # first call on the device: looks up the array's address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for x, y in zip(xs, ys):
        ed.apply_H_noalloc(ctx, x, y)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0  # nothing allocated or freed by the two calls
    for seed, x, y, y_ref in zip((1, 2), xs, ys, refs):
        err = (torch.linalg.norm(y - y_ref) / torch.linalg.norm(y_ref)).item()
        assert err <= TOL64, (name, seed, err)
        xo = np.zeros(len(okeys))
        xo[pos] = x.cpu().numpy()
        yo = oracle_mod.apply_H(m, okeys, xo)[pos]
        yg = y.cpu().numpy()
        assert np.linalg.norm(yg - yo) <= TOL64 * np.linalg.norm(yo), (name, seed)


def test_noalloc_rejects_oversized_sector(ed):
    from paper_2605_07621_gb300 import EDError, _lib

    ctx = ed.build_local_ops(ed.build_sectors(W.config_j1j2_4x7()))  # 40,116,600 states > 4,194,272
    st = _lib.load().ed_apply_H_noalloc(ctx.handle, ctypes.c_void_p(256), ctypes.c_void_p(1 << 40), None)
    assert st == _lib.ED_EINVAL
    assert b"static scratch holds" in _lib.load().ed_last_error()
    with pytest.raises(EDError, match="ED_EINVAL"):
        _lib.check(st)
