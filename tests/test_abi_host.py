"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function declared in include/ed.h, and builds the sector/block
structure of Eqs. (2)-(3) correctly (compared with the oracle's basis)."""
import os
import re
import subprocess
from math import comb

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def edlib():
    import importlib.util

    spec = importlib.util.spec_from_file_location("_ed_build", os.path.join(ROOT, "paper_2605_07621_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    import paper_2605_07621_gb300 as ed

    return ed


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(ed_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_exports_every_declared_symbol(edlib):
    from paper_2605_07621_gb300 import _lib

    declared = _declared_functions()
    assert {"ed_build_sectors", "ed_build_local_ops", "ed_apply_H", "ed_lanczos_ground", "ed_lanczos_gf"} <= declared
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ed_\w+)", out))
    assert declared <= exported, declared - exported
    bound = {s[0] for s in _lib.SIGNATURES}
    assert declared <= bound, declared - bound


@pytest.mark.parametrize("name", ["heis16", "hub12", "j1j2_4x4", "xxz_odd", "hub_small", "degenerate_cut"])
def test_blocks_and_keys_match_oracle(edlib, oracle_mod, name):
    if name == "heis16":
        m = W.config_heis16()
    elif name == "hub12":
        m = W.config_hub12()
    elif name == "j1j2_4x4":
        m = W.j1j2_torus(4, 4, cut_mask=0xFF)
    elif name == "xxz_odd":
        m = W.xxz_chain(11, 1.0, 0.5, n_up=4, cut_mask=0b10110100101)
    elif name == "hub_small":
        m = W.hubbard_chain(6, 1.0, 2.0, 2, 5)
    else:
        m = W.heisenberg_chain(8, cut_mask=0xFF)  # every site on side A
    ctx = edlib.build_sectors(m)
    s, dA, dB, off = ctx.blocks()
    D = oracle_mod.sector_dim(m)
    assert ctx.dim == D == int((dA * dB).sum())
    assert off[0] == 0 and np.all(off[1:] == np.cumsum(dA * dB)[:-1])
    if m.kind == "spin":
        nA = bin(m.cut_mask).count("1")
        nB = m.n_sites - nA
        for si, a, b in zip(s, dA, dB):
            assert a == comb(nA, si) and b == comb(nB, m.n_up - si)
    keys = ctx.state_keys()
    okeys = oracle_mod.sector_keys(m)
    np.testing.assert_array_equal(np.sort(keys), okeys)
    # rows ascend within each block (combinadic order of the side-local bit
    # words), columns too.  Side-local bits (ed_side_sites): on side A the
    # sites on a cross-cut bond come first (low bits), on side B last (high bits)
    if m.kind == "spin":
        inA = [(m.cut_mask >> i) & 1 for i in range(m.n_sites)]
        cut = [False] * m.n_sites
        for i, j in m.bonds:
            if inA[i] != inA[j]:
                cut[i] = cut[j] = True
        sa = [i for i in range(m.n_sites) if inA[i] and cut[i]] + [i for i in range(m.n_sites) if inA[i] and not cut[i]]
        sb = [i for i in range(m.n_sites) if not inA[i] and not cut[i]] + [i for i in range(m.n_sites) if not inA[i] and cut[i]]
        assert ctx.side_sites(0) == sa and ctx.side_sites(1) == sb

        def local(k, sites):
            return sum(((int(k) >> i) & 1) << p for p, i in enumerate(sites))

    for si, a, b, o in zip(s, dA, dB, off):
        blk = keys[o:o + a * b].reshape(a, b)
        if m.kind == "spin":
            assert np.all(np.diff([local(k, sa) for k in blk[:, 0]]) > 0)
            assert np.all(np.diff([local(k, sb) for k in blk[0, :]]) > 0)


def test_j1j2_4x8_structure(edlib):
    ctx = edlib.build_sectors(W.config_j1j2_4x8())
    s, dA, dB, off = ctx.blocks()
    assert ctx.dim == 601080390 and len(s) == 17
    assert dA.max() * dB.max() == 165636900
    w = dA * dB / ctx.dim
    assert abs(1.0 / np.sum(w ** 2) - 5.11) < 0.01
    # side B (columns x = 4..7): the 8 sites of the columns x = 5, 6 take the
    # low bits, the 8 sites on cross-cut bonds (x = 4, 7) the high bits
    assert sorted(ctx.side_sites(1)[:8]) == list(range(20, 28))
    assert sorted(ctx.side_sites(1)[8:]) == list(range(16, 20)) + list(range(28, 32))


def test_malformed_models_rejected(edlib):
    from paper_2605_07621_gb300 import EDError

    bad_bond = W.Model("spin", 4, [(0, 4)], jxy=1.0, jz=1.0, n_up=2, cut_mask=3)
    with pytest.raises(EDError, match="ED_EINVAL"):
        edlib.build_sectors(bad_bond)
    self_bond = W.Model("spin", 4, [(1, 1)], jxy=1.0, jz=1.0, n_up=2, cut_mask=3)
    with pytest.raises(EDError, match="ED_EINVAL"):
        edlib.build_sectors(self_bond)
    bad_sector = W.heisenberg_chain(6, n_up=7)
    with pytest.raises(EDError, match="ED_EINVAL"):
        edlib.build_sectors(bad_sector)
    no_cut = W.hubbard_chain(4)
    no_cut.spin_cut = False
    with pytest.raises(EDError, match="ED_EUNSUPPORTED"):
        edlib.build_sectors(no_cut)
    mask_out = W.heisenberg_chain(6, cut_mask=1 << 7)
    with pytest.raises(EDError, match="ED_EINVAL"):
        edlib.build_sectors(mask_out)


def test_dense_create_rejects_bad_arguments(edlib):
    """Argument checks of ed_dense_create run before any device call."""
    import ctypes

    from paper_2605_07621_gb300 import _lib as L

    lib = L.load()
    chi = np.array([2, 3], dtype=np.int64)
    h = [np.eye(2), np.eye(3)]
    HL = (ctypes.c_void_p * 2)(*[a.ctypes.data for a in h])
    delta = np.array([0], dtype=np.int32)  # a cross term must move the charge
    Lm = (ctypes.c_void_p * 2)()
    out = ctypes.c_void_p()
    assert lib.ed_dense_create(2, chi.ctypes.data, HL, HL, 1, delta.ctypes.data, Lm, Lm, ctypes.byref(out)) == L.ED_EINVAL
    bad = np.array([2, 0], dtype=np.int64)  # empty block
    assert lib.ed_dense_create(2, bad.ctypes.data, HL, HL, 0, None, None, None, ctypes.byref(out)) == L.ED_EINVAL
    assert not out.value
