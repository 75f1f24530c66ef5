"""GPU parity of H|psi> (through the C ABI) against the CPU oracle.

Tolerances: FP64 storage -> relative L2 <= 1e-12; FP32 storage (input is
the FP32 rounding of the FP64 vector, compared with the oracle applied to
the FP64 vector) -> relative L2 <= 1e-6.  Outputs are matched to the
oracle's ordering by bit-string key.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-6


@pytest.fixture(scope="module")
def ed():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_07621_gb300 as ed

    return ed


def _models():
    rng = np.random.default_rng(11)
    return {
        "heis16": W.config_heis16(),
        "hub12": W.config_hub12(),
        "j1j2_4x4": W.j1j2_torus(4, 4, cut_mask=0xFF),
        "j1j2_4x4_strip": W.j1j2_torus(4, 4, cut_mask=0b0011001100110011),
        "xxz_odd_cut": W.xxz_chain(11, 1.0, 0.5, n_up=4, cut_mask=0b10110100101),
        "xxz_n_up_1": W.xxz_chain(9, 0.7, 1.3, n_up=1),
        "all_on_A": W.heisenberg_chain(10, cut_mask=0x3FF),
        "all_on_B": W.heisenberg_chain(10, cut_mask=0),
        "hub_tp_eps": W.hubbard_chain(8, 1.0, 3.0, 3, 5, pbc=True, tp=0.27, eps=rng.uniform(-1, 1, 8)),
        "hub_2x3_torus": W.hubbard_torus(2, 3, 1.0, 5.0, 2, 3),
        "hub_open_3x4": W.hubbard_open_cluster(3, 4, 1.0, 6.0, tp=-0.2, eps=rng.uniform(-1, 1, 12), n_up=5, n_dw=7),
        "hub_empty_dw": W.hubbard_chain(7, 1.0, 2.0, 3, 0),
        "hub12_particle": W.hubbard_chain(12, 1.0, 4.0, 7, 6),
        "hub12_hole": W.hubbard_chain(12, 1.0, 4.0, 5, 6),
        "hub_rect_dyadic": W.hubbard_torus(2, 4, 1.0, 2.0, 3, 5),
        # couplings that are not dyadic: 128-bit integer weights (J2 = 0.3),
        # and a value range too wide for them (J2 = 3e-19: FP64 class weights)
        "j1j2_4x4_j2_03": W.j1j2_torus(4, 4, 1.0, 0.3, cut_mask=0xFF),
        "j1j2_4x4_wide_range": W.j1j2_torus(4, 4, 1.0, 3e-19, cut_mask=0xFF),
        "hub_site_U": W.Model("hubbard", 5, W.chain_bonds(5, True), t=1.0, U=[1.0, 2.0, 3.0, 1.0, 0.0],
                              eps=[0.1, -0.2, 0.3, 0.0, 0.5], n_up=2, n_dw=3, spin_cut=True),
        # Anderson impurity (star): one dyadic hybridisation value and disordered
        # bath energies (FP64: integer passes for the hopping, diagonal added in
        # FP64 afterwards), and eight distinct hybridisations (more value
        # classes than the class-sorted kernels take: the general CSR kernels).
        # hub_site_U above also has dyadic hopping and a non-dyadic diagonal.
        "qim_uniform_V": W.anderson_impurity(8, 3.0, -1.5, 0.5, W.impurity_bath(8, seed=11), 4, 5),
        "qim_distinct_V": W.anderson_impurity(8, 2.0, -0.7, rng.uniform(0.2, 0.9, 8), W.impurity_bath(8, seed=12),
                                              5, 3),
    }


MODELS = _models()


def _parity(ed, oracle_mod, m, dtype):
    import torch

    ctx = ed.build_local_ops(ed.build_sectors(m))
    keys = ctx.state_keys()
    okeys = oracle_mod.sector_keys(m)
    pos = oracle_mod.find_keys(m, okeys, keys)
    assert (pos >= 0).all()
    y_ref = oracle_mod.apply_H(m, okeys, W.start_values(okeys))[pos]
    x64 = torch.tensor(W.start_values(keys), device="cuda")
    x = x64.to(dtype)
    y = torch.full_like(x, float("nan"))
    ed.apply_H(ctx, x, y)
    torch.cuda.synchronize()
    yy = y.double().cpu().numpy()
    return np.linalg.norm(yy - y_ref) / np.linalg.norm(y_ref)


@pytest.mark.parametrize("name", list(MODELS))
def test_apply_fp64(ed, oracle_mod, name):
    import torch

    assert _parity(ed, oracle_mod, MODELS[name], torch.float64) <= TOL64


@pytest.mark.parametrize("name", list(MODELS))
def test_apply_fp32(ed, oracle_mod, name):
    import torch

    assert _parity(ed, oracle_mod, MODELS[name], torch.float32) <= TOL32


def test_random_vector_matches_input_generator(ed):
    import torch

    m = MODELS["hub_open_3x4"]
    ctx = ed.build_local_ops(ed.build_sectors(m))
    x = torch.empty(ctx.dim, dtype=torch.float64, device="cuda")
    ed.random_vector(ctx, x, seed=12345)
    ref = W.start_values(ctx.state_keys(), 12345)
    assert np.array_equal(x.cpu().numpy(), ref)


def test_apply_rejects_bad_args(ed):
    import torch

    ctx = ed.build_local_ops(ed.build_sectors(MODELS["heis16"]))
    x = torch.zeros(ctx.dim, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        ed.apply_H(ctx, x, torch.zeros(ctx.dim + 1, dtype=torch.float64, device="cuda"))
    with pytest.raises(ed.EDError, match="overlap"):
        from paper_2605_07621_gb300 import _lib

        _lib.check(_lib.load().ed_apply_H(ctx.handle, x.data_ptr(), x.data_ptr(), 0, None))


def _sampled_rows(ed, oracle_mod, m, n_chunks, chunk, seed=20260507):
    """H x at full size, x = key-indexed start values generated on the GPU;
    checked on n_chunks random chunks of consecutive rows against the
    oracle's row terms evaluated with the same key-indexed values."""
    import torch

    ctx = ed.build_local_ops(ed.build_sectors(m))
    D = ctx.dim
    out = {}
    for dt in (torch.float64, torch.float32):
        x = torch.empty(D, dtype=torch.float64, device="cuda")
        ed.random_vector(ctx, x, seed=seed)
        xd = x.to(dt)
        del x
        y = torch.empty_like(xd)
        ed.apply_H(ctx, xd, y)
        torch.cuda.synchronize()
        rng = np.random.default_rng(3)
        starts = np.sort(rng.integers(0, D - chunk, n_chunks))
        # include both ends of the vector
        starts[0] = 0
        starts[-1] = D - chunk
        idx = (starts[:, None] + np.arange(chunk)[None, :]).ravel()
        yg = y[torch.tensor(idx, device="cuda")].double().cpu().numpy()
        keys = np.concatenate([ctx.state_keys(int(s), chunk) for s in starts])
        diag, off, nk, nv = oracle_mod.row_terms(m, keys)
        xv = W.start_values(keys, seed)
        if dt == torch.float32:
            xv = xv.astype(np.float32).astype(np.float64)
            xn = W.start_values(nk, seed).astype(np.float32).astype(np.float64)
        else:
            xn = W.start_values(nk, seed)
        contrib = nv * xn
        yr = diag * xv + np.add.reduceat(np.concatenate([contrib, [0.0]]), off[:-1]) * (np.diff(off) > 0)
        out[dt] = np.linalg.norm(yg - yr) / np.linalg.norm(yr)
        del y, xd
        torch.cuda.empty_cache()
    return out


def test_hub4x4_sampled_rows(ed, oracle_mod):
    import torch

    err = _sampled_rows(ed, oracle_mod, W.config_hub4x4(), 200, 2000)
    assert err[torch.float64] <= TOL64
    assert err[torch.float32] <= TOL32


def test_j1j2_4x8_sampled_rows(ed, oracle_mod):
    import torch

    err = _sampled_rows(ed, oracle_mod, W.config_j1j2_4x8(), 300, 2000)
    assert err[torch.float64] <= TOL64
    assert err[torch.float32] <= TOL32


def test_j1j2_4x8_nondyadic_sampled_rows(ed, oracle_mod):
    """J2 = 0.3 (J2/2 = 0.15 is not a dyadic rational): the FP64 apply sums the
    fixed-point input exactly per value class and weights each class sum in
    FP64; sampled rows of the full 601,080,390-state vector against the oracle."""
    import torch

    err = _sampled_rows(ed, oracle_mod, W.j1j2_torus(8, 4, 1.0, 0.3, 16, 0xFFFF), 300, 2000)
    assert err[torch.float64] <= TOL64
    assert err[torch.float32] <= TOL32


def _dyadic_spin(m):
    """Every spin matrix element (J_xy/2, J_z/4) is a multiple of 2^-20, so
    the FP64 apply runs in exact fixed point."""
    vals = np.concatenate([np.atleast_1d(np.asarray(m.jxy, float)) / 2, np.atleast_1d(np.asarray(m.jz, float)) / 4])
    return bool(np.all(vals * 2.0 ** 20 == np.round(vals * 2.0 ** 20)))


CROSS_MODELS = ["heis16", "j1j2_4x4", "j1j2_4x4_strip", "xxz_odd_cut", "xxz_n_up_1"]


EXTRA_CROSS = {
    # 52 cross bonds: more than the class-sorted kernels take (general kernel)
    "j1j2_4x6_ragged": lambda: W.j1j2_torus(4, 6, cut_mask=0b101101001011010010110100),
    # 32 cross bonds, five on one B site: the row pass's general cross loop
    "j1j2_4x4_crowded": lambda: W.j1j2_torus(4, 4, cut_mask=25011),
    # 30 cross bonds, six on one B site, 3x6 torus
    "j1j2_3x6_crowded": lambda: W.j1j2_torus(3, 6, cut_mask=125720),
}


MORE_SPIN = {
    # odd side sizes, a one-bit low half, two-bit sides
    "xxz_9_cut5": lambda: W.xxz_chain(9, 1.0, 0.5, n_up=4, cut_mask=0b000011111),
    "heis_6_cut2": lambda: W.heisenberg_chain(6, 1.0, 3, True, 0b000011),
    "heis_5_cut2": lambda: W.heisenberg_chain(5, 1.0, 2, True, 0b00011),
    # four value classes (J1 = 1, J2 = 0.5, jz != jxy): every class slot in use
    "j1j2_xxz_4x4": lambda: W.Model("spin", 16, W.torus_j1j2_bonds(4, 4)[0] + W.torus_j1j2_bonds(4, 4)[1],
                                    jxy=[1.0] * 32 + [0.5] * 32, jz=[0.75] * 32 + [0.25] * 32, n_up=7,
                                    cut_mask=0xFF),
    # non-dyadic couplings: the FP64 policy of the Kronecker pass
    "j1j2_4x4_j2_03": lambda: W.j1j2_torus(4, 4, 1.0, 0.3, cut_mask=0xFF),
    # three value classes on the bonds between the halves (ladder with rungs)
    "ladder_2x6": lambda: W.Model("spin", 12, W.chain_bonds(6, True) + [(i + 6, (i + 1) % 6 + 6) for i in range(6)]
                                  + [(i, i + 6) for i in range(6)],
                                  jxy=[1.0] * 12 + [0.25] * 6, jz=[1.0] * 12 + [0.25] * 6, n_up=6,
                                  cut_mask=0b000111000111),
}


@pytest.mark.parametrize("name", CROSS_MODELS + list(EXTRA_CROSS) + list(MORE_SPIN))
def test_cross_term_models(ed, oracle_mod, name):
    """Spin models with cross-cut bonds (crowded cuts, odd side sizes, four
    value classes, non-dyadic couplings, ladders) against the oracle, FP64
    and FP32, with the row pass each one gets."""
    import torch

    if name in MODELS:
        m = MODELS[name]
    elif name in EXTRA_CROSS:
        m = EXTRA_CROSS[name]()
    else:
        m = MORE_SPIN[name]()
    okeys = oracle_mod.sector_keys(m)
    ctx = ed.build_local_ops(ed.build_sectors(m))
    keys = ctx.state_keys()
    pos = oracle_mod.find_keys(m, okeys, keys)
    y_ref = oracle_mod.apply_H(m, okeys, W.start_values(okeys))[pos]
    x64 = torch.tensor(W.start_values(keys), device="cuda")
    for dt, tol in ((torch.float64, TOL64), (torch.float32, TOL32)):
        x = x64.to(dt)
        y = torch.full_like(x, float("nan"))
        ed.apply_H(ctx, x, y)
        torch.cuda.synchronize()
        yy = y.double().cpu().numpy()
        assert np.linalg.norm(yy - y_ref) <= tol * np.linalg.norm(y_ref), (name, dt)


def test_j1j2_4x7_full_parity(ed, oracle_mod):
    """J1-J2 4x7 torus, Sz=0, cut 14|14 (40,116,600 states, 15 blocks up to
    3432 x 3432): FP64 and FP32, whole vector against the oracle."""
    import torch

    m = W.config_j1j2_4x7()
    okeys = oracle_mod.sector_keys(m)
    xo = W.start_values(okeys)
    y_ref0 = oracle_mod.apply_H(m, okeys, xo)
    del xo
    for flags in (ed.OPS_DEFAULT,):
        ctx = ed.build_local_ops(ed.build_sectors(m), flags)
        keys = ctx.state_keys()
        pos = oracle_mod.find_keys(m, okeys, keys)
        assert (pos >= 0).all()
        y_ref = y_ref0[pos]
        x64 = torch.empty(ctx.dim, dtype=torch.float64, device="cuda")
        ed.random_vector(ctx, x64)
        for dt, tol in ((torch.float64, TOL64), (torch.float32, TOL32)):
            x = x64.to(dt)
            y = torch.empty_like(x)
            ed.apply_H(ctx, x, y)
            torch.cuda.synchronize()
            yy = y.double().cpu().numpy()
            assert np.linalg.norm(yy - y_ref) <= tol * np.linalg.norm(y_ref), (flags, dt)
            del x, y
        del x64, ctx
        torch.cuda.empty_cache()


@pytest.mark.parametrize("name,mode", [("j1j2_4x4", "fixed"), ("j1j2_4x4_j2_03", "wide"),
                                       ("j1j2_4x4_wide_range", "classed"), ("hub_rect_dyadic", "fixed")])
def test_fp64_mode_selection(ed, name, mode):
    """Dyadic couplings take the exact 64-bit path, other couplings the
    128-bit integer weights, a value range beyond 2^55 the FP64 class
    weights; each of these contexts is also in the FP64 parity list."""
    ctx = ed.build_local_ops(ed.build_sectors(MODELS[name]))
    assert ctx.fp64_mode() == mode
