"""GPU Lanczos ground state, mixed-precision refinement and Green's function
(through the C ABI) against the oracle (stored values in tests/golden/ were
written by tests/golden/make_golden.py from the oracle only)."""
import json
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def ed():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_07621_gb300 as ed

    return ed


def _ctx(ed, m):
    return ed.build_local_ops(ed.build_sectors(m))


def test_heis16_150_steps_alpha_prefix(ed):
    """Heisenberg ring L=16: exactly 150 steps without reorthogonalisation
    from the key-indexed start vector; E0 and alpha_0..19 as the oracle."""
    g = _gold("heis16.json")
    ctx = _ctx(ed, W.config_heis16())
    r = ed.lanczos_ground(ctx, mode="f64", max_iter=150, fixed_iter=True)
    assert r.iterations == 150
    assert abs(r.e0 - g["e0"]) <= 1e-10 * abs(g["e0"])
    assert abs(r.e0 - g["e0_150_noreorth"]) <= 1e-10 * abs(g["e0"])
    assert np.abs(r.alpha[:20] - np.array(g["alpha_0_19"])).max() < 1e-11
    assert np.abs(r.beta[:20] - np.array(g["beta_1_20"])).max() < 1e-11


@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_hub12_ground_state(ed, mode):
    g = _gold("hub12.json")
    ctx = _ctx(ed, W.config_hub12())
    r = ed.lanczos_ground(ctx, mode=mode)
    assert r.converged
    assert abs(r.e0 - g["e0"]) <= 1e-10 * abs(g["e0"]), (r.e0, g["e0"])


def test_f32_mode_accuracy(ed):
    g = _gold("hub12.json")
    ctx = _ctx(ed, W.config_hub12())
    r = ed.lanczos_ground(ctx, mode="f32", tol=1e-7)
    assert abs(r.e0 - g["e0"]) <= 1e-6 * abs(g["e0"])


@pytest.mark.parametrize("name", ["j1j2_4x4", "hub_open_3x4"])
@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_small_models_e0(ed, name, mode):
    rng = np.random.default_rng(11)
    ms = {
        "j1j2_4x4": W.j1j2_torus(4, 4, cut_mask=0xFF),
        "hub_open_3x4": W.hubbard_open_cluster(3, 4, 1.0, 6.0, tp=-0.2, eps=rng.uniform(-1, 1, 12), n_up=5, n_dw=7),
    }
    e_ref = _gold("small_e0.json")["e0"][name]
    r = ed.lanczos_ground(_ctx(ed, ms[name]), mode=mode)
    assert abs(r.e0 - e_ref) <= 1e-10 * abs(e_ref)


def test_ground_vector(ed, oracle_mod):
    import torch

    m = W.config_hub12()
    ctx = _ctx(ed, m)
    psi = torch.empty(ctx.dim, dtype=torch.float64, device="cuda")
    r = ed.lanczos_ground(ctx, mode="mixed", psi0=psi)
    assert r.residual < 1e-6
    p = psi.cpu().numpy()
    assert abs(np.linalg.norm(p) - 1) < 1e-12
    # Rayleigh quotient with the oracle's H, matched by key
    keys = ctx.state_keys()
    okeys = oracle_mod.sector_keys(m)
    pos = oracle_mod.find_keys(m, okeys, keys)
    po = np.zeros(len(okeys))
    po[pos] = p
    rq = po @ oracle_mod.apply_H(m, okeys, po)
    assert abs(rq - r.e0) <= 1e-10 * abs(r.e0)


def test_lanczos_dimension_one(ed):
    m = W.xxz_chain(6, 1.0, 0.7, n_up=0)
    r = ed.lanczos_ground(_ctx(ed, m), mode="f64")
    assert r.converged and abs(r.e0 - 6 * 0.7 / 4) < 1e-14


def test_cut_independence_j1j2_4x4(ed):
    """The same lattice with three different entanglement cuts has the same spectrum."""
    es = []
    for mask in (0xFF, 0x0F0F, 0b0101101001011010):
        r = ed.lanczos_ground(_ctx(ed, W.j1j2_torus(4, 4, cut_mask=mask)), mode="f64")
        es.append(r.e0)
    assert max(es) - min(es) < 1e-10 * abs(es[0])


def _cf_green(g, omega, eta, m):
    """G(omega + i eta) from the first m oracle coefficients of both runs."""
    import oracle

    z = np.asarray(omega) + 1j * eta
    ap, bp = np.array(g["a_particle"][:m]), np.array(g["b_particle"][: m - 1])
    ah, bh = np.array(g["a_hole"][:m]), np.array(g["b_hole"][: m - 1])
    return (oracle.continued_fraction(z + g["e0"], g["w_particle"], ap, bp)
            - oracle.continued_fraction(g["e0"] - z, g["w_hole"], ah, bh))


@pytest.mark.parametrize("reorth", ["auto", "partial"])
def test_hub12_green_function(ed, reorth):
    """Hub12 G_00(omega) with full re-orthogonalisation (auto at this size) or
    the partial one; the checks are those of _hub12_gf_check."""
    _hub12_gf_check(ed, reorth)


def _hub12_gf_check(ed, reorth):
    """Hub12 G_00(omega), 2048 frequencies on [-15, 15], 300 Lanczos steps.

    The oracle's coefficients (500 steps, full reorthogonalisation) are
    stored; G follows from any prefix.  At eta = 0.5 a 300-step continued
    fraction is converged and the GPU must agree to 1e-9.  At eta = 0.05 the
    300-step fraction is itself only accurate to its truncation error (the
    oracle's 300- and 500-step values differ by ~1e-3) and later Lanczos
    coefficients are ill-conditioned, so the check there is agreement within
    twice that truncation spread.  The first coefficients and the weights are
    well conditioned and are compared tightly; coefficient k differs between
    two correct runs by roughly 1e-12 * 40^k (start vectors agreeing to
    rounding), so only k < 5 are compared one by one."""
    import torch

    g = _gold("hub12.json")
    ctx = _ctx(ed, W.config_hub12())
    psi = torch.empty(ctx.dim, dtype=torch.float64, device="cuda")
    r = ed.lanczos_ground(ctx, mode="f64", psi0=psi, tol=1e-14)
    assert abs(r.e0 - g["e0"]) <= 1e-10 * abs(g["e0"])
    omega = np.linspace(-15.0, 15.0, 2048)
    G5, co = ed.lanczos_gf(ctx, psi, r.e0, omega, 0.5, site=0, spin=0, n_iter=300, reorth=reorth)
    assert abs(co["particle"][0] - g["w_particle"]) < 1e-9
    assert abs(co["hole"][0] - g["w_hole"]) < 1e-9
    assert abs(co["particle"][0] + co["hole"][0] - 1.0) < 1e-9
    # later coefficients amplify the start vector's rounding-level differences
    # (about 40x per step here), so only the first five are compared one by one
    for side in ("particle", "hole"):
        assert np.abs(co[side][1][:5] - np.array(g["a_" + side][:5])).max() < 1e-9
        assert np.abs(co[side][2][:5] - np.array(g["b_" + side][:5])).max() < 1e-9
    ref5 = _cf_green(g, omega, 0.5, 300)
    assert np.abs(G5 - ref5).max() <= 1e-9 * np.abs(ref5).max()
    G05, _ = ed.lanczos_gf(ctx, psi, r.e0, omega, 0.05, site=0, spin=0, n_iter=300, reorth=reorth)
    ref300 = _cf_green(g, omega, 0.05, 300)
    spread = np.abs(ref300 - _cf_green(g, omega, 0.05, 500)).max()
    assert np.abs(G05 - ref300).max() <= 2.0 * spread
    assert G05.imag.max() <= 0.0  # retarded: -Im G / pi is a spectral density


@pytest.mark.parametrize("spin,site", [(0, 0), (1, 3)])
def test_green_function_lehmann(ed, oracle_mod, spin, site):
    import torch

    m = W.hubbard_chain(6, 1.0, 4.0, 3, 2, pbc=True, tp=0.1, eps=np.linspace(-0.5, 0.5, 6))
    omega = np.linspace(-8, 8, 321)
    Gref, e_dense = oracle_mod.lehmann_green_function(m, omega, 0.05, site=site, spin=spin)
    ctx = _ctx(ed, m)
    psi = torch.empty(ctx.dim, dtype=torch.float64, device="cuda")
    r = ed.lanczos_ground(ctx, mode="f64", psi0=psi, tol=1e-14, reorth=True)
    assert abs(r.e0 - e_dense) < 1e-11 * abs(e_dense)
    # n_iter above every shifted-sector dimension: the Krylov space is exhausted
    # and the continued fraction is exact (the driver reorthogonalises here)
    G, co = ed.lanczos_gf(ctx, psi, r.e0, omega, 0.05, site=site, spin=spin, n_iter=500)
    assert np.abs(G - Gref).max() < 1e-9 * np.abs(Gref).max()
    assert abs(co["particle"][0] + co["hole"][0] - 1.0) < 1e-12


@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_impurity_ground_state(ed, oracle_mod, mode):
    """Anderson impurity, 9 sites (15,876 states): E0 against the oracle's Lanczos."""
    m = W.anderson_impurity(8, 4.0, -2.0, 0.5, W.impurity_bath(8, seed=21), 4, 5)
    e_ref, _, _ = oracle_mod.ground_state(m, tol=1e-14)
    r = ed.lanczos_ground(_ctx(ed, m), mode=mode, tol=1e-13)
    assert r.converged and abs(r.e0 - e_ref) < 1e-10 * abs(e_ref)


def test_impurity_green_function_lehmann(ed, oracle_mod):
    """Impurity Green's function G_dd of a 6-site Anderson model against the
    Lehmann sum over dense eigenpairs (Krylov space exhausted: exact)."""
    import torch

    m = W.anderson_impurity(5, 3.0, -1.0, [0.3, 0.5, 0.4, 0.6, 0.35], W.impurity_bath(5, seed=8), 3, 3)
    omega = np.linspace(-6, 6, 241)
    Gref, e_dense = oracle_mod.lehmann_green_function(m, omega, 0.05, site=0, spin=0)
    ctx = _ctx(ed, m)
    psi = torch.empty(ctx.dim, dtype=torch.float64, device="cuda")
    r = ed.lanczos_ground(ctx, mode="f64", psi0=psi, tol=1e-14, reorth=True)
    assert abs(r.e0 - e_dense) < 1e-11 * abs(e_dense)
    G, co = ed.lanczos_gf(ctx, psi, r.e0, omega, 0.05, site=0, spin=0, n_iter=500)
    assert np.abs(G - Gref).max() < 1e-9 * np.abs(Gref).max()
    assert abs(co["particle"][0] + co["hole"][0] - 1.0) < 1e-12


def test_green_function_plain_recurrence_and_modes(ed):
    """Without re-orthogonalisation the well-conditioned quantities stay exact
    (weights, sum rule, first coefficients) and G stays causal; an unknown
    mode is rejected."""
    import ctypes

    import torch

    from paper_2605_07621_gb300 import _lib as L

    g = _gold("hub12.json")
    ctx = _ctx(ed, W.config_hub12())
    psi = torch.empty(ctx.dim, dtype=torch.float64, device="cuda")
    r = ed.lanczos_ground(ctx, mode="f64", psi0=psi, tol=1e-14)
    omega = np.linspace(-15.0, 15.0, 512)
    G, co = ed.lanczos_gf(ctx, psi, r.e0, omega, 0.05, site=0, spin=0, n_iter=300, reorth="none")
    assert abs(co["particle"][0] + co["hole"][0] - 1.0) < 1e-9
    for side in ("particle", "hole"):
        assert np.abs(co[side][1][:5] - np.array(g["a_" + side][:5])).max() < 1e-9
    assert G.imag.max() <= 0.0
    Gr = np.zeros(2 * len(omega))
    st = L.load().ed_lanczos_gf(ctx.handle, ctypes.c_void_p(psi.data_ptr()), r.e0, 0, 0, 10, omega.ctypes.data,
                                len(omega), 0.05, Gr.ctypes.data, None, None, None, None, None, None, 7, None)
    assert st == L.ED_EINVAL


@pytest.mark.parametrize("name,mode", [("heis16", "f64"), ("hub12", "f64"), ("hub12", "f32"),
                                       ("qim_small", "f64")])
def test_captured_steps_match_step_by_step(ed, name, mode):
    """Small sectors replay pairs of Lanczos steps from a captured CUDA graph;
    with profiling on the same run goes step by step.  Both must produce the
    same coefficients bit for bit (same kernels, same order)."""
    m = {"heis16": W.config_heis16(), "hub12": W.config_hub12(),
         "qim_small": W.anderson_impurity(8, 4.0, -2.0, 0.5, W.impurity_bath(8, seed=21), 4, 5)}[name]
    ctx = _ctx(ed, m)
    runs = []
    for prof in (False, True):
        ctx.profile(prof)
        r = ed.lanczos_ground(ctx, mode=mode, max_iter=61, fixed_iter=True)
        runs.append(r)
    ctx.profile(False)
    assert runs[0].iterations == runs[1].iterations == 61
    assert np.array_equal(runs[0].alpha, runs[1].alpha) and np.array_equal(runs[0].beta, runs[1].beta)
    assert runs[0].e0 == runs[1].e0


def test_captured_steps_on_a_user_stream(ed):
    """The captured steps run on the context's private stream, fenced against
    the caller's stream: on a user stream (and with work queued on it before
    the call) the coefficients equal those of the default-stream run."""
    import torch

    ctx = _ctx(ed, W.config_hub12())
    r0 = ed.lanczos_ground(ctx, mode="f64", max_iter=61, fixed_iter=True)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        junk = torch.randn(1 << 22, device="cuda")
        junk.mul_(2.0)  # queued ahead of the Lanczos run on the same stream
        r1 = ed.lanczos_ground(ctx, mode="f64", max_iter=61, fixed_iter=True, stream=s)
    s.synchronize()
    assert np.array_equal(r0.alpha, r1.alpha) and np.array_equal(r0.beta, r1.beta)
