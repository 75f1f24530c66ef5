"""Pins of the oracle's Lanczos and Green's-function code against brute force and closed forms."""
import numpy as np
import pytest
import scipy.linalg

import workloads as W


def test_lanczos_diagonal_closed_form(oracle_mod):
    d = np.linspace(-3.0, 5.0, 200)
    v0 = np.ones(200)
    a, b, _ = oracle_mod.lanczos(lambda x: d * x, v0, 120, reorth=True)
    e, _ = oracle_mod.tridiag_lowest(a, b[: len(a) - 1])
    assert abs(e - (-3.0)) < 1e-12


def test_tridiag_lowest_matches_dense(oracle_mod):
    rng = np.random.default_rng(5)
    a = rng.standard_normal(40)
    b = rng.uniform(0.1, 1.0, 39)
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    e, s = oracle_mod.tridiag_lowest(a, b)
    w = np.linalg.eigvalsh(T)
    assert abs(e - w[0]) < 1e-13
    assert np.linalg.norm(T @ s - e * s) < 1e-12


@pytest.mark.parametrize("name", ["heis12", "j1j2_4x3", "hub8", "hub_disorder"])
def test_lanczos_e0_vs_dense(oracle_mod, name):
    o = oracle_mod
    if name == "heis12":
        m = W.heisenberg_chain(12)
    elif name == "j1j2_4x3":
        m = W.j1j2_torus(4, 3, 1.0, 0.5)
    elif name == "hub8":
        m = W.hubbard_chain(8, 1.0, 4.0, 4, 4)
    else:
        m = W.hubbard_open_cluster(2, 4, 1.0, 3.0, tp=0.2, eps=np.linspace(-1, 1, 8), n_up=3, n_dw=4)
    keys = o.sector_keys(m)
    e_dense = np.linalg.eigvalsh(o.dense_H(m, keys))[0]
    e0, psi, _ = o.ground_state(m, keys, n_iter=200)
    assert abs(e0 - e_dense) < 1e-12 * max(1.0, abs(e_dense))
    r = o.apply_H(m, keys, psi) - e0 * psi
    assert np.linalg.norm(r) < 1e-8


def test_continued_fraction_two_level():
    """w0/(z - a0 - b1^2/(z - a1)) equals the 2x2 resolvent element."""
    import oracle

    a0, a1, b1 = 0.3, -1.1, 0.7
    T = np.array([[a0, b1], [b1, a1]])
    z = np.array([0.1 + 0.05j, -2.0 + 0.05j, 3.0 + 0.5j])
    ref = np.array([np.linalg.inv(zz * np.eye(2) - T)[0, 0] for zz in z])
    got = oracle.continued_fraction(z, 1.0, [a0, a1], [b1])
    assert np.abs(got - ref).max() < 1e-14


def test_gf_free_fermion_closed_form(oracle_mod):
    """U = 0 closed shell: G_00(z) = sum_k |u_k(0)|^2 / (z - eps_k) over all orbitals."""
    o = oracle_mod
    m = W.hubbard_chain(6, 1.0, 0.0, 3, 3, pbc=True)
    h = np.zeros((6, 6))
    for (i, j), t in zip(m.bonds, m.t):
        h[i, j] -= t
        h[j, i] -= t
    eps, u = np.linalg.eigh(h)
    omega = np.linspace(-4, 4, 101)
    eta = 0.1
    z = omega + 1j * eta
    ref = np.sum(np.abs(u[0, :]) ** 2 / (z[:, None] - eps[None, :]), axis=1)
    keys = o.sector_keys(m)
    e0, psi, _ = o.ground_state(m, keys, n_iter=200)
    assert abs(e0 - 2 * eps[:3].sum()) < 1e-12
    G = o.green_function(m, psi, e0, omega, eta, site=0, spin=0, n_iter=200, keys=keys)
    assert np.abs(G - ref).max() < 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("spin,site", [(0, 0), (1, 2)])
def test_gf_lehmann(oracle_mod, spin, site):
    o = oracle_mod
    m = W.hubbard_chain(6, 1.0, 4.0, 3, 3, pbc=True, tp=0.1)
    omega = np.linspace(-8, 8, 161)
    eta = 0.05
    G_ref, e_dense = o.lehmann_green_function(m, omega, eta, site=site, spin=spin)
    keys = o.sector_keys(m)
    e0, psi, _ = o.ground_state(m, keys, n_iter=300)
    assert abs(e0 - e_dense) < 1e-12 * abs(e_dense)
    G, co = o.green_function(m, psi, e0, omega, eta, site=site, spin=spin, n_iter=300, keys=keys,
                             return_coeffs=True)
    assert np.abs(G - G_ref).max() < 1e-10 * np.abs(G_ref).max()
    # sum rule: <c c^dag> + <c^dag c> = 1
    w = sum(v[0] for v in co.values())
    assert abs(w - 1.0) < 1e-12
    # spectral weight: -1/pi Im G integrates to ~1 on a wide grid (Lorentzian tails cut)
    wide = np.linspace(-400, 400, 400001)
    Gw = o.green_function(m, psi, e0, wide, eta, site=site, spin=spin, n_iter=300, keys=keys)
    A = -Gw.imag / np.pi
    assert abs(np.trapezoid(A, wide) - 1.0) < 2e-4
