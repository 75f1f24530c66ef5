"""Write the stored expected values under tests/golden/ from the oracle only.

    python tests/golden/make_golden.py                        # heis16, hub12, small models
    python tests/golden/make_golden.py j1j2_4x6 hub12_gf_start  # only the named entries

Every number written here comes from ``oracle/`` (full-sector exact
diagonalisation, FP64 Lanczos with full reorthogonalisation, continued
fractions) on the seeded workloads of ``workloads/``.  Nothing is taken from
the CUDA path.
"""
from __future__ import annotations

import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402

OUT = os.path.dirname(os.path.abspath(__file__))


def _oracle_rev():
    try:
        return subprocess.run(["git", "-C", ROOT, "log", "-1", "--format=%H", "--", "oracle"], capture_output=True,
                              text=True).stdout.strip()
    except Exception:
        return ""


def heis16():
    m = W.config_heis16()
    keys = oracle.sector_keys(m)
    e0, psi, _ = oracle.ground_state(m, keys, n_iter=300)
    v0 = W.start_values(keys, W.DEFAULT_SEED)
    mv = lambda x: oracle.apply_H(m, keys, x)
    a, b, _ = oracle.lanczos(mv, v0, 150, reorth=False)
    e150, _ = oracle.tridiag_lowest(a, b[: len(a) - 1])
    return {"config": "heis16", "e0": e0, "e0_150_noreorth": e150, "alpha_0_19": a[:20].tolist(),
            "beta_1_20": b[:20].tolist(), "seed": W.DEFAULT_SEED}


def hub12():
    """Hub12 ground state and the Lanczos coefficients of c^dag_{0 up} psi0 and
    c_{0 up} psi0 (500 steps each, full reorthogonalisation).  G(omega) at any
    eta and any truncation length follows from them."""
    m = W.config_hub12()
    keys = oracle.sector_keys(m)
    t = time.time()
    e0, psi, _ = oracle.ground_state(m, keys, n_iter=300, tol=1e-14)
    G, co = oracle.green_function(m, psi, e0, [0.0], 0.05, site=0, spin=0, n_iter=500, keys=keys, reorth=True,
                                  return_coeffs=True)
    return {"config": "hub12", "e0": e0, "site": 0, "spin": 0, "n_iter": 500,
            "w_particle": co["particle"][0], "a_particle": co["particle"][1].tolist(),
            "b_particle": co["particle"][2].tolist(),
            "w_hole": co["hole"][0], "a_hole": co["hole"][1].tolist(), "b_hole": co["hole"][2].tolist(),
            "seconds": time.time() - t}


def small_models():
    """E0 of small models used by the GPU driver tests (dense brute force)."""
    rng = np.random.default_rng(11)
    ms = {
        "j1j2_4x4": W.j1j2_torus(4, 4, cut_mask=0xFF),
        "hub_open_3x4": W.hubbard_open_cluster(3, 4, 1.0, 6.0, tp=-0.2, eps=rng.uniform(-1, 1, 12), n_up=5, n_dw=7),
    }
    out = {}
    for k, m in ms.items():
        keys = oracle.sector_keys(m)
        e0, _, _ = oracle.ground_state(m, keys, n_iter=400, tol=1e-14)
        out[k] = e0
    return out


def j1j2_4x6():
    """E0 of the J1-J2 Heisenberg model on the 4x6 torus (Lx=6, Ly=4, J2/J1 = 0.5,
    Sz=0: 2,704,156 states).  Plain Lanczos recurrence (no basis kept) from
    the seeded key-indexed start vector; the lowest Ritz value of every
    prefix is recorded so the stored E0 comes with its convergence history."""
    m = W.j1j2_torus(6, 4)
    keys = oracle.sector_keys(m)
    v0 = W.start_values(keys, W.DEFAULT_SEED)
    t = time.time()
    a, b, _ = oracle.lanczos(lambda x: oracle.apply_H(m, keys, x), v0, 260, reorth=False)
    ritz = [oracle.tridiag_lowest(a[:k], b[: k - 1])[0] for k in range(20, len(a) + 1, 20)]
    e0 = ritz[-1]
    return {"config": "j1j2_torus_6x4", "states": int(len(keys)), "e0": e0, "steps": int(len(a)),
            "ritz_every_20": ritz, "last_change": abs(ritz[-1] - ritz[-2]) / abs(e0), "seconds": time.time() - t,
            "seed": W.DEFAULT_SEED}


def hub12_gf_start():
    """Lanczos coefficients of c^dag_{0 up} v and c_{0 up} v for the Hub12 model
    with v = the normalised seeded key-indexed start vector (bit-for-bit the
    same input on any machine), 300 steps, full re-orthogonalisation; E0 is
    the stored Hub12 ground-state energy (any fixed shift serves)."""
    m = W.config_hub12()
    keys = oracle.sector_keys(m)
    with open(os.path.join(OUT, "hub12.json")) as f:
        e0 = json.load(f)["e0"]
    psi = W.start_values(keys, W.DEFAULT_SEED)
    psi = psi / np.linalg.norm(psi)
    t = time.time()
    _, co = oracle.green_function(m, psi, e0, [0.0], 0.05, site=0, spin=0, n_iter=300, keys=keys, reorth=True,
                                  return_coeffs=True)
    return {"config": "hub12", "e0_shift": e0, "site": 0, "spin": 0, "n_iter": 300, "start": "start_values/norm",
            "w_particle": co["particle"][0], "a_particle": co["particle"][1].tolist(),
            "b_particle": co["particle"][2].tolist(),
            "w_hole": co["hole"][0], "a_hole": co["hole"][1].tolist(), "b_hole": co["hole"][2].tolist(),
            "seconds": time.time() - t}


EXTRA = {"j1j2_4x6": j1j2_4x6, "hub12_gf_start": hub12_gf_start}


def main():
    rev = _oracle_rev()
    if len(sys.argv) > 1:
        # only the named extra entries, each to <name>.json
        for name in sys.argv[1:]:
            d = EXTRA[name]()
            d["oracle_rev"] = rev
            with open(os.path.join(OUT, f"{name}.json"), "w") as f:
                json.dump(d, f, indent=1)
            print(name, {k: v for k, v in d.items() if not isinstance(v, list)})
        return
    for name, fn in (("heis16", heis16), ("hub12", hub12)):
        d = fn()
        d["oracle_rev"] = rev
        with open(os.path.join(OUT, f"{name}.json"), "w") as f:
            json.dump(d, f, indent=1)
        print(name, d["e0"])
    d = {"e0": small_models(), "oracle_rev": rev}
    with open(os.path.join(OUT, "small_e0.json"), "w") as f:
        json.dump(d, f, indent=1)
    print(d)


if __name__ == "__main__":
    main()
