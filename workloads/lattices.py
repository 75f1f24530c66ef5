"""Lattices, couplings and symmetry sectors of the synthetic workloads.

A model is a K-local Hamiltonian on a finite lattice (the paper's Eq. (1))
given as a bond list plus per-bond and per-site couplings; this module only
*describes* such models.  Site i is bit i of a basis bit string.

Conventions (readings of the paper, which names the models but prints no
Hamiltonian normalisation):

* spin-1/2 XXZ:  H = sum_bonds [ jz S^z_i S^z_j + jxy/2 (S^+_i S^-_j + h.c.) ],
  S = sigma/2, bit 1 = spin up.  J1-J2: jxy = jz = J1 on nearest-neighbour
  bonds and J2 on both plaquette diagonals.
* Hubbard:  H = -sum_bonds,sigma t_b (c^dag_i c_j + h.c.) + sum_i U_i n_i,up n_i,dw
  + sum_i eps_i (n_i,up + n_i,dw).  A next-nearest-neighbour bond carries
  t_b = t' (it enters with the same minus sign as t).

Bonds are stored as a de-duplicated set of unordered pairs, so a ring of
length 2 or a torus of width 2 never counts a bond twice.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np


@dataclass
class Model:
    """Description of one lattice model, its target sector and its cut.

    kind      : "spin" (spin-1/2 XXZ) or "hubbard".
    n_sites   : number of lattice sites S.
    bonds     : (n_bonds, 2) int array of site pairs (i, j), i != j.
    jxy, jz   : per-bond spin couplings (spin models).
    t         : per-bond hopping amplitudes (Hubbard).
    U, eps    : per-site interaction and on-site energy (Hubbard).
    n_up      : spin: number of up spins (Sz = n_up - S/2); Hubbard: N_up.
    n_dw      : Hubbard: N_dw (ignored for spin models).
    cut_mask  : spin models: bit mask of the sites on side A of the
                entanglement cut (the rest form side B).
    spin_cut  : Hubbard models: the cut separates the spin-up from the
                spin-down degrees of freedom (A = up, B = down).
    """

    kind: str
    n_sites: int
    bonds: np.ndarray
    jxy: np.ndarray = None
    jz: np.ndarray = None
    t: np.ndarray = None
    U: np.ndarray = None
    eps: np.ndarray = None
    n_up: int = 0
    n_dw: int = 0
    cut_mask: int = 0
    spin_cut: bool = False
    name: str = ""
    meta: dict = field(default_factory=dict)

    def __post_init__(self):
        self.bonds = np.ascontiguousarray(np.asarray(self.bonds, dtype=np.int32).reshape(-1, 2))
        nb = len(self.bonds)
        z = np.zeros(nb)
        zs = np.zeros(self.n_sites)
        self.jxy = z.copy() if self.jxy is None else np.ascontiguousarray(np.broadcast_to(np.asarray(self.jxy, float), (nb,)))
        self.jz = z.copy() if self.jz is None else np.ascontiguousarray(np.broadcast_to(np.asarray(self.jz, float), (nb,)))
        self.t = z.copy() if self.t is None else np.ascontiguousarray(np.broadcast_to(np.asarray(self.t, float), (nb,)))
        self.U = zs.copy() if self.U is None else np.ascontiguousarray(np.broadcast_to(np.asarray(self.U, float), (self.n_sites,)))
        self.eps = zs.copy() if self.eps is None else np.ascontiguousarray(np.broadcast_to(np.asarray(self.eps, float), (self.n_sites,)))
        if self.kind not in ("spin", "hubbard"):
            raise ValueError(f"unknown model kind {self.kind!r}")

    @property
    def n_bonds(self) -> int:
        return len(self.bonds)

    def with_sector(self, n_up: int, n_dw: int | None = None) -> "Model":
        """Copy of this model targeting another symmetry sector."""
        m = Model(kind=self.kind, n_sites=self.n_sites, bonds=self.bonds.copy(), jxy=self.jxy.copy(),
                  jz=self.jz.copy(), t=self.t.copy(), U=self.U.copy(), eps=self.eps.copy(), n_up=n_up,
                  n_dw=self.n_dw if n_dw is None else n_dw, cut_mask=self.cut_mask, spin_cut=self.spin_cut,
                  name=self.name, meta=dict(self.meta))
        return m

    def with_cut(self, cut_mask: int) -> "Model":
        m = self.with_sector(self.n_up, self.n_dw)
        m.cut_mask = int(cut_mask)
        return m


def _dedup(pairs: Sequence[Tuple[int, int]]) -> List[Tuple[int, int]]:
    seen = set()
    out = []
    for i, j in pairs:
        if i == j:
            continue
        key = (min(i, j), max(i, j))
        if key in seen:
            continue
        seen.add(key)
        out.append((int(i), int(j)))
    return out


def chain_bonds(L: int, pbc: bool = True, reach: int = 1) -> List[Tuple[int, int]]:
    """Bonds (i, i+reach) of a chain of L sites, wrapped if pbc."""
    pairs = []
    for i in range(L):
        j = i + reach
        if j < L:
            pairs.append((i, j))
        elif pbc:
            pairs.append((i, j % L))
    return _dedup(pairs)


def square_torus_bonds(Lx: int, Ly: int) -> List[Tuple[int, int]]:
    """Nearest-neighbour bonds of an Lx x Ly torus, site i = x*Ly + y."""
    s = lambda x, y: (x % Lx) * Ly + (y % Ly)
    pairs = []
    for x in range(Lx):
        for y in range(Ly):
            pairs.append((s(x, y), s(x + 1, y)))
            pairs.append((s(x, y), s(x, y + 1)))
    return _dedup(pairs)


def torus_j1j2_bonds(Lx: int, Ly: int):
    """(J1 bonds, J2 bonds) of an Lx x Ly torus, site i = x*Ly + y.

    J1: horizontal and vertical neighbours; J2: both diagonals of every
    plaquette.  Each list is de-duplicated, and a pair that is both a J1 and
    a J2 neighbour (only possible on width-2 tori) is kept as J1 only.
    """
    s = lambda x, y: (x % Lx) * Ly + (y % Ly)
    j1 = []
    j2 = []
    for x in range(Lx):
        for y in range(Ly):
            j1.append((s(x, y), s(x + 1, y)))
            j1.append((s(x, y), s(x, y + 1)))
            j2.append((s(x, y), s(x + 1, y + 1)))
            j2.append((s(x, y), s(x + 1, y - 1)))
    j1 = _dedup(j1)
    seen = {(min(a, b), max(a, b)) for a, b in j1}
    j2 = [p for p in _dedup(j2) if (min(p), max(p)) not in seen]
    return j1, j2


def open_cluster_bonds(Lx: int, Ly: int):
    """(nearest-neighbour, diagonal) bonds of an open Lx x Ly cluster, i = x*Ly + y."""
    s = lambda x, y: x * Ly + y
    nn, nnn = [], []
    for x in range(Lx):
        for y in range(Ly):
            if x + 1 < Lx:
                nn.append((s(x, y), s(x + 1, y)))
            if y + 1 < Ly:
                nn.append((s(x, y), s(x, y + 1)))
            if x + 1 < Lx and y + 1 < Ly:
                nnn.append((s(x, y), s(x + 1, y + 1)))
            if x + 1 < Lx and y - 1 >= 0:
                nnn.append((s(x, y), s(x + 1, y - 1)))
    return _dedup(nn), _dedup(nnn)


# --------------------------------------------------------------------------- spin models

def xxz_chain(L: int, jxy: float = 1.0, jz: float = 1.0, n_up: int | None = None, pbc: bool = True,
              cut_mask: int | None = None, name: str = "") -> Model:
    bonds = chain_bonds(L, pbc)
    if n_up is None:
        n_up = L // 2
    if cut_mask is None:
        cut_mask = (1 << (L // 2)) - 1
    return Model("spin", L, bonds, jxy=jxy, jz=jz, n_up=n_up, n_dw=L - n_up, cut_mask=cut_mask,
                 name=name or f"xxz_chain_L{L}")


def heisenberg_chain(L: int, J: float = 1.0, n_up: int | None = None, pbc: bool = True,
                     cut_mask: int | None = None) -> Model:
    return xxz_chain(L, J, J, n_up, pbc, cut_mask, name=f"heisenberg_chain_L{L}")


def j1j2_torus(Lx: int, Ly: int, J1: float = 1.0, J2: float = 0.5, n_up: int | None = None,
               cut_mask: int | None = None) -> Model:
    """J1-J2 Heisenberg model on an Lx x Ly torus (site i = x*Ly + y).

    The default cut puts the columns x < Lx/2 on side A (sites 0 .. N/2-1),
    i.e. a cut across the long axis when Lx > Ly.
    """
    j1, j2 = torus_j1j2_bonds(Lx, Ly)
    n = Lx * Ly
    bonds = j1 + j2
    J = [J1] * len(j1) + [J2] * len(j2)
    if n_up is None:
        n_up = n // 2
    if cut_mask is None:
        cut_mask = (1 << ((Lx // 2) * Ly)) - 1
    return Model("spin", n, bonds, jxy=J, jz=J, n_up=n_up, n_dw=n - n_up, cut_mask=cut_mask,
                 name=f"j1j2_torus_{Lx}x{Ly}", meta={"Lx": Lx, "Ly": Ly, "J1": J1, "J2": J2,
                                                      "n_j1": len(j1), "n_j2": len(j2)})


# --------------------------------------------------------------------------- Hubbard models

def hubbard_chain(L: int, t: float = 1.0, U: float = 4.0, n_up: int | None = None, n_dw: int | None = None,
                  pbc: bool = True, tp: float = 0.0, eps=None) -> Model:
    nn = chain_bonds(L, pbc, 1)
    bonds = list(nn)
    tb = [t] * len(nn)
    if tp != 0.0:
        seen = {(min(a, b), max(a, b)) for a, b in nn}
        nnn = [p for p in chain_bonds(L, pbc, 2) if (min(p), max(p)) not in seen]
        bonds += nnn
        tb += [tp] * len(nnn)
    if n_up is None:
        n_up = L // 2
    if n_dw is None:
        n_dw = L // 2
    return Model("hubbard", L, bonds, t=tb, U=U, eps=0.0 if eps is None else eps, n_up=n_up, n_dw=n_dw,
                 spin_cut=True, name=f"hubbard_chain_L{L}")


def hubbard_torus(Lx: int, Ly: int, t: float = 1.0, U: float = 8.0, n_up: int | None = None,
                  n_dw: int | None = None) -> Model:
    bonds = square_torus_bonds(Lx, Ly)
    n = Lx * Ly
    return Model("hubbard", n, bonds, t=t, U=U, n_up=n // 2 if n_up is None else n_up,
                 n_dw=n // 2 if n_dw is None else n_dw, spin_cut=True, name=f"hubbard_torus_{Lx}x{Ly}")


def hubbard_open_cluster(Lx: int, Ly: int, t: float = 1.0, U: float = 4.0, tp: float = 0.0, eps=None,
                         n_up: int | None = None, n_dw: int | None = None) -> Model:
    nn, nnn = open_cluster_bonds(Lx, Ly)
    bonds = list(nn)
    tb = [t] * len(nn)
    if tp != 0.0:
        bonds += nnn
        tb += [tp] * len(nnn)
    n = Lx * Ly
    return Model("hubbard", n, bonds, t=tb, U=U, eps=0.0 if eps is None else eps,
                 n_up=n // 2 if n_up is None else n_up, n_dw=n // 2 if n_dw is None else n_dw,
                 spin_cut=True, name=f"hubbard_open_{Lx}x{Ly}")


def hubbard_dimer(t: float = 1.0, U: float = 4.0) -> Model:
    """Two sites, one bond, N_up = N_dw = 1."""
    return Model("hubbard", 2, [(0, 1)], t=t, U=U, n_up=1, n_dw=1, spin_cut=True, name="hubbard_dimer")


def anderson_impurity(n_bath: int, U: float, eps_d: float, V, eps_bath, n_up: int, n_dw: int) -> Model:
    """Single-impurity Anderson model in the star geometry: site 0 is the
    impurity (energy eps_d, interaction U), sites 1..n_bath the bath orbitals
    (energies eps_bath, no interaction), each coupled to the impurity by the
    hybridisation V_k (scalar or one per bath site):
        H = sum_s eps_d n_0s + U n_0u n_0d + sum_{k,s} eps_k n_ks
            + sum_{k,s} V_k (c^dag_0s c_ks + h.c.).
    In this package's Hubbard convention (-t per bond) the bonds carry t = -V_k.
    The cut is the spin cut (A = up electrons, B = down electrons).
    """
    Vk = np.broadcast_to(np.asarray(V, dtype=np.float64), (n_bath,))
    eb = np.asarray(eps_bath, dtype=np.float64)
    if eb.shape != (n_bath,):
        raise ValueError("eps_bath needs one energy per bath site")
    S = n_bath + 1
    bonds = [(0, k) for k in range(1, S)]
    Us = np.zeros(S)
    Us[0] = U
    eps = np.concatenate([[eps_d], eb])
    return Model("hubbard", S, bonds, t=[-float(v) for v in Vk], U=Us, eps=eps, n_up=n_up, n_dw=n_dw,
                 spin_cut=True, name=f"anderson_impurity_{n_bath}")


def impurity_bath(n_bath: int, half_width: float = 2.0, seed: int = 20260507) -> np.ndarray:
    """Particle-hole symmetric bath energies: n_bath // 2 seeded values
    U[0.05, half_width] and their negatives (a zero level when n_bath is odd),
    in ascending order."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(0.05, half_width, size=n_bath // 2)
    out = np.concatenate([-e, e, [0.0] * (n_bath % 2)])
    return np.sort(out)


def batched_hubbard_instances(n: int = 512, seed: int = 20260507) -> List[Model]:
    """The batched workload: independent Hubbard instances with a spin cut.

    Geometries: periodic rings L = 8..12 and open clusters 2x4, 2x5, 2x6,
    3x3, 3x4.  N_up and N_dw are uniform in [1, S-1], U ~ U[0, 8],
    t' ~ U[-0.3, 0.3] on next-nearest-neighbour bonds (ring: (i, i+2);
    cluster: plaquette diagonals), eps_i ~ U[-1, 1).  t = 1.
    """
    rng = np.random.default_rng(seed)
    geoms = [("ring", L, 0) for L in range(8, 13)] + [("open", 2, 4), ("open", 2, 5), ("open", 2, 6),
                                                      ("open", 3, 3), ("open", 3, 4)]
    out = []
    for k in range(n):
        g = geoms[int(rng.integers(len(geoms)))]
        if g[0] == "ring":
            S = g[1]
        else:
            S = g[1] * g[2]
        n_up = int(rng.integers(1, S))
        n_dw = int(rng.integers(1, S))
        U = float(rng.uniform(0.0, 8.0))
        tp = float(rng.uniform(-0.3, 0.3))
        eps = rng.uniform(-1.0, 1.0, size=S)
        if g[0] == "ring":
            m = hubbard_chain(S, 1.0, U, n_up, n_dw, pbc=True, tp=tp, eps=eps)
        else:
            m = hubbard_open_cluster(g[1], g[2], 1.0, U, tp=tp, eps=eps, n_up=n_up, n_dw=n_dw)
        m.name = f"batch{k}_{m.name}"
        m.meta.update({"U": U, "tp": tp, "geom": g})
        out.append(m)
    return out


# --------------------------------------------------------------------------- the named workloads

def config_heis16() -> Model:
    """Heisenberg S=1/2 ring L=16, J=1, Sz=0 (12,870 states), cut 8|8 (A = sites 0..7)."""
    m = heisenberg_chain(16, 1.0, 8, True, 0xFF)
    m.name = "heis16"
    return m


def config_hub12() -> Model:
    """Hubbard ring L=12, t=1, U=4, N_up = N_dw = 6 (924 x 924 states), spin cut."""
    m = hubbard_chain(12, 1.0, 4.0, 6, 6, True)
    m.name = "hub12"
    return m


def config_j1j2_4x8() -> Model:
    """J1-J2 Heisenberg on the 4x8 torus (Lx=8, Ly=4), J1=1, J2=0.5, Sz=0
    (601,080,390 states); cut 16|16 across the long axis, A = columns x=0..3."""
    m = j1j2_torus(8, 4, 1.0, 0.5, 16, 0xFFFF)
    m.name = "j1j2_4x8"
    return m


def config_hub4x4() -> Model:
    """Hubbard 4x4 torus, t=1, U=8, N_up = N_dw = 8 (12,870 x 12,870 states), spin cut."""
    m = hubbard_torus(4, 4, 1.0, 8.0, 8, 8)
    m.name = "hub4x4"
    return m


def config_j1j2_4x7() -> Model:
    """Smaller J1-J2 torus (Lx=7, Ly=4, 40,116,600 states, cut 14|14) used
    for detailed kernel profiles: same kernels, vectors still larger than L2."""
    m = j1j2_torus(7, 4, 1.0, 0.5, 14, (1 << 14) - 1)
    m.name = "j1j2_4x7"
    return m


def config_qim15() -> Model:
    """Anderson impurity with 14 bath orbitals (S = 15 sites), U = 4 at the
    impurity, eps_d = -U/2, V = 0.5 to every bath orbital, particle-hole
    symmetric seeded bath on [-2, 2]; N_up = 8, N_dw = 7 (6435 x 6435 =
    41,409,225 states), spin cut."""
    m = anderson_impurity(14, 4.0, -2.0, 0.5, impurity_bath(14), 8, 7)
    m.name = "qim15"
    return m


CONFIG_NAMES = ("heis16", "hub12", "j1j2_4x8", "hub4x4", "j1j2_4x7", "qim15")


def config_by_name(name: str) -> Model:
    return {"heis16": config_heis16, "hub12": config_hub12, "j1j2_4x8": config_j1j2_4x8,
            "hub4x4": config_hub4x4, "j1j2_4x7": config_j1j2_4x7, "qim15": config_qim15}[name]()
