"""Synthetic hydrogen-like molecules with s-only even-tempered basis sets.

Workload recipe (the paper's density-fitting section uses real molecules and basis
data that are not available here, so these stand in for them):

* centres have nuclear charge 1 and are drawn uniformly in a cube of side ``box`` by
  rejection sampling with a minimum separation of 1.4 bohr (numpy PCG64 stream);
* each centre carries 5 orbital s primitives with even-tempered exponents spanning
  [0.1, 10] and 15 auxiliary s primitives spanning [0.05, 50];
* basis functions are ordered centre-major, exponent ascending;
* an odd number of centres gets molecular charge +1 so that the restricted
  Hartree-Fock determinant has nocc = floor(n/2) doubly occupied orbitals.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def even_tempered(lo: float, hi: float, k: int) -> np.ndarray:
    """k exponents lo * (hi/lo)**(j/(k-1)), j = 0..k-1 (a geometric ladder)."""
    if k == 1:
        return np.array([lo], dtype=np.float64)
    j = np.arange(k, dtype=np.float64)
    return lo * (hi / lo) ** (j / (k - 1))


ORB_EXPONENTS = even_tempered(0.1, 10.0, 5)
AUX_EXPONENTS = even_tempered(0.05, 50.0, 15)


@dataclass
class Molecule:
    """Arrays describing one molecule and its two basis sets (all float64, C order)."""

    xyz: np.ndarray        # [natm, 3] nuclear positions (bohr)
    charges: np.ndarray    # [natm] nuclear charges
    ao_xyz: np.ndarray     # [nao, 3] centre of every orbital primitive
    ao_exp: np.ndarray     # [nao] orbital exponents
    aux_xyz: np.ndarray    # [naux, 3] centre of every auxiliary primitive
    aux_exp: np.ndarray    # [naux] auxiliary exponents
    nelec: int             # electron count (even)

    @property
    def natm(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def nao(self) -> int:
        return int(self.ao_exp.shape[0])

    @property
    def naux(self) -> int:
        return int(self.aux_exp.shape[0])

    @property
    def nocc(self) -> int:
        return self.nelec // 2


def make_geometry(n: int, box: float, seed, min_sep: float = 1.4, max_tries: int = 10_000_000) -> np.ndarray:
    """Rejection-sample n points uniformly in [0, box)^3 with pairwise distance >= min_sep."""
    rng = np.random.default_rng(seed)
    pts = np.empty((n, 3), dtype=np.float64)
    k = 0
    tries = 0
    while k < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError(f"could not place {n} centres in a {box} bohr cube")
        p = rng.uniform(0.0, box, size=3)
        if k == 0 or np.min(np.sum((pts[:k] - p) ** 2, axis=1)) >= min_sep * min_sep:
            pts[k] = p
            k += 1
    return pts


def molecule_from_geometry(xyz: np.ndarray, orb_exp=ORB_EXPONENTS, aux_exp=AUX_EXPONENTS,
                           charges=None, nelec=None) -> Molecule:
    """Attach the even-tempered basis sets to a geometry (centre-major ordering)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    n = xyz.shape[0]
    orb_exp = np.asarray(orb_exp, dtype=np.float64)
    aux_exp = np.asarray(aux_exp, dtype=np.float64)
    if charges is None:
        charges = np.ones(n, dtype=np.float64)
    charges = np.ascontiguousarray(charges, dtype=np.float64)
    if nelec is None:
        ztot = int(round(charges.sum()))
        nelec = ztot - (ztot % 2)
    return Molecule(
        xyz=xyz,
        charges=charges,
        ao_xyz=np.ascontiguousarray(np.repeat(xyz, len(orb_exp), axis=0)),
        ao_exp=np.ascontiguousarray(np.tile(orb_exp, n)),
        aux_xyz=np.ascontiguousarray(np.repeat(xyz, len(aux_exp), axis=0)),
        aux_exp=np.ascontiguousarray(np.tile(aux_exp, n)),
        nelec=int(nelec),
    )


def box_for(n: int) -> float:
    """Cube side at a density of one centre per 10 bohr^3."""
    return float((10.0 * n) ** (1.0 / 3.0))


def make_molecule(n: int, box: float | None = None, seed=0) -> Molecule:
    return molecule_from_geometry(make_geometry(n, box_for(n) if box is None else box, seed))


def config_c0() -> Molecule:
    """20 centres in a 6 bohr cube, seed 0: nao 100, naux 300, nocc 10."""
    return make_molecule(20, 6.0, 0)


def config_c1() -> Molecule:
    """300 centres at 1 per 10 bohr^3 (box 14.42 bohr), seed 0: nao 1500, naux 4500, nocc 150."""
    return make_molecule(300, box_for(300), 0)


def batch_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Centre counts drawn uniformly from {lo..hi} with default_rng(seed)."""
    return np.random.default_rng(seed).integers(lo, hi + 1, size=count)


def batch_molecules(count: int, lo: int, hi: int, seed: int) -> list[Molecule]:
    """count molecules; molecule i uses geometry seed (seed, i) and density 1 per 10 bohr^3."""
    sizes = batch_sizes(count, lo, hi, seed)
    return [make_molecule(int(n), box_for(int(n)), (seed, i)) for i, n in enumerate(sizes)]
