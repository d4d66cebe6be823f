"""Restricted Hartree-Fock with density-fitted J/K and Pulay DIIS (oracle, FP64, numpy).

TEST INFRASTRUCTURE ONLY.  The paper (arXiv 2506.06661) uses DF mean-field methods
(Section "Density fitting", the ``.density_fit()`` discussion) and names DIIS as the
default SCF accelerator (Section "Second-Order Self-Consistent Field") without printing
formulas, so this module follows the textbook definitions:

* Fock matrix F = h + J[D] - 1/2 K[D]; with D = 2 C_occ C_occ^T this is h + J - K[C_occ]
  where K[C] = sum_P (B_P C)(B_P C)^T;
* energy E = 1/2 tr(D (h + F)) + E_nuc;
* canonical orthogonalisation X = U s^-1/2 over eigenvalues s > lindep of S;
* DIIS error e = X^T (F D S - S D F) X, Pulay extrapolation over at most 8 vectors;
* an initial density ``dm0`` need not be idempotent nor carry the right electron count
  (Section "Initial Guess for Mean-field Methods"), so the first Fock matrix uses the
  general K[D] = sum_P B_P D B_P.

numpy.linalg.eigh / solve serve as library primitives for the dense eigenproblem and
the small DIIS linear system.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import (cholesky, df_j, df_k, df_k_dm, int1e, int2c, int3c, nuclear_repulsion, whiten)


@dataclass
class DFSystem:
    nao: int
    naux: int
    nelec: int
    S: np.ndarray
    h: np.ndarray
    enuc: float
    B: np.ndarray          # whitened 3-index tensor, packed [naux][npair]
    M: np.ndarray | None = None
    L: np.ndarray | None = None

    @property
    def nocc(self) -> int:
        return self.nelec // 2


def build_system(mol, keep_metric: bool = False) -> DFSystem:
    """Integrals, metric Cholesky and whitened B for a gen.Molecule."""
    S, T, V = int1e(mol.ao_xyz, mol.ao_exp, mol.xyz, mol.charges)
    M = int2c(mol.aux_xyz, mol.aux_exp)
    L = cholesky(M)
    B = whiten(L, int3c(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp))
    return DFSystem(nao=mol.nao, naux=mol.naux, nelec=mol.nelec, S=S, h=T + V,
                    enuc=nuclear_repulsion(mol.xyz, mol.charges), B=B,
                    M=M if keep_metric else None, L=L if keep_metric else None)


def canonical_orthogonalization(S: np.ndarray, lindep: float = 1e-8) -> np.ndarray:
    s, U = np.linalg.eigh(S)
    keep = s > lindep
    return U[:, keep] / np.sqrt(s[keep])


def occupied_from_fock(F: np.ndarray, X: np.ndarray, nocc: int):
    """Diagonalise X^T F X and return (C_occ, orbital energies) with C = X C'."""
    e, Cp = np.linalg.eigh(X.T @ F @ X)
    C = X @ Cp
    return C[:, :nocc], e


def core_guess(sysm: DFSystem, X: np.ndarray | None = None):
    if X is None:
        X = canonical_orthogonalization(sysm.S)
    C, e = occupied_from_fock(sysm.h, X, sysm.nocc)
    return C, e


@dataclass
class SCFResult:
    energy: float
    converged: bool
    iterations: int
    C_occ: np.ndarray
    D: np.ndarray
    mo_energy: np.ndarray
    history: list = field(default_factory=list)


class DIIS:
    """Pulay DIIS on (F, e) pairs; solves [[B, -1], [-1, 0]] [c, lam] = [0, -1]."""

    def __init__(self, space: int = 8):
        self.space = space
        self.F: list[np.ndarray] = []
        self.e: list[np.ndarray] = []

    def push(self, F: np.ndarray, e: np.ndarray) -> None:
        self.F.append(F)
        self.e.append(e)
        if len(self.F) > self.space:
            self.F.pop(0)
            self.e.pop(0)

    def extrapolate(self) -> np.ndarray:
        m = len(self.F)
        if m < 2:
            return self.F[-1]
        Bm = np.empty((m + 1, m + 1))
        for i in range(m):
            for j in range(m):
                Bm[i, j] = np.sum(self.e[i] * self.e[j])
        Bm[m, :m] = Bm[:m, m] = -1.0
        Bm[m, m] = 0.0
        rhs = np.zeros(m + 1)
        rhs[m] = -1.0
        try:
            c = np.linalg.solve(Bm, rhs)
        except np.linalg.LinAlgError:
            c = None
        if c is None or not np.all(np.isfinite(c)):
            # singular subspace: restart from the newest vector
            self.F, self.e = self.F[-1:], self.e[-1:]
            return self.F[-1]
        return sum(c[i] * self.F[i] for i in range(m))


def rhf(sysm: DFSystem, dm0: np.ndarray | None = None, diis_space: int = 8, conv_tol: float = 1e-8,
        conv_err: float = 1e-5, max_cycle: int = 100, lindep: float = 1e-8) -> SCFResult:
    """DF-RHF to |dE| < conv_tol and max|e| < conv_err."""
    nao, nocc = sysm.nao, sysm.nocc
    X = canonical_orthogonalization(sysm.S, lindep)
    if dm0 is None:
        C, _ = occupied_from_fock(sysm.h, X, nocc)
        D = 2.0 * C @ C.T
    else:
        C = None
        D = np.array(dm0, dtype=np.float64)
    diis = DIIS(diis_space)
    e_old = None
    hist = []
    converged = False
    mo_e = None
    it = 0
    for it in range(1, max_cycle + 1):
        J = df_j(sysm.B, nao, D)
        K = df_k(sysm.B, nao, C) if C is not None else 0.5 * df_k_dm(sysm.B, nao, D)
        F = sysm.h + J - K
        E = 0.5 * np.sum(D * (sysm.h + F)) + sysm.enuc
        FDS = F @ D @ sysm.S
        err = X.T @ (FDS - FDS.T) @ X
        emax = float(np.max(np.abs(err)))
        hist.append((E, emax))
        if e_old is not None and abs(E - e_old) < conv_tol and emax < conv_err:
            converged = True
            break
        diis.push(F, err)
        Fbar = diis.extrapolate()
        C, mo_e = occupied_from_fock(Fbar, X, nocc)
        D = 2.0 * C @ C.T
        e_old = E
    return SCFResult(energy=E, converged=converged, iterations=it, C_occ=C if C is not None else np.zeros((nao, 0)),
                     D=D, mo_energy=mo_e, history=hist)
