"""Finite-difference orbital Hessians from the oracle, shared by the stability tests.

Test infrastructure: the oracle's Fock build under exact orbital rotations exp(kappa)
(scipy.linalg.expm) of its canonical orbitals.  The energy's gradient with respect to a
(virtual, occupied) rotation kappa_ai is 4 F_ai in the rotated orbitals; central differences
of that gradient give the Hessian with an O(h^2) error, because the second-order terms of the
exponential map are occupied-occupied and virtual-virtual rotations, to which the energy is
invariant.  Second differences of the energy itself give the same matrix, more slowly.
"""
import numpy as np
from scipy.linalg import expm

import gen
import oracle
from oracle import scf as oscf


def fock(sysm, D):
    return sysm.h + oracle.df_j(sysm.B, sysm.nao, D) - 0.5 * oracle.df_k_dm(sysm.B, sysm.nao, D)


def energy(sysm, D):
    return 0.5 * np.sum(D * (sysm.h + fock(sysm, D))) + sysm.enuc


def canonical_orbitals(sysm, D):
    """(X, C') with C' the eigenvectors of X^T F[D] X in the canonical orthonormal basis X."""
    X = oscf.canonical_orthogonalization(sysm.S)
    _, Cp = np.linalg.eigh(X.T @ fock(sysm, D) @ X)
    return X, Cp


def rotated(X, Cp, nocc, kappa):
    """Orbitals X C' exp(A) with A = [[0, -kappa^T], [kappa, 0]] (kappa [nvir][nocc])."""
    nmo = Cp.shape[1]
    A = np.zeros((nmo, nmo))
    A[nocc:, :nocc] = kappa
    A[:nocc, nocc:] = -kappa.T
    return X @ Cp @ expm(A)


def fd_hessian(sysm, D, h=1e-4):
    """Hessian of the energy over (virtual, occupied) rotations, from central differences of
    the gradient 4 F_vo; returns (H, (X, C'))."""
    X, Cp = canonical_orbitals(sysm, D)
    nocc, nmo = sysm.nocc, Cp.shape[1]
    nvir = nmo - nocc

    def grad(kappa):
        C = rotated(X, Cp, nocc, kappa)
        Co = C[:, :nocc]
        return 4 * (C[:, nocc:].T @ fock(sysm, 2 * Co @ Co.T) @ Co)

    n = nvir * nocc
    H = np.zeros((n, n))
    for q in range(n):
        e = np.zeros(n)
        e[q] = h
        H[:, q] = ((grad(e.reshape(nvir, nocc)) - grad(-e.reshape(nvir, nocc))) / (2 * h)).ravel()
    assert np.abs(H - H.T).max() <= 1e-6 * np.abs(H).max()
    return 0.5 * (H + H.T), (X, Cp)


def fd_hessian_eigenvalues(sysm, D):
    return np.linalg.eigvalsh(fd_hessian(sysm, D)[0])


def energy_fd_hessian(sysm, D, h=1e-3):
    """The same Hessian from second differences of the energy (slow: four energies per entry)."""
    X, Cp = canonical_orbitals(sysm, D)
    nocc, nmo = sysm.nocc, Cp.shape[1]
    nvir = nmo - nocc
    n = nvir * nocc

    def e_of(k):
        Co = rotated(X, Cp, nocc, k.reshape(nvir, nocc))[:, :nocc]
        return energy(sysm, 2 * Co @ Co.T)

    e0 = e_of(np.zeros(n))
    H = np.zeros((n, n))
    I = np.eye(n) * h
    for p in range(n):
        H[p, p] = (e_of(I[p]) - 2 * e0 + e_of(-I[p])) / (h * h)
        for q in range(p):
            H[p, q] = H[q, p] = (e_of(I[p] + I[q]) - e_of(I[p] - I[q]) - e_of(-I[p] + I[q])
                                 + e_of(-I[p] - I[q])) / (4 * h * h)
    return H


def h10_ring(d=4.5):
    """Ten centres on a regular ring with neighbours d bohr apart (centred at (10, 10, 10))."""
    n = 10
    R = d / (2 * np.sin(np.pi / n))
    ang = 2 * np.pi * np.arange(n) / n
    xyz = np.stack([R * np.cos(ang), R * np.sin(ang), np.zeros(n)], 1) + 10.0
    return gen.molecules.molecule_from_geometry(xyz)


def escape(sysm, D, H, XC, angle=0.3):
    """Turn the orbitals by `angle` along the Hessian's lowest eigenvector and converge the
    oracle's SCF from there; returns its result."""
    X, Cp = XC
    nocc, nmo = sysm.nocc, Cp.shape[1]
    w, V = np.linalg.eigh(H)
    u = angle * V[:, 0].reshape(nmo - nocc, nocc)
    Co = rotated(X, Cp, nocc, u)[:, :nocc]
    return oscf.rhf(sysm, dm0=2 * Co @ Co.T)
