"""Pins for the oracle's density fitting, J/K and RHF (CPU only).

* exactness: when the auxiliary set holds every product Gaussian of the orbital basis,
  the fitted (mn|kl) = sum_P T_{P,mn} T_{P,kl} of the paper's DF equation is exact, so
  DF-J and DF-K must equal brute-force four-centre J and K;
* the solve form (mn|kl) = sum_PQ (P|mn)(M^-1)_PQ (Q|kl) (the paper's rewritten DF
  equation in the auxiliary-basis section) must give the same J and K as the Cholesky
  whitening;
* symmetry, tr(DJ) = sum_P d_P^2 >= 0, K positive semidefinite, K invariant under
  occupied rotations, the Lehtola diagonal error terms >= 0;
* H2 with one s function per centre has a symmetry-fixed orbital and a closed-form RHF
  energy, which the DF-RHF must reproduce with a product-complete auxiliary set.
"""
import numpy as np
import pytest
from scipy import linalg as sla

import gen
import oracle
from oracle import scf


def product_aux(xyz, ex):
    """Unique product Gaussians (exponent a+b at the product centre) of an orbital set."""
    seen, cx, ce = set(), [], []
    for i in range(len(ex)):
        for j in range(i + 1):
            p = ex[i] + ex[j]
            P = (ex[i] * xyz[i] + ex[j] * xyz[j]) / p
            key = (round(p, 12),) + tuple(np.round(P, 12))
            if key not in seen:
                seen.add(key)
                cx.append(P)
                ce.append(p)
    return np.array(cx), np.array(ce)


def tiny_product_complete():
    xyz0 = np.array([[0.0, 0.0, 0.0], [1.4, 0.2, -0.3], [-0.5, 1.6, 0.4]])
    mol = gen.molecule_from_geometry(xyz0, orb_exp=[0.4, 1.9], aux_exp=[1.0])
    ax, ae = product_aux(mol.ao_xyz, mol.ao_exp)
    mol.aux_xyz, mol.aux_exp = ax, ae
    return mol


def dens(nao, nocc, seed):
    rng = np.random.default_rng(seed)
    C = rng.standard_normal((nao, nocc)) * 0.3
    return C, 2.0 * C @ C.T


def test_cholesky_reconstructs_and_matches_library(c0_system):
    M, L = c0_system.M, c0_system.L
    assert np.allclose(np.triu(L, 1), 0.0)
    assert np.max(np.abs(L @ L.T - M)) <= 1e-12 * np.max(np.abs(M))
    Lnp = np.linalg.cholesky(M)
    assert np.max(np.abs(L - Lnp)) <= 1e-9 * np.max(np.abs(Lnp))


def test_cholesky_reports_singular_metric():
    mol = gen.make_molecule(3, 4.0, 7)
    xyz = np.vstack([mol.aux_xyz, mol.aux_xyz[:1]])
    ex = np.concatenate([mol.aux_exp, mol.aux_exp[:1]])
    with pytest.raises(oracle.NotPositiveDefinite) as ei:
        oracle.cholesky(oracle.int2c(xyz, ex))
    assert ei.value.pivot == len(ex) - 1


def test_whitening_solves_triangular_system(c0, c0_system):
    R = oracle.int3c(c0.ao_xyz, c0.ao_exp, c0.aux_xyz, c0.aux_exp)
    B = c0_system.B
    assert np.max(np.abs(c0_system.L @ B - R)) <= 1e-12 * np.max(np.abs(R))
    Bref = sla.solve_triangular(c0_system.L, R, lower=True)
    assert np.max(np.abs(B - Bref)) <= 1e-9 * np.max(np.abs(Bref))


def test_sampled_rows_match_packed_tensor(c0, c0_system):
    # int3c_rows is int3c read at (max(r, n), min(r, n)): bit for bit, first and last rows
    # included; df_b_rows gives the same rows of B as the pinned whitening
    rows = [0, 37, c0.nao - 1]
    R = oracle.int3c(c0.ao_xyz, c0.ao_exp, c0.aux_xyz, c0.aux_exp)
    Rr = oracle.int3c_rows(c0.ao_xyz, c0.ao_exp, c0.aux_xyz, c0.aux_exp, rows)
    n = np.arange(c0.nao)
    for t, r in enumerate(rows):
        a, b = np.maximum(r, n), np.minimum(r, n)
        assert np.array_equal(Rr[:, t, :], R[:, a * (a + 1) // 2 + b])
    Br = oracle.df_b_rows(c0.ao_xyz, c0.ao_exp, c0.aux_xyz, c0.aux_exp, c0_system.L, rows)
    for t, r in enumerate(rows):
        a, b = np.maximum(r, n), np.minimum(r, n)
        ref = c0_system.B[:, a * (a + 1) // 2 + b]
        assert np.max(np.abs(Br[:, t, :] - ref)) <= 1e-9 * np.max(np.abs(ref))
    # the sampled-row J and K formulas of the full-size GPU test, against the oracle's df_j /
    # df_k on the whole tensor: K among the rows, J of a density supported on the rows
    rng = np.random.default_rng(5)
    C = rng.standard_normal((c0.nao, 7)) / np.sqrt(c0.nao)
    Ds = np.zeros((c0.nao, c0.nao))
    for r in rows:
        v = 0.1 * rng.standard_normal(c0.nao)
        Ds[r, :] += v
        Ds[:, r] += v
    X = Br @ C
    Kref = np.einsum("pai,pbi->ab", X, X)
    d = sum(2.0 * Br[:, t, :] @ Ds[r, :] - Br[:, t, rows] @ Ds[r, rows] for t, r in enumerate(rows))
    Jref = np.einsum("p,pab->ab", d, Br[:, :, rows])
    K = oracle.df_k(c0_system.B, c0.nao, C)[np.ix_(rows, rows)]
    J = oracle.df_j(c0_system.B, c0.nao, Ds)[np.ix_(rows, rows)]
    assert np.max(np.abs(K - Kref)) <= 1e-11 * np.max(np.abs(K))
    assert np.max(np.abs(J - Jref)) <= 1e-11 * np.max(np.abs(J))


def test_aux_normalisation_invariance(c0, c0_system):
    """chol(Lam M Lam) = Lam L for positive diagonal Lam, so B does not depend on aux scaling."""
    lam = np.exp(np.random.default_rng(0).uniform(-2, 2, size=c0.naux))
    M = c0_system.M * lam[:, None] * lam[None, :]
    R = oracle.int3c(c0.ao_xyz, c0.ao_exp, c0.aux_xyz, c0.aux_exp) * lam[:, None]
    B2 = oracle.whiten(oracle.cholesky(M), R)
    assert np.max(np.abs(B2 - c0_system.B)) <= 1e-8 * np.max(np.abs(c0_system.B))


def test_df_is_exact_for_product_complete_aux():
    mol = tiny_product_complete()
    nao = mol.nao
    B = oracle.whiten(oracle.cholesky(oracle.int2c(mol.aux_xyz, mol.aux_exp)),
                      oracle.int3c(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp))
    eri = oracle.int4c(mol.ao_xyz, mol.ao_exp)
    C, D = dens(nao, 2, 11)
    J4, K4 = oracle.jk_4c(eri, D, C @ C.T)
    J = oracle.df_j(B, nao, D)
    K = oracle.df_k(B, nao, C)
    assert np.max(np.abs(J - J4)) <= 1e-8 * np.max(np.abs(J4))
    assert np.max(np.abs(K - K4)) <= 1e-8 * np.max(np.abs(K4))
    # diagonal error vanishes pair by pair
    delta = oracle.eri_diag(mol.ao_xyz, mol.ao_exp) - np.sum(B * B, axis=0)
    assert np.max(np.abs(delta)) <= 1e-8 * np.max(oracle.eri_diag(mol.ao_xyz, mol.ao_exp))


def test_df_jk_solve_form_matches_cholesky_form(c0, c0_system):
    nao = c0.nao
    R = oracle.int3c(c0.ao_xyz, c0.ao_exp, c0.aux_xyz, c0.aux_exp)
    C, D = dens(nao, c0.nocc, 12)
    J = oracle.df_j(c0_system.B, nao, D)
    K = oracle.df_k(c0_system.B, nao, C)
    Rf = np.stack([oracle.unpack(R[q], nao) for q in range(c0.naux)])   # [naux, nao, nao]
    MinvR = np.linalg.solve(c0_system.M, R)
    MinvRf = np.stack([oracle.unpack(MinvR[q], nao) for q in range(c0.naux)])
    g = np.einsum("qkl,kl->q", Rf, D)
    Jref = np.einsum("q,qmn->mn", np.linalg.solve(c0_system.M, g), Rf)
    X = np.einsum("qmn,ni->qmi", Rf, C)
    Y = np.einsum("qmn,ni->qmi", MinvRf, C)
    Kref = np.einsum("qmi,qni->mn", X, Y)
    # conditioning of M (~4e10) limits agreement between the two factorisations
    assert np.max(np.abs(J - Jref)) <= 1e-6 * np.max(np.abs(J))
    assert np.max(np.abs(K - Kref)) <= 1e-6 * np.max(np.abs(K))


def test_jk_symmetry_and_positivity(c0, c0_system):
    nao = c0.nao
    C, D = dens(nao, c0.nocc, 13)
    J = oracle.df_j(c0_system.B, nao, D)
    K = oracle.df_k(c0_system.B, nao, C)
    assert np.max(np.abs(J - J.T)) <= 1e-14 * np.max(np.abs(J))
    assert np.max(np.abs(K - K.T)) <= 1e-13 * np.max(np.abs(K))
    B = c0_system.B
    w = np.where(np.eye(nao, dtype=bool)[np.tril_indices(nao)], 1.0, 2.0)
    d = B @ (w * D[np.tril_indices(nao)])
    assert np.sum(D * J) == pytest.approx(np.sum(d * d), rel=1e-12)
    assert np.sum(D * K) >= 0.0
    assert np.min(np.linalg.eigvalsh(K)) >= -1e-12 * np.max(np.abs(K))


def test_k_invariant_under_occupied_rotation(c0, c0_system):
    nao = c0.nao
    C, _ = dens(nao, c0.nocc, 14)
    U, _ = np.linalg.qr(np.random.default_rng(15).standard_normal((c0.nocc, c0.nocc)))
    K1 = oracle.df_k(c0_system.B, nao, C)
    K2 = oracle.df_k(c0_system.B, nao, C @ U)
    assert np.max(np.abs(K1 - K2)) <= 1e-12 * np.max(np.abs(K1))


def test_general_density_k_matches_factorised(c0, c0_system):
    nao = c0.nao
    C, D = dens(nao, 4, 16)
    K1 = oracle.df_k(c0_system.B, nao, C)
    K2 = 0.5 * oracle.df_k_dm(c0_system.B, nao, D)
    assert np.max(np.abs(K1 - K2)) <= 1e-12 * np.max(np.abs(K1))


def test_lehtola_diagonal_error_nonnegative(c0, c0_system):
    delta = oracle.eri_diag(c0.ao_xyz, c0.ao_exp) - np.sum(c0_system.B ** 2, axis=0)
    assert np.min(delta) >= -1e-10 * np.max(np.abs(delta))


def h2_closed_form(a, R):
    xyz = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, R]])
    S, T, V = oracle.int1e(xyz, [a, a], xyz, np.ones(2))
    h = T + V
    eri = oracle.int4c(xyz, np.array([a, a]))
    s = S[0, 1]
    hgg = (h[0, 0] + h[0, 1]) / (1 + s)
    AAAA, AABB, AAAB, ABAB = eri[0, 0, 0, 0], eri[0, 0, 1, 1], eri[0, 0, 0, 1], eri[0, 1, 0, 1]
    gggg = (2 * AAAA + 2 * AABB + 8 * AAAB + 4 * ABAB) / (4 * (1 + s) ** 2)
    return 2 * hgg + gggg + 1.0 / R


@pytest.mark.parametrize("a,R", [(0.4, 1.4), (1.0, 2.0), (0.25, 0.9)])
def test_h2_rhf_closed_form(a, R):
    xyz = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, R]])
    mol = gen.molecule_from_geometry(xyz, orb_exp=[a], aux_exp=[2 * a])
    # product-complete aux: 2a at A, 2a at B, 2a at the midpoint
    mol.aux_xyz = np.array([[0, 0, 0], [0, 0, R], [0, 0, R / 2]], dtype=float)
    mol.aux_exp = np.array([2 * a, 2 * a, 2 * a])
    res = scf.rhf(scf.build_system(mol))
    assert res.converged
    assert res.energy == pytest.approx(h2_closed_form(a, R), abs=1e-11)


def test_scf_stationarity_and_idempotency(c0_system, c0_scf):
    s = c0_system
    D = c0_scf.D
    assert c0_scf.converged
    assert np.sum(D * s.S) == pytest.approx(s.nelec, abs=1e-10)
    assert np.max(np.abs(D @ s.S @ D - 2 * D)) <= 1e-10
    C = c0_scf.C_occ
    F = s.h + oracle.df_j(s.B, s.nao, D) - oracle.df_k(s.B, s.nao, C)
    comm = F @ D @ s.S - s.S @ D @ F
    assert np.max(np.abs(comm)) <= 1e-4


def _energy(s, C):
    D = 2 * C @ C.T
    J = oracle.df_j(s.B, s.nao, D)
    K = oracle.df_k(s.B, s.nao, C)
    return np.sum(D * s.h) + 0.5 * np.sum(D * J) - 0.5 * np.sum(D * K) + s.enuc


def test_scf_energy_is_variational_minimum(c0_system, c0_scf):
    s = c0_system
    X = scf.canonical_orthogonalization(s.S)
    _, Cp = np.linalg.eigh(X.T @ (s.h + oracle.df_j(s.B, s.nao, c0_scf.D) - oracle.df_k(s.B, s.nao, c0_scf.C_occ)) @ X)
    e0 = _energy(s, c0_scf.C_occ)
    assert e0 == pytest.approx(c0_scf.energy, abs=1e-9)
    rng = np.random.default_rng(3)
    nmo, nocc = Cp.shape[1], s.nocc
    for _ in range(3):
        kappa = np.zeros((nmo, nmo))
        kappa[nocc:, :nocc] = 1e-3 * rng.standard_normal((nmo - nocc, nocc))
        kappa = kappa - kappa.T
        U = sla.expm(kappa)
        Cr = X @ (Cp @ U)[:, :nocc]
        assert _energy(s, Cr) > e0
