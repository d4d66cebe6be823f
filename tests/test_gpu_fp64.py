"""GPU parity of the FP64 path against the CPU oracle (C-ABI through the binding).

Sizes: the 20-centre molecule (nao 100, naux 300, several tiles of every kernel) and
ragged molecules whose dimensions are not multiples of any tile.  Bar: 1e-10 relative
in max-norm for J and K (FP64 mode), tighter where the arithmetic allows it."""
import numpy as np
import pytest
import torch

import gen
import oracle
from oracle import scf as oscf

pytestmark = pytest.mark.gpu

dfscf = pytest.importorskip("paper_2506_06661_gb300")


def rel(a, b):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def ragged_molecule(n=7, seed=4, orb=(0.1, 10.0, 5), aux=(0.05, 50.0, 15), nelec=None):
    xyz = gen.make_geometry(n, 5.0, seed)
    return gen.molecule_from_geometry(xyz, gen.even_tempered(*orb), gen.even_tempered(*aux), nelec=nelec)


def test_boys_matches_oracle():
    rng = np.random.default_rng(0)
    t = np.concatenate([[0.0, 1e-300, 1e-12, 5e-4, 9.999e-4, 1e-3, 1.0001e-3, 0.5, 1.0, 10.0, 39.99, 40.0, 40.01,
                         100.0, 1e6], 10 ** rng.uniform(-8, 3, 4000)])
    got = dfscf.boys_f0(t).cpu().numpy()
    ref = oracle.boys_f0(t)
    assert np.max(np.abs(got - ref) / ref) <= 1e-14


def test_boys_empty_and_ragged():
    assert dfscf.boys_f0(np.zeros(0)).numel() == 0
    t = np.linspace(0, 50, 257)
    assert np.allclose(dfscf.boys_f0(t).cpu().numpy(), oracle.boys_f0(t), rtol=1e-14, atol=0)


@pytest.mark.parametrize("which", ["c0", "ragged"])
def test_int1e_matches_oracle(which, c0):
    mol = c0 if which == "c0" else ragged_molecule()
    S, T, V = dfscf.int1e(mol.ao_xyz, mol.ao_exp, mol.xyz, mol.charges)
    So, To, Vo = oracle.int1e(mol.ao_xyz, mol.ao_exp, mol.xyz, mol.charges)
    assert rel(S, So) <= 1e-14 and rel(T, To) <= 1e-14 and rel(V, Vo) <= 1e-13
    assert abs(dfscf.nuclear_repulsion(mol.xyz, mol.charges) - oracle.nuclear_repulsion(mol.xyz, mol.charges)) <= 1e-12


def test_metric_cholesky_matches_oracle(c0, c0_system):
    L, M = dfscf.metric_chol(c0.aux_xyz, c0.aux_exp, return_metric=True)
    assert rel(M, c0_system.M) <= 1e-14
    Lc = L.cpu().numpy()
    assert np.all(np.triu(Lc, 1) == 0.0)
    # backward error of the GPU factor, then agreement with the oracle's factor
    assert rel(Lc @ Lc.T, c0_system.M) <= 1e-13
    assert rel(Lc, c0_system.L) <= 1e-8


def test_metric_cholesky_reports_bad_pivot():
    mol = gen.make_molecule(3, 4.0, 7)
    xyz = np.vstack([mol.aux_xyz, mol.aux_xyz[:1]])
    ex = np.concatenate([mol.aux_exp, mol.aux_exp[:1]])
    with pytest.raises(dfscf.DFError) as ei:
        dfscf.metric_chol(xyz, ex)
    assert ei.value.code == dfscf.DF_ERR_NOT_SPD
    assert ei.value.pivot == len(ex) - 1


@pytest.fixture(scope="module")
def c0_gpu_B(c0):
    L = dfscf.metric_chol(c0.aux_xyz, c0.aux_exp)
    return dfscf.build_B(c0.ao_xyz, c0.ao_exp, c0.aux_xyz, c0.aux_exp, L, "fp64")


def test_build_B_matches_oracle(c0, c0_system, c0_gpu_B):
    got = torch.stack([dfscf.B_get_packed(c0_gpu_B, P) for P in range(c0.naux)])
    assert rel(got, c0_system.B) <= 1e-8
    # padding of every row is zero
    raw = c0_gpu_B.buf.view(torch.float64)[: c0.naux * c0_gpu_B.ld].view(c0.naux, c0_gpu_B.ld)
    assert torch.all(raw[:, c0.nao * (c0.nao + 1) // 2:] == 0)


def core_density(sysm):
    C, _ = oscf.core_guess(sysm)
    return C, 2 * C @ C.T


def test_jk_fp64_matches_oracle(c0, c0_system, c0_gpu_B):
    C, D = core_density(c0_system)
    J, K = dfscf.jk(c0_gpu_B, D, C)
    Jo = oracle.df_j(c0_system.B, c0.nao, D)
    Ko = oracle.df_k(c0_system.B, c0.nao, C)
    assert rel(J, Jo) <= 1e-10
    assert rel(K, Ko) <= 1e-10


@pytest.mark.parametrize("nocc,orb,aux,n", [(1, (0.1, 10.0, 5), (0.05, 50.0, 15), 7),
                                             (3, (0.2, 5.0, 3), (0.3, 20.0, 2), 9),
                                             (17, (0.1, 10.0, 5), (0.05, 50.0, 15), 13)])
def test_jk_fp64_ragged(nocc, orb, aux, n):
    """nao and naux not multiples of any tile; naux < nao in the second case."""
    mol = ragged_molecule(n, 11, orb, aux)
    sysm = oscf.build_system(mol)
    L = dfscf.metric_chol(mol.aux_xyz, mol.aux_exp)
    B = dfscf.build_B(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp, L, "fp64")
    rng = np.random.default_rng(nocc)
    C = rng.standard_normal((mol.nao, nocc)) * 0.3
    D = 2 * C @ C.T
    J, K = dfscf.jk(B, D, C)
    assert rel(J, oracle.df_j(sysm.B, mol.nao, D)) <= 1e-10
    assert rel(K, oracle.df_k(sysm.B, mol.nao, C)) <= 1e-10


def test_jk_only_j_or_only_k(c0, c0_system, c0_gpu_B):
    C, D = core_density(c0_system)
    J, K = dfscf.jk(c0_gpu_B, D, None)
    assert K is None and rel(J, oracle.df_j(c0_system.B, c0.nao, D)) <= 1e-10
    J, K = dfscf.jk(c0_gpu_B, None, C)
    assert J is None and rel(K, oracle.df_k(c0_system.B, c0.nao, C)) <= 1e-10


@pytest.mark.parametrize("n", [1, 2, 3, 7, 64, 129, 200, 400])
def test_eigh_matches_library(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    A = A + A.T
    w, Z = dfscf.eigh(A)
    w, Z = w.cpu().numpy(), Z.cpu().numpy()
    wr = np.linalg.eigvalsh(A)
    assert np.max(np.abs(w - wr)) <= 1e-12 * max(1.0, np.max(np.abs(wr)))
    assert np.max(np.abs(A @ Z - Z * w)) <= 1e-11 * max(1.0, np.max(np.abs(wr)))
    assert np.max(np.abs(Z.T @ Z - np.eye(n))) <= 1e-12


def test_eigh_full_spectrum_multi_sm_overlap():
    """Full spectrum above n = 160 runs on the multi-SM path: the overlap matrix of the
    80-centre molecule (eigenvalues from ~1e-5 to ~10, small ones clustered) and a
    density of rank 31 (a 269-fold zero eigenvalue)."""
    mol = gen.make_molecule(80, gen.molecules.box_for(80), 0)
    _, _, S, *_ = dfscf.core_guess(mol)
    S = S.cpu().numpy()
    rng = np.random.default_rng(31)
    C = 0.3 * rng.standard_normal((300, 31))
    for A in (S, 2 * C @ C.T):
        n = A.shape[0]
        w, Z = dfscf.eigh(A)
        w, Z = w.cpu().numpy(), Z.cpu().numpy()
        wr = np.linalg.eigvalsh(A)
        scale = max(1.0, np.max(np.abs(wr)))
        assert np.max(np.abs(w - wr)) <= 1e-12 * scale
        assert np.max(np.abs(A @ Z - Z * w)) <= 1e-11 * scale
        assert np.max(np.abs(Z.T @ Z - np.eye(n))) <= 1e-11


def test_scf_fp64_matches_oracle(c0, c0_scf):
    r = dfscf.scf_run(c0, precision="fp64")
    assert r.converged
    assert abs(r.energy - c0_scf.energy) <= 1e-9
    D = r.D.cpu().numpy()
    assert rel(D, c0_scf.D) <= 1e-5
    assert r.lumo > r.homo


def test_scf_accepts_converged_dm0(c0, c0_scf):
    # an idempotent dm0 starts from its orbitals; a non-idempotent one (the same density
    # mixed with half the core-guess density, same electron count) through the eager first
    # iteration; both reach the oracle's energy
    r = dfscf.scf_run(c0, dm0=c0_scf.D, precision="fp64")
    assert r.guess == 1 and r.converged and r.iterations <= 4
    assert abs(r.energy - c0_scf.energy) <= 1e-9
    _, Dc, *_ = dfscf.core_guess(c0)
    mix = 0.5 * c0_scf.D + 0.5 * Dc.cpu().numpy()
    r = dfscf.scf_run(c0, dm0=mix, precision="fp64")
    assert r.guess == 1 and r.converged
    assert abs(r.energy - c0_scf.energy) <= 1e-9


def test_scf_rejects_bad_dm0(c0, c0_scf):
    r = dfscf.scf_run(c0, dm0=3.0 * c0_scf.D, precision="fp64")
    assert r.guess == 2 and r.converged
    assert abs(r.energy - c0_scf.energy) <= 1e-9


def test_scf_nonidempotent_dm0_reaches_same_fixed_point(c0, c0_system, c0_scf):
    rng = np.random.default_rng(1)
    P = 0.003 * rng.standard_normal(c0_scf.D.shape)
    dm0 = c0_scf.D + 0.5 * (P + P.T)
    from oracle import mlp
    assert mlp.guess_is_valid(dm0, c0_system.S, c0_system.nelec)
    r = dfscf.scf_run(c0, dm0=dm0, precision="fp64")
    assert r.guess == 1 and r.converged
    assert abs(r.energy - c0_scf.energy) <= 1e-9


def test_scf_reports_noconv(c0):
    with pytest.raises(dfscf.DFError) as ei:
        dfscf.scf_run(c0, precision="fp64", max_cycle=3)
    assert ei.value.code == dfscf.DF_ERR_NOCONV


def test_jk_workspace_too_small(c0_gpu_B, c0):
    L = dfscf.lib()
    tiny = torch.empty(16, dtype=torch.uint8, device="cuda")
    D = torch.zeros(c0.nao, c0.nao, dtype=torch.float64, device="cuda")
    J = torch.empty_like(D)
    rc = L.df_jk(dfscf._ptr(c0_gpu_B.buf), c0.nao, c0.naux, 0, dfscf._ptr(D), None, 0, dfscf._ptr(J), None,
                 dfscf._ptr(tiny), 16, dfscf._stream())
    assert rc == dfscf.DF_ERR_NOMEM


@pytest.mark.parametrize("n,k", [(16, 1), (100, 11), (257, 40), (400, 41)])
def test_eigh_lowest_matches_library(n, k):
    rng = np.random.default_rng(n + k)
    A = rng.standard_normal((n, n))
    A = A + A.T
    w, Z = dfscf.eigh_lowest(A, k)
    w, Z = w.cpu().numpy(), Z.cpu().numpy()
    wr = np.linalg.eigvalsh(A)[:k]
    scale = max(1.0, np.max(np.abs(np.linalg.eigvalsh(A))))
    assert np.max(np.abs(w - wr)) <= 1e-12 * scale
    assert np.max(np.abs(A @ Z - Z * w)) <= 1e-10 * scale
    assert np.max(np.abs(Z.T @ Z - np.eye(k))) <= 1e-12


@pytest.mark.parametrize("n,k,ctas", [(257, 40, 1), (120, 100, 1), (300, 31, 4), (200, 21, 152)])
def test_eigh_lowest_forced_launch_shapes(n, k, ctas):
    """The one-CTA solver at sizes the default picks the cooperative grid for (grouped Sturm
    multisection with 2 and 1 lanes per eigenvalue), and cooperative grids of 4 and 152 CTAs."""
    lib = dfscf.lib()
    lib.df_tune_set(b"eig_ctas", ctas)
    try:
        rng = np.random.default_rng(n * k)
        A = rng.standard_normal((n, n))
        A = A + A.T
        w, Z = dfscf.eigh_lowest(A, k)
    finally:
        lib.df_tune_set(b"eig_ctas", 0)
    w, Z = w.cpu().numpy(), Z.cpu().numpy()
    ev = np.linalg.eigvalsh(A)
    scale = max(1.0, np.max(np.abs(ev)))
    assert np.max(np.abs(w - ev[:k])) <= 1e-12 * scale
    assert np.max(np.abs(A @ Z - Z * w)) <= 1e-10 * scale
    assert np.max(np.abs(Z.T @ Z - np.eye(k))) <= 1e-12


def test_eigh_lowest_near_degenerate_spectrum():
    """Pairs of eigenvalues 1e-9 apart: the vectors must still span the right subspace."""
    n, k = 60, 10
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.sort(np.concatenate([np.repeat(np.linspace(-3, -1, 5), 2) + np.tile([0, 1e-9], 5),
                                  np.linspace(0, 5, n - 10)]))
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    w, Z = dfscf.eigh_lowest(A, k)
    Z = Z.cpu().numpy()
    assert np.max(np.abs(Z.T @ Z - np.eye(k))) <= 1e-10
    P = Z @ Z.T
    Pref = Q[:, :k] @ Q[:, :k].T
    assert np.max(np.abs(P - Pref)) <= 1e-8


@pytest.mark.parametrize("n,nocc,ctas", [(60, 12, 0), (200, 40, 1), (400, 90, 0), (300, 64, 16)])
def test_eigh_lowest_of_negated_projector(n, nocc, ctas):
    """-2 V V^T (V orthonormal): an nocc-fold eigenvalue -2 and an (n - nocc)-fold 0.  Inverse
    iteration from distinct starts plus two Gram-Schmidt passes resolves an exactly degenerate
    cluster to ~1e-8 in the span (the vectors of the cluster come out nearly parallel before
    the re-orthogonalisation); eigenvalues and orthonormality stay at rounding level.  One-CTA
    and cooperative launches alike."""
    rng = np.random.default_rng(n + nocc)
    V, _ = np.linalg.qr(rng.standard_normal((n, nocc)))
    A = -2.0 * V @ V.T
    lib = dfscf.lib()
    lib.df_tune_set(b"eig_ctas", ctas)
    try:
        w, Z = dfscf.eigh_lowest(A, nocc + 1)
    finally:
        lib.df_tune_set(b"eig_ctas", 0)
    w, Z = w.cpu().numpy(), Z.cpu().numpy()
    assert np.max(np.abs(w[:nocc] + 2.0)) <= 1e-12 and abs(w[nocc]) <= 1e-12
    assert np.max(np.abs(Z.T @ Z - np.eye(nocc + 1))) <= 1e-11
    Zo = Z[:, :nocc]
    assert np.max(np.abs(Zo @ Zo.T - V @ V.T)) <= 1e-7
    assert np.max(np.abs(A @ Z - Z * w)) <= 2e-7


@pytest.mark.parametrize("n,rank", [(40, 5), (100, 10), (257, 31)])
def test_eigh_rank_deficient_density(n, rank):
    """A density-like matrix 2 C C^T: n - rank zero eigenvalues (a degenerate spectrum)."""
    rng = np.random.default_rng(n)
    C = 0.3 * rng.standard_normal((n, rank))
    A = 2 * C @ C.T
    w, Z = dfscf.eigh(A)
    w, Z = w.cpu().numpy(), Z.cpu().numpy()
    wr = np.linalg.eigvalsh(A)
    scale = np.max(np.abs(wr))
    assert np.max(np.abs(w - wr)) <= 1e-12 * scale
    assert np.max(np.abs(A @ Z - Z * w)) <= 1e-11 * scale
    assert np.max(np.abs(Z.T @ Z - np.eye(n))) <= 1e-12
