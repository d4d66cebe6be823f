"""Mixed-precision (split-BF16 x3 on tcgen05 tensor cores) J/K against the FP64 oracle.

Two references: the exact FP64 oracle, and a numpy emulation of the same split
arithmetic (hi = RN_bf16(x), lo = RN_bf16(x - hi), products hi*hi + hi*lo + lo*hi, the
half-transformed X rounded to FP32 before its own split).  The emulation isolates the
kernel's FP32 accumulation error from the split representation error."""
import numpy as np
import pytest
import torch

import gen
import oracle
from oracle import scf as oscf

pytestmark = pytest.mark.gpu
dfscf = pytest.importorskip("paper_2506_06661_gb300")


def bf16_rn(x):
    """Round float64 to the nearest bf16 value (8 significant bits, ties to even)."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.round(m * 256.0), e - 8)


def split(x):
    hi = bf16_rn(x)
    return hi, bf16_rn(x - hi)


def emulated_k(Bfull, C):
    """Bfull [naux, nao, nao]; returns K from split-BF16 x3 of both contractions."""
    Bh, Bl = split(Bfull)
    Ch, Cl = split(C)
    X = np.einsum("pmn,ni->pmi", Bh, Ch) + np.einsum("pmn,ni->pmi", Bh, Cl) + np.einsum("pmn,ni->pmi", Bl, Ch)
    Xh, Xl = split(X.astype(np.float32).astype(np.float64))
    return (np.einsum("pmi,pni->mn", Xh, Xh) + np.einsum("pmi,pni->mn", Xh, Xl)
            + np.einsum("pmi,pni->mn", Xl, Xh))


def rel(a, b):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def full_B(sysm):
    return np.stack([oracle.unpack(sysm.B[P], sysm.nao) for P in range(sysm.naux)])


@pytest.mark.parametrize("case", ["c0", "nocc1", "ragged17"])
def test_mixed_jk_parity(case, c0):
    if case == "c0":
        mol, nocc = c0, c0.nocc
    else:
        mol = gen.molecule_from_geometry(gen.make_geometry(7 if case == "nocc1" else 13, 5.0, 11))
        nocc = 1 if case == "nocc1" else 17
    sysm = oscf.build_system(mol)
    rng = np.random.default_rng(nocc)
    if case == "c0":
        C, _ = oscf.core_guess(sysm)
    else:
        C = 0.3 * rng.standard_normal((mol.nao, nocc))
    D = 2 * C @ C.T
    L = dfscf.metric_chol(mol.aux_xyz, mol.aux_exp)
    B = dfscf.build_B(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp, L, "mixed")
    J, K = dfscf.jk(B, D, C, precision="mixed")
    Jo = oracle.df_j(sysm.B, mol.nao, D)
    Ko = oracle.df_k(sysm.B, mol.nao, C)
    Ke = emulated_k(full_B(sysm), C)
    ej, ek, eke = rel(J, Jo), rel(K, Ko), rel(K, Ke)
    print(f"{case}: J rel {ej:.2e}  K rel (exact) {ek:.2e}  K rel (split emulation) {eke:.2e}")
    assert ej <= 2e-6
    # only the FP32 accumulation order differs from the emulation: sums of >= 128 terms
    # with cancellation, measured 2.3e-6 on the 20-centre molecule
    assert eke <= 1e-5
    assert ek <= 5e-5         # split-BF16 representation error vs exact FP64
    # the FP64 planes of a mixed B still give the exact FP64 result
    J64, K64 = dfscf.jk(B, D, C, precision="fp64")
    assert rel(J64, Jo) <= 1e-10 and rel(K64, Ko) <= 1e-10


def test_mixed_scf_energy_within_1e6(c0, c0_scf):
    r = dfscf.scf_run(c0, precision="mixed")
    assert r.converged and r.fp64_iterations >= 2
    assert abs(r.energy - c0_scf.energy) <= 1e-6
