"""Mixed-precision (split-BF16 on tcgen05 tensor cores) J/K against the FP64 oracle.

Two references: the exact FP64 oracle, and a numpy emulation of the same split
arithmetic: every operand row as two fixed-point planes (x rounded to the grids sigma 2^-7 and
sigma 2^-15, sigma the power of two above the row's max |x|) and BF16 roundings of the rest;
products pa*qb with a + b < planes, summed exactly; the half-transformed X split again from its
exact value.  The emulation isolates the kernel's FP32 accumulation error from the split
representation error."""
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


def row_planes(x, planes, axis):
    """Row-scaled planes of x along `axis` (the contraction index): two fixed-point planes on
    the grids sigma 2^-7 and sigma 2^-15 (sigma = power of two above the row's max |x|), then
    BF16 roundings of the remainder."""
    amax = np.max(np.abs(x), axis=axis, keepdims=True)
    _, e = np.frexp(amax)
    sig = np.where(amax > 0, np.ldexp(1.0, e), 0.0)
    safe = np.where(sig > 0, sig, 1.0)
    out, r = [], x
    for g in (128.0, 32768.0):
        h = np.where(sig > 0, np.round(r * g / safe) * safe / g, 0.0)
        out.append(h)
        r = r - h
    for _ in range(planes - 2):
        q = bf16_rn(r)
        out.append(q)
        r = r - q
    return out


def emulated_k(Bfull, C, planes):
    """Bfull [naux, nao, nao]; returns K from the split arithmetic of both contractions."""
    Bp = row_planes(Bfull, planes, axis=2)
    Cp = row_planes(C, planes, axis=0)
    # the kernel keeps X as the exact order-0 sum plus an FP32 higher-order sum (~2^-32 of X)
    X = sum(np.einsum("pmn,ni->pmi", Bp[a], Cp[b]) for a in range(planes) for b in range(planes - a))
    Xm = X.transpose(1, 0, 2).reshape(X.shape[1], -1)       # rows m, contraction over (P, i)
    Xp = row_planes(Xm, planes, axis=1)
    return sum(Xp[a] @ Xp[b].T for a in range(planes) for b in range(planes - a))


def rel(a, b):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def full_B(sysm):
    return np.stack([oracle.unpack(sysm.B[P], sysm.nao) for P in range(sysm.naux)])


@pytest.mark.parametrize("planes", [5, 4, 3])
@pytest.mark.parametrize("case", ["c0", "nocc1", "ragged17"])
def test_mixed_jk_parity(case, planes, c0):
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
    lib = dfscf.lib()
    lib.df_tune_set(b"mixed_planes", planes)
    try:
        L = dfscf.metric_chol(mol.aux_xyz, mol.aux_exp)
        B = dfscf.build_B(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp, L, "mixed")
        J, K = dfscf.jk(B, D, C, precision="mixed")
        # the FP64 planes of a mixed B still give the exact FP64 result
        J64, K64 = dfscf.jk(B, D, C, precision="fp64")
    finally:
        lib.df_tune_set(b"mixed_planes", 5)
    Jo = oracle.df_j(sysm.B, mol.nao, D)
    Ko = oracle.df_k(sysm.B, mol.nao, C)
    Ke = emulated_k(full_B(sysm), C, planes)
    ej, ek, eke, eemu = rel(J, Jo), rel(K, Ko), rel(K, Ke), rel(Ke, Ko)
    print(f"{case} planes {planes}: J rel {ej:.2e}  K rel (exact) {ek:.2e}  K rel (split emulation) {eke:.2e}"
          f"  emulation vs exact {eemu:.2e}")
    # J streams the FP64 rows in both modes
    assert ej <= 1e-10
    assert rel(J64, Jo) <= 1e-10 and rel(K64, Ko) <= 1e-10
    # bounds measured on GB300 with a margin of about 5x
    assert eke <= {5: 1e-7, 4: 1e-6, 3: 1e-6}[planes]
    assert ek <= {5: 1e-7, 4: 1e-6, 3: 2e-6}[planes]


def test_mixed_scf_energy_within_1e6(c0, c0_scf):
    r = dfscf.scf_run(c0, precision="mixed")
    assert r.converged and r.fp64_iterations >= 2
    assert abs(r.energy - c0_scf.energy) <= 1e-6


@pytest.mark.parametrize("n", [13, 27])
def test_syrk_k_box_16_matches_default(n):
    """The exchange SYRK with 16-element K boxes (32-byte swizzle, a deeper ring; knob
    syrk_bk) issues the same plane products in the same order as the 32-element boxes: K must
    agree to FP32-partial rounding and stay within the mixed tolerance of the FP64 oracle."""
    m = gen.make_molecule(n, gen.molecules.box_for(n), 31)
    sysm = oscf.build_system(m)
    rng = np.random.default_rng(n)
    C = 0.3 * rng.standard_normal((m.nao, max(2, m.nocc)))
    L = dfscf.metric_chol(m.aux_xyz, m.aux_exp)
    B = dfscf.build_B(m.ao_xyz, m.ao_exp, m.aux_xyz, m.aux_exp, L, "mixed")
    old = dfscf.lib().df_tune_get(b"syrk_bk")
    old_pair = dfscf.lib().df_tune_get(b"syrk_pair")
    try:
        assert dfscf.lib().df_tune_set(b"syrk_pair", 0) == 0   # the K box applies to the one-CTA SYRK
        assert dfscf.lib().df_tune_set(b"syrk_bk", 32) == 0
        _, K32 = dfscf.jk(B, None, C, precision="mixed", want_j=False)
        assert dfscf.lib().df_tune_set(b"syrk_bk", 16) == 0
        _, K16 = dfscf.jk(B, None, C, precision="mixed", want_j=False)
    finally:
        dfscf.lib().df_tune_set(b"syrk_bk", old)
        dfscf.lib().df_tune_set(b"syrk_pair", old_pair)
    Ko = oracle.df_k(sysm.B, m.nao, C)
    assert rel(K16, K32.cpu().numpy()) <= 1e-6
    assert rel(K16, Ko) <= 2e-6 and rel(K32, Ko) <= 2e-6


@pytest.mark.parametrize("n", [13, 27, 52])
def test_syrk_cta_pair_matches_default(n):
    """The exchange SYRK on CTA pairs (knob syrk_pair: cta_group::2, 256 x 128 blocks whose
    B operand is split between the two CTAs) forms the same plane products into the same four
    accumulators.  13 centres: one 128-row block, so the peer CTA's rows are all padding; 27:
    two blocks; 52: three blocks, an odd count.  K must agree with the one-CTA SYRK to FP32-partial
    rounding and stay within the mixed tolerance of the FP64 oracle."""
    m = gen.make_molecule(n, gen.molecules.box_for(n), 32)
    sysm = oscf.build_system(m)
    rng = np.random.default_rng(n + 1)
    C = 0.3 * rng.standard_normal((m.nao, max(2, m.nocc)))
    L = dfscf.metric_chol(m.aux_xyz, m.aux_exp)
    B = dfscf.build_B(m.ao_xyz, m.ao_exp, m.aux_xyz, m.aux_exp, L, "mixed")
    old = dfscf.lib().df_tune_get(b"syrk_pair")
    try:
        assert dfscf.lib().df_tune_set(b"syrk_pair", 0) == 0
        _, K1 = dfscf.jk(B, None, C, precision="mixed", want_j=False)
        assert dfscf.lib().df_tune_set(b"syrk_pair", 1) == 0
        _, K2 = dfscf.jk(B, None, C, precision="mixed", want_j=False)
    finally:
        dfscf.lib().df_tune_set(b"syrk_pair", old)
    Ko = oracle.df_k(sysm.B, m.nao, C)
    assert torch.isfinite(K2).all()
    assert rel(K2, K1.cpu().numpy()) <= 1e-6
    assert rel(K2, Ko) <= 2e-6 and rel(K1, Ko) <= 2e-6
