"""Long-range density fitting (df_lrdf_build / df_lrdf_jk) against the oracle.

J and K of the paper's LRDF equation, (mn|kl) ~ (mn|kl)^SR + sum_P T_P,mn T_P,kl with the
long-range metric, on a 10-centre molecule (nao 50, two diffuse auxiliary functions per centre) for two
range-separation parameters, at the FP64 parity tolerance (1e-10 relative, max-norm); and
for a large omega the long-range scheme must reduce to ordinary DF (df_jk).
"""
import numpy as np
import pytest

import gen
import oracle
from oracle import lrdf

pytestmark = pytest.mark.gpu
dfscf = pytest.importorskip("paper_2506_06661_gb300")


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module")
def mol10():
    # the long-range operator cannot tell tight auxiliary functions apart (its metric is
    # numerically singular for the 15-function set): LRDF takes a small, diffuse auxiliary
    # set, here two functions per centre (naux = nao / 2.5)
    xyz = gen.molecules.make_geometry(10, gen.molecules.box_for(10), 3)
    m = gen.molecule_from_geometry(xyz, aux_exp=gen.molecules.even_tempered(0.1, 0.6, 2))
    rng = np.random.default_rng(4)
    C = 0.3 * rng.standard_normal((m.nao, 5))
    return m, C, 2 * C @ C.T


@pytest.mark.parametrize("omega", [0.35, 1.2])
def test_lrdf_jk_matches_oracle(mol10, omega):
    m, C, D = mol10
    T = dfscf.lrdf_build(m.ao_xyz, m.ao_exp, m.aux_xyz, m.aux_exp, omega)
    J, K = dfscf.lrdf_jk(T, m.ao_xyz, m.ao_exp, omega, D, C)
    Jo, Ko = lrdf.lrdf_jk(m.ao_xyz, m.ao_exp, m.aux_xyz, m.aux_exp, omega, D, C)
    assert _rel(J.cpu().numpy(), Jo) <= 1e-10
    assert _rel(K.cpu().numpy(), Ko) <= 1e-10


def test_lrdf_reduces_to_df_for_large_omega(mol10):
    m, C, D = mol10
    T = dfscf.lrdf_build(m.ao_xyz, m.ao_exp, m.aux_xyz, m.aux_exp, 1e6)
    J, K = dfscf.lrdf_jk(T, m.ao_xyz, m.ao_exp, 1e6, D, C)
    L = dfscf.metric_chol(m.aux_xyz, m.aux_exp)
    B = dfscf.build_B(m.ao_xyz, m.ao_exp, m.aux_xyz, m.aux_exp, L, "fp64")
    Jd, Kd = dfscf.jk(B, D, C)
    assert _rel(J.cpu().numpy(), Jd.cpu().numpy()) <= 1e-8
    assert _rel(K.cpu().numpy(), Kd.cpu().numpy()) <= 1e-8


def test_lrdf_rejects_bad_omega(mol10):
    m, C, D = mol10
    with pytest.raises(dfscf.DFError) as e:
        dfscf.lrdf_build(m.ao_xyz, m.ao_exp, m.aux_xyz, m.aux_exp, 0.0)
    assert e.value.code == dfscf.DF_ERR_ARG
