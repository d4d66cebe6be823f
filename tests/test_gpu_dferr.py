"""DF-error diagnostics on the GPU (df_fit_residual) against the oracle.

sigma_mn = (mn|mn) - sum_PQ (P|mn)(M^-1)_PQ (Q|mn) (the residual of the paper's
auxiliary-basis optimisation, whose ordered-pair sum is Lehtola's Delta), and its Jacobian
contracted with d alpha / d theta for the two parameters (ln alpha_min, ln beta) of the
even-tempered auxiliary set on every centre.  A Gauss-Newton step on those two parameters,
taken with the GPU's residual and Jacobian, must match the oracle's step and lower sum sigma^2.
"""
import numpy as np
import pytest
import torch

import gen
import oracle
from oracle import dferr

pytestmark = pytest.mark.gpu
dfscf = pytest.importorskip("paper_2506_06661_gb300")


def etg_molecule(xyz, amin, beta, nk=6):
    ex = amin * beta ** np.arange(nk)
    mol = gen.molecule_from_geometry(np.asarray(xyz, dtype=float), orb_exp=[0.25, 1.1, 4.0], aux_exp=ex)
    k = np.tile(np.arange(nk), len(xyz)).astype(float)
    dalpha = np.stack([mol.aux_exp, k * mol.aux_exp], axis=1)  # d alpha / d (ln amin, ln beta)
    return mol, dalpha


XYZ3 = [[0.0, 0.0, 0.0], [1.5, 0.1, -0.2], [0.3, 1.7, 0.5]]


def test_residual_and_jacobian_match_oracle():
    mol, dalpha = etg_molecule(XYZ3, 0.3, 2.2)
    sig, jac, delta = dfscf.fit_residual(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp, dalpha)
    s_ora, j_ora = dferr.residual_jacobian(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp)
    jt = j_ora @ dalpha
    d = oracle.eri_diag(mol.ao_xyz, mol.ao_exp)
    assert np.abs(sig.cpu().numpy() - s_ora).max() <= 1e-10 * d.max()
    assert np.abs(jac.cpu().numpy() - jt).max() <= 1e-9 * np.abs(jt).max()
    assert abs(delta - dferr.delta_total(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp)) <= 1e-10 * d.max()


def test_residual_on_20_centres(c0):
    sig, jac, delta = dfscf.fit_residual(c0.ao_xyz, c0.ao_exp, c0.aux_xyz, c0.aux_exp)
    assert jac is None
    s_ora = dferr.residual(c0.ao_xyz, c0.ao_exp, c0.aux_xyz, c0.aux_exp)
    d = oracle.eri_diag(c0.ao_xyz, c0.ao_exp)
    # the 20-centre metric has cond 4e10: both sides subtract sum_P T^2 from (mn|mn)
    assert np.abs(sig.cpu().numpy() - s_ora).max() <= 1e-7 * d.max()
    assert sig.min().item() >= -1e-7 * d.max()
    assert delta > 0


def test_gauss_newton_step_on_even_tempered_parameters():
    theta = np.log([0.3, 2.2])

    def fit(th):
        mol, dalpha = etg_molecule(XYZ3, *np.exp(th))
        s, j, _ = dfscf.fit_residual(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp, dalpha)
        return s.cpu().numpy(), j.cpu().numpy(), mol, dalpha

    s0, J0, mol, dalpha = fit(theta)
    step = np.linalg.lstsq(J0, -s0, rcond=None)[0]
    so, jo = dferr.residual_jacobian(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp)
    step_ora = np.linalg.lstsq(jo @ dalpha, -so, rcond=None)[0]
    assert np.allclose(step, step_ora, rtol=1e-6, atol=1e-9)
    # the Gauss-Newton direction is a descent direction of sum sigma^2 (its directional
    # derivative 2 sigma^T J step is negative); backtrack until the sum drops
    f0 = float(s0 @ s0)
    assert float(s0 @ (J0 @ step)) < 0.0
    scale, f1 = 1.0, np.inf
    for _ in range(30):
        s1, _, _, _ = fit(theta + scale * step)
        f1 = float(s1 @ s1)
        if f1 < f0:
            break
        scale *= 0.5
    assert f1 < f0
