"""Pins for the oracle's DF-error diagnostics (CPU only).

* the exponent derivatives of the metric and the three-centre integrals equal central finite
  differences of the oracle's C integrals (an independent implementation of the values);
* the analytic Jacobian of the residual sigma_mn equals central finite differences of sigma;
* sigma_mn >= 0 (the Coulomb-metric fit never overestimates a diagonal integral) and sigma
  vanishes for an auxiliary set holding every product Gaussian;
* Delta through the solve form equals Delta through the Cholesky-whitened tensor B.
"""
import numpy as np
import pytest

import gen
import oracle
from oracle import dferr

from test_oracle_df import tiny_product_complete


def small_mol():
    xyz = np.array([[0.0, 0.0, 0.0], [1.5, 0.1, -0.2], [0.3, 1.7, 0.5]])
    return gen.molecule_from_geometry(xyz, orb_exp=[0.25, 1.1, 4.0], aux_exp=gen.molecules.even_tempered(0.2, 12.0, 5))


def test_boys_f1_is_minus_derivative_of_f0():
    t = np.array([0.0, 1e-5, 5e-4, 2e-3, 0.3, 2.0, 11.0, 35.0])
    h = 1e-6 * np.maximum(t, 1.0)
    f0p, _ = dferr.boys_f0_f1(t + h)
    f0m, _ = dferr.boys_f0_f1(np.maximum(t - h, 0.0))
    fd = (f0p - f0m) / (t + h - np.maximum(t - h, 0.0))
    _, f1 = dferr.boys_f0_f1(t)
    assert np.allclose(-fd, f1, rtol=1e-6, atol=1e-9)
    assert np.allclose(dferr.boys_f0_f1(t)[0], oracle.boys_f0(t), rtol=1e-13, atol=0)


def test_exponent_derivatives_match_finite_differences():
    mol = small_mol()
    m1 = dferr.metric_first_arg_derivative(mol.aux_xyz, mol.aux_exp)
    dv = dferr.int3c_aux_derivative(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp)
    for P in (0, 4, 7, 14):
        h = 1e-6 * mol.aux_exp[P]
        ep, em = mol.aux_exp.copy(), mol.aux_exp.copy()
        ep[P] += h
        em[P] -= h
        dM = (oracle.int2c(mol.aux_xyz, ep) - oracle.int2c(mol.aux_xyz, em)) / (2 * h)
        expect = m1[P].copy()
        expect[P] *= 2.0  # both functions of (P|P) carry alpha_P
        assert np.allclose(dM[P], expect, rtol=1e-6, atol=1e-9 * np.abs(expect).max())
        dR = (oracle.int3c(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, ep) -
              oracle.int3c(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, em)) / (2 * h)
        assert np.allclose(dR[P], dv[P], rtol=1e-6, atol=1e-9 * np.abs(dv[P]).max())


def test_residual_jacobian_matches_finite_differences():
    mol = small_mol()
    sigma, jac = dferr.residual_jacobian(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp)
    assert np.allclose(sigma, dferr.residual(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp), rtol=0, atol=1e-12)
    scale = np.abs(jac).max()
    for P in range(mol.naux):
        h = 1e-5 * mol.aux_exp[P]
        ep, em = mol.aux_exp.copy(), mol.aux_exp.copy()
        ep[P] += h
        em[P] -= h
        fd = (dferr.residual(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, ep) -
              dferr.residual(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, em)) / (2 * h)
        assert np.abs(fd - jac[:, P]).max() <= 1e-6 * scale, P


def test_residual_is_nonnegative_and_vanishes_when_exact(c0):
    s = dferr.residual(c0.ao_xyz, c0.ao_exp, c0.aux_xyz, c0.aux_exp)
    d = oracle.eri_diag(c0.ao_xyz, c0.ao_exp)
    assert np.min(s) >= -1e-9 * np.max(d)
    mol = tiny_product_complete()
    s0 = dferr.residual(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp)
    assert np.max(np.abs(s0)) <= 1e-8 * np.max(oracle.eri_diag(mol.ao_xyz, mol.ao_exp))


def test_delta_solve_form_equals_whitened_form(c0, c0_system):
    total = dferr.delta_total(c0.ao_xyz, c0.ao_exp, c0.aux_xyz, c0.aux_exp)
    nao = c0.nao
    w = np.array([1.0 if m == n else 2.0 for m in range(nao) for n in range(m + 1)])
    via_B = float(np.sum(w * (oracle.eri_diag(c0.ao_xyz, c0.ao_exp) - np.sum(c0_system.B ** 2, axis=0))))
    assert abs(total - via_B) <= 1e-8 * abs(total) + 1e-12
    assert total > 0
