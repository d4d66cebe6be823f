"""Pins for the oracle's long-range density fitting (CPU only).

* full-range limits: with no range separation the oracle's LR 2c/3c/4c integrals equal the
  oracle's C integrals (an independent implementation), and for w -> infinity LRDF J/K equal
  ordinary DF J/K;
* the erf(w r)/r closed form equals a quadrature of its defining representation
  erf(w r)/r = (2/sqrt(pi)) int_0^w exp(-t^2 r^2) dt over the Gaussian-kernel overlap
  (pi/(c+d))^(3/2) (pi/(rho+t^2))^(3/2) exp(-rho t^2 R^2/(rho+t^2));
* w -> 0: the short-range 4c tensor becomes the full one and the long-range one vanishes;
* with an auxiliary set holding every product Gaussian LRDF is exact at any w: J and K equal
  brute-force four-centre J and K.
"""
import numpy as np
import pytest
from scipy.integrate import quad

import gen
import oracle
from oracle import lrdf

from test_oracle_df import dens, tiny_product_complete


def mol6():
    xyz = np.array([[0.0, 0.0, 0.0], [1.5, 0.1, -0.2], [0.3, 1.7, 0.5], [2.2, 1.9, 0.4], [-1.1, 0.8, 1.3],
                    [0.9, -1.4, 1.0]])
    return gen.molecule_from_geometry(xyz, orb_exp=[0.3, 1.5], aux_exp=gen.molecules.even_tempered(0.2, 8.0, 4))


def test_full_range_limits_match_c_integrals():
    m = mol6()
    assert np.allclose(lrdf.int2c_lr(m.aux_xyz, m.aux_exp, None), oracle.int2c(m.aux_xyz, m.aux_exp), rtol=1e-13,
                       atol=0)
    assert np.allclose(lrdf.int3c_lr(m.ao_xyz, m.ao_exp, m.aux_xyz, m.aux_exp, None),
                       oracle.int3c(m.ao_xyz, m.ao_exp, m.aux_xyz, m.aux_exp), rtol=1e-12, atol=1e-15)
    assert np.allclose(lrdf.int4c_range(m.ao_xyz, m.ao_exp, None, "full"), oracle.int4c(m.ao_xyz, m.ao_exp),
                       rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("omega", [0.05, 0.4, 2.0])
def test_lr_metric_equals_quadrature(omega):
    m = mol6()
    M = lrdf.int2c_lr(m.aux_xyz, m.aux_exp, omega)
    for P, Q in ((0, 0), (1, 6), (3, 20), (9, 17)):
        c, d = m.aux_exp[P], m.aux_exp[Q]
        R2 = float(np.sum((m.aux_xyz[P] - m.aux_xyz[Q]) ** 2))
        rho = c * d / (c + d)
        NcNd = (2 * c / np.pi) ** 0.75 * (2 * d / np.pi) ** 0.75

        def g(t):
            return (np.pi / (c + d)) ** 1.5 * (np.pi / (rho + t * t)) ** 1.5 * np.exp(-rho * t * t * R2 / (rho + t * t))
        val = NcNd * 2 / np.sqrt(np.pi) * quad(g, 0.0, omega, epsabs=0, epsrel=1e-13, limit=200)[0]
        assert abs(M[P, Q] - val) <= 1e-11 * abs(val), (P, Q, M[P, Q], val)


def test_short_range_limits():
    m = mol6()
    full = oracle.int4c(m.ao_xyz, m.ao_exp)
    sr0 = lrdf.int4c_range(m.ao_xyz, m.ao_exp, 1e-7, "sr")
    assert np.abs(sr0 - full).max() <= 1e-6 * np.abs(full).max()
    lr0 = lrdf.int4c_range(m.ao_xyz, m.ao_exp, 1e-7, "lr")
    assert np.abs(lr0).max() <= 1e-6 * np.abs(full).max()
    srinf = lrdf.int4c_range(m.ao_xyz, m.ao_exp, 1e6, "sr")
    assert np.abs(srinf).max() <= 1e-6 * np.abs(full).max()


def test_lrdf_reduces_to_df_at_large_omega():
    m = mol6()
    C, D = dens(m.nao, 3, 5)
    J, K = lrdf.lrdf_jk(m.ao_xyz, m.ao_exp, m.aux_xyz, m.aux_exp, 1e7, D, C)
    B = oracle.whiten(oracle.cholesky(oracle.int2c(m.aux_xyz, m.aux_exp)),
                      oracle.int3c(m.ao_xyz, m.ao_exp, m.aux_xyz, m.aux_exp))
    Jd, Kd = oracle.df_j(B, m.nao, D), oracle.df_k(B, m.nao, C)
    assert np.abs(J - Jd).max() <= 1e-7 * np.abs(Jd).max()
    assert np.abs(K - Kd).max() <= 1e-7 * np.abs(Kd).max()


@pytest.mark.parametrize("omega", [0.3, 1.0])
def test_lrdf_exact_for_product_complete_aux(omega):
    m = tiny_product_complete()
    C, D = dens(m.nao, 2, 9)
    J, K = lrdf.lrdf_jk(m.ao_xyz, m.ao_exp, m.aux_xyz, m.aux_exp, omega, D, C)
    J4, K4 = oracle.jk_4c(oracle.int4c(m.ao_xyz, m.ao_exp), D, C @ C.T)
    assert np.abs(J - J4).max() <= 1e-8 * np.abs(J4).max()
    assert np.abs(K - K4).max() <= 1e-8 * np.abs(K4).max()
