"""Pins for the oracle's Boys function and s-type integrals (CPU only).

Every check compares against something other than the oracle's own formula: a numerical
quadrature of the defining integral, a closed form of a special case, or a relation
between two independently coded integral classes (the Gaussian product theorem of the
paper's overlap example: theta = ab/(a+b), X_p = (a X_a + b X_b)/(a+b)).
"""
import numpy as np
import pytest
from scipy import integrate, special

import oracle

PI = np.pi


def unit_charge(a):
    """Factor converting an L2-normalised s Gaussian into a unit-charge one."""
    return (a / PI) ** 1.5 / (2 * a / PI) ** 0.75


def test_boys_f0_definition_quadrature():
    ts = [0.0, 1e-12, 1e-6, 5e-4, 9.99e-4, 1e-3, 1.001e-3, 0.01, 0.3, 1.0, 2.5, 7.0, 20.0, 45.0, 120.0]
    got = oracle.boys_f0(ts)
    for t, g in zip(ts, got):
        ref, _ = integrate.quad(lambda u: np.exp(-t * u * u), 0.0, 1.0, epsabs=0, epsrel=2e-14, limit=200)
        assert abs(g - ref) <= 1e-14 * max(1.0, ref), (t, g, ref)


def test_boys_f0_limits():
    assert oracle.boys_f0(0.0)[0] == 1.0
    for t in (60.0, 200.0, 1e4):
        assert oracle.boys_f0(t)[0] == pytest.approx(0.5 * np.sqrt(PI / t), rel=1e-15)


def test_overlap_self_normalised_and_kinetic_closed_form():
    ex = np.array([0.1, 0.7, 3.0, 10.0])
    xyz = np.zeros((4, 3))
    S, T, _ = oracle.int1e(xyz, ex, np.zeros((1, 3)), np.zeros(1))
    assert np.allclose(np.diag(S), 1.0, rtol=0, atol=1e-15)
    # kinetic energy of a normalised s Gaussian: 3a/2
    assert np.allclose(np.diag(T), 1.5 * ex, rtol=1e-14)


def _hermite_3d(a, A, b, B, poly):
    """Gauss-Hermite product quadrature of poly(x,y,z) phi_a phi_b (exact for polynomials
    of moderate degree), following the paper's overlap quadrature: nodes u_n/sqrt(a+b)+X_p,
    weights w_n/sqrt(a+b), times exp(-theta (X_a-X_b)^2) per axis."""
    u, w = np.polynomial.hermite.hermgauss(20)
    p = a + b
    theta = a * b / p
    P = (a * A + b * B) / p
    pref = (2 * a / PI) ** 0.75 * (2 * b / PI) ** 0.75
    nodes = [u / np.sqrt(p) + P[k] for k in range(3)]
    wts = [w / np.sqrt(p) * np.exp(-theta * (A[k] - B[k]) ** 2) for k in range(3)]
    X, Y, Z = np.meshgrid(*nodes, indexing="ij")
    W = wts[0][:, None, None] * wts[1][None, :, None] * wts[2][None, None, :]
    return pref * np.sum(W * poly(X, Y, Z))


def test_overlap_and_kinetic_vs_gauss_hermite():
    rng = np.random.default_rng(5)
    xyz = rng.uniform(-1.5, 1.5, size=(6, 3))
    ex = np.array([0.1, 0.3162, 1.0, 3.162, 10.0, 0.55])
    S, T, _ = oracle.int1e(xyz, ex, np.zeros((1, 3)), np.zeros(1))
    for i in range(6):
        for j in range(6):
            a, b, A, B = ex[i], ex[j], xyz[i], xyz[j]
            s_ref = _hermite_3d(a, A, b, B, lambda x, y, z: 1.0)
            # T = 1/2 int grad(phi_a) . grad(phi_b), grad phi = -2a (r - A) phi
            t_ref = _hermite_3d(a, A, b, B, lambda x, y, z: 2 * a * b * (
                (x - A[0]) * (x - B[0]) + (y - A[1]) * (y - B[1]) + (z - A[2]) * (z - B[2])))
            assert S[i, j] == pytest.approx(s_ref, rel=1e-12, abs=1e-15)
            assert T[i, j] == pytest.approx(t_ref, rel=1e-11, abs=1e-14)


def test_nuclear_attraction_own_centre():
    ex = np.array([0.1, 1.0, 10.0])
    xyz = np.zeros((3, 3))
    _, _, V = oracle.int1e(xyz, ex, np.zeros((1, 3)), np.array([1.7]))
    assert np.allclose(np.diag(V), -2 * 1.7 * np.sqrt(2 * ex / PI), rtol=1e-14)


def test_nuclear_attraction_equals_point_charge_limit_of_3c():
    """V_ab(C) = -Z (unit point charge at C | ab); a steep unit-charge Gaussian tends to the point."""
    rng = np.random.default_rng(1)
    xyz = rng.uniform(-1, 1, size=(4, 3))
    ex = np.array([0.2, 0.9, 2.0, 6.0])
    C = np.array([[0.3, -0.2, 0.5]])
    _, _, V = oracle.int1e(xyz, ex, C, np.array([1.0]))
    c = 1e10
    R3 = oracle.int3c(xyz, ex, C, np.array([c]))[0] * unit_charge(c)
    Vp = oracle.unpack(R3, 4)
    assert np.allclose(V, -Vp, rtol=1e-8, atol=1e-12)


def test_metric_closed_form_unit_charges():
    rng = np.random.default_rng(2)
    xyz = rng.uniform(-2, 2, size=(5, 3))
    ex = np.array([0.05, 0.3, 1.0, 7.0, 50.0])
    M = oracle.int2c(xyz, ex)
    for i in range(5):
        for j in range(5):
            c, d = ex[i], ex[j]
            R = np.linalg.norm(xyz[i] - xyz[j])
            rho = c * d / (c + d)
            unit = special.erf(np.sqrt(rho) * R) / R if R > 0 else 2 * np.sqrt(rho / PI)
            assert M[i, j] * unit_charge(c) * unit_charge(d) == pytest.approx(unit, rel=1e-13)


def test_eri_self_closed_form():
    for a in (0.1, 1.0, 10.0):
        eri = oracle.int4c(np.zeros((1, 3)), np.array([a]))
        assert eri[0, 0, 0, 0] == pytest.approx(2 * np.sqrt(a / PI), rel=1e-14)


def test_3c_equals_2c_of_product_gaussian():
    """(c|ab) = S_ab * (c | unit-charge Gaussian of exponent a+b at the product centre)."""
    rng = np.random.default_rng(3)
    xyz = rng.uniform(-1.5, 1.5, size=(4, 3))
    ex = np.array([0.1, 0.8, 3.0, 10.0])
    aux_xyz = rng.uniform(-1.5, 1.5, size=(3, 3))
    aux_ex = np.array([0.05, 1.3, 40.0])
    R = oracle.int3c(xyz, ex, aux_xyz, aux_ex)
    S, _, _ = oracle.int1e(xyz, ex, np.zeros((1, 3)), np.zeros(1))
    for q in range(3):
        for i in range(4):
            for j in range(i + 1):
                p = ex[i] + ex[j]
                P = (ex[i] * xyz[i] + ex[j] * xyz[j]) / p
                M2 = oracle.int2c(np.array([aux_xyz[q], P]), np.array([aux_ex[q], p]))
                ref = S[i, j] * M2[0, 1] * unit_charge(p)
                assert R[q, i * (i + 1) // 2 + j] == pytest.approx(ref, rel=1e-13)


def test_4c_equals_coulomb_of_product_charges():
    rng = np.random.default_rng(4)
    xyz = rng.uniform(-1, 1, size=(3, 3))
    ex = np.array([0.3, 1.0, 4.0])
    eri = oracle.int4c(xyz, ex)
    S, _, _ = oracle.int1e(xyz, ex, np.zeros((1, 3)), np.zeros(1))
    for a in range(3):
        for b in range(3):
            for c in range(3):
                for d in range(3):
                    p, q = ex[a] + ex[b], ex[c] + ex[d]
                    P = (ex[a] * xyz[a] + ex[b] * xyz[b]) / p
                    Q = (ex[c] * xyz[c] + ex[d] * xyz[d]) / q
                    R = np.linalg.norm(P - Q)
                    rho = p * q / (p + q)
                    coul = special.erf(np.sqrt(rho) * R) / R if R > 1e-12 else 2 * np.sqrt(rho / PI)
                    assert eri[a, b, c, d] == pytest.approx(S[a, b] * S[c, d] * coul, rel=1e-12)


def test_nuclear_repulsion():
    xyz = np.array([[0, 0, 0], [0, 0, 2.0], [0, 3.0, 0]])
    z = np.array([1.0, 2.0, 1.0])
    ref = 1 * 2 / 2.0 + 1 * 1 / 3.0 + 2 * 1 / np.sqrt(13.0)
    assert oracle.nuclear_repulsion(xyz, z) == pytest.approx(ref, rel=1e-15)
