"""Pins of the oracle for Cartesian Gaussians of any angular momentum (oracle/angular.py).

Independent routes, none of which reuses the Hermite-expansion code under test:
* s functions: the closed forms of the s-only oracle (S, T, V, metric, three- and four-centre);
* F_n against adaptive quadrature of its defining integral;
* p and d functions as centre derivatives of s functions.  With g = exp(-a |r - A|^2),
  d g / dA_x = 2a (x - A_x) g and d^2 g / dA_x^2 = (4a^2 (x - A_x)^2 - 2a) g, so with the
  normalisations, an integral over p_x equals a^-1/2 d/dA_x of the s integral, d_xy equals
  a^-1 d^2/(dA_x dA_y), and d_xx equals (a sqrt 3)^-1 (d^2/dA_x^2 + 2a) of the s integral
  (central differences of the s-only closed forms);
* overlap and kinetic integrals by Gauss-Hermite quadrature about the product centre (the
  paper's Section "Numba JIT compilation": exact here, the integrands being polynomials
  times one Gaussian);
* rotation: p functions transform as a vector.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import roots_hermite

import gen
import oracle
from oracle import angular as ang

S0 = (0, 0, 0)
PX, PY, PZ = (1, 0, 0), (0, 1, 0), (0, 0, 1)
UNIT = [PX, PY, PZ]


def test_s_functions_match_the_closed_forms():
    mol = gen.make_molecule(3, 6.0, 1)
    orb, auxe = [0.3, 1.0], [0.2, 0.9]
    bas, aux = ang.basis(mol.xyz, orb, 0), ang.basis(mol.xyz, auxe, 0)
    ao_xyz, ao_exp = np.repeat(mol.xyz, 2, axis=0), np.tile(orb, 3)
    ax_xyz, ax_exp = np.repeat(mol.xyz, 2, axis=0), np.tile(auxe, 3)
    S, T, V = ang.int1e(bas, mol.xyz, mol.charges)
    So, To, Vo = oracle.int1e(ao_xyz, ao_exp, mol.xyz, mol.charges)
    for x, y in ((S, So), (T, To), (V, Vo), (ang.int2c(aux), oracle.int2c(ax_xyz, ax_exp)),
                 (ang.int4c(bas), oracle.int4c(ao_xyz, ao_exp))):
        assert np.abs(x - y).max() <= 1e-13 * np.abs(y).max()
    R = ang.int3c(bas, aux)
    Ro = oracle.int3c(ao_xyz, ao_exp, ax_xyz, ax_exp)
    Ru = np.array([oracle.unpack(Ro[P], len(bas)) for P in range(Ro.shape[0])])
    assert np.abs(R - Ru).max() <= 1e-13 * np.abs(Ru).max()


@pytest.mark.parametrize("n", range(7))
def test_boys_function_against_quadrature(n):
    for t in (0.0, 1e-6, 5e-4, 2e-3, 0.5, 3.0, 20.0, 60.0):
        ref = quad(lambda u: u ** (2 * n) * math.exp(-t * u * u), 0.0, 1.0, epsabs=0, epsrel=1e-13)[0]
        assert abs(ang.boys(n, t) - ref) <= 1e-12 * ref, (n, t)


# geometry and exponents of the derivative pins
A = np.array([0.1, -0.3, 0.2])
B = np.array([0.9, 0.4, -0.5])
C = np.array([-0.4, 0.8, 0.6])
D = np.array([0.5, -0.7, 1.1])
a, b, c, d = 0.7, 1.3, 0.45, 0.9
H = 1e-4


def _d1(f, X, k):
    e = np.zeros(3)
    e[k] = H
    return (f(X + e) - f(X - e)) / (2 * H)


def _d2(f, X, k, m):
    ek, em = np.zeros(3), np.zeros(3)
    ek[k], em[m] = H, H
    return (f(X + ek + em) - f(X + ek - em) - f(X - ek + em) + f(X - ek - em)) / (4 * H * H)


def _integrals():
    """Integrals with a p or d function on A (angular powers la), s elsewhere: name -> f(la, A)."""
    return {
        "overlap": lambda la, X: ang.overlap(X, a, la, B, b, S0),
        "kinetic": lambda la, X: ang.kinetic(X, a, la, B, b, S0),
        "nuclear": lambda la, X: ang.nuclear(X, a, la, B, b, S0, C, 1.0),
        "metric": lambda la, X: ang.coulomb(ang.single(X, a, la), ang.single(B, b, S0)),
        "3c orbital": lambda la, X: ang.coulomb(ang.single(C, c, S0), ang.pair(X, a, la, B, b, S0)),
        "4c": lambda la, X: ang.coulomb(ang.pair(X, a, la, B, b, S0), ang.pair(C, c, S0, D, d, S0)),
    }


@pytest.mark.parametrize("name", list(_integrals()))
def test_p_functions_are_centre_derivatives_of_s(name):
    f = _integrals()[name]
    for k, lv in enumerate(UNIT):
        fd = _d1(lambda X: f(S0, X), A, k) / math.sqrt(a)
        val = f(lv, A)
        assert abs(val - fd) <= 1e-8 * max(1.0, abs(val)), (name, k, val, fd)


def test_p_on_both_sides_and_on_the_auxiliary_function():
    # <p_x(A) | p_y(B)> = (ab)^-1/2 d^2 / (dA_x dB_y) <s | s>, and (p_z(C) | s s) for the metric side
    def s_s(XA, XB):
        return ang.overlap(XA, a, S0, XB, b, S0)
    e = np.zeros(3)
    e[1] = H
    fd = (_d1(lambda X: s_s(X, B + e), A, 0) - _d1(lambda X: s_s(X, B - e), A, 0)) / (2 * H) / math.sqrt(a * b)
    assert abs(ang.overlap(A, a, PX, B, b, PY) - fd) <= 1e-7
    f = lambda X, lc: ang.coulomb(ang.single(X, c, lc), ang.pair(A, a, S0, B, b, S0))  # noqa: E731
    fd = _d1(lambda X: f(X, S0), C, 2) / math.sqrt(c)
    assert abs(f(C, PZ) - fd) <= 1e-8


@pytest.mark.parametrize("name", ["overlap", "kinetic", "nuclear", "metric", "3c orbital"])
def test_d_functions_are_second_centre_derivatives_of_s(name):
    f = _integrals()[name]
    s0 = f(S0, A)
    dxx = (_d2(lambda X: f(S0, X), A, 0, 0) + 2 * a * s0) / (a * math.sqrt(3))
    dxy = _d2(lambda X: f(S0, X), A, 0, 1) / a
    assert abs(f((2, 0, 0), A) - dxx) <= 1e-6 * max(1.0, abs(dxx)), (name, f((2, 0, 0), A), dxx)
    assert abs(f((1, 1, 0), A) - dxy) <= 1e-6 * max(1.0, abs(dxy)), (name, f((1, 1, 0), A), dxy)


def _gh_1d(i, j, XA, XB, ea, eb, deriv_j=False):
    """One-dimensional overlap by Gauss-Hermite quadrature about the product centre; with
    deriv_j the right factor is replaced by -1/2 of its second derivative."""
    p = ea + eb
    theta = ea * eb / p
    Xp = (ea * XA + eb * XB) / p
    u, w = roots_hermite(12)
    x = u / math.sqrt(p) + Xp
    if deriv_j:
        xb = x - XB
        right = -0.5 * (j * (j - 1) * xb ** (j - 2) if j >= 2 else 0.0) + eb * (2 * j + 1) * xb ** j \
            - 2 * eb * eb * xb ** (j + 2)
    else:
        right = (x - XB) ** j
    return math.exp(-theta * (XA - XB) ** 2) * np.sum(w / math.sqrt(p) * (x - XA) ** i * right)


@pytest.mark.parametrize("la,lb", [((1, 0, 0), (0, 1, 0)), ((2, 0, 0), (1, 1, 0)), ((0, 1, 1), (0, 0, 2)),
                                   ((1, 1, 0), (1, 1, 0))])
def test_overlap_and_kinetic_against_gauss_hermite(la, lb):
    n = ang.norm(a, la) * ang.norm(b, lb)
    s1 = [_gh_1d(la[k], lb[k], A[k], B[k], a, b) for k in range(3)]
    t1 = [_gh_1d(la[k], lb[k], A[k], B[k], a, b, deriv_j=True) for k in range(3)]
    S = n * s1[0] * s1[1] * s1[2]
    T = n * (t1[0] * s1[1] * s1[2] + s1[0] * t1[1] * s1[2] + s1[0] * s1[1] * t1[2])
    assert abs(ang.overlap(A, a, la, B, b, lb) - S) <= 1e-13 * max(1.0, abs(S))
    assert abs(ang.kinetic(A, a, la, B, b, lb) - T) <= 1e-13 * max(1.0, abs(T))


def test_p_blocks_rotate_as_vectors():
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    Q *= np.sign(np.linalg.det(Q))
    S = np.array([[ang.overlap(A, a, li, B, b, lj) for lj in UNIT] for li in UNIT])
    Sr = np.array([[ang.overlap(Q @ A, a, li, Q @ B, b, lj) for lj in UNIT] for li in UNIT])
    assert np.abs(Sr - Q @ S @ Q.T).max() <= 1e-13
    M = np.array([[ang.coulomb(ang.single(A, a, li), ang.single(C, c, lj)) for lj in UNIT] for li in UNIT])
    Mr = np.array([[ang.coulomb(ang.single(Q @ A, a, li), ang.single(Q @ C, c, lj)) for lj in UNIT]
                   for li in UNIT])
    assert np.abs(Mr - Q @ M @ Q.T).max() <= 1e-13


def test_sp_metric_is_positive_definite_and_df_exact_with_a_complete_set():
    """With s and p orbital functions of exponent 0.8 on one centre, an auxiliary set holding
    every product Gaussian (exponent 1.6, s to d) makes density fitting exact: every fitted
    (mn|kl) equals the four-centre value."""
    cen = np.array([[0.0, 0.0, 0.0]])
    orb = [0.8]
    bas = ang.basis(cen, orb, 1)                      # s, px, py, pz on one centre
    aux = ang.basis(cen, [1.6], 2)                    # all products: s .. d at exponent 1.6
    M = ang.int2c(aux)
    assert np.linalg.eigvalsh(M)[0] > 0
    R = ang.int3c(bas, aux)
    E = ang.int4c(bas)
    L = np.linalg.cholesky(M)
    Bw = np.linalg.solve(L, R.reshape(len(aux), -1))
    fit = (Bw.T @ Bw).reshape(len(bas), len(bas), len(bas), len(bas))
    assert np.abs(fit - E).max() <= 1e-10 * np.abs(E).max()
