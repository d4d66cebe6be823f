"""Oracle for integrals over Cartesian Gaussians of any angular momentum (test
infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use this module; the CUDA
library shares no code with it.  Plain FP64 Python over small bases.

The functions are the paper's Cartesian Gaussian-type orbitals (arXiv 2506.06661, Section
"Numba JIT compilation", the |S| example), normalised:
    chi(r) = N (x - A_x)^lx (y - A_y)^ly (z - A_z)^lz exp(-a |r - A|^2),
    N = (2a/pi)^(3/4) (4a)^(L/2) / sqrt((2lx-1)!! (2ly-1)!! (2lz-1)!!),  L = lx + ly + lz.
The product of two of them separates into Cartesian factors with the Gaussian product theorem
(same passage).  The integrals follow the McMurchie-Davidson scheme (McMurchie and Davidson,
J. Comput. Phys. 26, 218 (1978)): each one-dimensional product is expanded in Hermite
Gaussians about P with coefficients E_t^{ij}, and the Coulomb integrals of Hermite Gaussians
R_{tuv} come from the Boys functions F_n.  These are the integrals the density fitting of the
paper's Section "Density fitting" needs beyond s functions: overlap, kinetic energy, nuclear
attraction, the metric (P|Q), the three-centre (P|mn) and, for tests, four-centre (mn|kl).
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np
from scipy.special import gammainc

PI = math.pi


def double_factorial(n: int) -> int:
    """n!! with (-1)!! = 0!! = 1."""
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


def norm(a: float, l) -> float:
    """Normalisation of the Cartesian primitive with exponent a and powers l = (lx, ly, lz)."""
    L = sum(l)
    den = 1
    for k in l:
        den *= double_factorial(2 * k - 1)
    return (2 * a / PI) ** 0.75 * (4 * a) ** (L / 2) / math.sqrt(den)


def boys(n: int, t: float) -> float:
    """F_n(t) = int_0^1 u^(2n) exp(-t u^2) du: the regularised lower incomplete gamma function
    (a library routine) for t >= 1e-3, F_n(t) = Gamma(n + 1/2) P(n + 1/2, t) / (2 t^(n + 1/2)),
    and the Maclaurin series sum_k (-t)^k / (k! (2n + 2k + 1)) below."""
    if t < 1e-3:
        s, term = 0.0, 1.0
        for k in range(12):
            s += term / (2 * n + 2 * k + 1)
            term *= -t / (k + 1)
        return s
    return math.gamma(n + 0.5) * gammainc(n + 0.5, t) / (2.0 * t ** (n + 0.5))


@lru_cache(maxsize=None)
def hermite_e(i: int, j: int, t: int, xab: float, a: float, b: float) -> float:
    """E_t^{ij}: coefficient of the Hermite Gaussian of order t about P in the product of the
    one-dimensional factors (x - A)^i e^{-a (x-A)^2} (x - B)^j e^{-b (x-B)^2}, xab = A - B."""
    p = a + b
    if t < 0 or t > i + j:
        return 0.0
    if i == 0 and j == 0:
        return math.exp(-(a * b / p) * xab * xab)
    if j == 0:
        xpa = -b / p * xab
        return (hermite_e(i - 1, j, t - 1, xab, a, b) / (2 * p) + xpa * hermite_e(i - 1, j, t, xab, a, b)
                + (t + 1) * hermite_e(i - 1, j, t + 1, xab, a, b))
    xpb = a / p * xab
    return (hermite_e(i, j - 1, t - 1, xab, a, b) / (2 * p) + xpb * hermite_e(i, j - 1, t, xab, a, b)
            + (t + 1) * hermite_e(i, j - 1, t + 1, xab, a, b))


@lru_cache(maxsize=None)
def hermite_r(t: int, u: int, v: int, n: int, p: float, x: float, y: float, z: float) -> float:
    """R^n_{tuv}: derivative of order (t, u, v) with respect to P of (-2p)^n F_n(p |P - C|^2),
    with (x, y, z) = P - C."""
    if t < 0 or u < 0 or v < 0:
        return 0.0
    if t == 0 and u == 0 and v == 0:
        return (-2 * p) ** n * boys(n, p * (x * x + y * y + z * z))
    if t > 0:
        return (t - 1) * hermite_r(t - 2, u, v, n + 1, p, x, y, z) + x * hermite_r(t - 1, u, v, n + 1, p, x, y, z)
    if u > 0:
        return (u - 1) * hermite_r(t, u - 2, v, n + 1, p, x, y, z) + y * hermite_r(t, u - 1, v, n + 1, p, x, y, z)
    return (v - 1) * hermite_r(t, u, v - 2, n + 1, p, x, y, z) + z * hermite_r(t, u, v - 1, n + 1, p, x, y, z)


def _f(v):
    return tuple(float(c) for c in v)


def _overlap_1d(i, j, xab, a, b):
    return hermite_e(i, j, 0, xab, a, b) * math.sqrt(PI / (a + b))


def overlap(A, a, la, B, b, lb) -> float:
    """<chi_A | chi_B> of two normalised Cartesian primitives."""
    A, B = _f(A), _f(B)
    s = 1.0
    for k in range(3):
        s *= _overlap_1d(la[k], lb[k], A[k] - B[k], a, b)
    return norm(a, la) * norm(b, lb) * s


def kinetic(A, a, la, B, b, lb) -> float:
    """<chi_A | -1/2 nabla^2 | chi_B>: the second derivative of the right factor in each
    direction, -1/2 d^2/dx^2 [x^j e^{-b x^2}] = -1/2 j(j-1) x^{j-2} + b(2j+1) x^j - 2b^2 x^{j+2}
    (x measured from B), times the overlaps of the other two directions."""
    A, B = _f(A), _f(B)
    s1 = [_overlap_1d(la[k], lb[k], A[k] - B[k], a, b) for k in range(3)]
    t1 = []
    for k in range(3):
        i, j, x = la[k], lb[k], A[k] - B[k]
        v = b * (2 * j + 1) * _overlap_1d(i, j, x, a, b) - 2 * b * b * _overlap_1d(i, j + 2, x, a, b)
        if j >= 2:
            v -= 0.5 * j * (j - 1) * _overlap_1d(i, j - 2, x, a, b)
        t1.append(v)
    t = t1[0] * s1[1] * s1[2] + s1[0] * t1[1] * s1[2] + s1[0] * s1[1] * t1[2]
    return norm(a, la) * norm(b, lb) * t


def nuclear(A, a, la, B, b, lb, C, Zc) -> float:
    """<chi_A | -Z / |r - C| | chi_B>."""
    A, B, C = _f(A), _f(B), _f(C)
    p = a + b
    P = [(a * A[k] + b * B[k]) / p for k in range(3)]
    pc = [P[k] - C[k] for k in range(3)]
    v = 0.0
    for t in range(la[0] + lb[0] + 1):
        et = hermite_e(la[0], lb[0], t, A[0] - B[0], a, b)
        for u in range(la[1] + lb[1] + 1):
            eu = hermite_e(la[1], lb[1], u, A[1] - B[1], a, b)
            for w in range(la[2] + lb[2] + 1):
                ew = hermite_e(la[2], lb[2], w, A[2] - B[2], a, b)
                v += et * eu * ew * hermite_r(t, u, w, 0, p, pc[0], pc[1], pc[2])
    return -Zc * 2 * PI / p * norm(a, la) * norm(b, lb) * v


def _pair(A, a, la, B, b, lb, scale):
    """(p, P, E) of a charge distribution chi_A chi_B: E[t][u][v] = E^x_t E^y_u E^z_v times
    `scale` (the product of the functions' normalisations)."""
    p = a + b
    P = tuple((a * A[k] + b * B[k]) / p for k in range(3))
    ex = [hermite_e(la[0], lb[0], t, A[0] - B[0], a, b) for t in range(la[0] + lb[0] + 1)]
    ey = [hermite_e(la[1], lb[1], t, A[1] - B[1], a, b) for t in range(la[1] + lb[1] + 1)]
    ez = [hermite_e(la[2], lb[2], t, A[2] - B[2], a, b) for t in range(la[2] + lb[2] + 1)]
    E = np.einsum("i,j,k->ijk", ex, ey, ez) * scale
    return p, P, E


def coulomb(d1, d2) -> float:
    """(d1 | 1/r12 | d2) of two charge distributions given as (p, P, E) from _pair."""
    p, P, E1 = d1
    q, Q, E2 = d2
    alpha = p * q / (p + q)
    pq = [P[k] - Q[k] for k in range(3)]
    s = 0.0
    for t, u, v in np.ndindex(*E1.shape):
        if E1[t, u, v] == 0.0:
            continue
        for t2, u2, v2 in np.ndindex(*E2.shape):
            e2 = E2[t2, u2, v2]
            if e2 == 0.0:
                continue
            sign = -1.0 if (t2 + u2 + v2) % 2 else 1.0
            s += E1[t, u, v] * sign * e2 * hermite_r(t + t2, u + u2, v + v2, 0, alpha, pq[0], pq[1], pq[2])
    return 2 * PI ** 2.5 / (p * q * math.sqrt(p + q)) * s


def single(A, a, la):
    """A lone normalised function as a charge distribution (its partner is the constant 1:
    exponent 0, no normalisation)."""
    return _pair(_f(A), a, la, _f(A), 0.0, (0, 0, 0), norm(a, la))


def pair(A, a, la, B, b, lb):
    return _pair(_f(A), a, la, _f(B), b, lb, norm(a, la) * norm(b, lb))


# ---- basis sets and integral matrices ----------------------------------------------------------
def cartesian_powers(l: int):
    """The (lx, ly, lz) with lx + ly + lz = l, lx descending, then ly descending."""
    return [(lx, ly, l - lx - ly) for lx in range(l, -1, -1) for ly in range(l - lx, -1, -1)]


def basis(centres, exponents, lmax: int):
    """Cartesian primitives on every centre: for each exponent, all components of angular
    momentum 0..lmax (centre-major, then exponent, then l, then component)."""
    out = []
    for A in np.asarray(centres, dtype=float):
        for a in exponents:
            for l in range(lmax + 1):
                for lv in cartesian_powers(l):
                    out.append((tuple(A), float(a), lv))
    return out


def int1e(bas, nuc_xyz, nuc_z):
    """(S, T, V) over a basis from basis()."""
    n = len(bas)
    S, T, V = np.zeros((n, n)), np.zeros((n, n)), np.zeros((n, n))
    for i, (A, a, la) in enumerate(bas):
        for j, (B, b, lb) in enumerate(bas[: i + 1]):
            S[i, j] = S[j, i] = overlap(A, a, la, B, b, lb)
            T[i, j] = T[j, i] = kinetic(A, a, la, B, b, lb)
            V[i, j] = V[j, i] = sum(nuclear(A, a, la, B, b, lb, C, z) for C, z in zip(nuc_xyz, nuc_z))
    return S, T, V


def int2c(aux):
    """The metric (P|Q) over an auxiliary basis from basis()."""
    n = len(aux)
    d = [single(*f) for f in aux]
    M = np.zeros((n, n))
    for i in range(n):
        for j in range(i + 1):
            M[i, j] = M[j, i] = coulomb(d[i], d[j])
    return M


def int3c(bas, aux):
    """(P|mn) as [naux][nao][nao]."""
    nb, na = len(bas), len(aux)
    d = [single(*f) for f in aux]
    out = np.zeros((na, nb, nb))
    for m in range(nb):
        for k in range(m + 1):
            pm = pair(*bas[m], *bas[k])
            for P in range(na):
                out[P, m, k] = out[P, k, m] = coulomb(d[P], pm)
    return out


def int4c(bas):
    """(mn|kl) as [nao]^4 (small bases only)."""
    n = len(bas)
    prs = {}
    for m in range(n):
        for k in range(m + 1):
            prs[(m, k)] = pair(*bas[m], *bas[k])
    out = np.zeros((n, n, n, n))
    keys = list(prs)
    for x, (m, k) in enumerate(keys):
        for (l, s) in keys[: x + 1]:
            v = coulomb(prs[(m, k)], prs[(l, s)])
            for a, b in ((m, k), (k, m)):
                for c, e in ((l, s), (s, l)):
                    out[a, b, c, e] = out[c, e, a, b] = v
    return out
