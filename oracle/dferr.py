"""Oracle for the density-fitting error diagnostics (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use this module; the
CUDA library shares no code with it.  Plain FP64 numpy, small sizes only.

Follows arXiv 2506.06661:
* Section "Density fitting", the Delta equation (Lehtola's diagonal error):
      Delta = sum_mn [(mn|mn) - sum_P T_{P,mn} T_{P,mn}];
* Section "Automatic Differentiation" (auxiliary-basis optimisation): the fitted integrals
  sum_PQ (P|mn) (M^-1)_PQ (Q|kl), the residual
      sigma_mn = (mn|mn) - sum_P C_{P,mn} (P|mn),  C = M^-1 (P|mn),
  and its Jacobian with respect to the auxiliary exponents alpha_P.  The paper differentiates
  with automatic differentiation; here the derivative is written out for s primitives:
      d sigma_mn / d alpha_P = -2 C_{P,mn} [d(P|mn)/d alpha_P - sum_Q m1_{PQ} C_{Q,mn}],
  where m1_{PQ} = d M_PQ / d alpha_P with alpha_Q held fixed (on the diagonal this is half the
  total derivative of M_PP, which is what the quadratic form needs).

The integrals are the closed forms of L2-normalised s primitives N_a = (2a/pi)^(3/4):
  (c|d)   = N_c N_d 2 pi^(5/2) / (c d sqrt(c + d)) F0(cd/(c+d) R^2),
  (c|ab)  = N_c N_a N_b 2 pi^(5/2) / (p c sqrt(p + c)) exp(-ab/p R_AB^2) F0(pc/(p+c) |P - C|^2),
with p = a + b and P = (aA + bB)/p; F0' = -F1, F1(t) = (F0(t) - exp(-t)) / (2t).
Their exponent derivatives follow by the product rule:
  d ln(N_c / (c sqrt(c + x))) / dc = 3/(4c) - 1/c - 1/(2(c + x)),
  d/dc [c x / (c + x)] = x^2 / (c + x)^2.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

from . import eri_diag, int2c, int3c

PI = np.pi


def boys_f0_f1(t):
    """F0(t) and F1(t) for t >= 0 (series below t = 1e-3, closed forms above)."""
    t = np.asarray(t, dtype=np.float64)
    small = t < 1e-3
    ts = np.where(small, 1.0, t)
    f0 = 0.5 * np.sqrt(PI / ts) * erf(np.sqrt(ts))
    f1 = (f0 - np.exp(-ts)) / (2.0 * ts)
    # Maclaurin series: F_m(t) = sum_k (-t)^k / (k! (2m + 2k + 1))
    s0 = np.zeros_like(t)
    s1 = np.zeros_like(t)
    term = np.ones_like(t)
    for k in range(10):
        s0 = s0 + term / (2 * k + 1)
        s1 = s1 + term / (2 * k + 3)
        term = term * (-t) / (k + 1)
    return np.where(small, s0, f0), np.where(small, s1, f1)


def _norm(a):
    return (2.0 * a / PI) ** 0.75


def metric_first_arg_derivative(aux_xyz, aux_exp):
    """m1[P][Q] = d (P|Q) / d alpha_P with alpha_Q fixed, for every P, Q (loops over pairs)."""
    aux_xyz = np.asarray(aux_xyz, dtype=np.float64)
    c_all = np.asarray(aux_exp, dtype=np.float64)
    n = c_all.size
    m1 = np.empty((n, n))
    for P in range(n):
        for Q in range(n):
            c, d = c_all[P], c_all[Q]
            R2 = float(np.sum((aux_xyz[P] - aux_xyz[Q]) ** 2))
            pref = _norm(c) * _norm(d) * 2.0 * PI ** 2.5 / (c * d * np.sqrt(c + d))
            T = c * d / (c + d) * R2
            f0, f1 = boys_f0_f1(T)
            val = pref * f0
            m1[P, Q] = val * (0.75 / c - 1.0 / c - 0.5 / (c + d)) + pref * (-f1) * d * d / (c + d) ** 2 * R2
    return m1


def int3c_aux_derivative(ao_xyz, ao_exp, aux_xyz, aux_exp):
    """d (P|mn) / d alpha_P as [naux][npair] (packed mn = m(m+1)/2 + n, m >= n)."""
    ao_xyz = np.asarray(ao_xyz, dtype=np.float64)
    a_all = np.asarray(ao_exp, dtype=np.float64)
    aux_xyz = np.asarray(aux_xyz, dtype=np.float64)
    c_all = np.asarray(aux_exp, dtype=np.float64)
    nao, naux = a_all.size, c_all.size
    out = np.empty((naux, nao * (nao + 1) // 2))
    for m in range(nao):
        for nu in range(m + 1):
            a, b = a_all[m], a_all[nu]
            p = a + b
            mu = a * b / p
            RAB2 = float(np.sum((ao_xyz[m] - ao_xyz[nu]) ** 2))
            Pc = (a * ao_xyz[m] + b * ao_xyz[nu]) / p
            ij = m * (m + 1) // 2 + nu
            for P in range(naux):
                c = c_all[P]
                RPC2 = float(np.sum((Pc - aux_xyz[P]) ** 2))
                pref = _norm(c) * _norm(a) * _norm(b) * 2.0 * PI ** 2.5 / (p * c * np.sqrt(p + c)) * np.exp(-mu * RAB2)
                T = p * c / (p + c) * RPC2
                f0, f1 = boys_f0_f1(T)
                val = pref * f0
                out[P, ij] = val * (0.75 / c - 1.0 / c - 0.5 / (p + c)) + pref * (-f1) * p * p / (p + c) ** 2 * RPC2
    return out


def residual(ao_xyz, ao_exp, aux_xyz, aux_exp):
    """sigma_mn = (mn|mn) - sum_PQ (P|mn) (M^-1)_PQ (Q|mn) for every packed pair."""
    v = int3c(ao_xyz, ao_exp, aux_xyz, aux_exp)
    M = int2c(aux_xyz, aux_exp)
    C = np.linalg.solve(M, v)
    return eri_diag(ao_xyz, ao_exp) - np.sum(C * v, axis=0)


def residual_jacobian(ao_xyz, ao_exp, aux_xyz, aux_exp):
    """(sigma [npair], jac [npair][naux]) with jac[mn][P] = d sigma_mn / d alpha_P."""
    v = int3c(ao_xyz, ao_exp, aux_xyz, aux_exp)
    M = int2c(aux_xyz, aux_exp)
    C = np.linalg.solve(M, v)
    sigma = eri_diag(ao_xyz, ao_exp) - np.sum(C * v, axis=0)
    dv = int3c_aux_derivative(ao_xyz, ao_exp, aux_xyz, aux_exp)
    m1 = metric_first_arg_derivative(aux_xyz, aux_exp)
    jac = -2.0 * C * (dv - m1 @ C)
    return sigma, jac.T.copy()


def delta_total(ao_xyz, ao_exp, aux_xyz, aux_exp):
    """Lehtola's Delta, summed over all ordered pairs (m, n): off-diagonal packed pairs twice."""
    sigma = residual(ao_xyz, ao_exp, aux_xyz, aux_exp)
    nao = len(ao_exp)
    w = np.array([1.0 if m == n else 2.0 for m in range(nao) for n in range(m + 1)])
    return float(np.sum(w * sigma))
