"""Oracle for long-range density fitting (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use this module; the
CUDA library shares no code with it.  Plain FP64 numpy, small sizes only.

Follows arXiv 2506.06661, Section "Density fitting", the long-range density fitting (LRDF)
paragraphs: the Coulomb operator splits as 1/r = erf(w r)/r + erfc(w r)/r; the long-range
part is density fitted with the long-range metric,
    M_PQ = (P|Q)^LR = L L^T,   T_{P,mn} = sum_Q (L^-1)_PQ (Q|mn)^LR,
and the short-range part is computed exactly:
    (mn|kl) ~ (mn|kl)^SR + sum_P T_{P,mn} T_{P,kl}.

For two s-type charge distributions with exponents p and q (reduced exponent
rho = pq/(p+q)) the erf(w r)/r interaction is the full Coulomb closed form with rho replaced
by rho_w = rho w^2 / (rho + w^2) in the Boys argument and the prefactor multiplied by
sqrt(w^2 / (rho + w^2)) (the long-range operator acts like a Gaussian of exponent w^2 folded
into the charge distributions).  The short-range integral is the full one minus the
long-range one.
"""
from __future__ import annotations

import numpy as np

from .dferr import boys_f0_f1

PI = np.pi


def _norm(a):
    return (2.0 * a / PI) ** 0.75


def _lr_factor(rho, omega):
    """(prefactor scale, argument scale) of the erf(w r)/r operator for reduced exponent rho."""
    if omega is None or np.isinf(omega):
        return np.ones_like(rho), np.ones_like(rho)
    f = omega * omega / (rho + omega * omega)
    return np.sqrt(f), f


def int2c_lr(aux_xyz, aux_exp, omega):
    """(P|Q) with the erf(w r)/r operator (omega None: full range)."""
    x = np.asarray(aux_xyz, dtype=np.float64)
    c = np.asarray(aux_exp, dtype=np.float64)
    R2 = np.sum((x[:, None, :] - x[None, :, :]) ** 2, axis=2)
    cc, dd = c[:, None], c[None, :]
    rho = cc * dd / (cc + dd)
    fs, fa = _lr_factor(rho, omega)
    pre = _norm(cc) * _norm(dd) * 2.0 * PI ** 2.5 / (cc * dd * np.sqrt(cc + dd))
    f0, _ = boys_f0_f1(rho * fa * R2)
    return pre * fs * f0


def _pairs(ao_xyz, ao_exp):
    x = np.asarray(ao_xyz, dtype=np.float64)
    a = np.asarray(ao_exp, dtype=np.float64)
    n = a.size
    m_idx, n_idx = [], []
    for m in range(n):
        for nu in range(m + 1):
            m_idx.append(m)
            n_idx.append(nu)
    m_idx, n_idx = np.array(m_idx), np.array(n_idx)
    am, an = a[m_idx], a[n_idx]
    p = am + an
    mu = am * an / p
    RAB2 = np.sum((x[m_idx] - x[n_idx]) ** 2, axis=1)
    P = (am[:, None] * x[m_idx] + an[:, None] * x[n_idx]) / p[:, None]
    K = _norm(am) * _norm(an) * np.exp(-mu * RAB2)
    return p, P, K


def int3c_lr(ao_xyz, ao_exp, aux_xyz, aux_exp, omega):
    """(Q|mn) with the erf(w r)/r operator as [naux][npair] (omega None: full range)."""
    p, P, K = _pairs(ao_xyz, ao_exp)
    x = np.asarray(aux_xyz, dtype=np.float64)
    c = np.asarray(aux_exp, dtype=np.float64)[:, None]
    R2 = np.sum((x[:, None, :] - P[None, :, :]) ** 2, axis=2)
    rho = p[None, :] * c / (p[None, :] + c)
    fs, fa = _lr_factor(rho, omega)
    pre = _norm(c) * K[None, :] * 2.0 * PI ** 2.5 / (p[None, :] * c * np.sqrt(p[None, :] + c))
    f0, _ = boys_f0_f1(rho * fa * R2)
    return pre * fs * f0


def int4c_range(ao_xyz, ao_exp, omega, part):
    """Full (nao^4) tensor of (mn|kl) for part 'full', 'lr' or 'sr' (= full - lr)."""
    p, P, K = _pairs(ao_xyz, ao_exp)
    n = len(ao_exp)
    pp, qq = p[:, None], p[None, :]
    rho = pp * qq / (pp + qq)
    R2 = np.sum((P[:, None, :] - P[None, :, :]) ** 2, axis=2)
    pre = K[:, None] * K[None, :] * 2.0 * PI ** 2.5 / (pp * qq * np.sqrt(pp + qq))
    full = pre * boys_f0_f1(rho * R2)[0]
    if part == "full":
        packed = full
    else:
        fs, fa = _lr_factor(rho, omega)
        lr = pre * fs * boys_f0_f1(rho * fa * R2)[0]
        packed = lr if part == "lr" else full - lr
    eri = np.empty((n, n, n, n))
    idx = {}
    k = 0
    for m in range(n):
        for nu in range(m + 1):
            idx[(m, nu)] = idx[(nu, m)] = k
            k += 1
    pair_of = np.array([[idx[(m, nu)] for nu in range(n)] for m in range(n)])
    eri[:] = packed[pair_of[:, :, None, None], pair_of[None, None, :, :]]
    return eri


def lrdf_jk(ao_xyz, ao_exp, aux_xyz, aux_exp, omega, D, C):
    """J[D] and K[C C^T] with the LRDF approximation of the paper's LRDF equation."""
    from . import cholesky, df_j, df_k, whiten
    n = len(ao_exp)
    L = cholesky(int2c_lr(aux_xyz, aux_exp, omega))
    T = whiten(L, int3c_lr(ao_xyz, ao_exp, aux_xyz, aux_exp, omega))
    sr = int4c_range(ao_xyz, ao_exp, omega, "sr")
    Pm = C @ C.T
    J = np.einsum("mnkl,kl->mn", sr, D) + df_j(T, n, D)
    K = np.einsum("mknl,kl->mn", sr, Pm) + df_k(T, n, C)
    return J, K
