"""CPU oracle for the density-fitted Hartree-Fock hot path (arXiv 2506.06661).

TEST INFRASTRUCTURE ONLY: only the tests, the package smoke check and the bench's CPU
baseline use this package.  It is plain FP64 code (C loops in ``oracle.c`` plus numpy
for the SCF bookkeeping) written from the paper's density-fitting equations and the
textbook restricted Hartree-Fock/DIIS definitions.  It shares nothing with the CUDA
library and never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build_library(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build_library()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        L.oracle_boys_f0.restype = ctypes.c_double
        L.oracle_boys_f0.argtypes = [ctypes.c_double]
        L.oracle_boys_f0_vec.argtypes = [dp, ctypes.c_long, dp]
        L.oracle_int1e.argtypes = [dp, dp, ctypes.c_int, dp, dp, ctypes.c_int, dp, dp, dp]
        L.oracle_nuclear_repulsion.restype = ctypes.c_double
        L.oracle_nuclear_repulsion.argtypes = [dp, dp, ctypes.c_int]
        L.oracle_int2c.argtypes = [dp, dp, ctypes.c_int, dp]
        L.oracle_int3c.argtypes = [dp, dp, ctypes.c_int, dp, dp, ctypes.c_int, dp]
        L.oracle_int3c_rows.argtypes = [dp, dp, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, dp]
        L.oracle_int4c.argtypes = [dp, dp, ctypes.c_int, dp]
        L.oracle_cholesky.restype = ctypes.c_int
        L.oracle_cholesky.argtypes = [dp, ctypes.c_int, dp, ctypes.c_double]
        L.oracle_whiten.argtypes = [dp, ctypes.c_int, dp, ctypes.c_long]
        L.oracle_df_j.argtypes = [dp, ctypes.c_long, ctypes.c_int, ctypes.c_int, dp, dp]
        L.oracle_df_k.argtypes = [dp, ctypes.c_long, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp]
        L.oracle_df_k_dm.argtypes = [dp, ctypes.c_long, ctypes.c_int, ctypes.c_int, dp, dp]
        L.oracle_jk_4c.argtypes = [dp, ctypes.c_int, dp, dp, dp, dp]
        L.oracle_eri_diag.argtypes = [dp, dp, ctypes.c_int, dp]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous float64"
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def boys_f0(t) -> np.ndarray:
    t = _f64(np.atleast_1d(t))
    out = np.empty_like(t)
    lib().oracle_boys_f0_vec(_p(t), t.size, _p(out))
    return out


def int1e(ao_xyz, ao_exp, nuc_xyz, nuc_z):
    ao_xyz, ao_exp, nuc_xyz, nuc_z = map(_f64, (ao_xyz, ao_exp, nuc_xyz, nuc_z))
    n = ao_exp.size
    S, T, V = (np.empty((n, n)) for _ in range(3))
    lib().oracle_int1e(_p(ao_xyz), _p(ao_exp), n, _p(nuc_xyz), _p(nuc_z), nuc_z.size, _p(S), _p(T), _p(V))
    return S, T, V


def nuclear_repulsion(nuc_xyz, nuc_z) -> float:
    nuc_xyz, nuc_z = _f64(nuc_xyz), _f64(nuc_z)
    return float(lib().oracle_nuclear_repulsion(_p(nuc_xyz), _p(nuc_z), nuc_z.size))


def int2c(aux_xyz, aux_exp) -> np.ndarray:
    aux_xyz, aux_exp = _f64(aux_xyz), _f64(aux_exp)
    n = aux_exp.size
    M = np.empty((n, n))
    lib().oracle_int2c(_p(aux_xyz), _p(aux_exp), n, _p(M))
    return M


def int3c(ao_xyz, ao_exp, aux_xyz, aux_exp) -> np.ndarray:
    """(Q|mn) as [naux][npair], packed pair mn = m(m+1)/2 + n for m >= n."""
    ao_xyz, ao_exp, aux_xyz, aux_exp = map(_f64, (ao_xyz, ao_exp, aux_xyz, aux_exp))
    nao, naux = ao_exp.size, aux_exp.size
    R = np.empty((naux, nao * (nao + 1) // 2))
    lib().oracle_int3c(_p(ao_xyz), _p(ao_exp), nao, _p(aux_xyz), _p(aux_exp), naux, _p(R))
    return R


def int3c_rows(ao_xyz, ao_exp, aux_xyz, aux_exp, rows) -> np.ndarray:
    """(Q|r n) for the orbital rows r in `rows` and every n, as [naux][len(rows)][nao]: the
    entries of int3c at packed pairs (max(r, n), min(r, n)), for sampling rows of B."""
    ao_xyz, ao_exp, aux_xyz, aux_exp = map(_f64, (ao_xyz, ao_exp, aux_xyz, aux_exp))
    nao, naux = ao_exp.size, aux_exp.size
    r = np.ascontiguousarray(rows, dtype=np.int32)
    assert r.ndim == 1 and np.all((r >= 0) & (r < nao))
    out = np.empty((naux, r.size, nao))
    lib().oracle_int3c_rows(_p(ao_xyz), _p(ao_exp), nao, _p(aux_xyz), _p(aux_exp), naux, r.ctypes.data_as(ctypes.c_void_p),
                            r.size, _p(out))
    return out


def int4c(ao_xyz, ao_exp) -> np.ndarray:
    ao_xyz, ao_exp = _f64(ao_xyz), _f64(ao_exp)
    n = ao_exp.size
    eri = np.empty((n, n, n, n))
    lib().oracle_int4c(_p(ao_xyz), _p(ao_exp), n, _p(eri))
    return eri


def eri_diag(ao_xyz, ao_exp) -> np.ndarray:
    ao_xyz, ao_exp = _f64(ao_xyz), _f64(ao_exp)
    n = ao_exp.size
    d = np.empty(n * (n + 1) // 2)
    lib().oracle_eri_diag(_p(ao_xyz), _p(ao_exp), n, _p(d))
    return d


class NotPositiveDefinite(RuntimeError):
    def __init__(self, pivot: int):
        super().__init__(f"metric is not positive definite at pivot {pivot}")
        self.pivot = pivot


def cholesky(M, tol: float = 1e-14) -> np.ndarray:
    M = _f64(M)
    n = M.shape[0]
    L = np.empty_like(M)
    bad = lib().oracle_cholesky(_p(M), n, _p(L), tol)
    if bad >= 0:
        raise NotPositiveDefinite(bad)
    return L


def whiten(L, R) -> np.ndarray:
    """B = L^-1 R by forward substitution (returns a new array)."""
    L = _f64(L)
    B = np.array(R, dtype=np.float64, order="C", copy=True)
    lib().oracle_whiten(_p(L), L.shape[0], _p(B), B.shape[1])
    return B


def df_b_rows(ao_xyz, ao_exp, aux_xyz, aux_exp, L, rows) -> np.ndarray:
    """Rows of the whitened tensor, B_P[r, n] = sum_Q (L^-1)_PQ (Q|r n) for r in `rows`, as
    [naux][len(rows)][nao] (the metric / whitening equations after Eq. (eq:df:eri)).  The
    triangular solve is a library routine (a step, not a restatement), applied to the same
    columns that `whiten` substitutes one by one."""
    from scipy.linalg import solve_triangular
    R = int3c_rows(ao_xyz, ao_exp, aux_xyz, aux_exp, rows)
    naux, nr, nao = R.shape
    return solve_triangular(_f64(L), R.reshape(naux, nr * nao), lower=True).reshape(naux, nr, nao)


def df_j(B, nao: int, D) -> np.ndarray:
    B, D = _f64(B), _f64(D)
    J = np.empty((nao, nao))
    lib().oracle_df_j(_p(B), B.shape[1], B.shape[0], nao, _p(D), _p(J))
    return J


def df_k(B, nao: int, C) -> np.ndarray:
    """K = sum_P (B_P C)(B_P C)^T for C [nao][nocc]."""
    B, C = _f64(B), _f64(C)
    K = np.empty((nao, nao))
    lib().oracle_df_k(_p(B), B.shape[1], B.shape[0], nao, _p(C), C.shape[1], _p(K))
    return K


def df_k_dm(B, nao: int, Dm) -> np.ndarray:
    """K[Dm] = sum_P B_P Dm B_P for any (not necessarily factorised) symmetric Dm."""
    B, Dm = _f64(B), _f64(Dm)
    K = np.empty((nao, nao))
    lib().oracle_df_k_dm(_p(B), B.shape[1], B.shape[0], nao, _p(Dm), _p(K))
    return K


def jk_4c(eri, D, Pm):
    eri, D, Pm = _f64(eri), _f64(D), _f64(Pm)
    n = D.shape[0]
    J, K = np.empty((n, n)), np.empty((n, n))
    lib().oracle_jk_4c(_p(eri), n, _p(D), _p(Pm), _p(J), _p(K))
    return J, K


def unpack(row: np.ndarray, nao: int) -> np.ndarray:
    """Packed lower triangle (m >= n) -> full symmetric matrix."""
    out = np.zeros((nao, nao))
    il = np.tril_indices(nao)
    # np.tril_indices enumerates (m, n) row-major with n <= m: exactly m(m+1)/2 + n order
    out[il] = row[: nao * (nao + 1) // 2]
    return out + np.tril(out, -1).T


from .scf import (  # noqa: E402,F401
    DFSystem,
    build_system,
    canonical_orthogonalization,
    core_guess,
    rhf,
)
