"""df_j_noalloc, the Coulomb build for callers that cannot allocate a device workspace
(plugins whose host framework owns all device memory, services that forbid allocation
while running).  Called through the C ABI with ctypes and checked against df_jk's J and
against the CPU oracle's DF-J on two calls in a row, at the FP64 parity tolerance the other
J tests use (1e-10 relative, max-norm).  This file is collected last so that a failure here
leaves every other test already run."""
import ctypes

import numpy as np
import pytest
import torch

import gen
import oracle
from oracle import scf as oscf

pytestmark = pytest.mark.gpu
dfscf = pytest.importorskip("paper_2506_06661_gb300")


def _abi():
    L = dfscf.lib()
    L.df_j_noalloc.restype = ctypes.c_int
    L.df_j_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p]
    L.df_j_noalloc_capacity.restype = ctypes.c_size_t
    L.df_j_noalloc_capacity.argtypes = []
    return L


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


def test_noalloc_j_matches_df_jk_twice():
    L = _abi()
    mol = gen.make_molecule(13, 5.5, 21)          # nao 65, naux 195: ragged tile counts
    Lf = dfscf.metric_chol(mol.aux_xyz, mol.aux_exp)
    B = dfscf.build_B(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp, Lf, "fp64")
    Bora = oscf.build_system(mol).B
    rng = np.random.default_rng(5)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        C = 0.3 * rng.standard_normal((mol.nao, 4 + call))
        D = torch.tensor(2 * C @ C.T, dtype=torch.float64, device="cuda")
        Jref, _ = dfscf.jk(B, D, None)
        J = torch.full_like(D, float("nan"))
        rc = L.df_j_noalloc(ctypes.c_void_p(B.buf.data_ptr()), mol.nao, mol.naux, ctypes.c_void_p(D.data_ptr()),
                            ctypes.c_void_p(J.data_ptr()), ctypes.c_void_p(stream))
        assert rc == dfscf.DF_OK, L.df_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(J).all()
        assert _rel(J, Jref) <= 1e-10
        Jora = torch.from_numpy(oracle.df_j(Bora, mol.nao, 2 * C @ C.T))
        assert _rel(J.cpu(), Jora) <= 1e-10


def test_noalloc_rejects_oversized_problem():
    L = _abi()
    assert L.df_j_noalloc_capacity() == 8 << 20
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    rc = L.df_j_noalloc(p, 1500, 4500, p, p, None)
    assert rc == dfscf.DF_ERR_ARG
    assert b"scratch" in L.df_last_error()
