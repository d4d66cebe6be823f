"""Error paths of the C ABI that need a GPU, triggered from the host only.

* A bounded device wait that runs out: the multi-SM eigensolver's grid barriers are told
  (knob "eig_barrier_extra") to wait for one arrival more than the grid provides, with a
  short poll limit, so every CTA gives up, raises the barrier's error flag and returns.
  The call must report DF_ERR_TIMEOUT, and an ordinary call in the same process must then
  give the right eigenpairs (the context stays usable).
* A non-finite Fock matrix: a NaN nuclear charge makes h, and with it F, non-finite; the
  SCF must stop with DF_ERR_NUMERIC.
No test here faults or hangs the GPU: every wait involved is bounded by a poll count.
"""
import numpy as np
import pytest
import torch

import gen

pytestmark = pytest.mark.gpu
dfscf = pytest.importorskip("paper_2506_06661_gb300")


def _knob(name, value):
    rc = dfscf.lib().df_tune_set(name.encode(), value)
    assert rc == dfscf.DF_OK, dfscf.lib().df_last_error()


def _sym(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    return A + A.T


def test_eigensolver_barrier_timeout_then_recovers():
    n, k = 200, 12   # n >= 160 takes the multi-SM path with its grid barriers
    A = _sym(n, 11)
    old = {name: dfscf.lib().df_tune_get(name.encode()) for name in ("eig_barrier_extra", "eig_barrier_polls")}
    try:
        _knob("eig_barrier_polls", 4096)
        _knob("eig_barrier_extra", 1)
        with pytest.raises(dfscf.DFError) as exc:
            dfscf.eigh_lowest(A, k)
        assert exc.value.code == dfscf.DF_ERR_TIMEOUT, exc.value.msg
        assert "timed out" in exc.value.msg
    finally:
        for name, v in old.items():
            _knob(name, v)
    torch.cuda.synchronize()
    w, Z = dfscf.eigh_lowest(A, k)
    wref = np.linalg.eigvalsh(A)[:k]
    assert np.max(np.abs(w.cpu().numpy() - wref)) <= 1e-10 * np.max(np.abs(wref))
    Zn = Z.cpu().numpy()
    assert np.max(np.abs(A @ Zn - Zn * w.cpu().numpy())) <= 1e-9 * np.max(np.abs(wref))


def test_full_eigh_barrier_timeout():
    n = 180
    A = _sym(n, 12)
    old = {name: dfscf.lib().df_tune_get(name.encode()) for name in ("eig_barrier_extra", "eig_barrier_polls")}
    try:
        _knob("eig_barrier_polls", 4096)
        _knob("eig_barrier_extra", 1)
        with pytest.raises(dfscf.DFError) as exc:
            dfscf.eigh(A)
        assert exc.value.code == dfscf.DF_ERR_TIMEOUT
    finally:
        for name, v in old.items():
            _knob(name, v)
    w, _ = dfscf.eigh(A)
    assert np.max(np.abs(w.cpu().numpy() - np.linalg.eigvalsh(A))) <= 1e-10 * np.max(np.abs(w.cpu().numpy()))


def test_nan_charge_stops_scf_with_numeric_error():
    mol = gen.make_molecule(6, gen.molecules.box_for(6), 4)
    mol.charges = mol.charges.copy()
    mol.charges[0] = float("nan")
    with pytest.raises(dfscf.DFError) as exc:
        dfscf.scf_run(mol, precision="fp64")
    assert exc.value.code == dfscf.DF_ERR_NUMERIC, exc.value.msg


def test_knob_range_is_checked():
    assert dfscf.lib().df_tune_set(b"eig_barrier_extra", 2) == dfscf.DF_ERR_ARG
    assert dfscf.lib().df_tune_set(b"eig_barrier_polls", 1) == dfscf.DF_ERR_ARG
