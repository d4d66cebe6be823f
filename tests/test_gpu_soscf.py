"""Newton (second-order) SCF steps after DIIS stalls (knob "soscf", on by default).

Four molecules of the 256-molecule batch workload (10-80 centres, seed 1) make plain Pulay
DIIS oscillate at max|e| ~ 1e-4 - 1e-3 for hundreds of iterations, on the GPU and in the CPU
oracle alike.  With the switch to Newton steps they must converge.  The SCF solution has a
plain definition that does not depend on the algorithm, so the converged density is checked
with the oracle's own Fock build: the orthogonal-basis commutator X^T (F D S - S D F) X
below the convergence threshold, the oracle's energy of that density equal to the GPU's,
the right electron count and an idempotent density.
"""
import numpy as np
import pytest

import gen
import oracle
from oracle import scf as oscf

pytestmark = pytest.mark.gpu
dfscf = pytest.importorskip("paper_2506_06661_gb300")


def batch_member(i, count=256, lo=10, hi=80, seed=1):
    n = int(gen.molecules.batch_sizes(count, lo, hi, seed)[i])
    return gen.make_molecule(n, gen.molecules.box_for(n), (seed, i))


def check_stationary(mol, D, energy, tol_err=2e-5):
    sysm = oscf.build_system(mol)
    D = D.cpu().numpy()
    J = oracle.df_j(sysm.B, mol.nao, D)
    K = 0.5 * oracle.df_k_dm(sysm.B, mol.nao, D)
    F = sysm.h + J - K
    E = 0.5 * np.sum(D * (sysm.h + F)) + sysm.enuc
    X = oscf.canonical_orthogonalization(sysm.S)
    FDS = F @ D @ sysm.S
    err = np.abs(X.T @ (FDS - FDS.T) @ X).max()
    assert err <= tol_err, err
    assert abs(E - energy) <= 1e-8, (E, energy)
    assert abs(np.sum(D * sysm.S) - mol.nelec) <= 1e-8
    DSD = D @ sysm.S @ D
    assert np.abs(DSD - 2 * D).max() <= 1e-6 * np.abs(D).max()
    return E


@pytest.mark.parametrize("idx", [147, 101])
def test_newton_steps_converge_where_diis_stalls(idx):
    m = batch_member(idx)
    old = dfscf.lib().df_tune_get(b"soscf")
    try:
        dfscf.lib().df_tune_set(b"soscf", 0)
        plain = dfscf.scf_run(m, precision="fp64", max_cycle=100, raise_on_noconv=False)
        assert not plain.converged      # the case this switch exists for
        dfscf.lib().df_tune_set(b"soscf", 1)
        r = dfscf.scf_run(m, precision="fp64", max_cycle=100)
    finally:
        dfscf.lib().df_tune_set(b"soscf", old)
    assert r.converged
    check_stationary(m, r.D, r.energy)
    rm = dfscf.scf_run(m, precision="mixed", max_cycle=100)
    assert rm.converged
    check_stationary(m, rm.D, rm.energy)
    print(f"molecule {idx}: fp64 {r.iterations} iterations, E {r.energy:.10f}; mixed {rm.iterations} "
          f"({rm.fp64_iterations} FP64), E {rm.energy:.10f}")


def test_batch_with_stalling_members_converges():
    """All four stalling members in one batch, both precisions: every one converges and the
    two precisions agree within 1e-6 Eh; the 40-centre member's density is checked with the
    oracle's Fock build (the 75-77-centre ones would take the CPU oracle minutes)."""
    idx = (7, 147, 226, 101)
    mols = [batch_member(i) for i in idx]
    res = {}
    for prec in ("fp64", "mixed"):
        out = dfscf.scf_run_batch(mols, slots=4, precision=prec, want_D=True, max_cycle=100)
        res[prec] = out.results
        for i, m, r, D in zip(idx, mols, out.results, out.D):
            assert r.converged, (i, prec)
            if i == 147:
                check_stationary(m, D, r.energy)
    for a, b in zip(res["fp64"], res["mixed"]):
        assert abs(a.energy - b.energy) <= 1e-6
