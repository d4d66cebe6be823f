"""Stability analysis of converged SCF solutions (knob "stability": scf_result.hess_min, by
Davidson's method on the Newton steps' Hessian products).

hess_min is the lowest eigenvalue of the orbital Hessian in the units of the gradient F_vo
(the energy's gradient with respect to a (virtual, occupied) rotation kappa is 4 F_vo, its
Hessian 4 H).  The pin does not use the GPU's Hessian products: on a 4-centre molecule the
oracle's canonical orbitals are rotated by exp(kappa) (scipy.linalg.expm), the oracle's Fock
matrix of each rotated density gives the gradient 4 F_vo, and central differences of that
gradient over every (virtual, occupied) pair give the full Hessian (the second-order terms of
the exponential map lie in the occupied-occupied and virtual-virtual blocks, to which the
energy is invariant, so the error is O(h^2)).  Its lowest eigenvalue must equal 4 hess_min.
At the ground state of the 20-centre molecule hess_min is positive in both precisions.

Knob "stability" = 2 leaves saddle points: on a ring of ten centres 4.5 bohr apart the
symmetric solution that DIIS reaches is a saddle (one negative eigenvalue, along bond
alternation).  The oracle steps off it along that eigenvector (0.3 rad, as the library) and
converges to the lower, alternating solution, whose finite-difference Hessian is positive;
the GPU must end there, stationary under the oracle's Fock build.
"""
import numpy as np
import pytest

import gen
from oracle import scf as oscf
from stability_fd import escape, fd_hessian, fd_hessian_eigenvalues, h10_ring

pytestmark = pytest.mark.gpu
dfscf = pytest.importorskip("paper_2506_06661_gb300")


def _with_knobs(fn, **knobs):
    old = {k: dfscf.lib().df_tune_get(k.encode()) for k in knobs}
    for k, v in knobs.items():
        dfscf.lib().df_tune_set(k.encode(), v)
    try:
        return fn()
    finally:
        for k, v in old.items():
            dfscf.lib().df_tune_set(k.encode(), v)


def test_hess_min_matches_finite_difference_hessian():
    mol = gen.make_molecule(4, gen.molecules.box_for(4), 2)
    sysm = oscf.build_system(mol)
    ref = oscf.rhf(sysm)
    assert ref.converged
    lam = fd_hessian_eigenvalues(sysm, ref.D)
    assert lam[0] > 0
    for prec in ("fp64", "mixed"):
        r = _with_knobs(lambda: dfscf.scf_run(mol, precision=prec), stability=1, stability_steps=200)
        assert r.converged and np.isfinite(r.hess_min)
        assert abs(4 * r.hess_min - lam[0]) <= 2e-6 * lam[-1], (prec, 4 * r.hess_min, lam[:3])


def test_ground_state_is_a_minimum(c0):
    for prec in ("fp64", "mixed"):
        r = _with_knobs(lambda: dfscf.scf_run(c0, precision=prec), stability=1)
        assert r.converged and r.hess_min > 0, (prec, r.hess_min)
        print(f"{prec}: hess_min {r.hess_min:.6e}")


def test_batch_members_report_hess_min():
    mols = [gen.make_molecule(n, gen.molecules.box_for(n), (3, n)) for n in (6, 9, 12)]
    out = _with_knobs(lambda: dfscf.scf_run_batch(mols, slots=2, precision="fp64"), stability=1)
    for m, r in zip(mols, out.results):
        single = _with_knobs(lambda: dfscf.scf_run(m, precision="fp64"), stability=1)
        assert r.converged and r.hess_min > 0
        assert abs(r.hess_min - single.hess_min) <= 1e-6 * max(1.0, abs(single.hess_min))


def test_stability_off_by_default(c0):
    r = dfscf.scf_run(c0, precision="fp64")
    assert np.isnan(r.hess_min)


@pytest.fixture(scope="module")
def ring_states():
    """The stretched ring's symmetric RHF solution (reached by DIIS from the core guess) is a
    saddle point: its Hessian has one negative eigenvalue, along bond alternation.  The oracle
    turns it by 0.3 rad along that eigenvector and converges to the lower, alternating
    solution, a minimum."""
    mol = h10_ring()
    sysm = oscf.build_system(mol)
    sad = oscf.rhf(sysm)
    assert sad.converged
    H, XC = fd_hessian(sysm, sad.D)
    lam_sad = np.linalg.eigvalsh(H)
    assert lam_sad[0] < -0.05          # 4 x (-0.0243)
    low = escape(sysm, sad.D, H, XC)
    assert low.converged and low.energy < sad.energy - 1e-3
    lam_low = fd_hessian_eigenvalues(sysm, low.D)
    assert lam_low[0] > 0
    return mol, sad, lam_sad, low, lam_low


def test_saddle_is_reported(ring_states):
    mol, sad, lam_sad, low, lam_low = ring_states
    r = _with_knobs(lambda: dfscf.scf_run(mol, precision="fp64"), stability=1, stability_steps=200)
    assert r.converged and r.stability_restarts == 0
    assert abs(r.energy - sad.energy) <= 1e-8, (r.energy, sad.energy)
    assert abs(4 * r.hess_min - lam_sad[0]) <= 2e-6 * lam_sad[-1], (4 * r.hess_min, lam_sad[:2])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_saddle_escape_reaches_the_minimum(ring_states, prec):
    mol, sad, lam_sad, low, lam_low = ring_states
    r = _with_knobs(lambda: dfscf.scf_run(mol, precision=prec), stability=2, stability_steps=200)
    assert r.converged
    assert abs(r.energy - low.energy) <= 1e-7, (prec, r.energy, low.energy, sad.energy)
    assert r.hess_min > 0 and abs(4 * r.hess_min - lam_low[0]) <= 1e-5 * lam_low[-1], (4 * r.hess_min, lam_low[:2])
    # FP64 DIIS keeps the ring's symmetry and stops at the saddle first; the mixed run may
    # break the symmetry on its own
    assert r.stability_restarts == 1 if prec == "fp64" else r.stability_restarts in (0, 1)
    from test_gpu_soscf import check_stationary
    check_stationary(mol, r.D, r.energy)


def test_batch_saddle_escape(ring_states):
    mol, sad, lam_sad, low, lam_low = ring_states
    other = gen.make_molecule(8, gen.molecules.box_for(8), 5)
    out = _with_knobs(lambda: dfscf.scf_run_batch([mol, other], slots=2, precision="fp64"), stability=2)
    r = out.results[0]
    assert r.converged and r.stability_restarts == 1
    assert abs(r.energy - low.energy) <= 1e-7 and r.hess_min > 0
    assert out.results[1].converged and out.results[1].hess_min > 0
