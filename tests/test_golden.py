"""Stored reference values of the 20-centre workload (tests/golden/oracle_c0.json, written by
tests/golden/make_golden.py from the oracle alone): the oracle must keep reproducing them (a
change of its arithmetic shows up here), and the GPU path must match them without running the
oracle."""
import json
import os

import numpy as np
import pytest

import gen
import oracle
from oracle import scf

GOLDEN = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_c0.json")))


def entries(d):
    return [(tuple(int(x) for x in k.split(",")), v) for k, v in d.items()]


def test_oracle_reproduces_golden(c0, c0_system, c0_scf):
    assert abs(c0_system.enuc - GOLDEN["e_nuc"]) <= 1e-12 * abs(GOLDEN["e_nuc"])
    assert abs(c0_scf.energy - GOLDEN["rhf_energy"]) <= 1e-10
    assert abs(c0_scf.iterations - GOLDEN["rhf_iterations"]) <= 1
    X = scf.canonical_orthogonalization(c0_system.S)
    C, _ = scf.occupied_from_fock(c0_system.h, X, c0_system.nocc)
    J = oracle.df_j(c0_system.B, c0.nao, 2.0 * C @ C.T)
    K = oracle.df_k(c0_system.B, c0.nao, C)
    for (i, j), v in entries(GOLDEN["core_guess_J"]):
        assert abs(J[i, j] - v) <= 1e-12 * max(1.0, abs(v))
    for (i, j), v in entries(GOLDEN["core_guess_K"]):
        assert abs(K[i, j] - v) <= 1e-12 * max(1.0, abs(v))
    for t, v in GOLDEN["boys_f0"].items():
        assert abs(float(oracle.boys_f0(np.array([float(t)]))[0]) - v) <= 4e-16 * v


@pytest.mark.gpu
def test_gpu_matches_golden(c0, c0_system):
    # the same inputs as the fixture: the oracle's core-guess orbitals (signs and rotations
    # inside the occupied space do not change J or K)
    dfscf = pytest.importorskip("paper_2506_06661_gb300")
    X = scf.canonical_orthogonalization(c0_system.S)
    C, _ = scf.occupied_from_fock(c0_system.h, X, c0_system.nocc)
    D = 2.0 * C @ C.T
    L = dfscf.metric_chol(c0.aux_xyz, c0.aux_exp)
    B = dfscf.build_B(c0.ao_xyz, c0.ao_exp, c0.aux_xyz, c0.aux_exp, L, "fp64")
    J, K = dfscf.jk(B, D, C, precision="fp64")
    J, K = J.cpu().numpy(), K.cpu().numpy()
    jmax = max(abs(v) for v in GOLDEN["core_guess_J"].values())
    kmax = max(abs(v) for v in GOLDEN["core_guess_K"].values())
    for (i, j), v in entries(GOLDEN["core_guess_J"]):
        assert abs(J[i, j] - v) <= 1e-10 * jmax
    for (i, j), v in entries(GOLDEN["core_guess_K"]):
        assert abs(K[i, j] - v) <= 1e-10 * kmax
    r = dfscf.scf_run(c0, precision="fp64")
    assert r.converged and abs(r.energy - GOLDEN["rhf_energy"]) <= 1e-9
