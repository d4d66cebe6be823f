"""Writes tests/golden/oracle_c0.json: reference values of the 20-centre parity workload
computed by the CPU oracle alone (plain FP64; nothing from the CUDA path), so that a change of
the oracle's arithmetic shows up as a changed fixture in review.

    python tests/golden/make_golden.py

Values: E_nuc; the DF-RHF energy (DIIS, |dE| < 1e-8, max|e| < 1e-5) and its iteration count;
J and K of the core-guess orbitals at a few entries (first, interior, last row); the Boys
function F0 at a few arguments across the series / erf / asymptotic ranges.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import gen  # noqa: E402
import oracle  # noqa: E402
from oracle import scf  # noqa: E402

ENTRIES = [(0, 0), (37, 12), (99, 0), (99, 99), (50, 51)]
BOYS_T = [0.0, 1e-6, 5e-4, 0.3, 2.0, 17.5, 45.0]


def main():
    mol = gen.config_c0()
    sysm = scf.build_system(mol)
    res = scf.rhf(sysm)
    X = scf.canonical_orthogonalization(sysm.S)
    C, _ = scf.occupied_from_fock(sysm.h, X, sysm.nocc)
    D = 2.0 * C @ C.T
    J = oracle.df_j(sysm.B, sysm.nao, D)
    K = oracle.df_k(sysm.B, sysm.nao, C)
    out = {
        "source": "oracle/ only (tests/golden/make_golden.py); workload gen.config_c0(): 20 centres, nao 100, "
                  "naux 300, nocc 10",
        "e_nuc": float(sysm.enuc),
        "rhf_energy": float(res.energy),
        "rhf_iterations": int(res.iterations),
        "core_guess_J": {f"{i},{j}": float(J[i, j]) for i, j in ENTRIES},
        "core_guess_K": {f"{i},{j}": float(K[i, j]) for i, j in ENTRIES},
        "boys_f0": {repr(t): float(oracle.boys_f0(np.array([t]))[0]) for t in BOYS_T},
    }
    with open(os.path.join(HERE, "oracle_c0.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
