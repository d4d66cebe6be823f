"""Incremental mixed-precision exchange in the SCF (knob "mixed_incremental").

With three BF16 planes per operand the mixed exchange of a 40-centre molecule has an error
floor that the plain mixed SCF wanders on before it switches to FP64.  The incremental mode
builds one FP64 base once max|e| < 1e-3 and then updates K from the change of the occupied
projector in mixed precision, so its error shrinks with the change: it must reach the
oracle's energy within 1e-6 Eh with no more iterations than the FP64 SCF needs plus a few,
and with at most a handful of FP64 Fock builds.
"""
import pytest

import gen
from oracle import scf as oscf

pytestmark = pytest.mark.gpu
dfscf = pytest.importorskip("paper_2506_06661_gb300")


def _set(name, v):
    assert dfscf.lib().df_tune_set(name.encode(), v) == dfscf.DF_OK, dfscf.lib().df_last_error()


@pytest.fixture(scope="module")
def mol40():
    m = gen.make_molecule(40, gen.molecules.box_for(40), 5)
    return m, oscf.rhf(oscf.build_system(m))


@pytest.fixture
def three_planes():
    old = {k: dfscf.lib().df_tune_get(k.encode()) for k in ("mixed_planes", "mixed_incremental")}
    _set("mixed_planes", 3)
    yield
    for k, v in old.items():
        _set(k, v)


def test_incremental_reaches_oracle_energy(mol40, three_planes):
    m, ref = mol40
    assert ref.converged
    _set("mixed_incremental", 1)
    r = dfscf.scf_run(m, precision="mixed", max_cycle=100)
    assert r.converged
    assert abs(r.energy - ref.energy) <= 1e-6, (r.energy, ref.energy)
    r64 = dfscf.scf_run(m, precision="fp64")
    assert abs(r.energy - r64.energy) <= 1e-6
    assert r.iterations <= r64.iterations + 6, (r.iterations, r64.iterations)
    # one base, the two final FP64 iterations, and at most a few rebuilt bases
    assert r.fp64_iterations <= 6, r.fp64_iterations


def test_plain_and_incremental_agree(mol40, three_planes):
    m, ref = mol40
    _set("mixed_incremental", 0)
    plain = dfscf.scf_run(m, precision="mixed", max_cycle=100)
    _set("mixed_incremental", 1)
    inc = dfscf.scf_run(m, precision="mixed", max_cycle=100)
    assert plain.converged and inc.converged
    assert abs(plain.energy - ref.energy) <= 1e-6 and abs(inc.energy - ref.energy) <= 1e-6
    print(f"plain mixed: {plain.iterations} iterations ({plain.fp64_iterations} FP64); "
          f"incremental: {inc.iterations} ({inc.fp64_iterations} FP64)")


def test_incremental_batch_matches_fp64():
    mols = [gen.make_molecule(n, gen.molecules.box_for(n), (13, i)) for i, n in enumerate([12, 30, 18, 25, 9])]
    ref = dfscf.scf_run_batch(mols, slots=3, precision="fp64").results
    out = dfscf.scf_run_batch(mols, slots=3, precision="mixed").results
    for a, b in zip(out, ref):
        assert a.converged and b.converged
        assert abs(a.energy - b.energy) <= 1e-6
