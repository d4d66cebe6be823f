"""Batched SCF (molecules of uneven size sharing a stream pool, graph-captured
iterations) against per-molecule oracle energies."""
import numpy as np
import pytest

import gen
from oracle import scf as oscf

pytestmark = pytest.mark.gpu
dfscf = pytest.importorskip("paper_2506_06661_gb300")


@pytest.fixture(scope="module")
def small_batch():
    sizes = [4, 9, 6, 12, 5, 8, 7]
    mols = [gen.make_molecule(n, gen.molecules.box_for(n), (9, i)) for i, n in enumerate(sizes)]
    ref = [oscf.rhf(oscf.build_system(m)).energy for m in mols]
    return mols, ref


@pytest.mark.parametrize("slots", [3, 16])
def test_batch_fp64_matches_oracle(small_batch, slots):
    mols, ref = small_batch
    out = dfscf.scf_run_batch(mols, slots=slots, precision="fp64", want_D=True)
    for m, r, e, D in zip(mols, out.results, ref, out.D):
        assert r.converged
        assert abs(r.energy - e) <= 1e-9
        Dn = D.cpu().numpy()
        S, _, _ = oscf.int1e(m.ao_xyz, m.ao_exp, m.xyz, m.charges)
        assert abs(np.sum(Dn * S) - m.nelec) <= 1e-8


def test_batch_mixed_within_1e6(small_batch):
    mols, ref = small_batch
    out = dfscf.scf_run_batch(mols, slots=4, precision="mixed")
    for r, e in zip(out.results, ref):
        assert r.converged and r.fp64_iterations >= 2
        assert abs(r.energy - e) <= 1e-6


def test_single_scf_matches_batch_of_one(small_batch):
    mols, ref = small_batch
    r1 = dfscf.scf_run(mols[3], precision="fp64")
    rb = dfscf.scf_run_batch([mols[3]], slots=1, precision="fp64").results[0]
    assert r1.iterations == rb.iterations
    assert abs(r1.energy - rb.energy) <= 1e-12
