"""Small cases of every major kernel path, run against the bounds-checking build of the
library (DFSCF_VARIANT=bounds) by tests/test_gpu_bounds.py.  Prints one JSON line with the
number of out-of-range indices the kernels recorded and the first one's location."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import gen  # noqa: E402
import paper_2506_06661_gb300 as dfscf  # noqa: E402
from paper_2506_06661_gb300 import guess  # noqa: E402


def main():
    assert dfscf.lib().df_bounds_checked() == 1, "not the bounds-checking build"
    rng = np.random.default_rng(0)
    # ragged sizes: 13 centres (nao 65, naux 195) and 27 centres (nao 135: two 128-row tiles)
    for n, seed in ((13, 1), (27, 2)):
        m = gen.make_molecule(n, gen.molecules.box_for(n), seed)
        L = dfscf.metric_chol(m.aux_xyz, m.aux_exp)
        C = 0.2 * rng.standard_normal((m.nao, max(1, m.nocc)))
        D = 2 * C @ C.T
        for prec in ("fp64", "mixed"):
            B = dfscf.build_B(m.ao_xyz, m.ao_exp, m.aux_xyz, m.aux_exp, L, prec)
            dfscf.jk(B, D, C, precision=prec)
            if prec == "fp64":
                dfscf.lib().df_tune_set(b"j_fp64_fma", 1)
                dfscf.jk(B, D, C, precision=prec)
                dfscf.lib().df_tune_set(b"j_fp64_fma", 0)
        for prec in ("fp64", "mixed"):
            dfscf.scf_run(m, precision=prec, raise_on_noconv=False)
    # batch with Newton steps on a stalling member (40 centres), incremental exchange on
    mols = [gen.make_molecule(k, gen.molecules.box_for(k), (5, k)) for k in (6, 11, 17)]
    n147 = int(gen.molecules.batch_sizes(256, 10, 80, 1)[147])
    mols.append(gen.make_molecule(n147, gen.molecules.box_for(n147), (1, 147)))
    dfscf.scf_run_batch(mols, slots=3, precision="mixed", raise_on_noconv=False)
    # DF error with its Jacobian, LRDF, the allocation-free J, the learned-guess kernels
    m = gen.make_molecule(5, gen.molecules.box_for(5), 3)
    k = np.tile(np.arange(15), m.natm).astype(float)
    dfscf.fit_residual(m.ao_xyz, m.ao_exp, m.aux_xyz, m.aux_exp, np.stack([m.aux_exp, k * m.aux_exp], axis=1))
    xyz = gen.molecules.make_geometry(6, gen.molecules.box_for(6), 4)
    ml = gen.molecule_from_geometry(xyz, aux_exp=gen.molecules.even_tempered(0.1, 0.6, 2))
    T = dfscf.lrdf_build(ml.ao_xyz, ml.ao_exp, ml.aux_xyz, ml.aux_exp, 0.4)
    C = 0.2 * rng.standard_normal((ml.nao, 3))
    dfscf.lrdf_jk(T, ml.ao_xyz, ml.ao_exp, 0.4, 2 * C @ C.T, C)
    model = guess.GuessModel.create(seed=1)
    guess.predict_density(model, m)
    torch.cuda.synchronize()
    count, where = dfscf.bounds_violations()
    print(json.dumps({"violations": count, "first": where}), flush=True)


if __name__ == "__main__":
    main()
