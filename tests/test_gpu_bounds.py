"""The bounds-checking build (-DDFSCF_BOUNDS_CHECK, libdfscf_bounds.so) runs small cases of
every major path (tests/bounds_workload.py): J and K in both precisions and both J
arithmetics on ragged sizes, FP64 and mixed SCF, a batch with Newton steps, the DF-error
Jacobian, LRDF, the allocation-free J and the learned-guess kernels.  The kernels' computed
indices are checked against their buffers' extents; none may fall outside.  It stands in for
a memory checker: a bad index is recorded and redirected inside the buffer, never faulted."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
dfscf = pytest.importorskip("paper_2506_06661_gb300")

HERE = os.path.dirname(os.path.abspath(__file__))


def test_no_out_of_range_index_in_checking_build():
    from paper_2506_06661_gb300 import build
    build.build(variant="bounds")
    env = dict(os.environ, DFSCF_VARIANT="bounds")
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_workload.py")], env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("{")][-1]
    out = json.loads(line)
    assert out["violations"] == 0, out["first"]


def test_normal_build_reports_no_checks():
    assert dfscf.lib().df_bounds_checked() == 0
    assert dfscf.bounds_violations() == (0, "")
