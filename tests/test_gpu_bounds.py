"""The bounds-checked debug build as the stand-in for a memory checker.

tests/bounds_suite.py runs the operator, hop, multi-field, conversion, solver (every mode,
register blocking, Schur, lattice batches, 10-real inner links), link-gradient and
domain-decomposition entry points on small and ragged lattices (2^4 aliases n+mu and n-mu;
6 x 4 x 10 x 2 has a ragged last tile) with liblq_checked.so, where every field access of the
kernels is checked against its field and an access out of range is skipped and counted.  The
suite runs in a child process (LQ_LIB_VARIANT=checked) so that it loads only the checked
library, and fails on the first operation after which lq_bounds_violations() is not zero or
whose result disagrees with the oracle.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_no_access_outside_the_fields():
    env = dict(os.environ, LQ_LIB_VARIANT="checked")
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_suite.py")], env=env, capture_output=True,
                       text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "bounds suite ok" in r.stdout


def test_normal_build_reports_no_checking(lqlib):
    if lqlib.checked():
        pytest.skip("this process uses the checked library")
    assert lqlib.bounds_violations() == (-1, None)
