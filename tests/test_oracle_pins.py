"""The FP64 oracle against closed forms, brute force and invariants."""
import pytest

import oracle.communicability as oc
from tests import pins


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda f: f.__name__)
def test_oracle_pin(check):
    check(oc)


def test_truncation_report_converges_to_dense():
    """The truncation report's converged e^A 1 equals the dense exponential."""
    import math

    import numpy as np

    import oracle.communicability as oc
    import oracle.truncation as ot
    from paper_1409_5000_gb300 import synth

    g = synth.er(300, 0.03, 17)
    th, y, m = ot.converged(g.n, g.row_ptr, g.col, 10)
    ref = oc.total_communicability_dense(g.n, g.row_ptr, g.col)
    assert np.max(np.abs(math.exp(th) * y - ref) / ref) < 1e-12
    nr, hd, mc = ot.errors(g, 5)
    assert nr > 1e-6 and mc >= 10  # m = 5 is far from converged here
