"""The bench workload at full size (ring16 to step 500, 5e8 rows), checked
through properties that hold at any size, in the launch configuration the
benchmark times (one paces_step per step, default tuning).

Per step: the propagation inside H_eff is unitary up to the series tolerance
and double-word rounding; truncation plus rescue never increases the norm;
the site populations sum to the norm (both exact integer sums); row, kept and
entry counts are consistent.
"""
import numpy as np
import pytest

from paper_2603_07341_gb300 import binding as B
from paper_2603_07341_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_ring16_full_size_invariants(libpaces):
    cfg = W.WORKLOADS["ring16"]
    s = B.Solver(**W.model_kwargs(cfg))
    s.set_state(*W.start_state(cfg))
    for _ in range(500):
        s.step(cfg["dt"], 1, cfg["theta"])
    rec = s.observables(1, 500)
    d = B.records_dict(rec, cfg["n_sites"])
    rows, kept, nnz = d["rows"], d["kept"], d["nnz"]
    assert rows[-1] > 4.5e8                                     # the bench window's size
    assert np.all(np.abs(d["norm"] - d["norm_phi0"]) <= 1e-12)  # unitary inside H_eff
    assert np.all(d["norm_phi0"] <= d["norm_before"] + 1e-14)   # Q and rescue never add weight
    assert np.all(np.abs(d["P"].sum(1) - d["norm"]) <= 1e-14)
    assert np.all(kept[1:] <= rows[:-1]) and np.all(kept <= rows)
    assert np.all(nnz >= rows) and np.all(nnz <= 5 * rows)      # diagonal + at most 4 moves
    assert np.all(d["terms"] >= 2) and np.all(d["terms"] <= 200)
    assert np.all(np.diff(d["time"]) > 0)
    s.close()
