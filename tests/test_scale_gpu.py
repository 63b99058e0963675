"""The bench workload at scale.

test_ring16_full_size_invariants: ring16 to step 500 (5e8 rows) in the launch
configuration the benchmark times (one paces_step per step, default tuning and
precision), checked through properties that hold at any size.  Per step: the
propagation inside H_eff is unitary up to the series tolerance; truncation
plus rescue never increases the norm; the site populations sum to the norm
(both exact integer sums); row, kept and entry counts are consistent.

test_one_step_at_1e7_rows_matches_oracle: a ring16 state of about 1e7 rows
from the middle of the trajectory, fed to the GPU and the oracle alike; one
step compared element by element (keys bit-exact in row order, amplitudes to
1e-10 normwise), which crosses multi-tile radix passes, grids of many waves
and candidate indices far above one launch.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2603_07341_gb300 import binding as B
from paper_2603_07341_gb300 import workloads as W
from tests.test_parity_gpu import compare_record, compare_state

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


def test_one_step_at_1e7_rows_matches_oracle(libpaces):
    cfg = W.WORKLOADS["ring16"]
    model = W.model_kwargs(cfg)
    start = W.start_state(cfg)
    gpu = B.Solver(**model)
    gpu.set_state(*start)
    for _ in range(300):
        gpu.step(cfg["dt"], 1, cfg["theta"])
        if gpu.num_rows() >= 1e7:
            break
    assert gpu.num_rows() >= 1e7
    site, occ, amps = gpu.state()
    ora = Oracle(**model)
    ora.set_state(*start)                 # psi(0), the reference of C(t)
    ora.load_state(site, occ, amps)
    del site, occ, amps
    _, a_before = ora.rows()
    theta = cfg["theta"]
    gpu.step(cfg["dt"], 1, theta)
    gkeep = gpu.keep()
    w = a_before.real ** 2 + a_before.imag ** 2
    okeep = w >= theta * theta
    diff = gkeep != okeep
    if diff.any():                        # only within rounding of theta^2
        band = np.abs(w - theta * theta) <= 1e-9 * theta * theta + 1e-10 * np.sum(w)
        assert np.all(band[diff])
        ora.step(cfg["dt"], theta, keep=gkeep.astype(np.uint8))
    else:
        ora.step(cfg["dt"], theta)
    n = compare_state(gpu, ora)
    assert n >= 1e7
    compare_record(gpu.observables(gpu.num_records() - 1, 1)[0], ora, cfg["n_sites"])
    gpu.close()
