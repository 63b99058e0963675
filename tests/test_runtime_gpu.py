"""Step replay as CUDA graphs, launch-shape tuning and the autotuner: none of
them may change results beyond the summation order of reductions."""
import numpy as np
import pytest

from paper_2603_07341_gb300 import autotune
from paper_2603_07341_gb300 import binding as B
from paper_2603_07341_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def solver(cfg, **kw):
    s = B.Solver(**W.model_kwargs(cfg, **kw.pop("over", {})), **kw)
    s.set_state(*W.start_state(cfg))
    return s


@pytest.mark.parametrize("max_rows", [0, 16])
def test_graph_replay_is_bitwise_identical(libpaces, max_rows):
    cfg = W.WORKLOADS["ring16"]
    a = solver(cfg, max_rows=max_rows)
    b = solver(cfg, max_rows=max_rows)
    b.set_tuning(use_graphs=1)
    assert b.tuning()["use_graphs"] == 1
    for n in (5, 8, 13, 9):          # chunks of several sizes, through capacity growth
        a.step(cfg["dt"], n, cfg["theta"])
        b.step(cfg["dt"], n, cfg["theta"])
    assert b.tuning()["use_graphs"] == 1          # capture succeeded: steps were replayed
    ta, aa = a.tuples()
    tb, ab = b.tuples()
    assert np.array_equal(ta, tb) and np.array_equal(aa, ab)
    assert np.array_equal(a.observables(), b.observables())


def test_tuning_knobs_keep_results(libpaces):
    cfg = W.WORKLOADS["ring16"]
    a = solver(cfg)
    b = solver(cfg)
    t = b.tuning()
    b.set_tuning(taylor_lanes_per_row=4, taylor_blocks_per_sm=1, grid_blocks_per_sm=4, chunk_blocks_per_sm=2)
    assert b.tuning()["taylor_lanes_per_row"] == 4
    with pytest.raises(B.PacesError):
        b.set_tuning(taylor_lanes_per_row=3)
    with pytest.raises(B.PacesError):
        b.set_tuning(taylor_blocks_per_sm=t["max_taylor_blocks_per_sm"] + 50)
    a.step(cfg["dt"], 30, cfg["theta"])
    b.step(cfg["dt"], 30, cfg["theta"])
    ta, aa = a.tuples()
    tb, ab = b.tuples()
    assert np.array_equal(ta, tb)
    assert np.max(np.abs(aa - ab)) <= 1e-13 * np.linalg.norm(aa)


@pytest.mark.parametrize("pct", [25, 70])
def test_table_load_keeps_results_bitwise(libpaces, pct):
    """The hash tables' size (their largest load) changes slot positions only:
    rows, their order and the amplitudes stay bit for bit, through capacity
    growth from a small start."""
    cfg = W.WORKLOADS["ring16"]
    a = solver(cfg, max_rows=64)
    b = B.Solver(**W.model_kwargs(cfg), max_rows=64)
    b.set_tuning(table_load_pct=pct)
    b.set_state(*W.start_state(cfg))
    assert b.tuning()["table_load_pct"] == pct
    with pytest.raises(B.PacesError):
        b.set_tuning(table_load_pct=10)
    for s in (a, b):
        s.step(cfg["dt"], 40, cfg["theta"])
    ta, aa = a.tuples()
    tb, ab = b.tuples()
    assert np.array_equal(ta, tb) and np.array_equal(aa, ab)


def test_autotuner_picks_valid_settings(libpaces, tmp_path):
    cfg = W.WORKLOADS["ring16"]
    model = W.model_kwargs(cfg)
    s = solver(cfg)
    ref = solver(cfg)
    s.step(cfg["dt"], 60, cfg["theta"])
    ref.step(cfg["dt"], 60, cfg["theta"])
    best, ms = autotune.autotune(s, model, cfg["dt"], cfg["theta"], steps=2,
                                 cache_path=str(tmp_path / "tune.json"))
    assert ms > 0 and best["taylor_lanes_per_row"] in (1, 4, 8)
    assert best["table_load_pct"] in (35, 50, 65)
    assert (tmp_path / "tune.json").exists()
    s.step(cfg["dt"], 5, cfg["theta"])
    ref.step(cfg["dt"], 5, cfg["theta"])
    ts, as_ = s.tuples()
    tr, ar = ref.tuples()
    assert np.array_equal(ts, tr)
    assert np.max(np.abs(as_ - ar)) <= 1e-12 * np.linalg.norm(ar)


def test_grid_barrier_time_limit_runs_out_safely(libpaces):
    """The propagator's grid barrier bounds every wait: a barrier that expects
    one arrival more than the grid has runs out after 1 ms and records the
    barrier error (5) instead of hanging; the context stays usable (a full
    barrier then completes, and a solver still steps)."""
    import torch
    assert B.selftest_barrier(0, 1.0) == 0
    assert B.selftest_barrier(1, 1.0) == 5
    assert B.selftest_barrier(0, 1.0) == 0
    torch.cuda.synchronize()
    cfg = W.WORKLOADS["ring4"]
    s = B.Solver(**W.model_kwargs(cfg))
    s.set_state(*W.start_state(cfg))
    s.step(cfg["dt"], 2, cfg["theta"])
    assert s.num_records() == 3


def test_fp64_rate_probe(libpaces):
    """The FP64 rate probe reports a positive rate no higher than the rate
    derived from the unit counts and the maximum clock (152 SMs x 2 FMA per
    clock x 2 flops x 2.07 GHz = 1.26 TFLOP/s), with a margin for the clock, and
    the same order of magnitude on a second call."""
    a = B.fp64_rate()
    b = B.fp64_rate()
    assert 0.05 < a < 1.4 and 0.05 < b < 1.4, (a, b)
    assert 0.5 < a / b < 2.0
