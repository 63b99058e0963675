"""The complex64-SpMV propagator (PACES_C64_SPMV) against the double-word path
and the FP64 oracle.  Terms n >= 3 run in FP32; the first two terms, the
accumulator, norms and truncation magnitudes stay double-word.  Stated bound:
every observable within 1e-6 of the double-word run over the horizon tested,
amplitudes within 1e-6 of the oracle (normwise)."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2603_07341_gb300 import binding as B
from paper_2603_07341_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def run(cfg, precision, nsteps, theta, **over):
    s = B.Solver(**W.model_kwargs(cfg, **over), precision=precision)
    s.set_state(*W.start_state(cfg))
    s.step(cfg["dt"], nsteps, theta)
    return s


@pytest.mark.parametrize("name,over,nsteps,theta", [
    ("dipolar6x6", {"m_init": 2}, 60, 1e-5),
    ("ring16", {}, 120, 1e-7),
    ("cube4", {"m_init": 2}, 20, 1e-5),
])
def test_c64_observables_within_1e6_of_double_word(libpaces, name, over, nsteps, theta):
    cfg = W.WORKLOADS[name]
    a = run(cfg, B.DW, nsteps, theta, **over)
    b = run(cfg, B.C64_SPMV, nsteps, theta, **over)
    ra = B.records_dict(a.observables(), cfg["n_sites"])
    rb = B.records_dict(b.observables(), cfg["n_sites"])
    for key in ("P", "nbar", "C", "norm"):
        err = np.max(np.abs(ra[key] - rb[key]))
        assert err <= 1e-6, (key, err)
    assert np.all(np.abs(ra["rows"] - rb["rows"]) <= 0.01 * ra["rows"])


def test_c64_amplitudes_against_oracle(libpaces):
    cfg = W.WORKLOADS["ring16"]
    model = W.model_kwargs(cfg)
    g = B.Solver(**model, precision=B.C64_SPMV)
    o = Oracle(**model)
    g.set_state(*W.start_state(cfg))
    o.set_state(*W.start_state(cfg))
    g.step(cfg["dt"], 1, cfg["theta"])     # the first step has no truncation: same rows
    o.step(cfg["dt"], cfg["theta"])
    tg, ag = g.tuples()
    to, ao = o.rows()
    assert np.array_equal(tg, to)
    assert np.max(np.abs(ag - ao)) <= 1e-6 * np.linalg.norm(ao)
