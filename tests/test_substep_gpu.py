"""Substepped propagation on the GPU against the oracle (App. C.1: the step's
exponential taken as s successive Taylor series of dt / s, the scaling the
paper names as its alternative propagator; App. I: past a threshold in dt a
single series fails and the norm explodes).

The number of series s = ceil(rho dt / xmax) comes from an integer bound rho on
||P H P|| that both sides compute exactly, so s and rho must be equal; the
amplitudes follow the usual bar (1e-10 normwise).
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2603_07341_gb300 import binding as B
from paper_2603_07341_gb300 import workloads as W
from tests.test_adjoint_gpu import _case, _ring_model
from tests.test_parity_gpu import compare_state, make_pair

pytestmark = pytest.mark.gpu
EPS4 = np.array([0.1, -0.2, 0.3, 0.0])


def _field(rec, name):
    return rec[:, B.OBS_FIELDS.index(name)]


@pytest.mark.parametrize("precision", [B.C128, B.DW], ids=["c128", "dw"])
def test_large_dt_substeps_lockstep(libpaces, precision):
    """ring4 over its full 2500-state space at dt = 3 (||H|| = 19.4): 8 series
    per step on both sides, amplitudes within 1e-10 of the oracle after every
    step, which the pins tie to the dense exp(-iHt) psi0."""
    cfg = W.WORKLOADS["ring4"]
    gpu, ora = make_pair(cfg, gpu_extra=dict(precision=precision), eps=EPS4)
    st = W.start_state(cfg)
    gpu.set_state(*st)
    ora.set_state(*st)
    for _ in range(6):
        gpu.step(3.0, 1, 0.0)
        ora.step(3.0, 0.0)
        compare_state(gpu, ora)
        rec = gpu.observables(gpu.num_records() - 1, 1)
        so = ora.stats()
        assert _field(rec, "substeps")[0] == so["substeps"] == 8
        assert _field(rec, "hbound")[0] == so["hbound"]
        assert abs(_field(rec, "terms")[0] - so["terms"]) <= so["substeps"]
        assert abs(_field(rec, "norm")[0] - 1.0) < 1e-12
        assert abs(rec[0, 3] - so["energy"]) <= 1e-10 * max(1.0, abs(so["energy"]))


@pytest.mark.parametrize("precision", [B.C128, B.DW], ids=["c128", "dw"])
def test_substeps_with_truncation_lockstep(libpaces, precision):
    """A truncated ring16 prefix with xmax = 0.25: several series per step
    while H_eff changes every step."""
    from tests.test_parity_gpu import lockstep
    cfg = W.WORKLOADS["ring16"]
    gpu, ora = make_pair(cfg, gpu_extra=dict(precision=precision), m_init=4, xmax=0.25)
    st = W.start_state(cfg)
    gpu.set_state(*st)
    ora.set_state(*st)
    lockstep(gpu, ora, 0.05, 1e-5, 12)
    assert ora.stats()["substeps"] >= 2
    rec = gpu.observables(1, 12)
    assert np.all(_field(rec, "substeps") >= 2)


def test_complex64_terms_with_substeps(libpaces):
    """The complex64 variant runs the same split: same series count, norm kept
    to its stated bound and amplitudes within 1e-6 of the FP64 run."""
    cfg = W.WORKLOADS["ring4"]
    model = W.model_kwargs(cfg, eps=EPS4)
    a = B.Solver(**model, precision=B.C64_SPMV)
    b = B.Solver(**model, precision=B.C128)
    st = W.start_state(cfg)
    for s in (a, b):
        s.set_state(*st)
        s.step(3.0, 4, 0.0)
    ra, rb = a.observables(1, 4), b.observables(1, 4)
    assert np.array_equal(_field(ra, "substeps"), _field(rb, "substeps"))
    assert np.max(np.abs(_field(ra, "norm") - 1.0)) < 1e-6
    _, aa = a.tuples()
    _, ab = b.tuples()
    assert np.max(np.abs(aa - ab)) < 1e-6


def test_too_many_series_is_reported(libpaces):
    """More than 1024 series per step is NOCONVERGE, and the state stays as the
    failed step regrew it (unpropagated)."""
    cfg = W.WORKLOADS["ring4"]
    gpu = B.Solver(**W.model_kwargs(cfg, eps=EPS4))
    gpu.set_state(*W.start_state(cfg))
    with pytest.raises(B.PacesError) as e:
        gpu.step(1000.0, 1, 0.0)
    assert e.value.code == 4


def test_single_series_when_disabled(libpaces):
    cfg = W.WORKLOADS["ring4"]
    gpu = B.Solver(**W.model_kwargs(cfg, eps=EPS4, xmax=-1.0))
    gpu.set_state(*W.start_state(cfg))
    gpu.step(0.5, 1, 0.0)
    assert _field(gpu.observables(1, 1), "substeps")[0] == 1


@pytest.mark.parametrize("precision", [B.C128, B.DW], ids=["c128", "dw"])
def test_gradient_through_substeps_matches_oracle(libpaces, precision):
    """The reverse pass runs the recurrence series by series (the oracle's
    adjoint through substeps is pinned to central differences)."""
    model = dict(_ring_model(), xmax=0.3)
    start = (np.array([0, 1], np.int32), np.array([[0] * 4, [1, 0, 0, 0]], np.int32), np.array([0.6, 0.8j]))
    gpu, _ = _case(model, start, 0.1, 2e-3, 17, 5, precision, 77)
    assert np.all(_field(gpu.observables(1, 17), "substeps") >= 2)
