"""The Lanczos propagator (App. C.3) on the GPU against the oracle's Lanczos.

exp(-i h H) v ~ ||v|| V_n exp(-i h T_n) e_1 over the same substeps as the
series; the oracle's decomposition is pinned to the paper's printed V_4, to the
dense exp(-iHt) psi0 and to the two-site breakdown.  Both sides stop on the
same residual estimate, so the Krylov dimension may differ by one; amplitudes
follow the usual bar (1e-10 normwise) and every observable is compared.
"""
import numpy as np
import pytest

from paper_2603_07341_gb300 import binding as B
from paper_2603_07341_gb300 import workloads as W
from tests.test_parity_gpu import compare_state, lockstep, make_pair

pytestmark = pytest.mark.gpu
EPS4 = np.array([0.1, -0.2, 0.3, 0.0])
LAN_G = dict(propagator=B.LANCZOS, kmax=30)
LAN_O = dict(propagator=1, kmax=30)


def _field(rec, name):
    return rec[:, B.OBS_FIELDS.index(name)]


def test_lanczos_ring4_full_trajectory(libpaces):
    cfg = W.WORKLOADS["ring4"]
    gpu, ora = make_pair(cfg, gpu_extra=LAN_G, ora_extra=LAN_O)
    st = W.start_state(cfg)
    gpu.set_state(*st)
    ora.set_state(*st)
    lockstep(gpu, ora, cfg["dt"], cfg["theta"], 200, check_every=10)
    rec = gpu.observables(1, 200)
    assert np.all(_field(rec, "terms") < 30)


def test_lanczos_ring16_prefix(libpaces):
    cfg = W.WORKLOADS["ring16"]
    gpu, ora = make_pair(cfg, gpu_extra=LAN_G, ora_extra=LAN_O)
    st = W.start_state(cfg)
    gpu.set_state(*st)
    ora.set_state(*st)
    lockstep(gpu, ora, cfg["dt"], cfg["theta"], 40, check_every=5)


def test_lanczos_dipolar_prefix(libpaces):
    """37 moves per state: the kernel's multi-lane rows."""
    cfg = W.WORKLOADS["dipolar6x6"]
    gpu, ora = make_pair(cfg, gpu_extra=LAN_G, ora_extra=LAN_O, m_init=2)
    st = W.start_state(cfg)
    gpu.set_state(*st)
    ora.set_state(*st)
    lockstep(gpu, ora, cfg["dt"], cfg["theta"], 4)


def test_lanczos_large_dt_substeps(libpaces):
    """dt = 3 over ring4's full space: 8 substeps on both sides."""
    cfg = W.WORKLOADS["ring4"]
    gpu, ora = make_pair(cfg, gpu_extra=LAN_G, ora_extra=LAN_O, eps=EPS4)
    st = W.start_state(cfg)
    gpu.set_state(*st)
    ora.set_state(*st)
    for _ in range(4):
        gpu.step(3.0, 1, 0.0)
        ora.step(3.0, 0.0)
        compare_state(gpu, ora)
        rec = gpu.observables(gpu.num_records() - 1, 1)
        so = ora.stats()
        assert _field(rec, "substeps")[0] == so["substeps"] == 8
        assert abs(_field(rec, "terms")[0] - so["terms"]) <= so["substeps"]
        assert abs(_field(rec, "norm")[0] - 1.0) < 1e-12


def test_lanczos_matches_the_series_on_the_gpu(libpaces):
    """The two propagators of one build agree to 1e-12 normwise step by step
    (both approximate exp(-i P H P dt) to 1e-15), with fewer Krylov vectors
    than series terms."""
    cfg = W.WORKLOADS["ring16"]
    model = W.model_kwargs(cfg)
    a = B.Solver(**model)
    b = B.Solver(**model, **LAN_G)
    st = W.start_state(cfg)
    for s in (a, b):
        s.set_state(*st)
    for _ in range(30):
        a.step(cfg["dt"], 1, cfg["theta"])
        b.step(cfg["dt"], 1, cfg["theta"])
    ta, aa = a.tuples()
    tb, ab = b.tuples()
    assert np.array_equal(ta, tb)
    assert np.max(np.abs(aa - ab)) <= 1e-12 * np.linalg.norm(aa)
    ra, rb = a.observables(1, 30), b.observables(1, 30)
    assert np.all(_field(rb, "terms") < _field(ra, "terms"))


def test_lanczos_too_few_vectors_is_reported(libpaces):
    """kmax = 2 cannot reach 1e-15 on ring4: NOCONVERGE, and the state stays
    as the failed step regrew it."""
    cfg = W.WORKLOADS["ring4"]
    gpu = B.Solver(**W.model_kwargs(cfg), propagator=B.LANCZOS, kmax=2)
    gpu.set_state(*W.start_state(cfg))
    with pytest.raises(B.PacesError) as e:
        gpu.step(cfg["dt"], 1, cfg["theta"])
    assert e.value.code == B.ERR_NOCONVERGE


def test_lanczos_rejected_combinations(libpaces):
    cfg = W.WORKLOADS["ring4"]
    model = W.model_kwargs(cfg)
    for bad in (dict(precision=B.DW), dict(precision=B.C64_SPMV), dict(kmax=B.MAX_KRYLOV + 1)):
        with pytest.raises(B.PacesError) as e:
            B.Solver(**model, **dict(LAN_G, **bad))
        assert e.value.code == B.ERR_INVALID
    gpu = B.Solver(**model, **LAN_G)
    with pytest.raises(B.PacesError) as e:
        gpu.record(4)
    assert e.value.code == B.ERR_UNSUPPORTED
