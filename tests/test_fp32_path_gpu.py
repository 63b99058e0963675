"""The complex64-SpMV propagator (PACES_C64_SPMV) against the plain FP64
single-instance form (PACES_C128, complex128 as in the paper) on the same GPU,
and against the FP64 oracle.  The terms of a series from two after the first
one below 2^-16 of the state's norm run in FP32 (never before term 3); the
leading terms, the accumulator, norms and truncation magnitudes stay
double-word.  Stated
bound: every observable (site populations P_s, phonon numbers <n_j>, the
autocorrelation C(t), the norm and the energy) within 1e-6 of the FP64 result
at every step of the horizon tested."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2603_07341_gb300 import binding as B
from paper_2603_07341_gb300 import workloads as W

pytestmark = pytest.mark.gpu
OBS_TOL = 1e-6


def run(cfg, precision, nsteps, theta, **over):
    s = B.Solver(**W.model_kwargs(cfg, **over), precision=precision)
    s.set_state(*W.start_state(cfg))
    s.step(cfg["dt"], nsteps, theta)
    return s


@pytest.mark.parametrize("name,over,nsteps,theta", [
    ("dipolar6x6", {"m_init": 2}, 60, 1e-5),
    ("ring16", {}, 120, 1e-7),
    ("cube4", {"m_init": 2}, 20, 1e-5),
    ("disorder12", {"eps": W.realisation_eps(W.WORKLOADS["disorder12"], 3)}, 80, 1e-5),
])
def test_c64_observables_within_1e6_of_fp64(libpaces, name, over, nsteps, theta):
    cfg = W.WORKLOADS[name]
    a = run(cfg, B.C128, nsteps, theta, **over)
    b = run(cfg, B.C64_SPMV, nsteps, theta, **over)
    ra = B.records_dict(a.observables(), cfg["n_sites"])
    rb = B.records_dict(b.observables(), cfg["n_sites"])
    for key in ("P", "nbar", "C", "norm", "energy"):
        err = np.max(np.abs(ra[key] - rb[key]))
        assert err <= OBS_TOL, (key, err)
    assert np.all(np.abs(ra["rows"] - rb["rows"]) <= 0.01 * ra["rows"])


def test_c64_observables_against_oracle(libpaces):
    """40 ring16 steps on the GPU in complex64 terms and in the oracle (FP64),
    each on its own: every observable within 1e-6 after every step.  Rows whose
    truncation decision flips between the two carry weight of order theta^2."""
    cfg = W.WORKLOADS["ring16"]
    model = W.model_kwargs(cfg)
    g = B.Solver(**model, precision=B.C64_SPMV)
    o = Oracle(**model)
    g.set_state(*W.start_state(cfg))
    o.set_state(*W.start_state(cfg))
    N = cfg["n_sites"]
    for k in range(40):
        g.step(cfg["dt"], 1, cfg["theta"])
        o.step(cfg["dt"], cfg["theta"])
        r = B.records_dict(g.observables(k + 1, 1), N)
        st = o.stats()
        P, nb = o.populations()
        assert np.max(np.abs(r["P"][0] - P)) <= OBS_TOL
        assert np.max(np.abs(r["nbar"][0] - nb)) <= OBS_TOL
        assert abs(r["C"][0] - (st["C_re"] + 1j * st["C_im"])) <= OBS_TOL
        assert abs(r["norm"][0] - st["norm"]) <= OBS_TOL
        assert abs(r["energy"][0] - st["energy"]) <= OBS_TOL * max(1.0, abs(st["energy"]))


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
