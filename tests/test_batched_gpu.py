"""Static-disorder ensembles evolved as one batched problem (the realisation
index is one more key digit).  Each realisation must match, row for row and in
order, the oracle run with that realisation's site energies, and its
observables must match the oracle's."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2603_07341_gb300 import binding as B
from paper_2603_07341_gb300 import workloads as W

pytestmark = pytest.mark.gpu
AMP_TOL = 1e-10


def ensemble(R, **over):
    cfg = W.WORKLOADS["disorder12"]
    eps = np.stack([W.realisation_eps(cfg, r) for r in range(R)])
    model = W.model_kwargs(cfg, **over)
    gb = B.Solver(**dict(model, eps=eps, batch=R))
    oras = [Oracle(**dict(model, eps=eps[r])) for r in range(R)]
    st = W.start_state(cfg)
    gb.set_state(*st)
    for o in oras:
        o.set_state(*st)
    return cfg, gb, oras


def split(gb):
    t, a = gb.tuples()
    return t[:, :-1], t[:, -1], a


def compare(gb, oras, R, N):
    t, real, a = split(gb)
    rec = B.records_dict(gb.observables(gb.num_records() - 1, 1), N, R)
    for r in range(R):
        sel = real == r
        to, ao = oras[r].rows()
        assert np.array_equal(t[sel], to), "realisation %d: rows differ" % r
        assert np.max(np.abs(a[sel] - ao)) <= AMP_TOL * np.linalg.norm(ao)
        st = oras[r].stats()
        P, nb = oras[r].populations()
        assert np.max(np.abs(rec["P"][0, r] - P)) <= 1e-10
        assert np.max(np.abs(rec["nbar"][0, r] - nb)) <= 1e-9
        assert abs(rec["C_r"][0, r] - (st["C_re"] + 1j * st["C_im"])) <= 1e-10


def test_ensemble_matches_oracle_per_realisation(libpaces):
    R, theta = 5, 1e-4
    cfg, gb, oras = ensemble(R, m_init=4)
    N = cfg["n_sites"]
    compare(gb, oras, R, N)
    for k in range(16):
        _, real_before, _ = split(gb)
        befores = [o.rows()[1] for o in oras]
        gb.step(cfg["dt"], 1, theta)
        keep = gb.keep()
        for r in range(R):
            kr = keep[real_before == r] if len(keep) else None
            a = befores[r]
            if kr is None:
                oras[r].step(cfg["dt"], theta)
                continue
            w = a.real * a.real + a.imag * a.imag
            diff = kr != (w >= theta * theta)
            if diff.any():
                band = np.abs(w - theta * theta) <= 1e-9 * theta * theta + 1e-10 * np.sum(w)
                assert np.all(band[diff])
                oras[r].step(cfg["dt"], theta, keep=kr.astype(np.uint8))
            else:
                oras[r].step(cfg["dt"], theta)
        if k % 5 == 4 or k == 15:
            compare(gb, oras, R, N)


def test_ensemble_equals_single_runs_on_the_gpu(libpaces):
    """Realisation r of the ensemble evolves exactly like a single run with
    eps^(r): same rows in the same order, amplitudes equal to the series
    tolerance (the ensemble stops its series on the ensemble's norms)."""
    R, theta, steps = 3, 1e-4, 12
    cfg, gb, _ = ensemble(R, m_init=4)
    gb.step(cfg["dt"], steps, theta)
    t, real, a = split(gb)
    for r in range(R):
        s = B.Solver(**W.model_kwargs(cfg, m_init=4, eps=W.realisation_eps(cfg, r)))
        s.set_state(*W.start_state(cfg))
        s.step(cfg["dt"], steps, theta)
        ts, as_ = s.tuples()
        sel = real == r
        assert np.array_equal(t[sel], ts)
        assert np.max(np.abs(a[sel] - as_)) <= 1e-13
