"""Piecewise-constant time-dependent Hamiltonians on the GPU (the extension of
Sec. 6: the Hamiltonian is adjusted at every time step, its coupling magnitudes
changing and its graph fixed), in lockstep with the oracle, whose updates are
pinned to the product of dense exponentials and to the global phase of a
uniform site-energy drive.  Steps after the first replay a captured CUDA graph,
so these tests also check that replays read the replaced coefficients."""
import math

import numpy as np
import pytest

from paper_2603_07341_gb300 import binding as B
from paper_2603_07341_gb300 import workloads as W
from tests.test_parity_gpu import compare_record, compare_state, make_pair

pytestmark = pytest.mark.gpu


def _drive(t, N):
    J = 1.0 + 0.3 * math.sin(1.3 * t)
    eps = 0.2 * np.cos(0.7 * t + np.arange(N))
    omega = np.full(N, 1.0 + 0.1 * math.sin(t))
    g = np.full(N, 1.0 + 0.2 * math.cos(t))
    return J, eps, omega, g


def _lockstep_driven(gpu, ora, dt, theta, nsteps, N):
    """Both sides take the same coefficients before every step; truncation
    decisions may differ only within the rounding band at the threshold
    (the oracle then adopts the GPU's), as in the undriven lockstep."""
    for k in range(nsteps):
        J, eps, omega, g = _drive(k * dt, N)
        gpu.set_coefficients(J, eps, omega, g)
        ora.set_coefficients(J, eps, omega, g)
        _, a_before = ora.rows()
        gpu.step(dt, 1, theta)
        gkeep = gpu.keep()
        keep = None
        if len(gkeep):
            w = a_before.real ** 2 + a_before.imag ** 2
            diff = gkeep != (w >= theta * theta)
            band = np.abs(w - theta * theta) <= 1e-9 * theta * theta + 1e-10 * np.sum(w)
            assert np.all(band[diff]), "truncation differs outside the rounding band"
            if diff.any():
                keep = gkeep.astype(np.uint8)
        ora.step(dt, theta, keep=keep)
        compare_state(gpu, ora)
        compare_record(gpu.observables(gpu.num_records() - 1, 1)[0], ora, N)


@pytest.mark.parametrize("precision", [B.C128, B.DW], ids=["c128", "dw"])
def test_driven_ring4_lockstep(libpaces, precision):
    cfg = W.WORKLOADS["ring4"]
    gpu, ora = make_pair(cfg, gpu_extra=dict(precision=precision))
    st = W.start_state(cfg)
    gpu.set_state(*st)
    ora.set_state(*st)
    _lockstep_driven(gpu, ora, cfg["dt"], cfg["theta"], 60, 4)


def test_driven_ring16_prefix_lockstep(libpaces):
    cfg = W.WORKLOADS["ring16"]
    gpu, ora = make_pair(cfg)
    st = W.start_state(cfg)
    gpu.set_state(*st)
    ora.set_state(*st)
    _lockstep_driven(gpu, ora, cfg["dt"], cfg["theta"], 30, 16)


def test_driven_ensemble_realisations(libpaces):
    """Ensembles take R x N site energies; each realisation follows its own
    oracle run."""
    cfg = W.WORKLOADS["disorder12"]
    R, N = 3, cfg["n_sites"]
    eps0 = np.stack([W.realisation_eps(cfg, r) for r in range(R)])
    model = W.model_kwargs(cfg)
    model.update(batch=R, eps=eps0)
    gpu = B.Solver(**model)
    from oracle.oracle import Oracle
    oras = [Oracle(**W.model_kwargs(cfg, eps=eps0[r])) for r in range(R)]
    st = W.start_state(cfg)
    gpu.set_state(*st)
    for o in oras:
        o.set_state(*st)
    for k in range(8):
        shift = 0.3 * math.cos(0.9 * k * cfg["dt"])
        gpu.set_coefficients(cfg["J"], eps=eps0 + shift)
        for r, o in enumerate(oras):
            o.set_coefficients(cfg["J"], eps=eps0[r] + shift)
        gpu.step(cfg["dt"], 1, cfg["theta"])
        for o in oras:
            o.step(cfg["dt"], cfg["theta"])
    tg, ag = gpu.tuples()
    for r, o in enumerate(oras):
        sel = tg[:, -1] == r
        to, ao = o.rows()
        assert np.array_equal(tg[sel][:, :-1], to)
        assert np.max(np.abs(ag[sel] - ao)) <= 1e-10 * np.linalg.norm(ao)


def test_unchanged_coefficients_leave_the_trajectory_bitwise(libpaces):
    cfg = W.WORKLOADS["ring16"]
    model = W.model_kwargs(cfg)
    a, b = B.Solver(**model), B.Solver(**model)
    st = W.start_state(cfg)
    for s in (a, b):
        s.set_state(*st)
    for _ in range(12):
        b.set_coefficients(cfg["J"], model["eps"], model["omega"], model["g"])
        a.step(cfg["dt"], 1, cfg["theta"])
        b.step(cfg["dt"], 1, cfg["theta"])
    ta, aa = a.tuples()
    tb, ab = b.tuples()
    assert np.array_equal(ta, tb) and np.array_equal(aa, ab)


def test_coefficient_updates_keep_the_move_graph(libpaces):
    cfg = W.WORKLOADS["ring4"]
    gpu = B.Solver(**W.model_kwargs(cfg))
    for J, g in ((0.0, None), (1.0, [1.0, 0.0, 1.0, 1.0]), (float("inf"), None)):
        with pytest.raises(B.PacesError) as e:
            gpu.set_coefficients(J, g=g)
        assert e.value.code == B.ERR_INVALID
    gpu.record(4)
    with pytest.raises(B.PacesError) as e:
        gpu.set_coefficients(0.5)
    assert e.value.code == B.ERR_UNSUPPORTED
