"""Host post-processing against the oracle's spectrum and closed forms."""
import numpy as np
import pytest

from oracle.oracle import absorption_spectrum as oracle_spectrum
from paper_2603_07341_gb300 import analysis as A
from paper_2603_07341_gb300 import workloads as W


def test_spectrum_matches_the_oracle():
    C = W.seeded_normal(402, 5).reshape(201, 2) @ np.array([1.0, 1j])
    grid = np.linspace(-3.0, 3.0, 25)
    assert np.allclose(A.absorption_spectrum(C, 0.05, grid), oracle_spectrum(C, 0.05, grid), atol=1e-12)


def test_spectrum_of_a_single_line_peaks_at_its_energy():
    """C(t) = e^{-i E t}: a Lorentzian of half width 1/tau at E."""
    E, dt, K = 0.7, 0.05, 4000
    C = np.exp(-1j * E * dt * np.arange(K + 1))
    grid = np.linspace(0.0, 1.4, 701)
    a = A.absorption_spectrum(C, dt, grid)
    assert abs(grid[np.argmax(a)] - E) <= 0.002
    half = a >= a.max() / 2
    width = grid[half].max() - grid[half].min()
    assert abs(width - 2 * A.INV_TAU) < 0.01


def test_rmsd_closed_forms():
    P = np.zeros((3, 5))
    P[0, 2] = 1.0                      # localised: 0
    P[1, 0] = P[1, 4] = 0.5            # two sites 4 apart, equal weight: 2
    P[2] = 0.2 * 0.9                   # uniform (norm 0.9): sqrt(2) for positions 0..4
    r = A.rmsd(P)
    assert np.allclose(r, [0.0, 2.0, np.sqrt(2.0)])
    assert np.allclose(A.rmsd(P[1], x=[0, 1, 2, 3, 8]), 4.0)


def test_differentiable_spectrum_equals_host_spectrum():
    """The torch spectrum of the autograd path and the host post-processing
    agree (same trapezoid weights, damping and sign convention)."""
    torch = pytest.importorskip("torch")
    from paper_2603_07341_gb300.autograd import spectrum
    from paper_2603_07341_gb300.analysis import absorption_spectrum
    K, dt = 64, 0.05
    k = np.arange(1, K + 1)
    C = np.exp(-0.7j * k * dt) * (1.0 - 0.004 * k) + 0.1 * np.exp(1.3j * k * dt)
    om = np.linspace(-6.0, 6.0, 257)
    A = spectrum(torch.from_numpy(np.stack([C.real, C.imag], 1)), 1.1, dt, om).numpy()
    ref = absorption_spectrum(np.concatenate([[1.1], C]), dt, om)
    assert np.max(np.abs(A - ref)) <= 1e-13
