"""Host post-processing of observables records.

absorption_spectrum: the linear absorption spectrum of an aggregate from the
    autocorrelation C(t) = <psi(0)|psi(t)> of the bright state (Eq.
    init_state_spec; the section on aggregates: A(w) proportional to the real
    part of the Fourier transform of <mu(t) mu(0)>), damped by e^{-t/tau} with
    1/tau = 0.0577 omega_0 (the appendix on quantum jumps), trapezoid weights
    on the step grid.
rmsd: the root-mean-square deviation of the exciton position (Eq. RMSD, read
    as the standard deviation of the position distribution P_s, normalised by
    sum_s P_s because truncation lowers the norm).
"""
from __future__ import annotations

import numpy as np

INV_TAU = 0.0577        # 1/tau in units of omega_0


def absorption_spectrum(C, dt, omega, inv_tau=INV_TAU):
    """A(w) = Re sum_k c_k C(t_k) e^{i w t_k} e^{-t_k / tau} dt, t_k = k dt, k = 0..K,
    c_k = 1/2 at both ends and 1 elsewhere.  C[k] is the record after step k
    (C[0] = 1 for a normalised psi(0)); for an ensemble pass the mean over
    realisations (the records' fixed C field)."""
    C = np.asarray(C, dtype=np.complex128).reshape(-1)
    omega = np.asarray(omega, dtype=np.float64).reshape(-1)
    K = len(C) - 1
    t = dt * np.arange(K + 1)
    c = np.ones(K + 1)
    if K > 0:
        c[0] = c[-1] = 0.5
    f = c * C * np.exp(-t * inv_tau) * dt
    return np.real(np.exp(1j * np.outer(omega, t)) @ f)


def rmsd(P, x=None):
    """sqrt(sum_s P_s (x_s - X)^2 / sum_s P_s), X = sum_s x_s P_s / sum_s P_s, for
    P of shape (..., N); x defaults to the positions 0..N-1 of a chain."""
    P = np.asarray(P, dtype=np.float64)
    x = np.arange(P.shape[-1], dtype=np.float64) if x is None else np.asarray(x, dtype=np.float64)
    norm = P.sum(-1)
    X = (P * x).sum(-1) / norm
    return np.sqrt((P * (x - X[..., None]) ** 2).sum(-1) / norm)
