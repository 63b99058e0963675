"""Differentiable trajectories: the GPU solver as a torch.autograd.Function.

The forward runs the co-evolving-subspace propagation (Sec. 3, Eq. taylor) on
the GPU for a Holstein model (Eq. holstein) whose parameters come from a
tensor p = [J, g, omega, eps_0 .. eps_{N-1}] (g and omega shared by all
sites), and returns the autocorrelation C(t_k) = <psi(0)|psi(t_k)> as a real
(nsteps, 2) tensor and the site populations P_s(t_k) as an (nsteps, N) tensor,
k = 1 .. nsteps.  The backward calls the library's reverse pass
(paces_record / paces_backward): the gradient of the recorded map, with the
subspace sequence and Taylor term counts held at their forward values.  Every
step of both passes runs in the CUDA library; this module only marshals
arguments.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B
from .analysis import INV_TAU


def _model(base: dict, p: np.ndarray) -> dict:
    N = int(base["n_sites"])
    m = dict(base)
    m["J"] = float(p[0])
    m["g"] = np.full(N, float(p[1]))
    m["omega"] = np.full(N, float(p[2]))
    m["eps"] = np.asarray(p[3:3 + N], dtype=np.float64).copy()
    return m


class Trajectory(torch.autograd.Function):
    """(p, model, start, dt, nsteps, theta, ckpt_every) -> (C, P)."""

    @staticmethod
    def forward(ctx, p, model, start, dt, nsteps, theta, ckpt_every):
        pv = p.detach().to("cpu", torch.float64).numpy()
        N = int(model["n_sites"])
        if pv.shape != (3 + N,):
            raise ValueError("p must hold 3 + n_sites values")
        solver = B.Solver(**_model(model, pv))
        solver.record(int(ckpt_every))
        solver.set_state(*start)
        solver.step(float(dt), int(nsteps), float(theta))
        rec = solver.observables(1, int(nsteps))
        C = np.ascontiguousarray(rec[:, [B.OBS_FIELDS.index("C_re"), B.OBS_FIELDS.index("C_im")]])
        P = np.ascontiguousarray(rec[:, B.OBS_FIXED:B.OBS_FIXED + N])
        ctx.solver = solver
        ctx.nsteps = int(nsteps)
        ctx.device = p.device
        return (torch.from_numpy(C).to(p.device), torch.from_numpy(P).to(p.device))

    @staticmethod
    def backward(ctx, gC, gP):
        solver = ctx.solver
        dC = None
        if gC is not None:
            g = gC.detach().to("cpu", torch.float64).numpy()
            dC = g[:, 0] + 1j * g[:, 1]
        dP = None if gP is None else gP.detach().to("cpu", torch.float64).numpy()
        grad = solver.backward(ctx.nsteps, dL_dC=dC, dL_dP=dP)
        solver.close()
        ctx.solver = None
        return torch.from_numpy(grad).to(ctx.device), None, None, None, None, None, None


def trajectory(p: torch.Tensor, model: dict, start, dt: float, nsteps: int, theta: float, ckpt_every: int = 20):
    """C (nsteps, 2) and P (nsteps, N) after each of nsteps steps, differentiable in p."""
    return Trajectory.apply(p, model, start, dt, nsteps, theta, ckpt_every)


def spectrum(C: torch.Tensor, c0: complex, dt: float, omega, inv_tau: float = INV_TAU) -> torch.Tensor:
    """Differentiable absorption spectrum A(w) = Re sum_k w_k C(t_k) e^{i w t_k}
    e^{-t_k / tau} dt over t_k = k dt, k = 0..K (trapezoid weights w_k: 1/2 at
    both ends), from C (K, 2) after steps 1..K and C(0) = c0 = <psi(0)|psi(0)>
    (the aggregates section; damping from the appendix on quantum jumps)."""
    K = C.shape[0]
    dev, dt_ = C.device, torch.float64
    t = dt * torch.arange(K + 1, device=dev, dtype=dt_)
    w = torch.ones(K + 1, device=dev, dtype=dt_)
    w[0] = w[-1] = 0.5
    damp = w * torch.exp(-t * inv_tau) * dt
    re = torch.cat([torch.tensor([float(np.real(c0))], device=dev, dtype=dt_), C[:, 0]])
    im = torch.cat([torch.tensor([float(np.imag(c0))], device=dev, dtype=dt_), C[:, 1]])
    om = torch.as_tensor(np.asarray(omega, dtype=np.float64), device=dev)
    ph = om[:, None] * t[None, :]
    # Re[(re + i im) (cos + i sin)] = re cos - im sin
    return (torch.cos(ph) * (re * damp)[None, :] - torch.sin(ph) * (im * damp)[None, :]).sum(1)


def population_spectrum_loss(p: torch.Tensor, model: dict, start, dt: float, nsteps: int, theta: float,
                             omega, A_target: torch.Tensor, ckpt_every: int = 20, site: int = 0) -> torch.Tensor:
    """L = P_site(T) + mean_w (A(w) - A_target(w))^2: the population of one
    site at the end plus the mean squared deviation of the absorption spectrum
    from a target, differentiable in p = [J, g, omega, eps_0 .. eps_{N-1}]."""
    C, P = trajectory(p, model, start, dt, nsteps, theta, ckpt_every)
    a = np.asarray(start[2], dtype=np.complex128)
    A = spectrum(C, complex(np.vdot(a, a)), dt, omega)
    return P[-1, site] + torch.mean((A - A_target) ** 2)


def seeded_target(model: dict, start, dt: float, nsteps: int, theta: float, omega, p0: np.ndarray,
                  rel: float = 0.05, seed: int = 12345):
    """Target spectrum for population_spectrum_loss: the spectrum of a forward
    run at parameters p0 (1 + rel z), z seeded normal draws, so that the loss
    has its minimum near, not at, p0."""
    from .workloads import seeded_normal
    pt = np.asarray(p0, dtype=np.float64) * (1.0 + rel * seeded_normal(len(p0), seed))
    sol = B.Solver(**_model(model, pt))
    try:
        sol.set_state(*start)
        sol.step(float(dt), int(nsteps), float(theta))
        rec = sol.observables(1, int(nsteps))
    finally:
        sol.close()
    C = torch.from_numpy(np.ascontiguousarray(rec[:, [B.OBS_FIELDS.index("C_re"), B.OBS_FIELDS.index("C_im")]]))
    a = np.asarray(start[2], dtype=np.complex128)
    return spectrum(C, complex(np.vdot(a, a)), dt, omega).detach()
