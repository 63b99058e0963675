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
