"""Seeded synthetic workloads shared by the tests, the benchmark and the smoke check.

This module only *describes* inputs: model parameters, the initial state and the
random site energies of the disorder ensemble.  It contains none of the
method's arithmetic, and it imports nothing from the rest of the package or
from the oracle, so both sides can take their inputs from here.

The five workloads stand in for the paper's parameterised model runs (the 1D
Holstein benchmark of Sec. 4 and the 1D/2D/3D aggregates of Sec. 5): they are
Holstein models (Eq. holstein) with omega = 1 (time in 1/omega_0) and a hard
phonon cap per site.  Choices the paper leaves open (m, m_init, theta, the
boundary of the disorder chain, the start states) are fixed here, each beside
its workload.
"""
from __future__ import annotations

import math

import numpy as np

# lattice and coupling kinds of the C interface
RING, CHAIN, OPEN2D, OPEN3D, EXPLICIT = 0, 1, 2, 3, 4
NEAREST, DIPOLAR = 0, 1

WORKLOADS = {
    # 1D Holstein ring N=4, K=4 (full space 4*5^4 = 2500), checked against expm
    "ring4": dict(n_sites=4, lattice_kind=RING, dims=(4, 1, 1), coupling_kind=NEAREST,
                  J=1.0, omega=1.0, g=1.0, eps=0.0, cap=4, m=2, m_init=-1,
                  dt=0.05, nsteps=200, theta=1e-8, start="site0"),
    # 1D Holstein ring N=16, K=8, g=1.5 -- the throughput workload
    "ring16": dict(n_sites=16, lattice_kind=RING, dims=(16, 1, 1), coupling_kind=NEAREST,
                   J=1.0, omega=1.0, g=1.5, eps=0.0, cap=8, m=2, m_init=10,
                   dt=0.02, nsteps=1000, theta=1e-7, start="site0"),
    # 2D 6x6 aggregate, all-pairs J0/r^3 with J0 = -1, S = 1 (g = 1), K = 6.  theta = 1e-4:
    # at 1e-6 (and 1e-5) H_eff outgrows the 288 GB of one GPU within ~100 steps
    "dipolar6x6": dict(n_sites=36, lattice_kind=OPEN2D, dims=(6, 6, 1), coupling_kind=DIPOLAR,
                       J=-1.0, omega=1.0, g=1.0, eps=0.0, cap=6, m=2, m_init=6,
                       dt=0.05, nsteps=2048, theta=1e-4, start="bright"),
    # disorder ensemble: 256 rings of N=12 with eps ~ N(0, 0.5 J), seeds 1000 + r.
    # theta = 1e-4 (2.7e6 rows per realisation; 1e-6 gives 3.7e7, 9.5e9 for the ensemble)
    "disorder12": dict(n_sites=12, lattice_kind=RING, dims=(12, 1, 1), coupling_kind=NEAREST,
                       J=1.0, omega=1.0, g=1.0, eps=0.0, cap=6, m=2, m_init=10,
                       dt=0.05, nsteps=2048, theta=1e-4, start="bright",
                       realisations=256, eps_sigma=0.5, seed0=1000),
    # the paper's 1D Holstein benchmark at g = 4 (1D parameter table): open chain
    # N = 25, d_pho = 64 (K = 63), J = omega = 1, m_init = 10, m = 2, dt = 0.05 to
    # t = 50, top-q_nom truncation with q_nom = 32e6, a Franck-Condon excitation on
    # the centre site
    "chain25": dict(n_sites=25, lattice_kind=CHAIN, dims=(25, 1, 1), coupling_kind=NEAREST,
                    J=1.0, omega=1.0, g=4.0, eps=0.0, cap=63, m=2, m_init=10,
                    dt=0.05, nsteps=1000, theta=0.0, q_nom=32_000_000, start="center"),
    # 3D 4x4x4 open cube, nearest-neighbour J = 1, K = 4 -- the gradient workload.
    # theta = 1e-4 (1e-5 and 1e-6 outgrow one GPU before step 80)
    "cube4": dict(n_sites=64, lattice_kind=OPEN3D, dims=(4, 4, 4), coupling_kind=NEAREST,
                  J=1.0, omega=1.0, g=1.0, eps=0.0, cap=4, m=2, m_init=6,
                  dt=0.05, nsteps=400, theta=1e-4, start="bright", ckpt_every=20),
}


def model_kwargs(cfg, **over):
    """Keyword arguments describing the model (common to both implementations)."""
    c = dict(cfg)
    c.update(over)
    N = c["n_sites"]
    arr = lambda v: np.broadcast_to(np.asarray(v, dtype=np.float64), (N,)).copy()
    out = dict(n_sites=N, lattice_kind=c["lattice_kind"], dims=tuple(c["dims"]),
               coupling_kind=c["coupling_kind"], J=float(c["J"]), eps=arr(c["eps"]),
               omega=arr(c["omega"]), g=arr(c["g"]),
               cap=np.broadcast_to(np.asarray(c["cap"], dtype=np.int32), (N,)).copy(),
               m=int(c["m"]), m_init=int(c["m_init"]))
    if "xmax" in c:          # substep bound of the propagator (library default otherwise)
        out["xmax"] = float(c["xmax"])
    return out


def describe(cfg):
    """One-line description of a workload."""
    kinds = {RING: "ring", CHAIN: "open chain", OPEN2D: "open 2D", OPEN3D: "open 3D", EXPLICIT: "explicit"}
    geo = "x".join(str(d) for d in cfg["dims"] if d > 1) if cfg["lattice_kind"] in (OPEN2D, OPEN3D) \
        else "N=%d" % cfg["n_sites"]
    coup = "J0/r^3 all pairs" if cfg["coupling_kind"] == DIPOLAR else "nearest-neighbour"
    trunc = ("q_nom=%d" % cfg["q_nom"]) if "q_nom" in cfg else ("theta=%g" % cfg["theta"])
    return ("Holstein %s %s, %s J=%g omega=%g g=%g K=%d, dt=%g %s, start %s"
            % (kinds[cfg["lattice_kind"]], geo, coup, cfg["J"], cfg["omega"], cfg["g"], cfg["cap"],
               cfg["dt"], trunc, cfg["start"]))


def start_state(cfg):
    """psi(0) in A form: (site[n], occ[n, N], amps[n] complex)."""
    N = cfg["n_sites"]
    kind = cfg["start"]
    if kind == "site0":
        return (np.zeros(1, dtype=np.int32), np.zeros((1, N), dtype=np.int32),
                np.ones(1, dtype=np.complex128))
    if kind == "center":        # |N // 2, vac>: a localised Franck-Condon excitation
        return (np.array([N // 2], dtype=np.int32), np.zeros((1, N), dtype=np.int32),
                np.ones(1, dtype=np.complex128))
    if kind == "bright":        # sum_s |s, vac> / sqrt(N)  (Eq. init_state_spec)
        return (np.arange(N, dtype=np.int32), np.zeros((N, N), dtype=np.int32),
                np.full(N, 1.0 / math.sqrt(N), dtype=np.complex128))
    raise ValueError(kind)


# --- seeded random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) and the
# --- Box-Muller transform.  Plain Python integers, identical on every machine.
_M64 = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in (0, 1]."""
        return ((self.next_u64() >> 11) + 1) * (1.0 / 9007199254740992.0)

    def normal_pair(self):
        u1, u2 = self.uniform(), self.uniform()
        rad = math.sqrt(-2.0 * math.log(u1))
        return rad * math.cos(2.0 * math.pi * u2), rad * math.sin(2.0 * math.pi * u2)


def disorder_energies(n_sites: int, sigma: float, seed: int) -> np.ndarray:
    """Site energies eps_s ~ N(0, sigma) for one realisation (seed = seed0 + r)."""
    rng = SplitMix64(seed)
    out = []
    while len(out) < n_sites:
        a, b = rng.normal_pair()
        out.extend((a, b))
    return np.asarray(out[:n_sites], dtype=np.float64) * sigma


def realisation_eps(cfg, r: int) -> np.ndarray:
    return disorder_energies(cfg["n_sites"], cfg["eps_sigma"] * cfg["J"], cfg["seed0"] + r)


def seeded_normal(n: int, seed: int) -> np.ndarray:
    """n standard normal draws from the same generator (targets, probe vectors)."""
    rng = SplitMix64(seed)
    out = []
    while len(out) < n:
        out.extend(rng.normal_pair())
    return np.asarray(out[:n], dtype=np.float64)
