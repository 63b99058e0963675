"""Python side of the CPU oracle (test infrastructure only).

Only the test suite, the package smoke check and the benchmark's CPU-baseline
leg import this module.  It wraps ``paces_oracle.c`` (plain FP64 C, compiled
here with gcc) and adds the host-side post-processing the paper applies to the
autocorrelation signal.  Nothing in it is shared with the CUDA product path.

Paper: paces, arXiv 2603.07341.  Model Eq. holstein; neighbour sets Eqs.
def_neighbor / def_neighbor_k / H_eff; step map of Sec. 3.4; Taylor propagator
App. C.1; spectrum from the damped autocorrelation (Sec. aggregates, App. E).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "paces_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

OR_OK, OR_INVALID, OR_NOMEM, OR_NOCONVERGE, OR_STATE = 0, 1, 3, 4, 6
ST_NAMES = ("norm", "norm_phi0", "energy", "C_re", "C_im", "rows", "kept", "nnz",
            "terms", "norm_before", "time", "substeps", "hbound")


MUTANTS = ("NO_RESCUE", "OPEN3D_AXES", "ENERGY_CONJ", "LANCZOS_NO_BETA")


def build_oracle(force: bool = False, mutant: str | None = None) -> str:
    """Compile the oracle with gcc (-ffp-contract=off: no FMA contraction).

    mutant: one of MUTANTS, for the pin tests only -- a second library with
    that planted mistake compiled in (the default build has none)."""
    lib = _LIB if mutant is None else _LIB.replace("liboracle.so", "liboracle_%s.so" % mutant.lower())
    if mutant is not None and mutant not in MUTANTS:
        raise ValueError(mutant)
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "paces_oracle.h"))):
        return lib
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared"]
    if mutant is not None:
        cmd.append("-DOR_MUTANT_%s" % mutant)
    subprocess.run(cmd + ["-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, lib)
    return lib


_libs = {}


def _load(mutant=None):
    if mutant not in _libs:
        lib = C.CDLL(build_oracle(mutant=mutant))
        P = C.c_void_p
        dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
        lib.or_create.restype = P
        lib.or_create.argtypes = [C.c_int, C.c_int, ip, C.c_int, C.c_double, dp, dp, dp, dp,
                                  ip, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int]
        lib.or_destroy.argtypes = [P]
        lib.or_set_xmax.argtypes = [P, C.c_double]
        lib.or_set_propagator.argtypes = [P, C.c_int, C.c_int]
        lib.or_last_krylov.argtypes = [P, dp, C.c_int]
        lib.or_set_coefficients.argtypes = [P, C.c_double, dp, dp, dp]
        lib.or_get_hopping.argtypes = [P, dp]
        lib.or_set_state.argtypes = [P, C.c_int, ip, ip, dp]
        lib.or_load_state.argtypes = [P, C.c_int, ip, ip, dp]
        lib.or_step.argtypes = [P, C.c_double, C.c_double, C.POINTER(C.c_ubyte), C.c_int]
        lib.or_step_nom.argtypes = [P, C.c_double, C.c_longlong, C.c_ulonglong]
        lib.or_nom_keep.argtypes = [P, C.c_longlong, C.c_ulonglong, C.POINTER(C.c_ubyte)]
        lib.or_tie_hash.restype = C.c_ulonglong
        lib.or_tie_hash.argtypes = [C.c_ulonglong, C.c_longlong, C.POINTER(C.c_int), C.c_int]
        lib.or_nrows.argtypes = [P]
        lib.or_get_rows.argtypes = [P, ip, dp]
        lib.or_level_offsets.argtypes = [P, ip, C.c_int]
        lib.or_last_keep.argtypes = [P, C.POINTER(C.c_ubyte), C.c_int]
        lib.or_build_hamiltonian.restype = C.c_long
        lib.or_build_hamiltonian.argtypes = [P, ip, ip, dp, dp]
        lib.or_stats.argtypes = [P, dp]
        lib.or_populations.argtypes = [P, dp, dp]
        lib.or_record.argtypes = [P, C.c_int]
        lib.or_backward.argtypes = [P, C.c_int, dp, dp, dp, dp]
        _libs[mutant] = lib
    return _libs[mutant]


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int)) if a is not None else None


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s failed with oracle status %d" % (what, code))
        self.code = code


class Oracle:
    """One FP64 instance of the co-evolving-subspace solver on the CPU.

    Parameters follow Eq. holstein: ``eps``, ``omega``, ``g`` per site, phonon
    caps ``cap`` (K_j = d_pho - 1), hopping ``J`` times the lattice pattern
    (ring / open chain / open 2D / open 3D nearest neighbour, or all pairs
    J / r^3).  ``m`` and ``m_init`` are the neighbour orders of Eq. H_eff
    (``m_init < 0``: closure).  ``xmax`` bounds rho dt / s, the length of each
    of the s Taylor series a step is split into (rho: largest absolute row sum
    of H over H_eff; ``xmax <= 0``: one series).  ``propagator`` 0 is the Taylor series
    (App. C.1), 1 the Lanczos decomposition (App. C.3) with at most ``kmax`` Krylov
    vectors per series.  ``mutant`` (pin tests only) selects a build with one planted
    mistake, see ``MUTANTS``.
    """

    def __init__(self, n_sites, lattice_kind=0, dims=(0, 0, 0), coupling_kind=0, J=1.0,
                 eps=None, omega=None, g=None, cap=None, m=2, m_init=10, tol=1e-15,
                 nmax=200, fixed_terms=0, J_explicit=None, xmax=8.0, propagator=0, kmax=30,
                 mutant=None):
        lib = _load(mutant)
        self.N = int(n_sites)
        N = self.N
        f = lambda v, d: np.ascontiguousarray(np.broadcast_to(
            np.asarray(d if v is None else v, dtype=np.float64), (N,)))
        self._eps, self._omega, self._g = f(eps, 0.0), f(omega, 1.0), f(g, 0.0)
        self._cap = np.ascontiguousarray(np.broadcast_to(
            np.asarray(4 if cap is None else cap, dtype=np.int32), (N,)))
        self._dims = np.asarray(list(dims) + [0] * (3 - len(dims)), dtype=np.int32)
        jx = None if J_explicit is None else np.ascontiguousarray(J_explicit, dtype=np.float64)
        self._h = lib.or_create(N, int(lattice_kind), _ip(self._dims), int(coupling_kind),
                                float(J), _dp(jx), _dp(self._eps), _dp(self._omega),
                                _dp(self._g), _ip(self._cap), int(m), int(m_init),
                                float(tol), int(nmax), int(fixed_terms))
        if not self._h:
            raise OracleError(OR_INVALID, "or_create")
        self._lib = lib
        lib.or_set_xmax(self._h, float(xmax))
        rc = lib.or_set_propagator(self._h, int(propagator), int(kmax))
        if rc:
            raise OracleError(rc, "or_set_propagator")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.or_destroy(h)
            self._h = None

    def set_coefficients(self, J, eps=None, omega=None, g=None):
        """Replace H's values between steps (piecewise-constant time dependence);
        the move graph is fixed (zeros of J and g stay zeros)."""
        f = lambda v: None if v is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(v, dtype=np.float64), (self.N,)))
        e, w, gg = f(eps), f(omega), f(g)
        rc = self._lib.or_set_coefficients(self._h, float(J), _dp(e), _dp(w), _dp(gg))
        if rc:
            raise OracleError(rc, "or_set_coefficients")

    def krylov_basis(self):
        """Lanczos vectors v_1..v_n of the last series of the last Lanczos step, [q, n]."""
        n = self._lib.or_last_krylov(self._h, None, 0)
        q = self.nrows()
        buf = np.zeros(2 * q * max(n, 1))
        self._lib.or_last_krylov(self._h, _dp(buf), n)
        v = buf[0::2] + 1j * buf[1::2]
        return v[: q * n].reshape(n, q).T.copy()

    def hopping(self):
        out = np.zeros((self.N, self.N))
        self._lib.or_get_hopping(self._h, _dp(out))
        return out

    def set_state(self, site, occ, amps):
        site = np.ascontiguousarray(site, dtype=np.int32)
        occ = np.ascontiguousarray(occ, dtype=np.int32).reshape(len(site), self.N)
        a = np.asarray(amps, dtype=np.complex128)
        ri = np.ascontiguousarray(np.stack([a.real, a.imag], 1).reshape(-1))
        rc = self._lib.or_set_state(self._h, len(site), _ip(site), _ip(occ), _dp(ri))
        if rc:
            raise OracleError(rc, "or_set_state")

    def load_state(self, site, occ, amps):
        """A mid-trajectory state taken as the current H_eff and vector."""
        site = np.ascontiguousarray(site, dtype=np.int32)
        occ = np.ascontiguousarray(occ, dtype=np.int32).reshape(len(site), self.N)
        a = np.asarray(amps, dtype=np.complex128)
        ri = np.ascontiguousarray(np.stack([a.real, a.imag], 1).reshape(-1))
        rc = self._lib.or_load_state(self._h, len(site), _ip(site), _ip(occ), _dp(ri))
        if rc:
            raise OracleError(rc, "or_load_state")

    def step(self, dt, theta, keep=None):
        kp, kl = None, 0
        if keep is not None:
            kb = np.ascontiguousarray(keep, dtype=np.uint8)
            kp, kl = kb.ctypes.data_as(C.POINTER(C.c_ubyte)), len(kb)
        rc = self._lib.or_step(self._h, float(dt), float(theta), kp, kl)
        if rc:
            raise OracleError(rc, "or_step")

    def step_nom(self, dt, q_nom, seed=0):
        """One step with top-q_nom truncation (seeded tie-break of equal weights)."""
        rc = self._lib.or_step_nom(self._h, float(dt), int(q_nom), int(seed) & ((1 << 64) - 1))
        if rc:
            raise OracleError(rc, "or_step_nom")

    def nom_keep(self, q_nom, seed=0):
        """Keep mask a top-q_nom step would apply to the current rows."""
        out = np.zeros(max(self.nrows(), 1), dtype=np.uint8)
        rc = self._lib.or_nom_keep(self._h, int(q_nom), int(seed) & ((1 << 64) - 1),
                                   out.ctypes.data_as(C.POINTER(C.c_ubyte)))
        if rc:
            raise OracleError(rc, "or_nom_keep")
        return out[: self.nrows()].astype(bool)

    def tie_hash(self, seed, t, tuple_):
        a = np.ascontiguousarray(tuple_, dtype=np.int32)
        return int(self._lib.or_tie_hash(int(seed) & ((1 << 64) - 1), int(t), _ip(a), len(a)))

    def nrows(self):
        return self._lib.or_nrows(self._h)

    def rows(self):
        q = self.nrows()
        t = np.zeros((q, self.N + 1), dtype=np.int32)
        a = np.zeros(2 * q)
        self._lib.or_get_rows(self._h, _ip(t), _dp(a))
        return t, a[0::2] + 1j * a[1::2]

    def level_offsets(self):
        buf = np.zeros(4096, dtype=np.int32)
        n = self._lib.or_level_offsets(self._h, _ip(buf), len(buf))
        return buf[:n].copy()

    def last_keep(self):
        n = self._lib.or_last_keep(self._h, None, 0)
        buf = np.zeros(max(n, 1), dtype=np.uint8)
        self._lib.or_last_keep(self._h, buf.ctypes.data_as(C.POINTER(C.c_ubyte)), n)
        return buf[:n].astype(bool)

    def hamiltonian(self):
        """(cnt[q], cols, vals, diag[q]) of P H P, entries of a row in move order."""
        nnz = self._lib.or_build_hamiltonian(self._h, None, None, None, None)
        q = self.nrows()
        cnt = np.zeros(q, dtype=np.int32)
        cols = np.zeros(max(nnz, 1), dtype=np.int32)
        vals = np.zeros(max(nnz, 1))
        diag = np.zeros(max(q, 1))
        self._lib.or_build_hamiltonian(self._h, _ip(cnt), _ip(cols), _dp(vals), _dp(diag))
        return cnt, cols[:nnz], vals[:nnz], diag[:q]

    def stats(self):
        st = np.zeros(len(ST_NAMES))
        self._lib.or_stats(self._h, _dp(st))
        return dict(zip(ST_NAMES, st))

    def populations(self):
        P, nb = np.zeros(self.N), np.zeros(self.N)
        self._lib.or_populations(self._h, _dp(P), _dp(nb))
        return P, nb

    def record(self, on=True):
        self._lib.or_record(self._h, 1 if on else 0)

    def backward(self, nsteps, dL_dc_final=None, dL_dC=None, dL_dP=None):
        """Gradient [J, g, omega, eps_0..eps_{N-1}] of a loss of the recorded steps.

        dL_dc_final: complex cotangent on the final rows (dL = Re(conj(g) dc));
        dL_dC: complex dL/dRe C_k + i dL/dIm C_k for recorded steps k = 0..nsteps-1;
        dL_dP: real dL/dP_s(t_k), shape (nsteps, N), of the site populations.
        """
        def ri(z):
            if z is None:
                return None
            z = np.asarray(z, dtype=np.complex128)
            return np.ascontiguousarray(np.stack([z.real, z.imag], 1).reshape(-1))
        a, b = ri(dL_dc_final), ri(dL_dC)
        p = None if dL_dP is None else np.ascontiguousarray(dL_dP, dtype=np.float64).reshape(-1)
        if p is not None and p.size != int(nsteps) * self.N:
            raise ValueError("dL_dP must hold nsteps * N values")
        grad = np.zeros(3 + self.N)
        rc = self._lib.or_backward(self._h, int(nsteps), _dp(a), _dp(b), _dp(p), _dp(grad))
        if rc:
            raise OracleError(rc, "or_backward")
        return grad


def absorption_spectrum(C_t, dt, omega_grid, inv_tau=0.0577):
    """A(w) = Re sum_k w_k C(t_k) exp(i w t_k) exp(-t_k / tau) dt, trapezoid weights.

    C_t[k] is the autocorrelation at t_k = k dt, k = 0..K (Sec. aggregates; the
    damping e^{-t/tau} with 1/tau = 0.0577 omega_0 of App. E).  Plain double loop.
    """
    C_t = np.asarray(C_t, dtype=np.complex128)
    K = len(C_t) - 1
    out = np.zeros(len(omega_grid))
    for iw, w in enumerate(omega_grid):
        acc = 0.0 + 0.0j
        for k in range(K + 1):
            t = k * dt
            wk = 0.5 if (k == 0 or k == K) else 1.0
            acc += wk * C_t[k] * np.exp(1j * w * t) * np.exp(-t * inv_tau) * dt
        out[iw] = acc.real
    return out
