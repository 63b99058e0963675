"""Thin ctypes binding of libpaces (include/paces.h): argument marshalling only.

Every step of the time-stepping path runs in the CUDA library.  PyTorch only
supplies the CUDA stream and device memory (through its caching allocator,
handed to the library as a paces_allocator).  If the library has not been
built, loading raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK, ERR_INVALID, ERR_KEY_WIDTH, ERR_CAPACITY, ERR_NOCONVERGE, ERR_CUDA, ERR_STATE, ERR_UNSUPPORTED = range(8)
RING, CHAIN, OPEN2D, OPEN3D, EXPLICIT = 0, 1, 2, 3, 4
NEAREST, DIPOLAR = 0, 1
C128, DW, C64_SPMV = 0, 1, 2
TAYLOR, LANCZOS = 0, 1
MAX_KRYLOV = 32
MAX_SITES, MAX_WORDS = 128, 4
OBS_FIELDS = ("time", "norm", "norm_phi0", "energy", "C_re", "C_im", "rows", "kept", "nnz", "terms",
              "norm_before", "substeps", "hbound")
OBS_FIXED = 14
STAGES = ("truncate", "expand", "hamiltonian", "propagate", "observe")

EXPORTED = (
    "paces_plan_layout", "paces_encode_keys", "paces_create", "paces_destroy", "paces_last_error",
    "paces_set_state", "paces_load_state", "paces_step", "paces_num_rows", "paces_get_state",
    "paces_get_levels", "paces_get_keep", "paces_get_hamiltonian", "paces_record_len",
    "paces_num_records", "paces_observables", "paces_profile", "paces_stage_stats",
    "paces_expand_noalloc", "paces_get_tuning", "paces_set_tuning", "paces_record", "paces_backward",
    "paces_step_nom", "paces_selftest_barrier", "paces_set_coefficients", "paces_fp64_rate",
)


class Params(C.Structure):
    _fields_ = [("n_sites", C.c_int32), ("lattice_kind", C.c_int32), ("dims", C.c_int32 * 3),
                ("coupling_kind", C.c_int32), ("J", C.c_double), ("J_explicit", C.POINTER(C.c_double)),
                ("eps", C.POINTER(C.c_double)), ("omega", C.POINTER(C.c_double)),
                ("g", C.POINTER(C.c_double)), ("phonon_cap", C.POINTER(C.c_int32)), ("m", C.c_int32),
                ("m_init", C.c_int32), ("precision", C.c_int32), ("fixed_terms", C.c_int32),
                ("taylor_tol", C.c_double), ("taylor_nmax", C.c_int32), ("max_rows", C.c_uint64),
                ("batch", C.c_int32), ("reserved0", C.c_int32), ("taylor_xmax", C.c_double),
                ("propagator", C.c_int32), ("krylov_max", C.c_int32)]


class Layout(C.Structure):
    _fields_ = [("n_sites", C.c_int32), ("words", C.c_int32), ("pow2", C.c_int32), ("reserved", C.c_int32),
                ("exciton_radix", C.c_uint64), ("site_word", C.c_int32 * MAX_SITES),
                ("site_stride", C.c_uint64 * MAX_SITES), ("site_radix", C.c_uint64 * MAX_SITES),
                ("batch_word", C.c_int32), ("reserved1", C.c_int32), ("batch_stride", C.c_uint64),
                ("batch_radix", C.c_uint64)]


class Tuning(C.Structure):
    _fields_ = [("taylor_lanes_per_row", C.c_int32), ("taylor_blocks_per_sm", C.c_int32),
                ("grid_blocks_per_sm", C.c_int32), ("chunk_blocks_per_sm", C.c_int32),
                ("use_graphs", C.c_int32), ("max_taylor_blocks_per_sm", C.c_int32),
                ("table_load_pct", C.c_int32), ("reserved", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN)]


class PacesError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("paces error %d: %s" % (code, msg))
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load libpaces.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError("libpaces.so is not built (%s); run paper_2603_07341_gb300.build.build()" % path)
    lib = C.CDLL(path)
    S = C.c_int
    P, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32)
    i64p = C.POINTER(C.c_int64)
    lib.paces_plan_layout.restype = S
    lib.paces_plan_layout.argtypes = [C.POINTER(Params), C.POINTER(Layout)]
    lib.paces_encode_keys.restype = S
    lib.paces_encode_keys.argtypes = [C.POINTER(Layout), C.c_int64, ip, ip, C.POINTER(C.c_uint64)]
    lib.paces_create.restype = S
    lib.paces_create.argtypes = [C.POINTER(Params), C.POINTER(Allocator), P, C.POINTER(P)]
    lib.paces_destroy.restype = S
    lib.paces_destroy.argtypes = [P]
    lib.paces_last_error.restype = C.c_char_p
    lib.paces_last_error.argtypes = [P]
    for fn in ("paces_set_state", "paces_load_state"):
        getattr(lib, fn).restype = S
        getattr(lib, fn).argtypes = [P, C.c_int64, ip, ip, dp]
    lib.paces_step.restype = S
    lib.paces_step.argtypes = [P, C.c_double, C.c_int64, C.c_double]
    lib.paces_step_nom.restype = S
    lib.paces_step_nom.argtypes = [P, C.c_double, C.c_int64, C.c_int64, C.c_uint64]
    lib.paces_num_rows.restype = S
    lib.paces_num_rows.argtypes = [P, i64p]
    lib.paces_get_state.restype = S
    lib.paces_get_state.argtypes = [P, C.c_int64, ip, ip, dp]
    lib.paces_get_levels.restype = S
    lib.paces_get_levels.argtypes = [P, i64p, C.c_int32, ip]
    lib.paces_get_keep.restype = S
    lib.paces_get_keep.argtypes = [P, C.POINTER(C.c_uint8), C.c_int64, i64p]
    lib.paces_get_hamiltonian.restype = S
    lib.paces_get_hamiltonian.argtypes = [P, ip, ip, dp, dp, C.c_int64, i64p]
    lib.paces_record_len.restype = C.c_int32
    lib.paces_record_len.argtypes = [P]
    lib.paces_num_records.restype = S
    lib.paces_num_records.argtypes = [P, i64p]
    lib.paces_observables.restype = S
    lib.paces_observables.argtypes = [P, C.c_int64, C.c_int64, dp]
    lib.paces_profile.restype = S
    lib.paces_profile.argtypes = [P, C.c_int32]
    lib.paces_stage_stats.restype = S
    lib.paces_stage_stats.argtypes = [P, dp, i64p, dp, C.c_int32]
    lib.paces_get_tuning.restype = S
    lib.paces_get_tuning.argtypes = [P, C.POINTER(Tuning)]
    lib.paces_set_tuning.restype = S
    lib.paces_set_tuning.argtypes = [P, C.POINTER(Tuning)]
    lib.paces_record.restype = S
    lib.paces_record.argtypes = [P, C.c_int32]
    lib.paces_backward.restype = S
    lib.paces_backward.argtypes = [P, C.c_int64, dp, dp, dp, dp]
    lib.paces_expand_noalloc.restype = S
    lib.paces_expand_noalloc.argtypes = [C.POINTER(Params), P, C.c_int64, P, C.c_int64, i64p, P]
    lib.paces_set_coefficients.restype = S
    lib.paces_set_coefficients.argtypes = [P, C.c_double, dp, dp, dp]
    lib.paces_selftest_barrier.restype = S
    lib.paces_selftest_barrier.argtypes = [C.c_int32, C.c_double, C.POINTER(C.c_int32)]
    lib.paces_fp64_rate.restype = S
    lib.paces_fp64_rate.argtypes = [C.POINTER(C.c_double)]
    _lib = lib
    return lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_int32))


def make_params(n_sites, lattice_kind=RING, dims=(0, 0, 0), coupling_kind=NEAREST, J=1.0, eps=None,
                omega=None, g=None, cap=None, m=2, m_init=10, precision=C128, fixed_terms=0, tol=0.0,
                nmax=0, max_rows=0, J_explicit=None, batch=1, xmax=0.0, propagator=0, kmax=0):
    """Build a Params struct; returns (struct, keepalive arrays).  For an
    ensemble (batch R > 1) eps is [R, N] (or broadcastable to it).  xmax: the
    substep bound (0: the library's 8; < 0: one Taylor series per step).
    propagator: TAYLOR or LANCZOS (kmax Krylov vectors at most; 0: 30)."""
    N = int(n_sites)
    R = max(1, int(batch))
    vec = lambda v: np.ascontiguousarray(np.broadcast_to(np.asarray(0.0 if v is None else v,
                                                                    dtype=np.float64), (N,)))
    epsv = np.ascontiguousarray(np.broadcast_to(np.asarray(0.0 if eps is None else eps, dtype=np.float64),
                                                (R, N)).reshape(-1)) if R > 1 else vec(eps)
    keep = dict(eps=epsv, omega=vec(omega), g=vec(g),
                cap=np.ascontiguousarray(np.broadcast_to(np.asarray(4 if cap is None else cap,
                                                                    dtype=np.int32), (N,))))
    if J_explicit is not None:
        keep["Jx"] = np.ascontiguousarray(J_explicit, dtype=np.float64).reshape(N * N)
    p = Params()
    p.n_sites = N
    p.lattice_kind = int(lattice_kind)
    d = list(dims) + [0] * (3 - len(dims))
    for i in range(3):
        p.dims[i] = int(d[i])
    p.coupling_kind = int(coupling_kind)
    p.J = float(J)
    p.J_explicit = _dp(keep.get("Jx"))
    p.eps, p.omega, p.g = _dp(keep["eps"]), _dp(keep["omega"]), _dp(keep["g"])
    p.phonon_cap = _ip(keep["cap"])
    p.m, p.m_init, p.precision, p.fixed_terms = int(m), int(m_init), int(precision), int(fixed_terms)
    p.taylor_tol, p.taylor_nmax, p.max_rows = float(tol), int(nmax), int(max_rows)
    p.batch = R
    p.taylor_xmax = float(xmax)
    p.propagator, p.krylov_max = int(propagator), int(kmax)
    return p, keep


def plan_layout(**model):
    """Host-only key layout of a model (no GPU needed)."""
    lib = load()
    p, keep = make_params(**model)
    L = Layout()
    rc = lib.paces_plan_layout(C.byref(p), C.byref(L))
    if rc:
        raise PacesError(rc, "paces_plan_layout")
    return L


def encode_keys(layout, site, occ):
    """Host-only encoding of A-form states into keys[n, words] (uint64)."""
    lib = load()
    site = np.ascontiguousarray(site, dtype=np.int32)
    occ = np.ascontiguousarray(occ, dtype=np.int32)
    out = np.zeros((len(site), layout.words), dtype=np.uint64)
    rc = lib.paces_encode_keys(C.byref(layout), len(site), _ip(site), _ip(occ),
                               out.ctypes.data_as(C.POINTER(C.c_uint64)))
    if rc:
        raise PacesError(rc, "paces_encode_keys")
    return out


def expand_noalloc(keys_in, max_out, stream=None, **model):
    """One expansion level with no device allocation inside the library.

    keys_in: CUDA tensor [n_in, words] of int64 holding uint64 keys (this
    wrapper allocates the output tensor with torch; the library call itself
    allocates nothing).  Returns the CUDA tensor [n_out, words]."""
    import torch
    lib = load()
    p, keep = make_params(**model)
    if not (torch.is_tensor(keys_in) and keys_in.is_cuda and keys_in.dtype == torch.int64 and keys_in.dim() == 2):
        raise ValueError("keys_in must be a 2-D int64 CUDA tensor [n_in, words]")
    words = plan_layout(**model).words
    if keys_in.shape[1] != words:
        raise ValueError("keys_in has %d words per key; this model's layout uses %d" % (keys_in.shape[1], words))
    keys_in = keys_in.contiguous()
    n_in = keys_in.shape[0]
    # the library works on the current device and that device's scratch array
    with torch.cuda.device(keys_in.device):
        out = torch.empty((int(max_out), words), dtype=torch.int64, device=keys_in.device)
        n = C.c_int64()
        st = stream if stream is not None else torch.cuda.current_stream(keys_in.device)
        rc = lib.paces_expand_noalloc(C.byref(p), C.c_void_p(keys_in.data_ptr()), n_in,
                                      C.c_void_p(out.data_ptr()), int(max_out), C.byref(n),
                                      C.c_void_p(st.cuda_stream))
    if rc:
        raise PacesError(rc, "paces_expand_noalloc")
    return out[: n.value]


class _TorchAllocator:
    """paces_allocator backed by torch's CUDA caching allocator."""

    def __init__(self, device):
        import torch
        self._torch = torch
        self._device = device

        def alloc(ctx, nbytes, stream):
            try:
                return self._torch.cuda.caching_allocator_alloc(int(nbytes), device=self._device,
                                                                stream=int(stream or 0))
            except Exception:     # out of memory: the library reports PACES_ERR_CAPACITY
                return None

        def free(ctx, ptr, nbytes, stream):
            self._torch.cuda.caching_allocator_delete(ptr)

        self._alloc_fn = ALLOC_FN(alloc)
        self._free_fn = FREE_FN(free)
        self.struct = Allocator(None, self._alloc_fn, self._free_fn)


class Solver:
    """One handle of the co-evolving-subspace solver on the current CUDA device."""

    def __init__(self, stream=None, torch_allocator=True, **model):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("paces needs a CUDA device")
        self._lib = load()
        self.N = int(model["n_sites"])
        self.batch = max(1, int(model.get("batch", 1)))
        self.ncols = self.N + (1 if self.batch > 1 else 0)
        self._params, self._keep = make_params(**model)
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._alloc = _TorchAllocator(self.device) if torch_allocator else None
        h = C.c_void_p()
        ap = C.byref(self._alloc.struct) if self._alloc else None
        rc = self._lib.paces_create(C.byref(self._params), ap, C.c_void_p(self.stream.cuda_stream),
                                    C.byref(h))
        if rc:
            raise PacesError(rc, "paces_create")
        self._h = h
        self.rec_len = self._lib.paces_record_len(h)

    # -- plumbing
    def _check(self, rc, what):
        if rc:
            raise PacesError(rc, "%s: %s" % (what, self._lib.paces_last_error(self._h).decode()))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.paces_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _state_args(N, site, occ, amps):
        site = np.ascontiguousarray(site, dtype=np.int32)
        occ = np.ascontiguousarray(occ, dtype=np.int32).reshape(len(site), N)
        a = np.asarray(amps, dtype=np.complex128).reshape(len(site))
        ri = np.ascontiguousarray(np.stack([a.real, a.imag], 1).reshape(-1))
        return site, occ, ri

    # -- API
    def set_state(self, site, occ, amps):
        s, o, a = self._state_args(self.N, site, occ, amps)
        self._check(self._lib.paces_set_state(self._h, len(s), _ip(s), _ip(o), _dp(a)), "set_state")

    def load_state(self, site, occ, amps):
        s, o, a = self._state_args(self.ncols, site, occ, amps)
        self._check(self._lib.paces_load_state(self._h, len(s), _ip(s), _ip(o), _dp(a)), "load_state")

    def step(self, dt, nsteps=1, theta=0.0):
        self._check(self._lib.paces_step(self._h, float(dt), int(nsteps), float(theta)), "step")

    def step_nom(self, dt, nsteps=1, q_nom=1, seed=0):
        """Steps with top-q_nom truncation (the paper's scheme; seeded tie-break)."""
        self._check(self._lib.paces_step_nom(self._h, float(dt), int(nsteps), int(q_nom),
                                             int(seed) & ((1 << 64) - 1)), "step_nom")

    def set_coefficients(self, J, eps=None, omega=None, g=None):
        """Replace H's values for the following steps (a Hamiltonian piecewise
        constant in time); None keeps an array.  The move graph is fixed: J and
        every g_s stay zero exactly where they were."""
        n = self.N * self.batch

        def f(v, k):
            if v is None:
                return None
            a = np.asarray(v, dtype=np.float64)
            a = a.reshape(-1) if a.size == k else a      # [R, N] site energies of an ensemble
            return np.ascontiguousarray(np.broadcast_to(a, (k,)))
        e, w, gg = f(eps, n), f(omega, self.N), f(g, self.N)
        self._check(self._lib.paces_set_coefficients(self._h, float(J), _dp(e), _dp(w), _dp(gg)),
                    "set_coefficients")

    def num_rows(self):
        n = C.c_int64()
        self._check(self._lib.paces_num_rows(self._h, C.byref(n)), "num_rows")
        return n.value

    def state(self):
        q = self.num_rows()
        site = np.zeros(q, dtype=np.int32)
        occ = np.zeros((q, self.ncols), dtype=np.int32)
        amps = np.zeros(2 * q)
        self._check(self._lib.paces_get_state(self._h, q, _ip(site), _ip(occ), _dp(amps)), "get_state")
        return site, occ, amps[0::2] + 1j * amps[1::2]

    def tuples(self):
        site, occ, amps = self.state()
        return np.concatenate([site[:, None], occ], 1), amps

    def levels(self):
        buf = np.zeros(300, dtype=np.int64)
        n = C.c_int32()
        self._check(self._lib.paces_get_levels(self._h, buf.ctypes.data_as(C.POINTER(C.c_int64)), len(buf),
                                               C.byref(n)), "get_levels")
        return buf[: n.value].copy()

    def keep(self):
        n = C.c_int64()
        self._check(self._lib.paces_get_keep(self._h, None, 0, C.byref(n)), "get_keep")
        out = np.zeros(max(n.value, 1), dtype=np.uint8)
        self._check(self._lib.paces_get_keep(self._h, out.ctypes.data_as(C.POINTER(C.c_uint8)), n.value,
                                             C.byref(n)), "get_keep")
        return out[: n.value].astype(bool)

    def hamiltonian(self):
        nnz = C.c_int64()
        self._check(self._lib.paces_get_hamiltonian(self._h, None, None, None, None, 0, C.byref(nnz)),
                    "get_hamiltonian")
        q = self.num_rows()
        cnt = np.zeros(q, dtype=np.int32)
        cols = np.zeros(max(nnz.value, 1), dtype=np.int32)
        vals = np.zeros(max(nnz.value, 1))
        diag = np.zeros(max(q, 1))
        self._check(self._lib.paces_get_hamiltonian(self._h, _ip(cnt), _ip(cols), _dp(vals), _dp(diag),
                                                    nnz.value, C.byref(nnz)), "get_hamiltonian")
        return cnt, cols[: nnz.value], vals[: nnz.value], diag[:q]

    def num_records(self):
        n = C.c_int64()
        self._check(self._lib.paces_num_records(self._h, C.byref(n)), "num_records")
        return n.value

    def observables(self, first=0, count=None):
        if count is None:
            count = self.num_records() - first
        out = np.zeros((count, self.rec_len))
        self._check(self._lib.paces_observables(self._h, int(first), int(count), _dp(out)), "observables")
        return out

    def tuning(self):
        t = Tuning()
        self._check(self._lib.paces_get_tuning(self._h, C.byref(t)), "get_tuning")
        return {f: getattr(t, f) for f, _ in Tuning._fields_ if f != "reserved"}

    def set_tuning(self, **kw):
        t = Tuning()
        self._check(self._lib.paces_get_tuning(self._h, C.byref(t)), "get_tuning")
        for k, v in kw.items():
            if k == "max_taylor_blocks_per_sm":
                continue
            setattr(t, k, int(v))
        self._check(self._lib.paces_set_tuning(self._h, C.byref(t)), "set_tuning")

    def profile(self, on=True):
        self._check(self._lib.paces_profile(self._h, 1 if on else 0), "profile")

    def record(self, ckpt_every=20):
        """Record the following steps for backward(); a checkpoint every ckpt_every steps (0: stop)."""
        self._check(self._lib.paces_record(self._h, int(ckpt_every)), "record")

    def backward(self, nsteps, dL_dc_final=None, dL_dC=None, dL_dP=None):
        """dL/d[J, g, omega, eps_0..eps_{N-1}] of a loss of the recorded steps.

        dL_dc_final: complex cotangent on the current rows (state() order);
        dL_dC: complex dL/dRe C_k + i dL/dIm C_k, one per recorded step;
        dL_dP: real dL/dP_s(t_k), shape (nsteps, N)."""
        def ri(z, n):
            if z is None:
                return None
            z = np.asarray(z, dtype=np.complex128).reshape(-1)
            if z.size != n:
                raise ValueError("cotangent has %d entries, expected %d" % (z.size, n))
            return np.ascontiguousarray(np.stack([z.real, z.imag], 1).reshape(-1))
        nsteps = int(nsteps)
        a = ri(dL_dc_final, self.num_rows()) if dL_dc_final is not None else None
        c = ri(dL_dC, nsteps)
        p = None
        if dL_dP is not None:
            p = np.ascontiguousarray(dL_dP, dtype=np.float64).reshape(-1)
            if p.size != nsteps * self.N:
                raise ValueError("dL_dP must hold nsteps * N values")
        grad = np.zeros(3 + self.N)
        self._check(self._lib.paces_backward(self._h, nsteps, _dp(a), _dp(c), _dp(p), _dp(grad)), "backward")
        return grad

    def stage_stats(self, reset=False):
        ms = np.zeros(5)
        launches = np.zeros(6, dtype=np.int64)
        by = np.zeros(5)
        self._check(self._lib.paces_stage_stats(self._h, _dp(ms), launches.ctypes.data_as(C.POINTER(C.c_int64)),
                                                _dp(by), 1 if reset else 0), "stage_stats")
        return ms, launches, by


def records_dict(rec, N, batch=1):
    """Split observables records into named columns: P[:, N] and nbar[:, N], or
    for an ensemble P[:, R, N], nbar[:, R, N] and C_r[:, R]."""
    d = {name: rec[:, i] for i, name in enumerate(OBS_FIELDS)}
    d["C"] = rec[:, 4] + 1j * rec[:, 5]
    R = max(1, int(batch))
    if R == 1:
        d["P"] = rec[:, OBS_FIXED:OBS_FIXED + N]
        d["nbar"] = rec[:, OBS_FIXED + N:OBS_FIXED + 2 * N]
        return d
    o = OBS_FIXED
    d["P"] = rec[:, o:o + R * N].reshape(-1, R, N)
    d["nbar"] = rec[:, o + R * N:o + 2 * R * N].reshape(-1, R, N)
    c = rec[:, o + 2 * R * N:o + 2 * R * N + 2 * R].reshape(-1, R, 2)
    d["C_r"] = c[:, :, 0] + 1j * c[:, :, 1]
    return d


def selftest_barrier(extra_arrivals, timeout_ms=1.0):
    """Run the bounded grid barrier on the current device (paces_selftest_barrier):
    returns the device error code it recorded (0: completed, 5: a wait ran out)."""
    lib = load()
    err = C.c_int32(-1)
    rc = lib.paces_selftest_barrier(int(extra_arrivals), float(timeout_ms), C.byref(err))
    if rc:
        raise PacesError(rc, "paces_selftest_barrier")
    return int(err.value)


def fp64_rate():
    """FP64 FMA rate the current device sustains, TFLOP/s (paces_fp64_rate)."""
    lib = load()
    v = C.c_double()
    rc = lib.paces_fp64_rate(C.byref(v))
    if rc:
        raise PacesError(rc, "paces_fp64_rate")
    return v.value
