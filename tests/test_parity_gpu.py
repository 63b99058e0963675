"""GPU path (through the C ABI) against the CPU oracle, element by element.

Bars: basis keys bit-exact and in the same row order after every expansion;
P H P entries identical; amplitudes within 1e-10 of the oracle's, normwise
(max_i |c_i - c_i^ref| <= 1e-10 ||c^ref||).  Truncation decisions may differ
only for rows whose weight sits within rounding of theta^2; the oracle then
adopts the GPU's mask (lockstep protocol).
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2603_07341_gb300 import binding as B
from paper_2603_07341_gb300 import workloads as W

pytestmark = pytest.mark.gpu
AMP_TOL = 1e-10


def make_pair(cfg, gpu_extra=None, ora_extra=None, **over):
    model = W.model_kwargs(cfg, **over)
    g = B.Solver(**model, **(gpu_extra or {}))
    o = Oracle(**model, **(ora_extra or {}))
    return g, o


def compare_state(gpu, ora, tol=AMP_TOL):
    tg, ag = gpu.tuples()
    to, ao = ora.rows()
    assert tg.shape == to.shape, (tg.shape, to.shape)
    assert np.array_equal(tg, to), "key sets or row order differ"
    if len(ao):
        err = np.max(np.abs(ag - ao))
        assert err <= tol * max(np.linalg.norm(ao), 1e-300), err
    return len(ao)


def compare_record(rec, ora, N, tol=1e-10):
    st = ora.stats()
    P, nb = ora.populations()
    scale = max(st["norm"], 1e-300)
    assert rec[B.OBS_FIELDS.index("rows")] == st["rows"]
    assert rec[B.OBS_FIELDS.index("kept")] == st["kept"]
    assert rec[B.OBS_FIELDS.index("nnz")] == st["nnz"]
    assert abs(rec[B.OBS_FIELDS.index("terms")] - st["terms"]) <= 1
    for name in ("norm", "norm_phi0", "norm_before"):
        assert abs(rec[B.OBS_FIELDS.index(name)] - st[name]) <= tol * scale, name
    assert abs(rec[3] - st["energy"]) <= tol * max(1.0, abs(st["energy"]))
    assert abs(rec[4] - st["C_re"]) <= tol and abs(rec[5] - st["C_im"]) <= tol
    assert np.max(np.abs(rec[B.OBS_FIXED:B.OBS_FIXED + N] - P)) <= tol * scale
    assert np.max(np.abs(rec[B.OBS_FIXED + N:B.OBS_FIXED + 2 * N] - nb)) <= tol * scale * 10


def lockstep(gpu, ora, dt, theta, nsteps, check_every=1):
    """Advance both one step at a time; returns the number of adopted rows."""
    adopted = 0
    N = gpu.N
    for k in range(nsteps):
        _, a_before = ora.rows()
        gpu.step(dt, 1, theta)
        gkeep = gpu.keep()
        if len(gkeep):
            assert len(gkeep) == len(a_before)
            w = a_before.real * a_before.real + a_before.imag * a_before.imag
            okeep = w >= theta * theta
            diff = gkeep != okeep
            if diff.any():
                band = np.abs(w - theta * theta) <= 1e-9 * theta * theta + 1e-10 * np.sum(w)
                assert np.all(band[diff]), "truncation differs outside the rounding band"
                adopted += int(diff.sum())
                ora.step(dt, theta, keep=gkeep.astype(np.uint8))
            else:
                ora.step(dt, theta)
        else:
            ora.step(dt, theta)
        if k % check_every == 0 or k == nsteps - 1:
            compare_state(gpu, ora)
            rec = gpu.observables(gpu.num_records() - 1, 1)[0]
            compare_record(rec, ora, N)
    return adopted


# smaller initial balls where the oracle would otherwise need minutes
SET_STATE_CASES = [("ring4", {}), ("ring16", {}), ("dipolar6x6", {"m_init": 2}),
                   ("disorder12", {"eps": W.realisation_eps(W.WORKLOADS["disorder12"], 0)}),
                   ("cube4", {"m_init": 3})]


@pytest.mark.parametrize("name,over", SET_STATE_CASES, ids=[c[0] for c in SET_STATE_CASES])
def test_initial_expansion_keys_bitexact(libpaces, name, over):
    """H_eff(0) = ball of radius m_init (Eq. H_eff): same states, same BFS order,
    same level boundaries."""
    cfg = W.WORKLOADS[name]
    gpu, ora = make_pair(cfg, **over)
    st = W.start_state(cfg)
    gpu.set_state(*st)
    ora.set_state(*st)
    compare_state(gpu, ora)
    lv = gpu.levels()
    olv = ora.level_offsets()
    assert list(lv) == list(olv[: len(lv)]) and len(lv) in (len(olv), len(olv) - 1)


@pytest.mark.parametrize("precision", [B.DW, B.C128], ids=["dw", "c128"])
@pytest.mark.parametrize("name,over", SET_STATE_CASES, ids=[c[0] for c in SET_STATE_CASES])
def test_hamiltonian_parity(libpaces, name, over, precision):
    """P_m H P_m: per-row counts, columns and values in move order, diagonal
    (in FP64 within 2^-50 relative: eps_s + sum_j omega_j n_j summed in another
    order; within the double-word rounding, 2^-47 relative, when the diagonal is
    held as a double-word)."""
    cfg = W.WORKLOADS[name]
    gpu, ora = make_pair(cfg, gpu_extra=dict(precision=precision), **over)
    st = W.start_state(cfg)
    gpu.set_state(*st)
    ora.set_state(*st)
    cg, colg, vg, dg = gpu.hamiltonian()
    co, colo, vo, do = ora.hamiltonian()
    assert np.array_equal(cg, co)
    assert np.array_equal(colg, colo)
    assert np.array_equal(vg, vo)
    if precision == B.C128:
        assert np.all(np.abs(dg - do) <= 2.0 ** -50 * np.abs(do))
    else:
        assert np.all(np.abs(dg - do) <= 2.0 ** -47 * np.abs(do))


@pytest.mark.parametrize("precision", [B.DW, B.C128], ids=["dw", "c128"])
def test_ring4_full_trajectory(libpaces, precision):
    """Config ring4: 200 steps of dt = 0.05 at theta = 1e-8 in lockstep."""
    cfg = W.WORKLOADS["ring4"]
    gpu, ora = make_pair(cfg, gpu_extra=dict(precision=precision))
    gpu.set_state(*W.start_state(cfg))
    ora.set_state(*W.start_state(cfg))
    lockstep(gpu, ora, cfg["dt"], cfg["theta"], cfg["nsteps"], check_every=10)
    assert gpu.num_records() == cfg["nsteps"] + 1


@pytest.mark.parametrize("precision", [B.DW, B.C128], ids=["dw", "c128"])
def test_ring16_trajectory_prefix(libpaces, precision):
    """Config ring16 (the throughput workload): the first 40 steps in lockstep."""
    cfg = W.WORKLOADS["ring16"]
    gpu, ora = make_pair(cfg, gpu_extra=dict(precision=precision))
    gpu.set_state(*W.start_state(cfg))
    ora.set_state(*W.start_state(cfg))
    lockstep(gpu, ora, cfg["dt"], cfg["theta"], 40, check_every=5)


def test_dipolar_trajectory_prefix(libpaces):
    cfg = W.WORKLOADS["dipolar6x6"]
    gpu, ora = make_pair(cfg, m_init=2)
    gpu.set_state(*W.start_state(cfg))
    ora.set_state(*W.start_state(cfg))
    lockstep(gpu, ora, cfg["dt"], 1e-4, 6, check_every=2)


@pytest.mark.parametrize("r", [0, 1])
def test_disorder_realisation_trajectory(libpaces, r):
    cfg = W.WORKLOADS["disorder12"]
    eps = W.realisation_eps(cfg, r)
    gpu, ora = make_pair(cfg, eps=eps, m_init=4)
    gpu.set_state(*W.start_state(cfg))
    ora.set_state(*W.start_state(cfg))
    lockstep(gpu, ora, cfg["dt"], cfg["theta"], 25, check_every=5)


def test_cube_trajectory_prefix(libpaces):
    cfg = W.WORKLOADS["cube4"]
    gpu, ora = make_pair(cfg, m_init=2)
    gpu.set_state(*W.start_state(cfg))
    ora.set_state(*W.start_state(cfg))
    lockstep(gpu, ora, cfg["dt"], 1e-4, 4, check_every=1)


# ---------------------------------------------------------------- closed forms on the GPU path
def test_gpu_two_site_rabi(libpaces):
    g = B.Solver(n_sites=2, lattice_kind=B.RING, J=1.0, eps=[0.3, -0.2], omega=1.0, g=0.0, cap=1, m=2,
                 m_init=-1)
    g.set_state([0], [[0, 0]], [1.0])
    g.step(0.05, 100, 0.0)
    rec = B.records_dict(g.observables(), 2)
    t = rec["time"]
    Om = math.sqrt(0.5 ** 2 + 4.0)
    assert np.max(np.abs(rec["P"][:, 1] - 4.0 / Om ** 2 * np.sin(Om * t / 2) ** 2)) < 1e-12


def test_gpu_independent_boson(libpaces):
    """N = 1 (exciton radix 1), J = 0: the displaced-oscillator closed form."""
    g = B.Solver(n_sites=1, lattice_kind=B.RING, J=0.0, omega=1.0, g=1.0, cap=40, m=2, m_init=-1)
    g.set_state([0], [[0]], [1.0])
    g.step(0.05, 200, 0.0)
    rec = B.records_dict(g.observables(), 1)
    t = rec["time"]
    c = np.exp((np.exp(-1j * t) - 1) + 1j * t)
    assert np.max(np.abs(rec["C"] - c)) < 1e-11
    assert np.max(np.abs(rec["nbar"][:, 0] - 2 * (1 - np.cos(t)))) < 1e-10


# ---------------------------------------------------------------- edge cases
def test_invalid_states_are_rejected(libpaces):
    g = B.Solver(n_sites=3, lattice_kind=B.RING, J=1.0, omega=1.0, g=1.0, cap=2, m=2, m_init=1)
    for site, occ in (([3], [[0, 0, 0]]), ([0], [[0, 3, 0]]), ([0, 0], [[0, 0, 0], [0, 0, 0]]), ([], [])):
        with pytest.raises(B.PacesError) as e:
            g.set_state(site, np.asarray(occ, dtype=np.int32).reshape(len(site), 3), [1.0] * len(site))
        assert e.value.code == B.ERR_INVALID
    with pytest.raises(B.PacesError) as e:
        g.step(0.05, 1, 0.0)
    assert e.value.code == B.ERR_STATE


def test_frozen_single_state(libpaces):
    """J = 0, g = 0: H_eff stays one row and the phase is exp(-i eps t)."""
    g = B.Solver(n_sites=3, lattice_kind=B.RING, J=0.0, eps=[0.0, 0.7, 0.0], omega=1.0, g=0.0, cap=2, m=2,
                 m_init=3)
    g.set_state([1], [[0, 0, 0]], [1.0])
    g.step(0.1, 30, 1e-6)
    rec = B.records_dict(g.observables(), 3)
    assert np.all(rec["rows"] == 1)
    assert np.max(np.abs(rec["C"] - np.exp(-0.7j * rec["time"]))) < 1e-12


def test_capacity_grows_and_matches(libpaces):
    """Start with the minimum capacity; the library grows and redoes the step."""
    cfg = W.WORKLOADS["ring16"]
    gpu, ora = make_pair(cfg, gpu_extra=dict(max_rows=16), m_init=6)
    gpu.set_state(*W.start_state(cfg))
    ora.set_state(*W.start_state(cfg))
    lockstep(gpu, ora, cfg["dt"], 1e-9, 12, check_every=4)
    assert gpu.num_rows() > 4096


def test_noconvergence_reported_and_recoverable(libpaces):
    cfg = W.WORKLOADS["ring4"]
    gpu = B.Solver(**W.model_kwargs(cfg), nmax=14)
    gpu.set_state(*W.start_state(cfg))
    gpu.step(0.05, 3, 1e-8)
    with pytest.raises(B.PacesError) as e:
        gpu.step(2.0, 2, 1e-8)
    assert e.value.code == B.ERR_NOCONVERGE
    assert gpu.num_records() == 4
    gpu.step(0.05, 2, 1e-8)          # the state is usable again
    assert gpu.num_records() == 6


def test_second_order_series_breaks_unitarity(libpaces):
    """App. C.2 negative control on the GPU path: two terms only, norm grows."""
    cfg = W.WORKLOADS["ring4"]
    gpu = B.Solver(**W.model_kwargs(cfg), fixed_terms=2)
    gpu.set_state(*W.start_state(cfg))
    gpu.step(0.05, 100, 1e-8)
    rec = B.records_dict(gpu.observables(), 4)
    assert rec["norm"][-1] > 1.0 + 1e-4 and np.all(rec["terms"][1:] == 2)


def test_load_state_continues_bitwise(libpaces):
    """A state exported and loaded again continues exactly like the original."""
    cfg = W.WORKLOADS["ring16"]
    a = B.Solver(**W.model_kwargs(cfg, m_init=4))
    b = B.Solver(**W.model_kwargs(cfg, m_init=4))
    a.set_state(*W.start_state(cfg))
    a.step(cfg["dt"], 10, cfg["theta"])
    b.load_state(*a.state())
    a.step(cfg["dt"], 5, cfg["theta"])
    b.step(cfg["dt"], 5, cfg["theta"])
    ta, aa = a.tuples()
    tb, ab = b.tuples()
    assert np.array_equal(ta, tb) and np.array_equal(aa, ab)


def test_holstein_chain_full_space_nonzeros_at_scale(libpaces):
    """App. C figures at full size: L = 9, d_pho = 5 has 9 * 5^9 = 17,578,125
    states and d^L[(5L-2) - 2L/d] = 76,953,125 stored entries of P H P."""
    L, d = 9, 5
    g = B.Solver(n_sites=L, lattice_kind=B.CHAIN, J=1.0, omega=1.0, g=0.8, cap=d - 1, m=2, m_init=-1)
    g.set_state([0], [[0] * L], [1.0])
    assert g.num_rows() == L * d ** L
    g.step(0.01, 1, 0.0)
    rec = B.records_dict(g.observables(), L)
    assert rec["nnz"][-1] == d ** L * (5 * L - 2) - 2 * L * d ** (L - 1) == 76953125
    assert abs(rec["norm"][-1] - 1.0) < 1e-12


def test_threshold_band_kept_set_exact(libpaces):
    """Truncation keeps exactly the rows with re^2 + im^2 >= theta^2 evaluated in
    FP64 with the products and the sum rounded separately (the oracle's rule),
    for amplitudes planted on theta^2, within and just outside 2^-14 of it (the
    band in which the kernel stops trusting its 20-bit magnitudes and runs the
    FP64 test), far from it, at zero, and at subnormal and large magnitudes.
    Every state of the 4-site ring is loaded, so no row is missing."""
    import itertools
    cfg = W.WORKLOADS["ring4"]
    N, K = cfg["n_sites"], cfg["cap"]
    occ1 = np.array(list(itertools.product(range(K + 1), repeat=N)), dtype=np.int32)
    site = np.repeat(np.arange(N, dtype=np.int32), len(occ1))
    occ = np.tile(occ1, (N, 1))
    n = len(site)
    rng = np.random.default_rng(11)
    offs = np.array([0.0, 2.0 ** -10, 2.0 ** -13, 2.0 ** -14 * 1.001, 2.0 ** -14, 2.0 ** -14 * 0.999,
                     2.0 ** -15, 2.0 ** -20, 2.0 ** -30, 1e-12, 1e-15, 2.0 ** -52, 2.0 ** -53])
    offs = np.concatenate([offs, -offs[1:]])
    for theta in (1e-7, 3.1e-4, 1e-2):
        w = theta * theta * (1.0 + np.resize(offs, n))
        w[::7] = theta * theta * np.exp(rng.normal(0.0, 4.0, len(w[::7])))   # far from the band
        ang = rng.uniform(0.0, 2.0 * np.pi, n)
        x, y = np.sqrt(w) * np.cos(ang), np.sqrt(w) * np.sin(ang)
        x[0], y[0] = theta, 0.0                   # exactly on theta^2
        x[1], y[1] = 0.0, -theta
        x[2], y[2] = 0.0, 0.0
        x[3], y[3] = 5e-324, 0.0                  # subnormal
        x[4], y[4] = 1e-300, 1e-300
        x[5], y[5] = 30.0, -40.0                  # large
        x[6], y[6] = np.nextafter(theta, 0.0), 0.0
        amps = x + 1j * y
        g = B.Solver(**W.model_kwargs(cfg))
        g.load_state(site, occ, amps)
        g.step(cfg["dt"], 1, theta)
        keep = g.keep()
        expect = (x * x + y * y) >= theta * theta
        assert len(keep) == n
        assert np.array_equal(keep, expect), (theta, np.flatnonzero(keep != expect)[:10])
        g.close()
