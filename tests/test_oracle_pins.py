"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check compares the oracle with something other than itself: a dense
Kronecker-product Hamiltonian exponentiated by eigendecomposition, textbook
closed forms, the paper's printed worked examples (tests/golden), invariants,
and finite differences.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle.oracle import Oracle, OracleError, absorption_spectrum
from paper_2603_07341_gb300 import workloads as W
from tests.dense_model import dense_holstein, dense_index, propagator, ring_hop

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def oracle_for(cfg, **over):
    kw = W.model_kwargs(cfg, **over)
    extra = {k: over[k] for k in ("tol", "nmax", "fixed_terms") if k in over}
    return Oracle(**kw, **extra)


def state_vector(o, D, strides, dim):
    t, a = o.rows()
    v = np.zeros(dim, dtype=np.complex128)
    v[dense_index(t, D, strides)] = a
    return v


# ---------------------------------------------------------------- whole step vs expm
def test_ring4_full_space_matches_dense_expm():
    """Config ring4 (full space 2500).  With theta = 0 every step keeps the whole
    space, so the trajectory is exp(-iHt) psi0 to the series tolerance (Sec. 3.5:
    the only error sources are Q, P_m and the series cutoff).  At the workload's
    theta = 1e-8 the early steps truncate; the end state stays within 1e-6."""
    cfg = W.WORKLOADS["ring4"]
    N = cfg["n_sites"]
    H, D, strides = dense_holstein(ring_hop(N, cfg["J"]), [0.0] * N, [1.0] * N, [1.0] * N, [4] * N)
    U = propagator(H)
    for theta, tol in ((0.0, 1e-11), (cfg["theta"], 1e-6)):
        o = oracle_for(cfg)
        o.set_state(*W.start_state(cfg))
        assert o.nrows() == 4 * 5 ** 4
        psi0 = state_vector(o, D, strides, H.shape[0])
        for k in range(1, cfg["nsteps"] + 1):
            o.step(cfg["dt"], theta)
            if theta == 0.0:
                assert o.stats()["rows"] == 2500
            if k % 50 == 0:
                err = np.linalg.norm(state_vector(o, D, strides, H.shape[0]) - U(k * cfg["dt"], psi0))
                assert err <= tol, (theta, k, err)


def test_threshold_to_zero_converges():
    """Starting from the full space (m_init = closure), the error against the exact
    evolution falls steadily as the threshold goes to zero and reaches the series
    tolerance (Sec. 4.2: fidelity grows with the kept set; Sec. 3.5 error sources)."""
    cfg = W.WORKLOADS["ring4"]
    N = cfg["n_sites"]
    H, D, strides = dense_holstein(ring_hop(N, 1.0), [0.0] * N, [1.0] * N, [1.0] * N, [4] * N)
    U = propagator(H)
    errs = []
    thetas = (1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-8, 1e-10)
    for th in thetas:
        o = oracle_for(cfg)
        o.set_state(*W.start_state(cfg))
        psi0 = state_vector(o, D, strides, H.shape[0])
        for _ in range(60):
            o.step(0.05, th)
        errs.append(np.linalg.norm(state_vector(o, D, strides, H.shape[0]) - U(3.0, psi0)))
    assert all(errs[i + 1] < 0.5 * errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-9


@pytest.mark.parametrize("m", [1, 2])
def test_restriction_error_order_and_bound(m):
    """Eq. epsilon_Pm / App. F: one step restricted to the radius-m ball errs by
    O(dt^{m+1}) and stays under sum_{l>m} (2^{l-m}-1)/l! (alpha dt)^l, alpha <= ||H||."""
    N = 4
    H, D, strides = dense_holstein(ring_hop(N, 1.0), [0.0] * N, [1.0] * N, [1.0] * N, [4] * N)
    alpha = np.max(np.abs(np.linalg.eigvalsh(H)))
    U = propagator(H)
    errs = []
    dts = (0.04, 0.02, 0.01)
    for dt in dts:
        o = Oracle(N, W.RING, J=1.0, omega=1.0, g=1.0, cap=4, m=m, m_init=m)
        o.set_state([0], [[0] * N], [1.0])
        psi0 = state_vector(o, D, strides, H.shape[0])
        o.step(dt, 0.0)
        err = np.linalg.norm(state_vector(o, D, strides, H.shape[0]) - U(dt, psi0))
        bound = sum((2.0 ** (l - m) - 1.0) / math.factorial(l) * (alpha * dt) ** l
                    for l in range(m + 1, 60))
        assert err <= bound, (dt, err, bound)
        errs.append(err)
    for a, b in zip(errs, errs[1:]):
        assert abs(math.log2(a / b) - (m + 1)) < 0.15, errs


# ---------------------------------------------------------------- closed forms
def test_two_site_rabi():
    """N = 2, g = 0: P_1 = (4J^2/Omega^2) sin^2(Omega t / 2), Omega^2 = Delta^2 + 4J^2.
    The ring of two sites has a single bond (pairs are de-duplicated)."""
    for eps in ((0.0, 0.0), (0.3, -0.2)):
        J = 1.0
        o = Oracle(2, W.RING, J=J, eps=eps, omega=1.0, g=0.0, cap=1, m=2, m_init=-1)
        o.set_state([0], [[0, 0]], [1.0])
        assert o.hopping()[0, 1] == J
        delta = eps[0] - eps[1]
        Om = math.sqrt(delta ** 2 + 4 * J * J)
        for k in range(1, 101):
            o.step(0.05, 0.0)
            t = 0.05 * k
            P, nbar = o.populations()
            assert abs(P[1] - 4 * J * J / Om ** 2 * math.sin(Om * t / 2) ** 2) < 1e-12
            assert np.all(nbar == 0.0)
        t_, _ = o.rows()
        assert np.all(t_[:, 1:] == 0)       # g = 0: the phonon vacuum sector is kept


def test_independent_boson_autocorrelation():
    """N = 1, J = 0 (displaced oscillator, Fig. 2 of the paper with the textbook
    solution): C(t) = exp[(g/w)^2 (e^{-iwt} - 1) + i g^2 t / w],
    <n>(t) = 2 (g/w)^2 (1 - cos wt).  Cap K = 40 leaves a Poisson tail < 1e-20."""
    g, w = 1.0, 1.0
    o = Oracle(1, W.RING, J=0.0, omega=w, g=g, cap=40, m=2, m_init=-1)
    o.set_state([0], [[0]], [1.0])
    assert o.nrows() == 41
    for k in range(1, 201):
        o.step(0.05, 0.0)
        t = 0.05 * k
        st = o.stats()
        c_exact = np.exp((g / w) ** 2 * (np.exp(-1j * w * t) - 1) + 1j * g * g * t / w)
        assert abs(st["C_re"] + 1j * st["C_im"] - c_exact) < 1e-11
        _, nbar = o.populations()
        assert abs(nbar[0] - 2 * (g / w) ** 2 * (1 - math.cos(w * t))) < 1e-10


def test_electronic_spectrum_g0_and_dipolar_pattern():
    """g = 0: C(t) = sum_k |<k|mu>|^2 e^{-i E_k t} over the N x N exciton matrix
    (the exact diagonalisation the paper uses for its g = 0 spectra).  Entries
    of the all-pairs J0/r^3 pattern are checked against hand values."""
    J0 = -1.0
    o = Oracle(9, W.OPEN2D, dims=(3, 3, 1), coupling_kind=W.DIPOLAR, J=J0, omega=1.0, g=0.0,
               cap=2, m=2, m_init=-1)
    h = o.hopping()
    assert h[0, 1] == J0 and h[0, 3] == J0                      # r = 1
    assert abs(h[0, 4] - J0 / (2.0 * math.sqrt(2.0))) < 1e-16   # r = sqrt 2
    assert abs(h[0, 2] - J0 / 8.0) < 1e-16                      # r = 2
    assert abs(h[0, 8] - J0 / (8.0 * math.sqrt(8.0))) < 1e-16   # r = sqrt 8
    assert np.allclose(h, h.T) and np.all(np.diag(h) == 0)
    mu = np.full(9, 1 / 3.0)
    o.set_state(np.arange(9), np.zeros((9, 9), dtype=np.int32), mu)
    E, V = np.linalg.eigh(h)
    w = np.abs(V.T @ mu) ** 2
    for k in range(1, 81):
        o.step(0.05, 0.0)
        st = o.stats()
        c_exact = np.sum(w * np.exp(-1j * E * 0.05 * k))
        assert abs(st["C_re"] + 1j * st["C_im"] - c_exact) < 1e-12


def test_dimer_bright_line_shift():
    """App. G.1: without vibrations the dimer's bright state absorbs at the bare
    transition shifted by exactly J: C(t) = e^{-iJt}."""
    for J in (0.55, -0.55):
        o = Oracle(2, W.RING, J=J, omega=1.0, g=0.0, cap=2, m=2, m_init=-1)
        o.set_state([0, 1], [[0, 0], [0, 0]], [1 / math.sqrt(2)] * 2)
        for k in range(1, 41):
            o.step(0.05, 0.0)
            st = o.stats()
            assert abs(st["C_re"] + 1j * st["C_im"] - np.exp(-1j * J * 0.05 * k)) < 1e-13


# ---------------------------------------------------------------- worked examples
def test_tb_neighbour_sets_worked_example():
    """Paper's TB example: |N0| = 2, |N1| = 3, |N2| = 4 and a 7-state ball of
    radius 2, {n-3..n+3}; N1 of {n-1, n+1} is {n-2, n, n+2}."""
    gd = gold("tb_neighbour_sets.json")
    L, n = 21, 10
    hop = np.zeros((L, L))
    for a in range(L - 1):
        hop[a, a + 1] = hop[a + 1, a] = 1.0
    supp = np.zeros(L)
    supp[[n - 1, n + 1]] = 1.0
    sets = [set(np.nonzero(np.linalg.matrix_power(hop, k) @ supp)[0]) for k in range(3)]
    assert [len(s) for s in sets] == [gd["N0"], gd["N1"], gd["N2"]]
    for mi, expect in ((1, gd["N1_first_example"]), (2, gd["ball_m2_offsets"])):
        o = Oracle(L, W.CHAIN, J=1.0, omega=1.0, g=0.0, cap=0, m=2, m_init=mi)
        o.set_state([n - 1, n + 1], np.zeros((2, L), dtype=np.int32), [2 ** -0.5] * 2)
        t, _ = o.rows()
        ball = set(t[:, 0].tolist())
        assert ball == set.union(*sets[: mi + 1])
        if mi == 1:
            assert set(t[2:, 0] - n) == set(expect)
        else:
            assert len(ball) == gd["ball_m2"] and sorted(b - n for b in ball) == expect
        assert list(o.level_offsets()[: mi + 2]) == ([0, 2, 5] if mi == 1 else [0, 2, 5, 7])


@pytest.mark.parametrize("L,d", [(3, 4), (4, 3), (2, 6)])
def test_holstein_nonzero_count_formula(L, d):
    """App. C: the full-space open Holstein chain has d^L[(5L-2) - 2L/d] stored
    entries, counting every diagonal; the TB chain has 3L - 2."""
    o = Oracle(L, W.CHAIN, J=1.0, omega=1.0, g=0.8, cap=d - 1, m=2, m_init=-1)
    o.set_state([0], [[0] * L], [1.0])
    assert o.nrows() == L * d ** L
    cnt, cols, vals, diag = o.hamiltonian()
    assert len(cols) + o.nrows() == d ** L * (5 * L - 2) - 2 * L * d ** (L - 1)
    tb = Oracle(L, W.CHAIN, J=1.0, omega=1.0, g=0.0, cap=0, m=2, m_init=-1)
    tb.set_state([0], [[0] * L], [1.0])
    c2, cols2, _, _ = tb.hamiltonian()
    assert tb.nrows() == L and len(cols2) + L == 3 * L - 2


def test_paper_sparsity_numbers():
    """App. C printed figures for L = 9, d_pho = 5: 587 MiB of 64-bit nonzeros and
    2248 TiB dense, from the density formula."""
    gd = gold("sparsity_appC.json")
    L, d = gd["L"], gd["d_pho"]
    dim = L * d ** L
    density = ((5 * L - 2) - 2 * L / d) / (L * L * d ** L)
    nnz = round(density * dim * dim)
    assert nnz == gd["nonzero_count_from_density"]
    assert round(nnz * 8 / 2 ** 20) == gd["nonzeros_MiB"]
    assert math.floor(dim * dim * 8 / 2 ** 40) == gd["dense_TiB"]


# ---------------------------------------------------------------- invariants
def test_norm_and_energy_conservation_inside_steps():
    """Sec. 3.5 / Fig. error_sources: the propagator is unitary to machine precision
    inside H_eff (norm to 1e-13) and conserves c^dag H_P c; with the full space kept
    the energy is constant across steps."""
    cfg = W.WORKLOADS["ring4"]
    o = oracle_for(cfg, eps=np.array([0.1, -0.2, 0.3, 0.0]))
    o.set_state(np.arange(4), np.zeros((4, 4), dtype=np.int32), [0.5] * 4)
    E0 = None
    for _ in range(40):
        o.step(0.05, 0.0)
        st = o.stats()
        assert abs(st["norm"] - st["norm_phi0"]) < 1e-13
        E0 = st["energy"] if E0 is None else E0
        assert abs(st["energy"] - E0) < 1e-12 * max(1.0, abs(E0))
    assert abs(E0) > 0.05


def test_truncation_never_increases_norm():
    cfg = W.WORKLOADS["ring16"]
    o = oracle_for(cfg, m_init=4)
    o.set_state(*W.start_state(cfg))
    for _ in range(15):
        o.step(0.02, 1e-4)
        st = o.stats()
        assert st["norm_phi0"] <= st["norm_before"] + 1e-15
        assert st["kept"] <= st["rows"]


def test_sign_of_J_invariance_on_bipartite_ring():
    """J -> -J leaves populations and phonon numbers unchanged for a localised
    start on a bipartite lattice (App. H; gauge |s> -> (-1)^s |s>)."""
    cfg = W.WORKLOADS["ring4"]
    res = []
    for J in (1.0, -1.0):
        o = oracle_for(cfg, J=J, m_init=3)
        o.set_state(*W.start_state(cfg))
        for _ in range(60):
            o.step(0.05, 1e-6)
        res.append(o.populations())
    assert np.allclose(res[0][0], res[1][0], atol=1e-13, rtol=0)
    assert np.allclose(res[0][1], res[1][1], atol=1e-13, rtol=0)


def test_second_order_taylor_breaks_unitarity():
    """App. C.2: cutting the series at N_series = m = 2 makes the norm grow."""
    cfg = W.WORKLOADS["ring4"]
    good = oracle_for(cfg)
    bad = oracle_for(cfg, fixed_terms=2)
    for o in (good, bad):
        o.set_state(*W.start_state(cfg))
        for _ in range(100):
            o.step(0.05, 1e-8)
    assert abs(good.stats()["norm"] - 1.0) < 1e-12
    assert bad.stats()["norm"] > 1.0 + 1e-4


def test_taylor_nonconvergence_is_reported():
    """App. I: a step too large for the series is an error, not a silent result."""
    cfg = W.WORKLOADS["ring4"]
    o = oracle_for(cfg, nmax=6)
    o.set_state(*W.start_state(cfg))
    with pytest.raises(OracleError) as e:
        o.step(0.5, 1e-8)
    assert e.value.code == 4


def test_invalid_inputs_rejected():
    o = Oracle(3, W.RING, J=1.0, omega=1.0, g=1.0, cap=2, m=2, m_init=1)
    for site, occ in (([3], [[0, 0, 0]]), ([0], [[0, 3, 0]]), ([0, 0], [[0, 0, 0]] * 2)):
        with pytest.raises(OracleError):
            o.set_state(site, occ, [1.0] * len(site))


# ---------------------------------------------------------------- spectrum
def test_spectrum_of_single_line_matches_geometric_sum():
    """A(w) of C(t) = e^{-iEt}: the trapezoid sum is a geometric series with a
    closed form; the damping is e^{-t/tau}, 1/tau = 0.0577 (App. E)."""
    E, dt, K = 0.3, 0.05, 400
    C_t = np.exp(-1j * E * dt * np.arange(K + 1))
    grid = np.linspace(-2, 2, 41)
    A = absorption_spectrum(C_t, dt, grid)
    for w, a in zip(grid, A):
        z = (1j * (w - E) - 0.0577) * dt
        s = (1 - np.exp(z * (K + 1))) / (1 - np.exp(z)) - 0.5 * (1 + np.exp(z * K))
        assert abs(a - (s * dt).real) < 1e-11


# ---------------------------------------------------------------- gradients
def _loss_run(params, keeps=None, record=False, nsteps=12, theta=2e-3, xmax=8.0):
    J, g, w, eps = params
    o = Oracle(3, W.RING, J=J, eps=eps, omega=w, g=g, cap=2, m=1, m_init=1, xmax=xmax)
    o.set_state([0, 1], [[0, 0, 0], [0, 0, 0]], [0.8, 0.6j])
    if record:
        o.record(True)
    Cs, masks, Ps = [], [], []
    for k in range(nsteps):
        kp = None if keeps is None or k == 0 else keeps[k]
        o.step(0.1, theta, kp)
        masks.append(o.last_keep() if k > 0 else None)
        st = o.stats()
        Cs.append(st["C_re"] + 1j * st["C_im"])
        Ps.append(o.populations()[0])
    Cs, Ps = np.array(Cs), np.array(Ps)
    target = 0.3 * np.exp(-0.5j * np.arange(nsteps))
    P, _ = o.populations()
    L = P[0] + np.sum(np.abs(Cs - target) ** 2)
    return L, o, masks, Cs, target, Ps


@pytest.mark.parametrize("xmax", [8.0, 0.3], ids=["one-series", "substeps"])
def test_adjoint_matches_finite_differences(xmax):
    """Adjoint of the truncated Taylor map with the subspace sequence held fixed
    agrees with central differences of the same replayed map (extension; the paper
    has no gradient: parity pinned by finite differences); also when every step
    is split into several series."""
    eps = W.seeded_normal(3, 7) * 0.2
    base = (0.4, 0.7, 1.1, eps)
    L0, o, masks, Cs, target, _ = _loss_run(base, record=True, xmax=xmax)
    assert (o.stats()["substeps"] > 1) == (xmax < 1.0)
    t, a = o.rows()
    dL_dc = np.where(t[:, 0] == 0, 2.0 * a, 0.0)
    grad = o.backward(len(Cs), dL_dc_final=dL_dc, dL_dC=2.0 * (Cs - target))
    assert sum(m is not None and (~m).any() for m in masks) > 3   # truncation was active

    def perturbed(p, h):
        J, g, w, e = base
        e = e.copy()
        if p == 0: J += h
        elif p == 1: g += h
        elif p == 2: w += h
        else: e[p - 3] += h
        return (J, g, w, e)

    for p in range(3 + 3):
        h = 1e-5
        lp = _loss_run(perturbed(p, h), keeps=masks, xmax=xmax)[0]
        lm = _loss_run(perturbed(p, -h), keeps=masks, xmax=xmax)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(grad[p] - fd) <= 1e-6 * max(1.0, abs(fd)), (p, grad[p], fd)


def test_adjoint_population_cotangents_match_finite_differences():
    """Loss sum_k sum_s a_ks P_s(t_k)^2 of the site populations after every
    step: the P_s cotangent 2 c_i dL/dP_s of the adjoint against central
    differences of the replayed map (extension; parity pinned by FD)."""
    eps = W.seeded_normal(3, 11) * 0.3
    base = (0.5, 0.9, 1.0, eps)
    a = W.seeded_normal(12 * 3, 12).reshape(12, 3)
    _, o, masks, _, _, Ps = _loss_run(base, record=True)
    grad = o.backward(len(Ps), dL_dP=2.0 * a * Ps)
    assert sum(m is not None and (~m).any() for m in masks) > 3

    def loss(params):
        Ps = _loss_run(params, keeps=masks)[5]
        return float(np.sum(a * Ps * Ps))

    J, g, w, e = base
    for p in range(3 + 3):
        h = 1e-5
        vals = []
        for sgn in (1, -1):
            q = [J, g, w, e.copy()]
            if p < 3:
                q[p] += sgn * h
            else:
                q[3][p - 3] += sgn * h
            vals.append(loss(tuple(q)))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(grad[p] - fd) <= 1e-6 * max(1.0, abs(fd)), (p, grad[p], fd)


# ---------------------------------------------------------------- top-q_nom truncation
def test_tie_hash_mixer_is_splitmix64():
    """The tie-break hash folds the SplitMix64 output function (Steele, Lea &
    Flood 2014): checked against the separately written generator of the
    workload module."""
    o = Oracle(2, W.RING, J=1.0, cap=1, m=1, m_init=0)
    for seed in (0, 1, 12345, (1 << 64) - 7):
        assert o.tie_hash(seed, 0, [0]) == W.SplitMix64(seed).next_u64()
        a, b = 3, 11
        inner = W.SplitMix64(seed ^ a).next_u64()
        assert o.tie_hash(seed, 0, [a, b]) == W.SplitMix64(inner ^ b).next_u64()
    g = 0x9E3779B97F4A7C15
    assert o.tie_hash(5, 3, [2]) == W.SplitMix64(((5 + 3 * g) & ((1 << 64) - 1)) ^ 2).next_u64()


def _basis(nstates, N=4, cap=3):
    """The first nstates tuples of an enumeration of the ring basis."""
    out = []
    for s in range(N):
        for occ in np.ndindex(*([cap + 1] * N)):
            out.append((s,) + occ)
            if len(out) == nstates:
                return np.array(out, dtype=np.int32)
    return np.array(out, dtype=np.int32)


def test_top_q_keeps_the_heaviest_rows():
    tup = _basis(40)
    amp = W.seeded_normal(80, 91).reshape(40, 2) @ np.array([1.0, 1j])
    o = Oracle(4, W.RING, J=1.0, g=1.0, cap=3, m=1, m_init=0)
    o.set_state(tup[:, 0], tup[:, 1:], amp)
    t, a = o.rows()
    w = a.real * a.real + a.imag * a.imag
    assert len(np.unique(w)) == len(w)
    for q_nom in (1, 7, 25, 39):
        keep = o.nom_keep(q_nom)
        cut = np.sort(w)[::-1][q_nom - 1]
        assert np.array_equal(keep, w >= cut), q_nom
    assert o.nom_keep(40).all() and o.nom_keep(1000).all()


def test_top_q_tie_break_is_unbiased():
    """Eight states of exactly equal weight compete for two places: over 400
    seeds each is kept about 100 times (App. D: randomise degenerate states at
    the cutoff), and the four heavier states are always kept."""
    tup = _basis(12)
    amp = np.concatenate([np.full(4, 0.4), np.full(8, 0.1)]).astype(np.complex128)
    o = Oracle(4, W.RING, J=1.0, g=1.0, cap=3, m=1, m_init=0)
    o.set_state(tup[:, 0], tup[:, 1:], amp)
    t, a = o.rows()
    heavy = np.abs(a) > 0.2
    counts = np.zeros(len(a))
    for seed in range(400):
        keep = o.nom_keep(6, seed)
        assert keep.sum() == 6 and keep[heavy].all()
        counts += keep
    tied = counts[~heavy]
    assert np.all((tied >= 60) & (tied <= 140)), tied
    assert tied.sum() == 800


def test_step_nom_equals_the_same_mask_as_override():
    cfg = W.WORKLOADS["ring4"]
    mk = lambda: Oracle(**W.model_kwargs(cfg))
    a, b = mk(), mk()
    for o in (a, b):
        o.set_state(*W.start_state(cfg))
        o.step(0.1, 0.0)
    for k in range(6):
        keep = b.nom_keep(60, 77)
        a.step_nom(0.1, 60, 77)
        b.step(0.1, 0.0, keep=keep.astype(np.uint8))
        ta, ca = a.rows()
        tb, cb = b.rows()
        assert np.array_equal(ta, tb) and np.array_equal(ca, cb)
        assert a.stats()["kept"] == 60


def test_kept_set_is_in_ascending_basis_order():
    """After a truncating step the first |M| rows are the kept states in
    ascending basis order (n_{N-1} most significant, then down to n_0, then
    s), and they are exactly the states of the previous step that reached
    theta (Sec. 3.3: truncation, then regrowth appended after M)."""
    cfg = W.WORKLOADS["ring4"]
    o = Oracle(**W.model_kwargs(cfg))
    o.set_state(*W.start_state(cfg))
    for k in range(6):
        t_prev, a_prev = o.rows()
        o.step(0.1, 2e-3)
        if k == 0:
            continue
        kept = int(o.stats()["kept"])
        t, _ = o.rows()
        M = t[:kept]
        order = np.lexsort([M[:, c] for c in range(M.shape[1])])   # last column is primary
        assert np.array_equal(order, np.arange(kept))
        w = np.abs(a_prev) ** 2
        want = {tuple(r) for r in t_prev[w >= 2e-3 ** 2]}
        assert {tuple(r) for r in M} == want


# ---------------------------------------------------------------- rescue, 3D geometry, energy value
def _ring4_dense():
    N = 4
    eps = np.array([0.1, -0.2, 0.3, 0.0])
    H, D, strides = dense_holstein(ring_hop(N, 1.0), eps, [1.0] * N, [1.0] * N, [4] * N)
    return eps, H, D, strides


def _rescue_run(mutant=None, nsteps=60):
    """ring4 with m = 30, a radius from which every kept set reaches the whole
    2500-state space, truncated hard (theta = 1e-2).  Rescue (Sec. 3.3,
    post-adaptation detruncation) gives every dropped amplitude back, so the
    trajectory is exp(-iHt) psi0 although most rows fall below theta."""
    eps, H, D, strides = _ring4_dense()
    U = propagator(H)
    o = Oracle(4, W.RING, J=1.0, eps=eps, omega=1.0, g=1.0, cap=4, m=30, m_init=-1, mutant=mutant)
    o.set_state([0], [[0] * 4], [1.0])
    psi0 = state_vector(o, D, strides, H.shape[0])
    kept = []
    for k in range(1, nsteps + 1):
        o.step(0.05, 1e-2)
        st = o.stats()
        assert st["rows"] == 2500
        kept.append(st["kept"])
    err = np.linalg.norm(state_vector(o, D, strides, H.shape[0]) - U(nsteps * 0.05, psi0))
    return err, kept


def test_rescue_restores_every_dropped_amplitude():
    err, kept = _rescue_run()
    assert max(kept[1:]) < 2500 and min(kept[1:]) < 500, kept      # truncation really dropped rows
    assert err <= 1e-11, err


def test_rescue_pin_fails_without_rescue():
    err, _ = _rescue_run(mutant="NO_RESCUE")
    assert err > 1e-3, err


def _cubic_adjacency(dims):
    """Open simple-cubic nearest neighbours from the coordinates, built here:
    site j = x + d0 (y + d1 z)."""
    d0, d1, d2 = dims
    coords = [(x, y, z) for z in range(d2) for y in range(d1) for x in range(d0)]
    N = len(coords)
    A = np.zeros((N, N))
    for a, ca in enumerate(coords):
        for b, cb in enumerate(coords):
            if sum(abs(u - v) for u, v in zip(ca, cb)) == 1:
                A[a, b] = 1.0
    assert coords[1] == (1, 0, 0) and coords[d0] == (0, 1, 0) and coords[d0 * d1] == (0, 0, 1)
    return A


@pytest.mark.parametrize("dims", [(2, 2, 2), (3, 2, 2), (2, 3, 4)])
def test_open3d_hopping_matches_hand_built_lattice(dims):
    """Eq. holstein on the open simple-cubic aggregates of Sec. 5: J_ab = J
    for nearest neighbours.  Every site of the 2x2x2 cube is a corner with
    three neighbours."""
    N = int(np.prod(dims))
    o = Oracle(N, W.OPEN3D, dims=dims, J=0.7, omega=1.0, g=0.0, cap=1, m=1, m_init=1)
    A = _cubic_adjacency(dims)
    assert np.array_equal(o.hopping(), 0.7 * A)
    if dims == (2, 2, 2):
        assert np.all(A.sum(1) == 3)


def test_open3d_pin_fails_on_exchanged_axes():
    o = Oracle(12, W.OPEN3D, dims=(3, 2, 2), J=1.0, omega=1.0, g=0.0, cap=1, m=1, m_init=1,
               mutant="OPEN3D_AXES")
    assert not np.array_equal(o.hopping(), _cubic_adjacency((3, 2, 2)))


def test_open3d_g0_autocorrelation_matches_eigh():
    """g = 0 on the 3x2x2 aggregate: the phonons stay in vacuum and
    C(t) = sum_k |<k|mu>|^2 exp(-i E_k t) from eigh of the exciton matrix built
    from the hand-made lattice (bright state mu = sum_s |s>/sqrt(N))."""
    dims = (3, 2, 2)
    N = 12
    A = _cubic_adjacency(dims)
    E, V = np.linalg.eigh(-1.0 * A)
    mu = np.ones(N) / np.sqrt(N)
    w = (V.T @ mu) ** 2
    o = Oracle(N, W.OPEN3D, dims=dims, J=-1.0, omega=1.0, g=0.0, cap=2, m=2, m_init=2)
    o.set_state(np.arange(N), np.zeros((N, N), dtype=np.int32), mu)
    dt = 0.05
    for k in range(1, 81):
        o.step(dt, 1e-12)
        st = o.stats()
        C = st["C_re"] + 1j * st["C_im"]
        assert abs(C - np.sum(w * np.exp(-1j * E * k * dt))) < 1e-12


def _energy_run(mutant=None):
    """The energy record of a step is <c'|P H P|c'> with c' the rescued state
    entering the propagator (Sec. 3.5).  c' is rebuilt here from the previous
    step's rows restricted to the new H_eff, and E compared with c'^dag H c'
    for the dense Kronecker-product H (P c' = c', so P H P gives the same)."""
    eps, H, D, strides = _ring4_dense()
    o = Oracle(4, W.RING, J=1.0, eps=eps, omega=1.0, g=1.0, cap=4, m=2, m_init=2, mutant=mutant)
    o.set_state([0, 1], [[0] * 4, [1, 0, 0, 0]], [0.6, 0.8j])
    worst = 0.0
    prev = state_vector(o, D, strides, H.shape[0])
    for _ in range(25):
        o.step(0.05, 2e-3)
        t, _ = o.rows()
        cp = np.zeros_like(prev)
        idx = dense_index(t, D, strides)
        cp[idx] = prev[idx]
        E_ref = float(np.real(np.vdot(cp, H @ cp)))
        worst = max(worst, abs(o.stats()["energy"] - E_ref) / max(1.0, abs(E_ref)))
        prev = state_vector(o, D, strides, H.shape[0])
    return worst


def test_energy_value_is_the_expectation_in_the_rescued_state():
    assert _energy_run() < 1e-13


def test_energy_pin_fails_on_a_dropped_conjugate():
    assert _energy_run(mutant="ENERGY_CONJ") > 1e-3


# ---------------------------------------------------------------- substepping (App. C.1, App. I)
def _ring4_state_after(dt, nsteps, xmax):
    eps, H, D, strides = _ring4_dense()
    o = Oracle(4, W.RING, J=1.0, eps=eps, omega=1.0, g=1.0, cap=4, m=2, m_init=-1, xmax=xmax)
    o.set_state([0], [[0] * 4], [1.0])
    psi0 = state_vector(o, D, strides, H.shape[0])
    for _ in range(nsteps):
        o.step(dt, 0.0)
    return o, state_vector(o, D, strides, H.shape[0]), propagator(H)(nsteps * dt, psi0)


def test_large_dt_substeps_match_dense_expm():
    """App. I: past a threshold in dt the single-series step fails and the norm
    explodes (here dt = 3 on the full ring4 space, ||H|| = 19.4: the norm
    grows past 1e100).  Split into s = ceil(rho dt / 8) series (App. C.1's
    scaling), the same steps equal exp(-iHt) psi0 to 1e-12."""
    o, v, ref = _ring4_state_after(3.0, 10, 8.0)
    st = o.stats()
    assert st["substeps"] == math.ceil(st["hbound"] * 3.0 / 8.0) and st["substeps"] >= 8
    assert np.linalg.norm(v - ref) <= 1e-12
    o1, v1, _ = _ring4_state_after(3.0, 10, 0.0)
    assert o1.stats()["substeps"] == 1 and o1.stats()["norm"] > 1e100


@pytest.mark.parametrize("dt", [0.05, 0.5, 1.5])
def test_substeps_are_exact_at_moderate_dt(dt):
    o, v, ref = _ring4_state_after(dt, 6, 8.0)
    assert np.linalg.norm(v - ref) <= 1e-12


def test_hbound_bounds_the_restricted_norm():
    """rho (largest row sum of |eps_s| + sum_j |omega_j| n_j + the absolute
    off-diagonal elements of H over H_eff, each term rounded up to 2^-20) is an
    upper bound of ||P H P||_2; checked against that sum taken from the dense H
    (off-diagonal part) and the tuples (diagonal part)."""
    eps, H, D, strides = _ring4_dense()
    o = Oracle(4, W.RING, J=1.0, eps=eps, omega=1.0, g=1.0, cap=4, m=2, m_init=2)
    o.set_state([0], [[0] * 4], [1.0])
    for _ in range(8):
        o.step(0.05, 1e-3)
        t, _ = o.rows()
        idx = dense_index(t, D, strides)
        HP = H[np.ix_(idx, idx)]
        rho = o.stats()["hbound"]
        off = np.abs(H[idx]).sum(1) - np.abs(H[idx, idx])
        rowsum = np.max(off + np.abs(eps[t[:, 0]]) + t[:, 1:].sum(1))
        assert np.max(np.abs(np.linalg.eigvalsh(HP))) <= rho
        assert rowsum <= rho <= rowsum + 12 * 2.0 ** -20


def test_load_state_continues_the_trajectory_exactly():
    """A state taken from step k and loaded into a fresh oracle (with the same
    psi(0)) continues bit for bit as the uninterrupted run: the test
    infrastructure the GPU parity at scale relies on."""
    cfg = W.WORKLOADS["ring16"]
    a = oracle_for(cfg, m_init=4)
    a.set_state(*W.start_state(cfg))
    for _ in range(6):
        a.step(0.02, 1e-5)
    t, amp = a.rows()
    b = oracle_for(cfg, m_init=4)
    b.set_state(*W.start_state(cfg))
    b.load_state(t[:, 0], t[:, 1:], amp)
    for _ in range(3):
        a.step(0.02, 1e-5)
        b.step(0.02, 1e-5)
        ta, aa = a.rows()
        tb, ab = b.rows()
        assert np.array_equal(ta, tb) and np.array_equal(aa, ab)
        sa, sb = a.stats(), b.stats()
        assert all(sa[k] == sb[k] for k in sa if k != "time")     # b's clock started at its set_state


# ---------------------------------------------------------------- Lanczos propagator (App. C.3)
def _lanczos_tb_basis(mutant=None):
    """Lanczos vectors of one step from psi' = (|n-1> + |n> + |n+1>)/sqrt(3) on an
    open tight-binding chain (g = 0, eps = 0, J = 1), rows n-4..n+4."""
    N, n = 21, 10
    o = Oracle(N, W.CHAIN, J=1.0, g=0.0, omega=1.0, cap=0, m=2, m_init=-1, propagator=1, kmax=30,
               mutant=mutant)
    o.set_state([n - 1, n, n + 1], np.zeros((3, N), dtype=np.int32), np.ones(3) / math.sqrt(3.0))
    o.step(0.05, 0.0)
    V = o.krylov_basis()
    t, _ = o.rows()
    sites = list(t[:, 0])
    g = gold("lanczos_V4_appC3.json")
    idx = [sites.index(n + d) for d in g["rows_offset"]]
    outside = [i for i in range(len(sites)) if i not in idx]
    return V, idx, outside, g


def test_lanczos_basis_matches_the_paper_V4():
    """App. C.3 prints V_4 for this state: the first four Lanczos vectors of the
    oracle equal it entry by entry (24 non-zeros) and vanish off rows n-4..n+4."""
    V, idx, outside, g = _lanczos_tb_basis()
    ref = np.array([[a * math.sqrt(b) for a, b in row] for row in g["entries_as_a_sqrt_b"]]) / g["scale"]
    assert V.shape[1] >= 4
    assert np.max(np.abs(V[idx, :4] - ref)) <= 1e-14
    assert np.count_nonzero(np.abs(ref) > 0) == g["nonzeros"]
    assert np.max(np.abs(V[outside, :4])) == 0.0
    # orthonormal basis
    G = V.conj().T @ V
    assert np.max(np.abs(G - np.eye(V.shape[1]))) <= 1e-13


def test_lanczos_pin_fails_without_the_beta_term():
    V, idx, _, g = _lanczos_tb_basis(mutant="LANCZOS_NO_BETA")
    ref = np.array([[a * math.sqrt(b) for a, b in row] for row in g["entries_as_a_sqrt_b"]]) / g["scale"]
    assert np.max(np.abs(V[idx, :4] - ref)) > 1e-2


@pytest.mark.parametrize("dt,nsteps", [(0.05, 40), (0.5, 6), (3.0, 4)])
def test_lanczos_full_space_matches_dense_expm(dt, nsteps):
    """ring4 with its whole 2500-state space every step (theta = 0): the Lanczos
    step exp(-i h H) v ~ beta_0 V_n exp(-i h T_n) e_1 equals exp(-iHt) psi0 to
    1e-12; at dt = 3 the step splits into the same substeps as the series."""
    eps, H, D, strides = _ring4_dense()
    U = propagator(H)
    o = Oracle(4, W.RING, J=1.0, eps=eps, omega=1.0, g=1.0, cap=4, m=2, m_init=-1, propagator=1, kmax=40)
    o.set_state([0], [[0] * 4], [1.0])
    psi0 = state_vector(o, D, strides, H.shape[0])
    for _ in range(nsteps):
        o.step(dt, 0.0)
    st = o.stats()
    assert st["substeps"] == max(1, math.ceil(st["hbound"] * dt / 8.0))
    assert st["terms"] <= 40 * st["substeps"]
    v = state_vector(o, D, strides, H.shape[0])
    assert np.linalg.norm(v - U(nsteps * dt, psi0)) <= 1e-12
    assert abs(st["energy"] - np.vdot(v, H @ v).real) <= 1e-10     # E of c', conserved by the step


def test_lanczos_two_site_breakdown_is_exact():
    """N = 2, g = 0: the Krylov space of |0> is two-dimensional, so the
    recurrence ends (beta_2 = 0) after two vectors and the step is exact:
    P_1 = sin^2(J t)."""
    o = Oracle(2, W.RING, J=1.0, omega=1.0, g=0.0, cap=1, m=2, m_init=-1, propagator=1, kmax=10)
    o.set_state([0], [[0, 0]], [1.0])
    for k in range(1, 61):
        o.step(0.1, 0.0)
        assert o.stats()["terms"] <= 2
        P, _ = o.populations()
        assert abs(P[1] - math.sin(0.1 * k) ** 2) < 1e-13


def test_lanczos_agrees_with_the_series_on_a_truncated_trajectory():
    """Both propagators approximate the same exp(-i P H P dt) to 1e-15 per step;
    on a truncated ring16 prefix the rows stay identical and the amplitudes
    within 1e-12 normwise."""
    cfg = W.WORKLOADS["ring16"]
    kw = W.model_kwargs(cfg, m_init=4)
    a, b = Oracle(**kw), Oracle(**kw, propagator=1, kmax=30)
    for o in (a, b):
        o.set_state(*W.start_state(cfg))
    for _ in range(12):
        a.step(0.02, 1e-5)
        b.step(0.02, 1e-5)
        ta, aa = a.rows()
        tb, ab = b.rows()
        assert np.array_equal(ta, tb)
        assert np.max(np.abs(aa - ab)) <= 1e-12 * np.linalg.norm(aa)
    assert b.stats()["terms"] < a.stats()["terms"]


def test_lanczos_rejects_recording_and_bad_dimensions():
    with pytest.raises(OracleError):
        Oracle(2, W.RING, J=1.0, g=0.0, cap=1, propagator=1, kmax=0)
    o = Oracle(2, W.RING, J=1.0, g=0.0, cap=1, propagator=1, kmax=8)
    o.record(True)
    o.set_state([0], [[0, 0]], [1.0])
    with pytest.raises(OracleError):
        o.step(0.05, 0.0)


# ---------------------------------------------------------------- piecewise-constant time dependence (Sec. 6)
def _drive(t):
    """Coefficients of a driven ring4 at time t: J, eps, omega, g."""
    return (1.0 + 0.3 * math.sin(1.3 * t), np.array([0.1, -0.2, 0.3, 0.0]) * math.cos(0.7 * t),
            np.full(4, 1.0 + 0.1 * math.sin(t)), np.full(4, 1.0 + 0.2 * math.cos(t)))


def test_piecewise_constant_H_matches_the_product_of_dense_exponentials():
    """H replaced before every step (the paper's extension to Hamiltonians that
    are piecewise constant in time): over ring4's full space (theta = 0) the
    state is U_K ... U_1 psi0 (phonon cap 3: 1024 states), U_k = exp(-i H(t_k) dt) from the dense Kronecker
    H of that step's coefficients."""
    dt, K = 0.05, 30
    J, eps, omega, g = _drive(0.0)
    o = Oracle(4, W.RING, J=J, eps=eps, omega=omega, g=g, cap=3, m=2, m_init=-1)
    o.set_state([0], [[0] * 4], [1.0])
    H0, D, strides = dense_holstein(ring_hop(4, J), eps, omega, g, [3] * 4)
    psi = state_vector(o, D, strides, H0.shape[0])
    for k in range(K):
        J, eps, omega, g = _drive(k * dt)
        o.set_coefficients(J, eps, omega, g)
        o.step(dt, 0.0)
        H, _, _ = dense_holstein(ring_hop(4, J), eps, omega, g, [3] * 4)
        psi = propagator(H)(dt, psi)
    assert np.linalg.norm(state_vector(o, D, strides, H0.shape[0]) - psi) <= 1e-12


def test_uniform_site_energy_drive_is_a_global_phase():
    """eps_s(t) = f(t) on every site adds f(t) times the identity: the truncated
    trajectory keeps its rows, populations and phonon numbers, and C(t) picks up
    exp(-i sum_k f(t_k) dt)."""
    cfg = W.WORKLOADS["ring16"]
    kw = W.model_kwargs(cfg, m_init=4)
    a, b = Oracle(**kw), Oracle(**kw)
    for o in (a, b):
        o.set_state(*W.start_state(cfg))
    phase = 0.0
    for k in range(15):
        f = 0.5 * math.cos(2.0 * k * 0.02)
        b.set_coefficients(cfg["J"], eps=np.full(16, f))
        phase += f * 0.02
        a.step(0.02, 1e-5)
        b.step(0.02, 1e-5)
        ta, _ = a.rows()
        tb, _ = b.rows()
        assert np.array_equal(ta, tb)
        Pa, na = a.populations()
        Pb, nb = b.populations()
        assert np.max(np.abs(Pa - Pb)) <= 1e-12 and np.max(np.abs(na - nb)) <= 1e-11
        sa, sb = a.stats(), b.stats()
        Ca, Cb = sa["C_re"] + 1j * sa["C_im"], sb["C_re"] + 1j * sb["C_im"]
        assert abs(Cb - Ca * np.exp(-1j * phase)) <= 1e-12


def test_coefficient_updates_keep_the_move_graph():
    o = Oracle(4, W.RING, J=1.0, omega=1.0, g=1.0, cap=4, m=2, m_init=2)
    for bad in (dict(J=0.0), dict(J=1.0, g=[1.0, 0.0, 1.0, 1.0]), dict(J=float("nan"))):
        with pytest.raises(OracleError):
            o.set_coefficients(**bad)
    o.set_coefficients(0.5, g=[2.0] * 4)
    o.record(True)
    with pytest.raises(OracleError):
        o.set_coefficients(1.0)
