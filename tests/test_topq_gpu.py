"""Top-q_nom truncation (the paper's scheme) on the GPU against the oracle.

The GPU's amplitudes agree with the oracle's to rounding (the propagator sums
in another order), so the kept sets may differ only for rows whose weight
sits within rounding of the cut; there the oracle adopts the GPU's mask (the
lockstep protocol of the threshold parity tests).  Degenerate weights are resolved by the seeded tie hash, checked
against the oracle's implementation of the same published generator.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2603_07341_gb300 import binding as B
from paper_2603_07341_gb300 import workloads as W

pytestmark = pytest.mark.gpu
AMP_TOL = 1e-10


def _ring16(**over):
    cfg = W.WORKLOADS["ring16"]
    return cfg, W.model_kwargs(cfg, **over)


def _lockstep_nom(gpu, ora, dt, q_nom, seed, nsteps):
    adopted = 0
    for k in range(nsteps):
        t_before, a_before = ora.rows()
        okeep = ora.nom_keep(q_nom, seed) if k > 0 else None
        gpu.step_nom(dt, 1, q_nom, seed)
        if k == 0:
            ora.step_nom(dt, q_nom, seed)
        else:
            gkeep = gpu.keep()
            assert len(gkeep) == len(okeep)
            diff = gkeep != okeep
            if diff.any():
                w = np.abs(a_before) ** 2
                wcut = np.sort(w)[::-1][q_nom - 1]
                band = np.abs(w - wcut) <= 1e-12 * wcut + 1e-300
                assert np.all(band[diff]), "mask differs away from the cut"
                adopted += int(diff.sum())
                ora.step(dt, 0.0, keep=gkeep.astype(np.uint8))
            else:
                ora.step_nom(dt, q_nom, seed)
            rec = gpu.observables(gpu.num_records() - 1, 1)[0]
            if len(okeep) > q_nom:
                assert rec[B.OBS_FIELDS.index("kept")] == q_nom
        tg, ag = gpu.tuples()
        to, ao = ora.rows()
        assert np.array_equal(tg, to), "rows differ at step %d" % k
        assert np.max(np.abs(ag - ao)) <= AMP_TOL * np.linalg.norm(ao)
    return adopted


@pytest.mark.parametrize("precision", [B.C128, B.DW])
def test_topq_lockstep_ring16(libpaces, precision):
    cfg, model = _ring16(m_init=6)
    gpu = B.Solver(**model, precision=precision)
    ora = Oracle(**model)
    gpu.set_state(*W.start_state(cfg))
    ora.set_state(*W.start_state(cfg))
    adopted = _lockstep_nom(gpu, ora, cfg["dt"], 3000, 12345, 25)
    assert adopted <= 25
    rec = gpu.observables(1, 25)
    rows, kept = rec[:, 6], rec[:, 7]
    assert np.all(kept[1:] <= 3000) and np.any(kept[1:] == 3000)
    assert np.all(rows[1:] >= kept[1:])            # q_true >= q_nom after regrowth


def _degenerate_state(n_heavy=5, n_tied=16, N=4, cap=3):
    tup = []
    for s in range(N):
        for occ in np.ndindex(*([cap + 1] * N)):
            tup.append((s,) + occ)
    tup = np.array(tup[: n_heavy + n_tied], dtype=np.int32)
    amp = np.concatenate([np.full(n_heavy, 0.3), np.full(n_tied, 0.05)]).astype(np.complex128)
    return tup, amp


@pytest.mark.parametrize("precision", [B.C128, B.DW])
def test_topq_degenerate_weights_follow_the_tie_hash(libpaces, precision):
    """load_state (a mid-trajectory state; the next step truncates) with
    sixteen states of identical weight competing for places: the kept rows
    are the ones the published tie hash orders first."""
    cfg = dict(W.WORKLOADS["ring4"], cap=3)
    model = W.model_kwargs(cfg, m_init=1)
    tup, amp = _degenerate_state()
    helper = Oracle(**model)
    w = amp.real * amp.real + amp.imag * amp.imag
    for seed in (0, 1, 99, 2 ** 63 + 5):
        gpu = B.Solver(**model, precision=precision)
        gpu.load_state(tup[:, 0], tup[:, 1:], amp)
        gpu.step_nom(0.01, 1, 9, seed)
        keep = gpu.keep()
        # t = index of the record the step writes: 0 after a bare load_state
        tk = np.array([(helper.tie_hash(seed, 0, list(t)) & 0xFFFFFFFF00000000) | (0xFFFFFFFF - i)
                       for i, t in enumerate(tup)], dtype=np.uint64)
        order = sorted(range(len(w)), key=lambda i: (-w[i], -int(tk[i])))
        want = np.zeros(len(w), bool)
        want[order[:9]] = True
        assert np.array_equal(keep, want), seed
        gpu.close()


def test_topq_small_state_keeps_everything(libpaces):
    cfg, model = _ring16(m_init=2)
    gpu = B.Solver(**model)
    gpu.set_state(*W.start_state(cfg))
    gpu.step_nom(cfg["dt"], 3, 10 ** 9, 7)
    rec = gpu.observables(1, 3)
    assert np.array_equal(rec[1:, 7], rec[:-1, 6])          # kept = all rows of the previous step


def test_topq_graph_replay_is_bitwise(libpaces):
    cfg, model = _ring16(m_init=6)
    runs = []
    for graphs in (0, 1):
        s = B.Solver(**model)
        s.set_tuning(use_graphs=graphs)
        s.set_state(*W.start_state(cfg))
        s.step_nom(cfg["dt"], 20, 2000, 3)
        runs.append(s.tuples())
        s.close()
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])


def test_topq_gradient_replays_its_masks(libpaces):
    cfg = dict(W.WORKLOADS["ring4"], cap=3, g=0.8, J=0.6)
    model = W.model_kwargs(cfg, eps=W.seeded_normal(4, 21) * 0.3, m_init=2)
    gpu = B.Solver(**model, precision=B.C128)
    ora = Oracle(**model)
    start = (np.array([0, 1], np.int32), np.zeros((2, 4), np.int32), np.array([0.8, 0.6j]))
    gpu.record(4)
    gpu.set_state(*start)
    ora.set_state(*start)
    ora.record(True)
    _lockstep_nom(gpu, ora, 0.1, 40, 5, 14)
    dC = W.seeded_normal(28, 3).reshape(14, 2) @ np.array([1.0, 1j])
    g_gpu = gpu.backward(14, dL_dC=dC)
    g_ora = ora.backward(14, dL_dC=dC)
    assert np.all(np.abs(g_gpu - g_ora) <= 1e-9 * np.maximum(1.0, np.abs(g_ora)))


def test_topq_invalid_arguments(libpaces):
    cfg, model = _ring16(m_init=2)
    s = B.Solver(**model)
    s.set_state(*W.start_state(cfg))
    with pytest.raises(B.PacesError) as e:
        s.step_nom(0.02, 1, 0, 1)
    assert e.value.code == B.ERR_INVALID
    s.close()
    s = B.Solver(**model, batch=2)
    s.set_state(*W.start_state(cfg))
    with pytest.raises(B.PacesError) as e:
        s.step_nom(0.02, 1, 100, 1)
    assert e.value.code == B.ERR_UNSUPPORTED


@pytest.mark.parametrize("precision", [B.C128, B.DW])
def test_topq_paper_benchmark_chain_prefix(libpaces, precision):
    """The paper's g = 4 benchmark shape (open chain N = 25, K = 63, three-word
    keys) at a small q_nom: lockstep with the oracle over the first steps."""
    cfg = W.WORKLOADS["chain25"]
    model = W.model_kwargs(cfg, m_init=4)
    gpu = B.Solver(**model, precision=precision)
    ora = Oracle(**model)
    gpu.set_state(*W.start_state(cfg))
    ora.set_state(*W.start_state(cfg))
    _lockstep_nom(gpu, ora, cfg["dt"], 1500, 2603073410, 10)


def test_qtrue_over_qnom_matches_the_papers_1d_estimate(libpaces):
    """For the 1D Holstein chain the paper finds q_true ~ 2^(m-1) 2.5 q_nom
    (Sec. 3.3, after Eq. qtrue: about 170e6 rows at q_nom = 32e6, m = 2).  The
    chain25 model at a smaller q_nom, once truncation is active: the ratio of
    regrown to kept rows stays near 5."""
    cfg = W.WORKLOADS["chain25"]
    s = B.Solver(**W.model_kwargs(cfg))
    s.set_state(*W.start_state(cfg))
    s.step_nom(cfg["dt"], 250, 2_000_000, 1)
    rec = s.observables(231, 20)
    rows, kept = rec[:, 6], rec[:, 7]
    assert np.all(kept == 2_000_000)
    ratio = rows / kept
    assert np.all((ratio > 4.0) & (ratio < 7.0)), ratio
