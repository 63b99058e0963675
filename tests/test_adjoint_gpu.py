"""Reverse pass (gradient extension) of the GPU path against the oracle's adjoint.

The oracle's adjoint is pinned to central differences of the replayed map
(tests/test_oracle_pins.py).  Here the GPU gradient of the same recorded map
-- same subspace sequence: the oracle adopts the GPU's truncation mask where
the two differ within rounding of theta^2 -- must agree with it to 1e-9
relative (FP64 adjoint over double-word or FP64 forward amplitudes), and
the full-size gradient workload (4x4x4 cube) is checked by a directional
derivative against central differences of the GPU forward itself.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2603_07341_gb300 import binding as B
from paper_2603_07341_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GRAD_TOL = 1e-9


def _lockstep(gpu, ora, dt, theta, nsteps):
    """Advance both one step at a time, the oracle adopting the GPU mask."""
    for k in range(nsteps):
        _, a_before = ora.rows()
        gpu.step(dt, 1, theta)
        gkeep = gpu.keep()
        if len(gkeep) and k > 0:
            w = np.abs(a_before) ** 2
            diff = gkeep != (w >= theta * theta)
            if diff.any():
                band = np.abs(w - theta * theta) <= 1e-9 * theta * theta + 1e-10 * np.sum(w)
                assert np.all(band[diff])
                ora.step(dt, theta, keep=gkeep.astype(np.uint8))
                continue
        ora.step(dt, theta)


def _cotangents(q, nsteps, N, seed):
    z = W.seeded_normal(2 * q + 2 * nsteps + nsteps * N, seed)
    dfin = z[0:2 * q:2] + 1j * z[1:2 * q:2]
    o = 2 * q
    dC = z[o:o + 2 * nsteps:2] + 1j * z[o + 1:o + 2 * nsteps:2]
    dP = z[o + 2 * nsteps:].reshape(nsteps, N)
    return dfin, dC, dP


def _case(model, start, dt, theta, nsteps, every, precision, seed):
    gpu = B.Solver(**model, precision=precision)
    ora = Oracle(**model)
    gpu.record(every)
    gpu.set_state(*start)
    ora.set_state(*start)
    ora.record(True)
    _lockstep(gpu, ora, dt, theta, nsteps)
    tg, ag = gpu.tuples()
    to, ao = ora.rows()
    assert np.array_equal(tg, to)
    dfin, dC, dP = _cotangents(len(ag), nsteps, model["n_sites"], seed)
    g_gpu = gpu.backward(nsteps, dL_dc_final=dfin, dL_dC=dC, dL_dP=dP)
    g_ora = ora.backward(nsteps, dL_dc_final=dfin, dL_dC=dC, dL_dP=dP)
    err = np.abs(g_gpu - g_ora)
    assert np.all(err <= GRAD_TOL * np.maximum(1.0, np.abs(g_ora))), (g_gpu, g_ora)
    return gpu, g_gpu


def _ring_model():
    eps = W.seeded_normal(4, 21) * 0.3
    cfg = dict(W.WORKLOADS["ring4"], cap=3, g=0.8, J=0.6)
    return W.model_kwargs(cfg, eps=eps, m_init=2)


@pytest.mark.parametrize("precision", [B.DW, B.C128])
def test_ring_gradient_matches_oracle(libpaces, precision):
    model = _ring_model()
    start = (np.array([0, 1], np.int32), np.zeros((2, 4), np.int32), np.array([0.8, 0.6j]))
    gpu, _ = _case(model, start, 0.1, 2e-3, 23, 5, precision, 31)
    kept = gpu.observables(1, 23)[:, B.OBS_FIELDS.index("kept")]
    rows = gpu.observables(1, 23)[:, B.OBS_FIELDS.index("rows")]
    assert np.any(kept[1:] < rows[:-1])          # truncation was active


def test_cube_gradient_matches_oracle(libpaces):
    """2x2x2 open cube, per-site energies: every eps_s bin and several segments."""
    eps = W.seeded_normal(8, 41) * 0.2
    cfg = dict(W.WORKLOADS["cube4"], n_sites=8, dims=(2, 2, 2), cap=2)
    model = W.model_kwargs(cfg, eps=eps, m_init=2)
    _case(model, W.start_state(cfg), 0.05, 1e-3, 16, 4, B.DW, 51)


def test_backward_restores_state_and_is_deterministic(libpaces):
    model = _ring_model()
    start = (np.array([0], np.int32), np.zeros((1, 4), np.int32), np.array([1.0 + 0j]))
    a = B.Solver(**model)
    b = B.Solver(**model)
    a.record(3)
    for s in (a, b):
        s.set_state(*start)
        s.step(0.1, 10, 2e-3)
    t0, c0 = a.tuples()
    rec0 = a.observables()
    dfin, dC, dP = _cotangents(len(c0), 10, 4, 61)
    g1 = a.backward(10, dL_dc_final=dfin, dL_dC=dC, dL_dP=dP)
    g2 = a.backward(10, dL_dc_final=dfin, dL_dC=dC, dL_dP=dP)
    assert np.array_equal(g1, g2)                      # bit for bit
    t1, c1 = a.tuples()
    assert np.array_equal(t0, t1) and np.array_equal(c0, c1)
    assert np.array_equal(rec0, a.observables())
    a.record(0)
    a.step(0.1, 5, 2e-3)
    b.step(0.1, 5, 2e-3)
    ta, ca = a.tuples()
    tb, cb = b.tuples()
    assert np.array_equal(ta, tb) and np.array_equal(ca, cb)


def test_backward_errors(libpaces):
    model = _ring_model()
    start = (np.array([0], np.int32), np.zeros((1, 4), np.int32), np.array([1.0 + 0j]))
    s = B.Solver(**model)
    s.set_state(*start)
    s.step(0.1, 3, 2e-3)
    with pytest.raises(B.PacesError) as e:
        s.backward(3)
    assert e.value.code == B.ERR_STATE
    s.record(2)
    s.step(0.1, 4, 2e-3)
    with pytest.raises(B.PacesError) as e:
        s.backward(3)
    assert e.value.code == B.ERR_INVALID
    with pytest.raises(B.PacesError) as e:
        s.set_tuning(grid_blocks_per_sm=2)
    assert e.value.code == B.ERR_STATE
    assert np.all(np.isfinite(s.backward(4)))
    s.close()
    s = B.Solver(**model, precision=B.C64_SPMV)
    with pytest.raises(B.PacesError) as e:
        s.record(2)
    assert e.value.code == B.ERR_UNSUPPORTED
    s.close()
    s = B.Solver(**model, batch=2)
    with pytest.raises(B.PacesError) as e:
        s.record(2)
    assert e.value.code == B.ERR_UNSUPPORTED


def test_autograd_function_matches_oracle(libpaces):
    import torch
    from paper_2603_07341_gb300.autograd import trajectory
    model = _ring_model()
    start = (np.array([0, 2], np.int32), np.zeros((2, 4), np.int32), np.array([0.6, 0.8j]))
    nsteps, dt, theta = 15, 0.1, 2e-3
    N = 4
    p0 = np.concatenate([[model["J"], model["g"][0], model["omega"][0]], model["eps"]])
    p = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    a = torch.from_numpy(W.seeded_normal(nsteps * N, 71).reshape(nsteps, N))
    target = torch.from_numpy(np.stack([0.3 * np.cos(0.5 * np.arange(nsteps)),
                                        -0.3 * np.sin(0.5 * np.arange(nsteps))], 1))
    C, P = trajectory(p, model, start, dt, nsteps, theta, ckpt_every=4)
    loss = torch.sum(a * P * P) + torch.sum((C - target) ** 2)
    loss.backward()
    # the oracle on the same map (no mask differences expected at this size: checked)
    ora = Oracle(**model)
    ora.set_state(*start)
    ora.record(True)
    Cs, Ps, rows = [], [], []
    for _ in range(nsteps):
        ora.step(dt, theta)
        st = ora.stats()
        Cs.append([st["C_re"], st["C_im"]])
        Ps.append(ora.populations()[0])
        rows.append(st["rows"])
    Cs, Ps = np.array(Cs), np.array(Ps)
    assert np.allclose(Cs, C.detach().numpy(), atol=1e-12)
    assert np.allclose(Ps, P.detach().numpy(), atol=1e-12)
    dC = 2.0 * (Cs - target.numpy())
    g_ora = ora.backward(nsteps, dL_dC=dC[:, 0] + 1j * dC[:, 1], dL_dP=2.0 * a.numpy() * Ps)
    g = p.grad.numpy()
    assert np.all(np.abs(g - g_ora) <= GRAD_TOL * np.maximum(1.0, np.abs(g_ora))), (g, g_ora)


def test_cube4_directional_derivative_at_scale(libpaces):
    """The 4x4x4 gradient workload (theta = 1e-4, 40 steps, checkpoints every
    20): grad . v against central differences of the GPU forward along a
    seeded direction v, with the row and kept counts of every step unchanged
    by the perturbation (so the subspace sequence is the recorded one)."""
    cfg = W.WORKLOADS["cube4"]
    nsteps, dt, theta = 40, cfg["dt"], cfg["theta"]
    N = cfg["n_sites"]
    base = W.model_kwargs(cfg)
    p0 = np.concatenate([[cfg["J"], cfg["g"], cfg["omega"]], np.zeros(N)])
    v = W.seeded_normal(3 + N, 81)
    v /= np.linalg.norm(v)
    a = W.seeded_normal(nsteps * N, 82).reshape(nsteps, N)

    def run(p, record):
        m = dict(base, J=float(p[0]), g=np.full(N, p[1]), omega=np.full(N, p[2]), eps=p[3:].copy())
        s = B.Solver(**m)
        if record:
            s.record(cfg["ckpt_every"])
        s.set_state(*W.start_state(cfg))
        s.step(dt, nsteps, theta)
        rec = s.observables(1, nsteps)
        P = rec[:, B.OBS_FIXED:B.OBS_FIXED + N]
        C = rec[:, 4] + 1j * rec[:, 5]
        L = float(np.sum(a * P) + np.sum(np.abs(C) ** 2))
        return s, L, P, C, rec[:, [B.OBS_FIELDS.index("rows"), B.OBS_FIELDS.index("kept")]]

    s, L0, P, C, counts = run(p0, True)
    assert counts[-1, 0] > 10000
    g = s.backward(nsteps, dL_dC=2.0 * C, dL_dP=a)
    s.close()
    h = 1e-6
    sp, Lp, _, _, cp = run(p0 + h * v, False)
    sm, Lm, _, _, cm = run(p0 - h * v, False)
    sp.close()
    sm.close()
    if not (np.array_equal(cp, counts) and np.array_equal(cm, counts)):
        pytest.skip("the perturbation moved a row across theta")
    fd = (Lp - Lm) / (2 * h)
    assert abs(g @ v - fd) <= 1e-6 * max(1.0, abs(fd)), (g @ v, fd)


def test_cube4_population_spectrum_loss_gradient(libpaces):
    """The gradient workload's loss -- site-0 population at T plus the mean
    squared deviation of the absorption spectrum from a seeded target (the
    spectrum of a run at parameters perturbed by 5% seeded noise) -- through
    the autograd function: grad . v against central differences of the same
    loss along a seeded direction (4x4x4 cube, theta = 1e-4, 40 steps,
    checkpoints every 20)."""
    import torch
    from paper_2603_07341_gb300.autograd import population_spectrum_loss, seeded_target
    cfg = W.WORKLOADS["cube4"]
    nsteps, dt, theta = 40, cfg["dt"], cfg["theta"]
    N = cfg["n_sites"]
    model = W.model_kwargs(cfg)
    start = W.start_state(cfg)
    p0 = np.concatenate([[cfg["J"], cfg["g"], cfg["omega"]], np.zeros(N)])
    omega = np.linspace(-6.0, 6.0, 1024)
    A_t = seeded_target(model, start, dt, nsteps, theta, omega, p0 + np.r_[0, 0, 0, 0.01 * np.ones(N)])
    p = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    L = population_spectrum_loss(p, model, start, dt, nsteps, theta, omega, A_t, ckpt_every=cfg["ckpt_every"])
    L.backward()
    g = p.grad.numpy()
    v = W.seeded_normal(3 + N, 91)
    v /= np.linalg.norm(v)
    h = 1e-6
    with torch.no_grad():
        Lp = float(population_spectrum_loss(torch.tensor(p0 + h * v), model, start, dt, nsteps, theta, omega, A_t))
        Lm = float(population_spectrum_loss(torch.tensor(p0 - h * v), model, start, dt, nsteps, theta, omega, A_t))
    fd = (Lp - Lm) / (2 * h)
    assert np.isfinite(g).all() and abs(g @ v - fd) <= 1e-5 * max(1.0, abs(fd)), (g @ v, fd)
