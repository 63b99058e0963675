"""Throughput of the paces per-timestep hot path on GB300.

Workload (default): the 1D Holstein ring N = 16, K = 8 phonons per site,
J = omega = 1, g = 1.5, dt = 0.02, theta = 1e-7, start |site 0, vacuum>, 1000
steps (synthetic; the parameterised model stands in for the paper's 1D Holstein
benchmark).  One bench step is one time step: truncation, m = 2 levels of
expansion with hash de-duplication and rescue, the P H P build, the Taylor
propagation and the observables.  The timed window is the last K steps of the
1000-step trajectory (the largest subspaces): the trajectory is first advanced,
untimed, to step 1000 - K - W, then W warm-up steps run, then K timed steps.

Metric: H-applied amplitudes/s = sum over timed steps of (Taylor terms x rows of
H_eff) / device time, with steps/s alongside.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the workload
on its own GPU (the single-instance path does not shard); value is the sum of
the ranks' units over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2603_07341_gb300 import workloads as W  # noqa: E402

METRIC = "H-applied amplitudes/s"
TIE_SEED = 2603073410                 # seed of the top-q_nom tie hash (workloads with q_nom)
UNIT = "amplitudes/s"
REF_SKIP = 60                         # reference arm: untimed oracle steps before its warm-up
FALLBACK_HBM_GBS = 6800.0
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # SMs x FP64 FMA/clk/SM x 2 flop x max SM clock (GHz)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(dist, ms, units, t_host, all_units, device):
    """Replicas: the slowest rank's times and the sum of all ranks' units."""
    if dist is None:
        return ms, units, t_host, all_units
    import torch
    tt = torch.tensor([ms, units, t_host, all_units], dtype=torch.float64, device=device)
    mx = tt.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(tt, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(tt[1]), float(mx[2]), float(tt[3])


def sol_precision(model):
    return {0: "c128", 1: "dw", 2: "c64"}[int(model.get("precision", 0))]


def taylor_counts(rec, h_words):
    """Units, FP64 flops and algorithmic bytes of the propagator over records.

    Bytes per row and term: 1 (entry count) + 8 (diagonal) + 16 (x_i) + 16
    (phi_n written) + 32 (r read and written; 16 written in term 1, where
    r = x + phi_1) and 5 per off-diagonal entry (column and coefficient id).
    FP64 flops per row and term of the FP64 kernel: 4 per off-diagonal entry
    (two FMAs), 5 for the diagonal (dt/n times d, two FMAs), 2 for r += phi_n."""
    q = rec[:, 6]
    nnz_off = rec[:, 8] - q
    terms = rec[:, 9]
    units = float(np.sum(terms * q))
    bytes_ = float(np.sum(q * 57.0 + nnz_off * 5.0 + (terms - 1) * (q * 73.0 + nnz_off * 5.0)))
    flops = float(np.sum(terms * (q * 7.0 + nnz_off * 4.0)))
    return units, bytes_, flops


def library_source_hash():
    """sha256[:16] over the code of the library's CUDA sources, comments and
    whitespace removed: the propagator's traffic also depends on the row order
    the other stages produce, but not on how the code is commented."""
    import re
    d = os.path.join(ROOT, "paper_2603_07341_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h")):
            src = open(os.path.join(d, name)).read()
            src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
            src = re.sub(r"//[^\n]*", " ", src)
            h.update(name.encode())
            h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def traffic_scaled(kernel, alg_bytes_per_launch):
    """DRAM bytes per launch of the propagator at the bench window, scaled from
    a one-kernel ncu capture of a small case of the same workload (inputs above
    L2, a few GB on the device): the capture's ratio of DRAM to algorithmic
    bytes times this window's algorithmic bytes.  None unless the summary in
    profiles/ was taken on the current library source."""
    path = os.path.join(ROOT, "profiles", "%s_ring16_small_traffic.md" % kernel)
    if not os.path.exists(path):
        return None, None
    fields = {}
    for line in open(path):
        if ":" in line and line.startswith("- "):
            k, v = line[2:].rsplit(":", 1)
            fields[k.strip()] = v.strip()
    if fields.get("library source sha256[:16]") != library_source_hash():
        return None, None
    try:
        ratio = float(fields["dram bytes per launch"]) / float(fields["algorithmic bytes per launch"])
    except (KeyError, ValueError, ZeroDivisionError):
        return None, None
    return ratio * alg_bytes_per_launch, "scaled: DRAM/algorithmic ratio %.3f of a %s capture (%s) times " \
        "this window's algorithmic bytes" % (ratio, kernel, fields.get("case", "small case"))


def cpu_info():
    """Host core count and CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None and os.path.exists("/proc/cpuinfo"):
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                model = line.split(":", 1)[1].strip()
                break
    import platform
    return os.cpu_count() or 1, "%s (%s)" % (model or "unknown", platform.machine())


def oracle_model(cfg):
    """The oracle's model: one realisation (the first) of an ensemble."""
    if "realisations" in cfg:
        return W.model_kwargs(cfg, eps=W.realisation_eps(cfg, 0))
    return W.model_kwargs(cfg)


def oracle_step(o, cfg):
    if "q_nom" in cfg:
        o.step_nom(cfg["dt"], cfg["q_nom"], TIE_SEED)
    else:
        o.step(cfg["dt"], cfg["theta"])


def _oracle_run(args):
    """One oracle process: psi(0), then `skip` untimed steps, then timed steps
    until `budget_s` seconds or `max_steps` steps.  Returns (units, seconds,
    timed steps, final rows)."""
    name, skip, budget_s, max_steps = args
    sys.path.insert(0, ROOT)
    from oracle.oracle import Oracle
    cfg = W.WORKLOADS[name]
    o = Oracle(**oracle_model(cfg))
    o.set_state(*W.start_state(cfg))
    for _ in range(skip):
        oracle_step(o, cfg)
    units, steps, rows = 0.0, 0, 0
    t0 = time.perf_counter()
    while True:
        oracle_step(o, cfg)
        st = o.stats()
        units += st["terms"] * st["rows"]
        rows = int(st["rows"])
        steps += 1
        el = time.perf_counter() - t0
        if (budget_s and el > budget_s) or (max_steps and steps >= max_steps):
            break
    return units, el, steps, rows


def oracle_replicas(name, procs, skip=0, budget_s=None, max_steps=None):
    """The oracle (single-threaded C) as it stands, run as `procs` independent
    processes, one per host core, started with spawn; aggregate units/s =
    the processes' units over the slowest process's time."""
    if procs <= 1:
        return [_oracle_run((name, skip, budget_s, max_steps))]
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_oracle_run, [(name, skip, budget_s, max_steps)] * procs)


def cpu_baseline(name, budget_s=15.0):
    """The oracle on this host: one process, then one per core, each timed
    from psi(0) for about budget_s seconds."""
    cores, model = cpu_info()
    one = oracle_replicas(name, 1, budget_s=budget_s)[0]
    allc = oracle_replicas(name, cores, budget_s=budget_s) if cores > 1 else [one]
    v_all = sum(r[0] for r in allc) / max(r[1] for r in allc)
    return {"value": v_all, "unit": UNIT, "cores": len(allc), "kind": "oracle",
            "cpu_model": model, "nproc": cores,
            "value_1core": one[0] / one[1],
            "sample": "oracle steps 1..%d of %s from psi(0) (%.1f s, final rows %d) in each of %d processes, "
                      "one per core; 1-core rate from one process alone (steps 1..%d)"
                      % (min(r[2] for r in allc), name, max(r[1] for r in allc), allc[0][3], len(allc), one[2])}


def ensemble_model(cfg, realisations=None, block=None):
    """Model keyword arguments; a disorder ensemble gets batch R and its eps
    table, or, with block = (lo, hi), the realisations lo..hi-1 of it."""
    model = W.model_kwargs(cfg)
    if "realisations" in cfg:
        R = int(realisations or cfg["realisations"])
        lo, hi = block if block is not None else (0, R)
        model["batch"] = hi - lo
        model["eps"] = np.stack([W.realisation_eps(cfg, r) for r in range(lo, hi)])
    return model


def run_trajectory(B, model, cfg, start_state, end, first_timed, K, barrier, clk=None):
    """set_state, then `end` steps one at a time, each followed by the read-back
    of its observables record; steps first_timed+1 .. first_timed+K are timed
    with CUDA events on the solver's stream (stage timing on)."""
    import torch
    sol = B.Solver(**model)
    stream = sol.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    all_units = 0.0
    barrier()
    t_host0 = time.perf_counter()
    sol.set_state(*start_state)
    for k in range(end):
        if k == first_timed:
            barrier()
            sol.profile(True)
            sol.stage_stats(reset=True)
            if clk is not None:
                clk.__enter__()
            # a profiler started with --profile-from-start off sees the timed steps only
            torch.cuda.profiler.start()
            e0.record(stream)
        if "q_nom" in cfg:
            sol.step_nom(cfg["dt"], 1, cfg["q_nom"], TIE_SEED)
        else:
            sol.step(cfg["dt"], 1, cfg["theta"])
        r = sol.observables(sol.num_records() - 1, 1)[0]
        all_units += r[9] * r[6]
        if k + 1 == first_timed + K:
            e1.record(stream)
    barrier()
    torch.cuda.profiler.stop()
    t_host = time.perf_counter() - t_host0
    if clk is not None:
        clk.__exit__(None, None, None)
    sol.profile(False)
    stage_ms, launches, stage_bytes = sol.stage_stats(reset=True)
    return {"solver": sol, "ms": e0.elapsed_time(e1), "t_host": t_host, "all_units": all_units,
            "rec": sol.observables(first_timed + 1, K), "rec_all": sol.observables(0, sol.num_records()),
            "stage_ms": stage_ms, "launches": launches, "stage_bytes": stage_bytes}


def observable_errors(B, rec, ref, N, R_rec=1, R_ref=1, r_rec=0, r_ref=0):
    """Largest absolute differences of P_s, <n_j>, C, norm and energy between two
    record blocks (realisation r of an ensemble block, or the single model)."""
    a = B.records_dict(rec, N, R_rec)
    b = B.records_dict(ref, N, R_ref)
    pick = lambda d, key, R, r: d[key] if R == 1 else d[key][:, r]
    Ca = a["C"] if R_rec == 1 else a["C_r"][:, r_rec]
    Cb = b["C"] if R_ref == 1 else b["C_r"][:, r_ref]
    out = {"P": float(np.max(np.abs(pick(a, "P", R_rec, r_rec) - pick(b, "P", R_ref, r_ref)))),
           "nbar": float(np.max(np.abs(pick(a, "nbar", R_rec, r_rec) - pick(b, "nbar", R_ref, r_ref)))),
           "C": float(np.max(np.abs(Ca - Cb)))}
    if R_rec == 1 and R_ref == 1:
        out["norm"] = float(np.max(np.abs(a["norm"] - b["norm"])))
        out["energy"] = float(np.max(np.abs(a["energy"] - b["energy"])))
    return out


def spectrum_error(B, rec_all, ref_all, cfg):
    """Largest |A(w) - A_ref(w)| over the spectrum grid (1024 points on [-6, 6]),
    relative to max |A_ref|, of the absorption spectra of two whole
    trajectories (records from step 0)."""
    from paper_2603_07341_gb300.analysis import absorption_spectrum
    w = np.linspace(-6.0, 6.0, 1024)
    C = lambda r: r[:, B.OBS_FIELDS.index("C_re")] + 1j * r[:, B.OBS_FIELDS.index("C_im")]
    A, Ar = absorption_spectrum(C(rec_all), cfg["dt"], w), absorption_spectrum(C(ref_all), cfg["dt"], w)
    return float(np.max(np.abs(A - Ar)) / np.max(np.abs(Ar)))


def compare_variants(B, args, cfg, model, start_state, end, first_timed, K, barrier, main):
    """The plain FP64 single-instance form next to the measured one: throughput
    over the same timed window, the largest observable differences over those
    steps and the spectrum difference over the whole trajectory."""
    N = cfg["n_sites"]
    units = lambda rec: float(np.sum(rec[:, 9] * rec[:, 6]))
    out = {}
    R = int(model.get("batch", 1))
    if R == 1:
        recs, alls = {}, {}
        forms = [f for f in ("c128", "c64", "dw") if f == "c128" or f in args.compare_forms.split(",")]
        prec = {"c128": B.C128, "c64": B.C64_SPMV, "dw": B.DW}
        for name in forms:
            p = prec[name]
            if p == model["precision"]:
                recs[name], alls[name] = main["rec"], main["rec_all"]
                continue
            run = run_trajectory(B, dict(model, precision=p), cfg, start_state, end, first_timed, K, barrier)
            run["solver"].close()
            recs[name], alls[name] = run["rec"], run["rec_all"]
            out[name] = {"value": units(run["rec"]) / (run["ms"] / 1e3), "ms_per_step": run["ms"] / K}
        for name in forms:
            if name == "c128":
                continue
            d = out.setdefault(name, {})
            d["max_abs_err_vs_c128"] = observable_errors(B, recs[name], recs["c128"], N)
            d["max_abs_err_vs_c128_whole_run"] = observable_errors(B, alls[name][1:], alls["c128"][1:], N)
            d["spectrum_rel_err_vs_c128"] = spectrum_error(B, alls[name], alls["c128"], cfg)
        out["reference_form"] = "c128: plain FP64 single instance, same steps"
        return out
    # ensemble: single-instance FP64 runs of a sample of realisations
    S = min(R, max(1, args.compare_sample))
    tot_units, tot_ms, errs = 0.0, 0.0, []
    for r in range(S):
        m = dict(model, batch=1, eps=np.asarray(model["eps"])[r].copy(), precision=B.C128)
        run = run_trajectory(B, m, cfg, start_state, end, first_timed, K, barrier)
        run["solver"].close()
        tot_units += units(run["rec"])
        tot_ms += run["ms"]
        errs.append(observable_errors(B, main["rec"], run["rec"], N, R_rec=R, R_ref=1, r_rec=r))
    out["single_c128"] = {"value": tot_units / (tot_ms / 1e3), "ms_per_step_per_realisation": tot_ms / K / S,
                          "sample": "realisations 0..%d, one solver each, run one after another" % (S - 1)}
    out["max_abs_err_vs_single_c128"] = {k: max(e[k] for e in errs) for k in errs[0]}
    out["reference_form"] = "c128: plain FP64 single instance per realisation"
    return out


def gradient_run(B, cfg, model, nsteps):
    """Forward (recorded, checkpoints every ckpt_every steps) and reverse pass of
    the whole trajectory for the loss L = P_0(T) + mean_w (A(w) - A_target(w))^2,
    A_target the spectrum at seeded perturbed parameters; host-clock times of
    both passes and the gradient dL/d[J, g, omega, eps_0 ..]."""
    import torch
    from paper_2603_07341_gb300 import autograd as AG
    N = cfg["n_sites"]
    base = dict(model)
    p0 = np.concatenate([[cfg["J"], cfg["g"], cfg["omega"]], np.full(N, float(cfg["eps"]))])
    start = W.start_state(cfg)
    w = np.linspace(-6.0, 6.0, 1024)
    ck = int(cfg.get("ckpt_every", 20))
    A_t = AG.seeded_target(base, start, cfg["dt"], nsteps, cfg["theta"], w, p0)
    p = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L = AG.population_spectrum_loss(p, base, start, cfg["dt"], nsteps, cfg["theta"], w, A_t, ckpt_every=ck)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    L.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    g = p.grad.numpy()
    return {"steps": nsteps, "ckpt_every": ck, "loss": float(L.detach()), "forward_s": t1 - t0,
            "backward_s": t2 - t1, "dL_dJ_g_omega": [float(x) for x in g[:3]],
            "dL_deps_norm": float(np.linalg.norm(g[3:])),
            "loss_form": "P_0(T) + mean over 1024 points on [-6, 6] of (A - A_target)^2, A_target at "
                         "p0 (1 + 0.05 z), z seeded normal (seed 12345)"}


def run_reference(args, cfg):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    # the oracle as it stands, one process per host core: W warm-up steps then
    # K timed steps from psi(0) in each (the oracle cannot reach the GPU window
    # in minutes)
    cores, cpu_model = cpu_info()
    skip = REF_SKIP + args.warmup
    runs = oracle_replicas(args.workload, cores, skip=skip, max_steps=args.steps)
    el = max(r[1] for r in runs)
    v = sum(r[0] for r in runs) / el
    sample = "oracle steps %d..%d of %s from psi(0) (steps 1..%d untimed) in each of %d processes (one per " \
        "core), final rows %d" % (skip + 1, skip + args.steps, args.workload, skip, len(runs), runs[0][3])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": len(runs), "kind": "oracle", "nproc": cores,
                             "cpu_model": cpu_model, "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ring16", choices=sorted(W.WORKLOADS))
    ap.add_argument("--end-step", type=int, default=500,
                    help="last timed step (the ring16 trajectory has 1000; 0 = the whole trajectory)")
    ap.add_argument("--precision", default="c128", choices=["c128", "dw", "c64"])
    ap.add_argument("--propagator", default="taylor", choices=["taylor", "lanczos"],
                    help="a6 propagator: the Taylor series (App. C.1) or the Lanczos decomposition (App. C.3)")
    ap.add_argument("--kmax", type=int, default=16, help="Lanczos: most Krylov vectors per series")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--realisations", type=int, default=0, help="ensemble size (0: the workload's)")
    ap.add_argument("--compare", action="store_true",
                    help="also time the plain FP64 single-instance form and report observable errors "
                         "(on by default for a single instance on one GPU)")
    ap.add_argument("--no-compare", action="store_true", help="skip the comparison run")
    ap.add_argument("--compare-sample", type=int, default=4)
    ap.add_argument("--compare-forms", default="c64", help="forms the comparison runs next to c128 (c64, dw)")
    ap.add_argument("--gradient", action="store_true",
                    help="also time the reverse pass of the whole trajectory (workloads with ckpt_every): "
                         "the site-0 population at T plus the spectrum mean squared error against a seeded "
                         "target, through autograd.population_spectrum_loss")
    ap.add_argument("--replicas", action="store_true",
                    help="ensembles under several ranks: every rank runs all realisations instead of a block")
    args = ap.parse_args()
    cfg = W.WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, cfg)

    import torch
    ws, rank, local = dist_setup()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_07341_gb300 import binding as B

    K, Wm = args.steps, args.warmup
    end = args.end_step or cfg["nsteps"]
    start = max(0, end - K - Wm)
    prec = {"dw": B.DW, "c128": B.C128, "c64": B.C64_SPMV}
    # an ensemble under several ranks is sharded: rank k evolves its block of
    # realisations; the disorder-averaged C(t) is one all-reduce at the end
    R_all = int(args.realisations or cfg.get("realisations", 1))
    shard = R_all > 1 and ws > 1 and not args.replicas
    block = None
    if shard:
        from paper_2603_07341_gb300.sharding import shard_range
        block = shard_range(R_all, ws, rank)
    model = ensemble_model(cfg, args.realisations, block)
    model["precision"] = prec[args.precision]
    if args.propagator == "lanczos":
        model["propagator"], model["kmax"] = B.LANCZOS, args.kmax
    R = int(model.get("batch", 1))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # psi(0) in pinned host memory; every step goes through the public API and
    # reads its observables record back to the host (end to end, host clock)
    site, occ, amps = W.start_state(cfg)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    site_p, occ_p = pin(site), pin(occ)
    amps_p = pin(np.stack([amps.real, amps.imag], 1).reshape(-1))
    first_timed = start + Wm
    clk = ClockSampler(local)
    run = run_trajectory(B, model, cfg, (site_p, occ_p, amps_p[0::2] + 1j * amps_p[1::2]), end, first_timed, K,
                         barrier, clk)
    sol, ms, t_host, all_units, rec = run["solver"], run["ms"], run["t_host"], run["all_units"], run["rec"]
    stage_ms, launches, stage_bytes = run["stage_ms"], run["launches"], run["stage_bytes"]
    units, tbytes, tflops = taylor_counts(rec, sol)
    ens = None
    if shard:
        from paper_2603_07341_gb300.sharding import run_sharded_ensemble
        nrec = sol.num_records()
        R_loc = int(model["batch"])
        allrec = sol.observables(0, nrec)
        C_loc = B.records_dict(allrec, cfg["n_sites"], R_loc)["C_r"] if R_loc > 1 else \
            (allrec[:, 4] + 1j * allrec[:, 5]).reshape(-1, 1)
        C_mean, _, _ = run_sharded_ensemble(R_all, nrec - 1, lambda lo, hi: C_loc, device="cuda")
        ens = {"realisations": R_all, "block": list(block), "C_mean_final": [float(C_mean[-1].real),
                                                                             float(C_mean[-1].imag)],
               "collective": "one all-reduce (sum) of sum_r C_r(t) over %d records" % nrec}
    t_max, total_units, t_host, all_units = reduce_over_ranks(dist, ms, units, t_host, all_units, "cuda")
    value = total_units / (t_max / 1e3)

    # roofline of the dominant kernel (the propagator), live CUDA events per launch
    peak_gbs, peak_kind = peaks()
    tay_ms = stage_ms[3] / K
    achieved_gbs = tbytes / K / (tay_ms / 1e3) / 1e9
    achieved_tf = tflops / K / (tay_ms / 1e3) / 1e12
    frac_hbm = achieved_gbs / peak_gbs
    frac_fp64 = achieved_tf / FP64_PEAK_TFLOPS
    kern = {"c128": "k_taylor_f64", "dw": "k_taylor_dw", "c64": "k_taylor_c64"}[sol_precision(model)]
    if args.propagator == "lanczos":
        # the library's own count of the Lanczos passes' algorithmic bytes
        kern = "k_lanczos_f64"
        tbytes = float(stage_bytes[3])
        achieved_gbs = tbytes / K / (tay_ms / 1e3) / 1e9
        frac_hbm, frac_fp64 = achieved_gbs / peak_gbs, 0.0
    traffic, traffic_note = traffic_scaled(kern, tbytes / K) if args.workload == "ring16" else (None, None)
    if sol_precision(model) == "c128" and frac_fp64 > frac_hbm and args.propagator == "taylor":
        roof = {"bound": "alu", "achieved": achieved_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s (FP64)",
                "frac": frac_fp64, "traffic": traffic,
                "peak_kind": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz",
                "hbm_achieved_gbs": achieved_gbs, "hbm_frac": frac_hbm, "hbm_peak_gbs": peak_gbs}
        # the FP64 rate this GPU sustains on independent FMA chains, measured
        # after the timed steps (paces_fp64_rate), next to the derived peak
        fp64_meas = B.fp64_rate()
        roof["fp64_measured_tflops"] = fp64_meas
        roof["frac_of_measured_fp64"] = achieved_tf / fp64_meas if fp64_meas > 0 else None
    else:
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": peak_gbs, "unit": "GB/s",
                "frac": frac_hbm, "traffic": traffic, "peak_kind": peak_kind + " (copy), sustained",
                "fp64_achieved_tflops": achieved_tf, "fp64_frac": frac_fp64}
    roof["traffic_note"] = traffic_note
    roof["kernel"] = kern + " (one cooperative launch per time step)"
    roof["algorithmic_bytes_per_launch"] = tbytes / K

    e2e = {"value": all_units / t_host, "unit": UNIT,
           "h2d_bytes_per_step": (site.nbytes + occ.nbytes + amps_p.nbytes) / end,
           "d2h_bytes_per_step": sol.rec_len * 8,
           "note": "host clock over the whole run from psi(0) in pinned host memory: set_state, then "
                   "%d x (paces_step(1) + read-back of that step's observables record); units over all "
                   "%d steps" % (end, end)}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, args.cpu_budget)

    grad = None
    if args.gradient and rank == 0:
        grad = gradient_run(B, cfg, model, end)
    variants = None
    # by default a single instance on one GPU is also run in complex64 terms over
    # the same steps: its throughput and observable errors against this run
    compare = args.compare or (ws == 1 and R == 1 and not args.no_compare and args.propagator == "taylor")
    if compare:
        sol.close()
        variants = compare_variants(B, args, cfg, model, (site_p, occ_p, amps_p[0::2] + 1j * amps_p[1::2]), end,
                                    first_timed, K, barrier, run)
    if rank == 0:
        q = rec[:, 6]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": Wm,
            "ms_per_step": t_max / K, "higher_is_better": True, "scaling": "strong" if shard else "weak",
            "vs_baseline": None,
            "dtype": {"dw": "f32x2 (double-word FP32, 48-bit significand)", "c128": "f64",
                      "c64": "f32 terms, f32x2 accumulator"}[sol_precision(model)],
            "data": "synthetic",
            "config": {"workload": "%s: %s, timed steps %d..%d of %d%s" % (
                           args.workload, W.describe(cfg), start + Wm + 1, start + Wm + K, cfg["nsteps"],
                           ", Lanczos propagator (at most %d Krylov vectors)" % args.kmax
                           if args.propagator == "lanczos" else ""),
                       "rows_mean": float(np.mean(q)), "rows_max": float(np.max(q)),
                       "nnz_mean": float(np.mean(rec[:, 8])), "terms_mean": float(np.mean(rec[:, 9])),
                       "parallelism": ("realisations sharded over %d ranks" % ws) if shard else
                                      ("replicas" if ws > 1 else "single GPU"),
                       "l2": "no flush between steps; per-step working set %.0f MB vs 129 MB L2"
                             % (np.max(q) * (16 * 4 + 8 * 2 + 16 * 2 + 4 * 4 + 5 * 4 + 9) / 1e6)},
            "steps_per_s": K / (t_max / 1e3),
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches[:5].sum()),
            "wall_s_whole_run": t_host,
            "stages_ms_per_step": {n: float(m / K) for n, m in zip(B.STAGES, stage_ms)},
            "stage_algorithmic_gbs": {n: (float(b / (m / 1e3) / 1e9) if m > 0 else None)
                                      for n, b, m in zip(B.STAGES, stage_bytes, stage_ms)},
            "clocks": clk.summary(),
        }
        if R > 1 or shard:
            line["config"]["realisations"] = R_all if shard else R
            line["config"]["units"] = "rows of all realisations x Taylor terms"
        if variants is not None:
            line["variants"] = variants
        if grad is not None:
            line["gradient"] = grad
        if ens is not None:
            line["ensemble"] = ens
        print(json.dumps(line))
    sol.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
