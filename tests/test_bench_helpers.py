"""Host-side helpers of bench.py: the propagator traffic scaled from a stored
small-case capture is reported only for the library code it was captured on
(comments ignored); the CPU description; the variant comparison's error
figures; the replica reduction lives in test_bench_ranks."""
import os
import shutil

import bench


def test_scaled_traffic_is_keyed_on_code(tmp_path, monkeypatch):
    """A summary in the committed format gives DRAM/algorithmic bytes of the
    small case, applied to the window's algorithmic bytes, and only for the
    library code it names."""
    src = os.path.join(bench.ROOT, "paper_2603_07341_gb300", "csrc")
    shutil.copytree(src, tmp_path / "paper_2603_07341_gb300" / "csrc")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.library_source_hash()
    prof = tmp_path / "profiles" / "k_taylor_f64_ring16_small_traffic.md"
    prof.write_text("# summary\n\n- library source sha256[:16]: %s\n- case: ring16 step 180\n"
                    "- dram bytes per launch: 30000000000\n- algorithmic bytes per launch: 25000000000\n" % h)
    t, note = bench.traffic_scaled("k_taylor_f64", 4.0e11)
    assert abs(t - 1.2 * 4.0e11) < 1.0 and "ring16 step 180" in note
    assert bench.traffic_scaled("k_taylor_dw", 4.0e11) == (None, None)
    prof.write_text(prof.read_text().replace(h, "0" * 16))
    assert bench.traffic_scaled("k_taylor_f64", 4.0e11) == (None, None)


def test_cpu_info_reports_cores_and_model():
    cores, model = bench.cpu_info()
    assert cores >= 1 and isinstance(model, str) and model


def test_taylor_counts_per_row_and_term():
    """Two records: 10 rows with 30 stored entries (20 off the diagonal) and 3
    terms, then 20 rows with 60 entries and 2 terms."""
    import numpy as np
    rec = np.zeros((2, 12))
    rec[0, 6], rec[0, 8], rec[0, 9] = 10, 30, 3
    rec[1, 6], rec[1, 8], rec[1, 9] = 20, 60, 2
    units, bytes_, flops = bench.taylor_counts(rec, 1)
    assert units == 10 * 3 + 20 * 2
    assert bytes_ == (10 * 57 + 20 * 5 + 2 * (10 * 73 + 20 * 5)) + (20 * 57 + 40 * 5 + 1 * (20 * 73 + 40 * 5))
    assert flops == 3 * (10 * 7 + 20 * 4) + 2 * (20 * 7 + 40 * 4)


def test_source_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_2603_07341_gb300", "csrc")
    fake = tmp_path / "paper_2603_07341_gb300" / "csrc"
    shutil.copytree(src, fake, ignore=shutil.ignore_patterns("*.o"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.library_source_hash()
    f = fake / "kern_taylor.cu"
    text = f.read_text()
    f.write_text("// a comment line\n" + text.replace("namespace paces {", "namespace paces {  /* note */", 1))
    assert bench.library_source_hash() == h0
    f.write_text(text + "\nstatic int extra_symbol = 1;\n")
    assert bench.library_source_hash() != h0


def test_ensemble_model_and_oracle_model():
    cfg = bench.W.WORKLOADS["disorder12"]
    m = bench.ensemble_model(cfg, 3)
    assert m["batch"] == 3 and m["eps"].shape == (3, cfg["n_sites"])
    assert (m["eps"][1] == bench.W.realisation_eps(cfg, 1)).all()
    om = bench.oracle_model(cfg)
    assert (om["eps"] == bench.W.realisation_eps(cfg, 0)).all()
    assert "batch" not in bench.ensemble_model(bench.W.WORKLOADS["ring16"])


def test_autograd_parameter_vector_maps_onto_the_model():
    """p = [J, g, omega, eps_0 .. eps_{N-1}]: J scales the hopping pattern, g and
    omega are shared by all sites, eps per site."""
    import numpy as np
    from paper_2603_07341_gb300.autograd import _model
    base = bench.W.model_kwargs(bench.W.WORKLOADS["ring4"])
    p = np.array([0.7, 1.3, 0.9, 0.1, -0.2, 0.3, -0.4])
    m = _model(base, p)
    assert m["J"] == 0.7
    assert np.all(m["g"] == 1.3) and np.all(m["omega"] == 0.9)
    assert np.array_equal(m["eps"], p[3:])
    assert m["n_sites"] == base["n_sites"] and m["cap"] is base["cap"]


def test_variant_errors_are_the_largest_differences():
    """The comparison block of the bench (a variant against the complex128 run)
    reports, per observable, the largest absolute difference over the records,
    and the spectrum difference relative to the reference spectrum's peak; an
    identical run reports zeros."""
    import numpy as np
    from paper_2603_07341_gb300 import binding as B
    N, T = 3, 40
    rng = np.random.default_rng(5)
    ref = rng.normal(size=(T, B.OBS_FIXED + 2 * N))
    ref[:, 0] = 0.05 * np.arange(T)                      # time
    var = ref.copy()
    var[7, B.OBS_FIXED + 1] += 3e-9                      # P_1 at one step
    var[11, B.OBS_FIXED + N + 2] -= 5e-10                # <n_2> at another
    var[20, 4] += 4e-8                                   # Re C
    var[21, 5] -= 3e-8                                   # Im C (a different step)
    var[30, 3] += 1e-7                                   # energy
    e = bench.observable_errors(B, var, ref, N)
    assert abs(e["P"] - 3e-9) < 1e-15 and abs(e["nbar"] - 5e-10) < 1e-15
    assert abs(e["C"] - 4e-8) < 1e-15 and abs(e["energy"] - 1e-7) < 1e-14 and e["norm"] == 0.0
    z = bench.observable_errors(B, ref, ref, N)
    assert all(v == 0.0 for v in z.values())
    cfg = {"dt": 0.05}
    assert bench.spectrum_error(B, ref, ref, cfg) == 0.0
    assert 0.0 < bench.spectrum_error(B, var, ref, cfg) < 1e-6
