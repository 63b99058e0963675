"""Host-side helpers of bench.py: the stored propagator traffic is reported
only for the library code it was captured on (comments ignored) and the bench
window it was captured at; the replica reduction lives in test_bench_ranks."""
import os
import shutil

import bench


def test_stored_traffic_is_keyed_on_code_and_window(tmp_path, monkeypatch):
    """A summary in the committed format is read back only for the library
    code it names and the window it was taken at."""
    src = os.path.join(bench.ROOT, "paper_2603_07341_gb300", "csrc")
    shutil.copytree(src, tmp_path / "paper_2603_07341_gb300" / "csrc")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.library_source_hash()
    prof = tmp_path / "profiles" / "k_taylor_dw_ring16_traffic.md"
    prof.write_text("# summary\n\n- library source sha256[:16]: %s\n- window end step: 500\n"
                    "- dram bytes per launch: 699490000000\n" % h)
    assert bench.traffic_from_profile(500) == 699490000000.0
    assert bench.traffic_from_profile(499) is None
    prof.write_text(prof.read_text().replace(h, "0" * 16))
    assert bench.traffic_from_profile(500) is None


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
