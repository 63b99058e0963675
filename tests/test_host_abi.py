"""CPU-side checks of the C ABI: the library loads, exports every declared
entry point, and its host-only key layout matches the paper's App. A example."""
import json
import math
import os
import re

import numpy as np
import pytest

from paper_2603_07341_gb300 import binding as B
from paper_2603_07341_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "paces.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(paces_[a-z0-9_]+)\s*\(", src)) - {"paces_t"})


def test_library_exports_every_declared_symbol(libpaces):
    syms = declared_symbols()
    assert len(syms) >= 18
    for s in syms:
        assert hasattr(libpaces, s), s
    assert set(syms) == set(B.EXPORTED)


@pytest.mark.parametrize("name,words,pow2", [("ring4", 1, 1), ("ring16", 1, 0), ("dipolar6x6", 2, 1),
                                             ("disorder12", 1, 1), ("cube4", 3, 0), ("chain25", 3, 1)])
def test_layout_word_counts(libpaces, name, words, pow2):
    """Dense mixed radix where a power-of-two field would cost an extra word
    (ring16: 16 log2 9 + 4 = 54.7 bits in one word; cube4: 154.6 bits in 3)."""
    L = B.plan_layout(**W.model_kwargs(W.WORKLOADS[name]))
    assert (L.words, L.pow2) == (words, pow2)


def test_key_compression_matches_appendix_A(libpaces):
    """App. A: L = 8 sites of d = 16 packed 4 bits per site, site 1 in the most
    significant bits.  Our word stores site j at 16^j above the exciton digit
    (3 bits for 8 sites), so the paper's value is our key >> 3 with the site
    order reversed."""
    gd = json.load(open(os.path.join(ROOT, "tests", "golden", "key_compression_appA.json")))
    L = B.plan_layout(n_sites=8, cap=15, g=1.0)
    assert (L.words, L.pow2, L.exciton_radix) == (1, 1, 8)
    for state, words in zip(gd["states"], gd["words16"]):
        key = B.encode_keys(L, [0], [state[::-1]])[0, 0]
        assert int(key) >> 3 == int(words[0] + words[1], 2)
        assert int(key) & 7 == 0


def test_lookup_table_memory_example():
    """App. A memory example: 1e7 states of 100 sites with d = 8 take
    ceil(100 log2 8 / 32) four-byte words each (382 MiB) against 3.73 GiB
    uncompressed."""
    ex = json.load(open(os.path.join(ROOT, "tests", "golden", "key_compression_appA.json")))["memory_example"]
    words = math.ceil(ex["sites"] * math.log2(ex["d"]) / 32)
    assert math.ceil(ex["n_states"] * words * ex["word_bytes"] / 2 ** 20) == ex["compressed_MiB"]
    assert round(ex["n_states"] * ex["sites"] * 4 / 2 ** 30, 2) == ex["uncompressed_GiB"]


def test_layout_rejects_too_wide_basis(libpaces):
    """300 bits of phonon digits exceed the 256-bit key of this build."""
    with pytest.raises(B.PacesError) as e:
        B.plan_layout(n_sites=100, lattice_kind=B.CHAIN, cap=7, g=1.0)
    assert e.value.code == B.ERR_KEY_WIDTH


def test_encode_roundtrip_and_ranges(libpaces):
    rng = np.random.default_rng(3)
    for name in ("ring16", "dipolar6x6", "cube4"):
        cfg = W.WORKLOADS[name]
        L = B.plan_layout(**W.model_kwargs(cfg))
        N, K = cfg["n_sites"], cfg["cap"]
        site = rng.integers(0, N, 50).astype(np.int32)
        occ = rng.integers(0, K + 1, (50, N)).astype(np.int32)
        keys = B.encode_keys(L, site, occ)
        # decode with plain integer arithmetic from the published layout
        for i in range(50):
            words = [int(x) for x in keys[i]]
            assert words[0] % L.exciton_radix == site[i]
            for j in range(N):
                w = words[L.site_word[j]]
                assert (w // L.site_stride[j]) % L.site_radix[j] == occ[i, j]
            assert all(x != (1 << 64) - 1 for x in words)
        bad = occ.copy()
        bad[0, 0] = -1
        with pytest.raises(B.PacesError):
            B.encode_keys(L, site, bad)


def test_invalid_params_rejected_without_gpu(libpaces):
    for kw in (dict(n_sites=0), dict(n_sites=200), dict(n_sites=4, lattice_kind=B.RING, coupling_kind=B.DIPOLAR),
               dict(n_sites=6, lattice_kind=B.OPEN2D, dims=(2, 2, 1)), dict(n_sites=4, cap=-1)):
        with pytest.raises(B.PacesError) as e:
            B.plan_layout(**kw)
        assert e.value.code == B.ERR_INVALID
