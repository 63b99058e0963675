"""The expansion entry point that allocates nothing, against the regular path.

Callers that cannot allocate device memory (a framework that owns all of it,
a loop that must never enter an allocator) use paces_expand_noalloc, whose
working memory is a fixed array inside the library.  Its output must equal,
key for key and in order, the rows paces_set_state builds with m_init = 1,
including on consecutive calls that reuse the array with different inputs.
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2603_07341_gb300 import binding as B
from paper_2603_07341_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def regular_rows(model, site, occ, amps, m_init):
    s = B.Solver(**dict(model, m_init=m_init))
    s.set_state(site, occ, amps)
    t, _ = s.tuples()
    s.close()
    return t


def keys_of(model, tuples):
    L = B.plan_layout(**model)
    return B.encode_keys(L, tuples[:, 0], tuples[:, 1:]), L.words


def check_case(model, site, occ, amps, base_radius):
    import torch
    inp = regular_rows(model, site, occ, amps, base_radius)
    want = regular_rows(model, site, occ, amps, base_radius + 1)
    kin, words = keys_of(model, inp)
    kwant, _ = keys_of(model, want)
    dev = torch.from_numpy(kin.view(np.int64)).cuda()
    out = B.expand_noalloc(dev, max_out=len(kwant) + 17, **model)
    got = out.cpu().numpy().view(np.uint64)
    assert got.shape == kwant.shape
    assert np.array_equal(got, kwant)
    return len(got)


def test_noalloc_expansion_matches_regular_path_on_consecutive_calls(libpaces):
    ring = W.model_kwargs(W.WORKLOADS["ring16"])
    dip = W.model_kwargs(W.WORKLOADS["dipolar6x6"])
    cube = W.model_kwargs(W.WORKLOADS["cube4"])
    n1 = check_case(ring, *W.start_state(W.WORKLOADS["ring16"]), base_radius=4)
    n2 = check_case(dip, *W.start_state(W.WORKLOADS["dipolar6x6"]), base_radius=1)
    n3 = check_case(cube, *W.start_state(W.WORKLOADS["cube4"]), base_radius=1)
    n4 = check_case(ring, *W.start_state(W.WORKLOADS["ring16"]), base_radius=4)
    assert n1 == n4 and min(n1, n2, n3) > 100


def test_noalloc_rejects_requests_beyond_its_array(libpaces):
    import torch
    ring = W.model_kwargs(W.WORKLOADS["ring16"])
    big = torch.zeros((3_000_000, 1), dtype=torch.int64, device="cuda")
    with pytest.raises(B.PacesError) as e:
        B.expand_noalloc(big, max_out=4_000_000, **ring)
    assert e.value.code == B.ERR_CAPACITY
    small = torch.zeros((1, 1), dtype=torch.int64, device="cuda")
    with pytest.raises(B.PacesError) as e:
        B.expand_noalloc(small, max_out=2, **ring)      # the level has more than one new state
    assert e.value.code == B.ERR_CAPACITY
