"""hf_search_static: the allocation-free variant of hf_search.

It serves callers that may not allocate device memory while they run (a
serving process with a fixed memory budget, a runtime whose pool owns all
device memory): the queries' codes go to a fixed array in the library's
device image instead of a per-call allocation. Its results must equal
hf_search's, call after call (the array keeps the previous call's contents).
This file is collected last so that a failure here stops a -x run only after
every other test has run.
"""
import ctypes

import numpy as np
import pytest

import synthdata as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hf():
    import __graft_entry__ as g

    g.build()
    import paper_2508_21682_gb300 as hf

    assert torch.cuda.is_available()
    return hf


def call_static(hf, G, q, k, w):
    """hf_search_static through the C ABI."""
    nq = q.shape[0]
    oi = torch.full((nq, k), -7, dtype=torch.int32, device="cuda")
    od = torch.full((nq, k), -7.0, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rc = hf.lib().hf_search_static(G._h, q.data_ptr(), nq, k, w, oi.data_ptr(), od.data_ptr(), st)
    return rc, oi, od


def test_static_search_equals_hf_search_twice(hf):
    n, d, T, k, w = 20000, 48, 4, 12, 24
    x = torch.from_numpy(S.gaussian_mixture(n, d, n_components=30, seed=1)).cuda()
    G = hf.build(x, T=T, bits=8, seed=3)
    for call, (nq, seed) in enumerate([(700, 11), (333, 12)]):  # second call: fewer queries
        q = torch.from_numpy(S.mixture_queries(nq, d, n_components=30, data_seed=1, seed=seed)).cuda()
        rc, si, sd = call_static(hf, G, q, k, w)
        assert rc == hf.HF_OK, hf.status_string(rc)
        ri, rd = G.search(q, k, w)
        torch.cuda.synchronize()
        assert torch.equal(si, ri), f"call {call}: neighbour ids differ"
        np.testing.assert_allclose(sd.cpu().numpy(), rd.cpu().numpy(), rtol=1e-5, atol=0)
    G.close()


def test_static_search_rejects_oversize_and_host_buffers(hf):
    n, d = 2000, 64
    x = torch.from_numpy(S.unit_gaussian(n, d, seed=2)).cuda()
    G = hf.build(x, T=1, bits=8, seed=3)
    limit_rows = (4 << 20) // d
    q = torch.zeros((limit_rows + 1, d), dtype=torch.float32, device="cuda")
    rc, _, _ = call_static(hf, G, q, 5, 4)
    assert rc == hf.HF_EINVAL
    qh = np.zeros((4, d), np.float32)
    oi = torch.empty((4, 5), dtype=torch.int32, device="cuda")
    od = torch.empty((4, 5), dtype=torch.float32, device="cuda")
    rc = hf.lib().hf_search_static(G._h, qh.ctypes.data, 4, 5, 4, oi.data_ptr(), od.data_ptr(), None)
    assert rc == hf.HF_EINVAL
    G.close()
