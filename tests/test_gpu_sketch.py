"""Parity of the second-stage sketch filter (sketch form, mode 3) against the
oracle (oracle/sketch.py), through the C ABI.

* Sketch bits: sign of <bf16 x_i, bf16 r_j> with FP32 accumulation on the
  tensor cores. Bits are compared with the float64 oracle wherever the
  inner product is farther from 0 than the FP32 summation bound
  d * 2^-24 * sum_m |x_im r_jm|; nearer than that, either bit is correct.
* Graph on integer-valued points and projections: every inner product and
  squared distance is an exact integer in FP32, so the sketches, the Hamming
  top-k2, the exact re-rank and its index tie-breaks are decided identically
  on both sides and the lists must be identical, element by element.
* Graph on the Gaussian mixture at the workload's dimension: a bit nearer to
  its decision boundary than the bound may flip. Rows whose point and
  candidates all carry the oracle's sketches are compared with the oracle's
  lists; the rest are checked for validity.
"""
import numpy as np
import pytest

import oracle as O
import synthdata as S
from oracle import sketch as OS
from _helpers import check_lists

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hf():
    import __graft_entry__ as g

    g.build()
    import paper_2508_21682_gb300 as hf

    assert torch.cuda.is_available()
    return hf


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def ambiguous_bits(x, R):
    """bool [n][bits]: inner products within the FP32 summation bound of 0."""
    xb, rb = O.budget.bf16(x), O.budget.bf16(R)
    dots = xb @ rb.T
    bound = x.shape[1] * 2.0 ** -24 * (np.abs(xb) @ np.abs(rb).T)
    return np.abs(dots) <= bound


def unpack(sk, bits):
    out = np.zeros((sk.shape[0], bits), bool)
    for j in range(bits):
        out[:, j] = (sk[:, j // 64] >> np.uint64(j % 64)) & np.uint64(1)
    return out


@pytest.mark.parametrize("n,d,bits,dev_r", [
    (20011, 384, 384, True),   # workload shape, ragged last row tile
    (5003, 100, 128, False),   # d padded to 128 columns, host projection
    (777, 384, 1024, True),    # widest sketch: 4 column tiles of 256
    (130, 33, 64, True),       # one 64-bit word, two row tiles
])
def test_sketch_bits(hf, n, d, bits, dev_r):
    x = S.gaussian_mixture(n, d, n_components=40, seed=6)
    R = S.sketch_projection(bits, d, seed=7)
    G = hf.build(cuda(x), T=1, bits=8, seed=1)
    G.set_sketch(cuda(R) if dev_r else R)
    got = unpack(G.sketches(), bits)
    want = OS.sketch_dots(x, R) > 0
    amb = ambiguous_bits(x, R)
    bad = (got != want) & ~amb
    assert not bad.any(), f"{bad.sum()} sketch bits differ outside the FP32 bound"
    assert amb.mean() < 1e-3
    G.close()


def test_sketch_rejects_bad_lengths(hf):
    x = S.unit_gaussian(100, 16, seed=1)
    G = hf.build(cuda(x), T=1, bits=8, seed=1)
    for bits in (32, 96, 2048):
        with pytest.raises(hf.HFError):
            G.set_sketch(S.sketch_projection(bits, 16))
    with pytest.raises(hf.HFError):  # sketch form before the sketches exist
        G.set_option("mode", 3)
        G.knn_graph(5, 8)
    G.set_sketch(S.sketch_projection(64, 16))
    G.set_option("sketch_k2", 100)
    with pytest.raises(hf.HFError):  # the graph's band lists hold at most 64
        G.knn_graph(5, 8)
    with pytest.raises(hf.HFError):
        G.set_option("sketch_k2", 1025)
    G.close()


@pytest.mark.parametrize("n,d,T,w,k,k2,bits", [
    (5003, 384, 6, 16, 15, 60, 384),   # the workload's k, k2 and sketch length; ragged tail
    (3001, 64, 4, 40, 10, 20, 128),    # two bands of offsets, 32-slot lists
    (2000, 24, 3, 9, 15, 8, 64),       # k2 < k: k candidates kept
    (40, 8, 2, 30, 5, 60, 64),         # n < 2w + 1: every candidate kept
])
def test_sketch_graph_exact_on_integer_points(hf, n, d, T, w, k, k2, bits):
    x = S.small_integer_points(n, d, seed=3)
    R = S.small_integer_projection(bits, d, seed=4)
    G = hf.build(cuda(x), T=T, bits=8, seed=5)
    F = O.Forest(x, T=T, bits=8, seed=5)
    G.set_sketch(cuda(R))
    assert np.array_equal(G.sketches(), OS.sketches(x, R))
    G.set_option("mode", 3)
    G.set_option("sketch_k2", k2)
    gi, gd = G.knn_graph(k, w)
    oi, od = OS.knn_graph_sketch(F, k, w, OS.sketches(x, R), max(k2, k))
    assert np.array_equal(gi.cpu().numpy().astype(np.int64), oi)
    assert np.array_equal(gd.cpu().numpy().astype(np.float64), od)
    G.close()


def test_sketch_graph_gaussian_workload_shape(hf):
    """The library's sketches may differ from the oracle's only in bits within
    the FP32 bound (checked first). Rows whose point and candidates all have
    the oracle's sketches must then match the oracle's graph (up to float32
    near-ties of the final distances); the few other rows are checked for
    validity: exact distances of listed pairs, order, no repeats or self,
    candidates only."""
    n, d, T, w, k, k2, bits = 20000, 384, 8, 32, 15, 60, 384
    x = S.gaussian_mixture(n, d, n_components=100, seed=9)
    R = S.sketch_projection(bits, d, seed=10)
    G = hf.build(cuda(x), T=T, bits=8, seed=11)
    F = O.Forest(x, T=T, bits=8, seed=11)
    G.set_sketch(cuda(R))
    G.set_option("mode", 3)
    G.set_option("sketch_k2", k2)
    gi, gd = G.knn_graph(k, w)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    sk = OS.sketches(x, R)
    skg = G.sketches()
    flipped = unpack(skg, bits) != unpack(sk, bits)
    assert not (flipped & ~ambiguous_bits(x, R)).any()
    moved = flipped.any(axis=1)
    oi, od = OS.knn_graph_sketch(F, k, w, sk, k2)
    cand = O.candidate_sets(F, w)
    touched = moved | np.array([moved[c[c >= 0]].any() for c in cand])
    strict = np.flatnonzero(~touched)
    assert strict.size >= n // 2, f"only {strict.size} rows with the oracle's sketches throughout"
    check_lists(x, gi[strict], gd[strict], oi[strict], od[strict], owners=strict, cand=cand[strict],
                min_equal=0.99)
    loose = np.flatnonzero(touched)
    if loose.size:
        li = gi[loose].astype(np.int64)
        ok = li >= 0
        true = O.sq_dist_fp64(x, np.broadcast_to(loose[:, None], li.shape), np.where(ok, li, -1))
        assert np.all(np.abs(gd[loose][ok] - true[ok]) <= 1e-5 * true[ok] + 1e-30)
        for r, i in enumerate(loose):
            row = li[r][ok[r]]
            assert len(set(row.tolist())) == row.size and i not in set(row.tolist())
            assert set(row.tolist()) <= set(cand[i][cand[i] >= 0].tolist())
            dd = gd[loose[r]][ok[r]]
            assert np.all((dd[1:] > dd[:-1]) | ((dd[1:] == dd[:-1]) & (row[1:] > row[:-1])))
    # the whole graph against the oracle's: nearly the same neighbours
    same = np.mean([len(set(a[a >= 0]) & set(b[b >= 0])) / max(1, (b >= 0).sum()) for a, b in zip(gi, oi)])
    assert same >= 0.995
    G.close()


def test_sketch_k2_all_candidates_equals_graph(hf):
    """k2 >= 2 w T keeps every candidate: the sketch form returns the graph of
    Algorithm 2 without its second stage (the graph oracle)."""
    n, d, T, w, k = 3000, 48, 2, 16, 10
    x = S.unit_gaussian(n, d, seed=12)
    G = hf.build(cuda(x), T=T, bits=8, seed=13)
    F = O.Forest(x, T=T, bits=8, seed=13)
    G.set_sketch(cuda(S.sketch_projection(64, d, seed=14)))
    G.set_option("mode", 3)
    G.set_option("sketch_k2", 64)
    gi, gd = G.knn_graph(k, w)
    oi, od = O.knn_graph(F, k, w)
    check_lists(x, gi.cpu().numpy(), gd.cpu().numpy(), oi, od, owners=np.arange(n), cand=O.candidate_sets(F, w))
    G.close()


# ---------------------------------------------------------------- search side
@pytest.mark.parametrize("n,d,T,w,k,k2,h,nq", [
    (5003, 64, 4, 20, 10, 60, 2, 300),      # Table 1's h; two-slot Hamming list
    (4001, 40, 3, 64, 30, 300, 2, 200),     # k = 30, k2 = 300 (16-slot list)
    (3001, 24, 2, 300, 15, 1000, 1, 100),   # the largest k2
    (2000, 36, 3, 16, 5, 7, 0, 150),        # no expansion, k2 < 32
    (70, 8, 2, 30, 40, 50, 3, 20),          # k > 32, windows wider than the set
])
def test_sketch_search_exact_on_integer_points(hf, n, d, T, w, k, k2, h, nq):
    x = S.small_integer_points(n, d, seed=7)
    q = S.small_integer_points(nq, d, seed=8)
    R = S.small_integer_projection(128, d, seed=9)
    G = hf.build(cuda(x), T=T, bits=8, seed=10)
    F = O.Forest(x, T=T, bits=8, seed=10)
    G.set_sketch(cuda(R))
    G.set_option("mode", 3)
    G.set_option("sketch_k2", k2)
    G.set_option("expand_h", h)
    gi, gd = G.search(cuda(q), k, w)
    oi, od = OS.search_sketch(F, q, k, w, OS.sketches(x, R), OS.sketches(q, R), k2, h)
    assert np.array_equal(gi.cpu().numpy().astype(np.int64), oi)
    assert np.array_equal(gd.cpu().numpy().astype(np.float64), od)
    # a second call reuses the master layout
    gi2, _ = G.search(cuda(q), k, w)
    assert np.array_equal(gi2.cpu().numpy(), gi.cpu().numpy())
    G.close()


def test_sketch_search_gaussian_workload_shape(hf):
    """Table 1's k, k2 and h on mixture data at d = 384; rows whose query and
    candidates all carry the oracle's sketches are compared with the oracle."""
    n, d, T, w, k, k2, h, nq, bits = 20000, 384, 8, 50, 30, 300, 2, 400, 384
    x = S.gaussian_mixture(n, d, n_components=100, seed=12)
    q = S.mixture_queries(nq, d, n_components=100, data_seed=12, seed=13)
    R = S.sketch_projection(bits, d, seed=14)
    G = hf.build(cuda(x), T=T, bits=8, seed=15)
    F = O.Forest(x, T=T, bits=8, seed=15)
    G.set_sketch(cuda(R))
    G.set_option("mode", 3)
    G.set_option("sketch_k2", k2)
    G.set_option("expand_h", h)
    gi, gd = G.search(cuda(q), k, w)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    sk, qsk = OS.sketches(x, R), OS.sketches(q, R)
    flipped = unpack(G.sketches(), bits) != unpack(sk, bits)
    assert not (flipped & ~ambiguous_bits(x, R)).any()
    moved = flipped.any(axis=1)
    # the query sketches are not exported: a query within the bound of a
    # decision anywhere is compared loosely
    qmoved = ambiguous_bits(q, R).any(axis=1)
    oi, od = OS.search_sketch(F, q, k, w, sk, qsk, k2, h)
    cand = O.search_candidates(F, q, w)
    touched = qmoved | np.array([moved[c[c >= 0]].any() for c in cand])
    strict = np.flatnonzero(~touched)
    assert strict.size >= nq // 2, f"only {strict.size} strict rows"
    check_lists(x, gi[strict], gd[strict], oi[strict], od[strict], queries=q[strict], min_equal=0.99)
    same = np.mean([len(set(a[a >= 0]) & set(b[b >= 0])) / max(1, (b >= 0).sum()) for a, b in zip(gi, oi)])
    assert same >= 0.99
    G.close()


def test_sketch_search_without_filters_is_the_search(hf):
    n, d, T, w, k = 4000, 32, 3, 10, 8
    x = S.unit_gaussian(n, d, seed=16)
    q = S.unit_gaussian(100, d, seed=17)
    G = hf.build(cuda(x), T=T, bits=8, seed=18)
    F = O.Forest(x, T=T, bits=8, seed=18)
    G.set_sketch(cuda(S.sketch_projection(64, d, seed=19)))
    G.set_option("mode", 3)
    G.set_option("sketch_k2", 2 * w * T)
    G.set_option("expand_h", 0)
    gi, gd = G.search(cuda(q), k, w)
    oi, od = O.search(F, q, k, w)
    check_lists(x, gi.cpu().numpy(), gd.cpu().numpy(), oi, od, queries=q)
    with pytest.raises(hf.HFError):  # no scratch-free sketch form
        G.search_static(cuda(q), k, w)
    G.close()
