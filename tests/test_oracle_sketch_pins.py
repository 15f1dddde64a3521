"""Pins of the sketch-stage oracle (oracle/sketch.py), no GPU.

The sketches are pinned to closed forms (R = identity gives the coordinate
signs; one non-zero row sets one named bit; -x gives the complement; the
Hamming fraction of long sketches estimates angle / pi, the collision
probability of sign random projections), the Hamming count to a bit-by-bit
count over Python integers, and the graph with its second stage to a
pure-Python brute force on tiny inputs and to the pinned graph oracle when k2
keeps every candidate. Planted mistakes in the oracle fail these pins.
"""
import math

import numpy as np
import pytest

import oracle as O
import synthdata as S
from oracle import sketch as OS


def test_pack_bits_one_bit_per_position():
    B = 192
    for j in (0, 1, 63, 64, 100, 191):
        bits = np.zeros((1, B), bool)
        bits[0, j] = True
        w = OS.pack_bits(bits)
        want = np.zeros(B // 64, np.uint64)
        want[j // 64] = np.uint64(1) << np.uint64(j % 64)
        assert np.array_equal(w[0], want)


def test_identity_projection_gives_coordinate_signs():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((50, 64)).astype(np.float32)
    x[3, 7] = 0.0  # a zero coordinate gives a clear bit
    sk = OS.sketches(x, np.eye(64, dtype=np.float32))
    for i in range(50):
        v = int(sk[i, 0])
        for j in range(64):
            assert ((v >> j) & 1) == (1 if x[i, j] > 0 else 0)


def test_single_row_sets_named_bit():
    d, B = 10, 128
    x = np.abs(np.random.default_rng(1).standard_normal((4, d))).astype(np.float32) + 0.1
    for j in (0, 70, 127):
        R = np.zeros((B, d), np.float32)
        R[j] = 1.0  # <x, r_j> > 0 for positive x, every other row gives 0
        sk = OS.sketches(x, R)
        want = np.zeros(B // 64, np.uint64)
        want[j // 64] = np.uint64(1) << np.uint64(j % 64)
        assert all(np.array_equal(sk[i], want) for i in range(4))


def test_negated_points_give_complement():
    x = S.unit_gaussian(200, 48, seed=3)
    R = S.sketch_projection(256, 48, seed=4)
    dots = OS.sketch_dots(x, R)
    assert np.all(dots != 0)
    a, b = OS.sketches(x, R), OS.sketches(-x, R)
    assert np.array_equal(a ^ b, np.full_like(a, np.uint64(0xFFFFFFFFFFFFFFFF)))
    assert np.all(OS.hamming(a, b) == 256)


def test_hamming_counts_bits():
    rng = np.random.default_rng(9)
    a = rng.integers(0, 2 ** 63, size=(30, 3), dtype=np.int64).astype(np.uint64) * np.uint64(2) + np.uint64(1)
    b = rng.integers(0, 2 ** 63, size=(30, 3), dtype=np.int64).astype(np.uint64)
    h = OS.hamming(a, b)
    for i in range(30):
        want = sum(bin(int(a[i, w]) ^ int(b[i, w])).count("1") for w in range(3))
        assert h[i] == want
    assert np.all(OS.hamming(a, a) == 0)


def test_hamming_fraction_estimates_angle():
    """Sign random projection: P(bit differs) = angle(x, y) / pi, so over 8192
    Gaussian rows the Hamming fraction is within a few standard errors of it."""
    d, B = 32, 8192
    rng = np.random.default_rng(11)
    x = rng.standard_normal((40, d))
    y = x + rng.uniform(0.1, 3.0, size=(40, 1)) * rng.standard_normal((40, d))
    R = S.sketch_projection(B, d, seed=12)
    hx, hy = OS.sketches(x, R), OS.sketches(y, R)
    frac = OS.hamming(hx, hy) / B
    xb, yb = O.budget.bf16(x), O.budget.bf16(y)
    cos = np.sum(xb * yb, 1) / np.linalg.norm(xb, axis=1) / np.linalg.norm(yb, axis=1)
    theta = np.arccos(np.clip(cos, -1, 1)) / math.pi
    se = np.sqrt(theta * (1 - theta) / B)
    assert np.all(np.abs(frac - theta) < 5 * se + 1e-3)


def _brute_graph(x, sigmas, sk, k, w, k2):
    """Pure-Python Algorithm 2 with the sketch stage."""
    n = x.shape[0]
    pos = [{int(p): r for r, p in enumerate(sig)} for sig in sigmas]
    out = []
    for i in range(n):
        cset = set()
        for t, sig in enumerate(sigmas):
            r = pos[t][i]
            for q in range(max(0, r - w), min(n, r + w + 1)):
                if q != r:
                    cset.add(int(sig[q]))
        def ham(j):
            return sum(bin(int(sk[i, u]) ^ int(sk[j, u])).count("1") for u in range(sk.shape[1]))
        c2 = sorted(cset, key=lambda j: (ham(j), j))[:k2]
        def dist(j):
            return sum((float(x[i, m]) - float(x[j, m])) ** 2 for m in range(x.shape[1]))
        top = sorted(c2, key=lambda j: (dist(j), j))[:k]
        out.append(top + [-1] * (k - len(top)))
    return np.array(out, dtype=np.int64)


def _case(n=60, d=6, T=3, bits=64, seed=0):
    x = S.unit_gaussian(n, d, seed=seed + 20)
    f = O.Forest(x, T=T, bits=4, seed=seed + 21)
    sk = OS.sketches(x, S.sketch_projection(bits, d, seed=seed + 22))
    return x, f, sk


@pytest.mark.parametrize("k,w,k2", [(3, 2, 4), (4, 5, 6), (5, 3, 5), (2, 1, 1)])
def test_graph_equals_brute_force(k, w, k2):
    x, f, sk = _case()
    gi, gd = OS.knn_graph_sketch(f, k, w, sk, k2)
    want = _brute_graph(x, f.sigma, sk, k, w, k2)
    assert np.array_equal(gi, want)
    # distances are those of the listed points
    xd = x.astype(np.float64)
    for i in range(x.shape[0]):
        for c in range(k):
            j = gi[i, c]
            if j >= 0:
                assert gd[i, c] == pytest.approx(np.sum((xd[i] - xd[j]) ** 2), rel=1e-12)
            else:
                assert gd[i, c] == np.inf


def test_k2_keeping_every_candidate_is_the_graph():
    x, f, sk = _case(n=300, d=8, T=4, bits=128, seed=3)
    w = 6
    gi, gd = OS.knn_graph_sketch(f, 5, w, sk, k2=2 * w * 4)
    ri, rd = O.knn_graph(f, 5, w)
    assert np.array_equal(gi, ri)
    assert np.array_equal(gd, rd)


def test_planted_mistakes_fail_the_pins(monkeypatch):
    """Each planted mistake in the oracle changes its graph on the tiny case."""
    x, f, sk = _case(bits=128)
    k, w, k2 = 3, 4, 4
    want = _brute_graph(x, f.sigma, sk, k, w, k2)
    assert np.array_equal(OS.knn_graph_sketch(f, k, w, sk, k2)[0], want)
    real = OS.hamming

    def last_word_dropped(a, b):  # one word of the sketch forgotten
        return real(np.asarray(a)[..., :1], np.asarray(b)[..., :1])

    def candidate_bit_added(a, b):  # a term that depends on the candidate
        return real(a, b) + (np.asarray(b)[..., 0] & np.uint64(1)).astype(np.int64)

    def point_distance(a, b):  # ranking by something else than the XOR count
        return (np.asarray(a)[..., 0] & np.uint64(0xFF)).astype(np.int64) - (np.asarray(b)[..., 0] & np.uint64(0xFF)).astype(np.int64)

    for bad in (last_word_dropped, candidate_bit_added, point_distance):
        monkeypatch.setattr(OS, "hamming", bad)
        assert not np.array_equal(OS.knn_graph_sketch(f, k, w, sk, k2)[0], want), bad.__name__
    monkeypatch.setattr(OS, "hamming", real)
    # sketches with the sign flipped or the comparison made >= differ from the
    # pinned ones on the identity case
    xi = np.array([[1.0, -1.0, 0.0] + [0.0] * 61], np.float32)
    assert int(OS.sketches(xi, np.eye(64, dtype=np.float32))[0, 0]) == 1
    assert int(OS.pack_bits(OS.sketch_dots(xi, np.eye(64, dtype=np.float32)) >= 0)[0, 0]) != 1


# ---------------------------------------------------------------- search side
def _brute_search(x, f, queries, sk, qsk, k, w, k2, h):
    """Pure-Python Algorithm 1 with both filters."""
    n = x.shape[0]
    qc = O.query_codes(f, queries)
    sig0 = [int(v) for v in f.sigma[0]]
    pos0 = {p: r for r, p in enumerate(sig0)}
    out = []
    for j in range(queries.shape[0]):
        cset = set()
        for t in range(f.T):
            p = int(O.locate(f, t, qc[j:j + 1])[0])
            for q in range(max(0, p - w), min(n, p + w)):
                cset.add(int(f.sigma[t][q]))
        def ham(c):
            return sum(bin(int(qsk[j, u]) ^ int(sk[c, u])).count("1") for u in range(sk.shape[1]))
        c2 = sorted(cset, key=lambda c: (ham(c), c))[:k2]
        ex = set()
        for c in c2:
            for o in range(-h, h + 1):
                r = pos0[c] + o
                if 0 <= r < n:
                    ex.add(sig0[r])
        def dist(c):
            return sum((float(queries[j, m]) - float(x[c, m])) ** 2 for m in range(x.shape[1]))
        top = sorted(ex, key=lambda c: (dist(c), c))[:k]
        out.append(top + [-1] * (k - len(top)))
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("k,w,k2,h", [(3, 2, 4, 1), (5, 4, 3, 2), (4, 3, 8, 0), (2, 1, 1, 5)])
def test_search_equals_brute_force(k, w, k2, h):
    x, f, sk = _case(n=80, bits=128)
    R = S.sketch_projection(128, 6, seed=22)
    q = S.unit_gaussian(12, 6, seed=40)
    qsk = OS.sketches(q, R)
    gi, gd = OS.search_sketch(f, q, k, w, sk, qsk, k2, h)
    assert np.array_equal(gi, _brute_search(x, f, q, sk, qsk, k, w, k2, h))
    xd, qd = x.astype(np.float64), q.astype(np.float64)
    for j in range(12):
        for c in range(k):
            if gi[j, c] >= 0:
                assert gd[j, c] == pytest.approx(np.sum((qd[j] - xd[gi[j, c]]) ** 2), rel=1e-12)


def test_search_without_filters_is_the_search():
    """k2 keeping every candidate and h = 0: Algorithm 1's first stage alone."""
    x, f, sk = _case(n=400, d=8, T=3, bits=64, seed=5)
    q = S.unit_gaussian(30, 8, seed=41)
    qsk = OS.sketches(q, S.sketch_projection(64, 8, seed=27))
    w = 7
    gi, gd = OS.search_sketch(f, q, 6, w, sk, qsk, k2=2 * w * 3, h=0)
    ri, rd = O.search(f, q, 6, w)
    assert np.array_equal(gi, ri) and np.array_equal(gd, rd)


def test_search_expansion_over_the_whole_order_is_exact():
    """h >= n: any one surviving candidate brings every point, so the result
    is the exact k nearest of each query (brute force)."""
    x, f, sk = _case(n=150, d=5, T=1, bits=64, seed=6)
    q = S.unit_gaussian(10, 5, seed=42)
    qsk = OS.sketches(q, S.sketch_projection(64, 5, seed=28))
    gi, gd = OS.search_sketch(f, q, 7, 2, sk, qsk, k2=1, h=150)
    xd, qd = x.astype(np.float64), q.astype(np.float64)
    for j in range(10):
        dd = np.sum((xd - qd[j]) ** 2, axis=1)
        want = np.lexsort((np.arange(150), dd))[:7]
        assert np.array_equal(gi[j], want)


def test_master_expand_positions():
    x, f, sk = _case(n=50, d=4, T=2, bits=64, seed=7)
    pos0, sig0 = f.position(0), f.sigma[0]
    c2 = np.array([[int(sig0[0]), int(sig0[25]), -1]])
    ex = OS.master_expand(f, c2, 2)
    # first candidate at position 0: offsets -2, -1 fall off the order
    assert list(ex[0, :5]) == [-1, -1, int(sig0[0]), int(sig0[1]), int(sig0[2])]
    assert list(ex[0, 5:10]) == [int(sig0[p]) for p in range(23, 28)]
    assert np.all(ex[0, 10:] == -1)
    assert pos0[sig0[25]] == 25


def test_planted_expansion_mistakes_fail(monkeypatch):
    x, f, sk = _case(n=80, bits=128)
    q = S.unit_gaussian(12, 6, seed=40)
    qsk = OS.sketches(q, S.sketch_projection(128, 6, seed=22))
    k, w, k2, h = 4, 3, 3, 2
    want = _brute_search(x, f, q, sk, qsk, k, w, k2, h)
    real = OS.master_expand

    def other_order(forest, c2, hh):  # expansion in order 1, not the master order
        class V:
            n = forest.n
            sigma = [forest.sigma[1]]
            def position(self, t):
                return forest.position(1)
        return real(V(), c2, hh)

    def no_centre(forest, c2, hh):  # the candidate itself left out
        e = real(forest, c2, hh).reshape(c2.shape[0], c2.shape[1], 2 * hh + 1)
        e[:, :, hh] = -1
        return e.reshape(c2.shape[0], -1)

    for bad in (other_order, no_centre):
        monkeypatch.setattr(OS, "master_expand", bad)
        assert not np.array_equal(OS.search_sketch(f, q, k, w, sk, qsk, k2, h)[0], want), bad.__name__
