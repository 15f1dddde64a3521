"""Pins the CPU oracle to facts that do not come from the oracle itself.

Each test checks the oracle against a closed form, an invariant of Hilbert
curves, a hand-derived fixture, a published generator output, or a brute-force
restatement on tiny inputs. ``test_pins_catch_planted_mistakes`` plants
mistakes in a copy of the key transform and checks that the curve pins fail.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import synthdata as S


# ---------------------------------------------------------------- helpers
def grid(d, b):
    return np.array(list(itertools.product(range(1 << b), repeat=d)), dtype=np.int64)


def key_int(keys, d, b):
    """Full key rows as Python ints (drops the zero padding)."""
    out = []
    for row in keys:
        v = 0
        for w in row:
            v = (v << 64) | int(w)
        out.append(v >> (64 * len(row) - d * b))
    return out


def curve_order(transpose, d, b):
    pts = grid(d, b)
    k = key_int(O.pack_key(transpose(pts, b), b), d, b)
    return pts, k


def textbook_xy2d(side, x, y):
    """Rotation-based 2-D Hilbert index (the common textbook formulation)."""
    dd = 0
    s = side // 2
    while s > 0:
        rx = 1 if x & s else 0
        ry = 1 if y & s else 0
        dd += s * s * ((3 * rx) ^ ry)
        if ry == 0:
            if rx == 1:
                x, y = side - 1 - x, side - 1 - y
            x, y = y, x
        s //= 2
    return dd


def check_curve(transpose, dims=(1, 2, 3), bits=(1, 2, 3, 4)):
    """Bijection onto [0, 2^(d b)) and unit steps between consecutive points."""
    for d in dims:
        for b in bits:
            pts, k = curve_order(transpose, d, b)
            if sorted(k) != list(range(1 << (d * b))):
                return False
            order = np.argsort(np.array(k, dtype=object).astype(np.int64))
            p = pts[order]
            if not np.all(np.abs(np.diff(p, axis=0)).sum(axis=1) == 1):
                return False
    return True


# ---------------------------------------------------------------- curve
def test_curve_bijection_and_unit_steps():
    assert check_curve(O.skilling_transpose)


@pytest.mark.parametrize("d,b", [(2, 3), (3, 2), (3, 4), (4, 2)])
def test_curve_starts_at_origin_ends_on_axis(d, b):
    pts, k = curve_order(O.skilling_transpose, d, b)
    order = np.argsort(np.array(k, dtype=np.int64))
    assert tuple(pts[order[0]]) == (0,) * d
    assert tuple(pts[order[-1]]) == ((1 << b) - 1,) + (0,) * (d - 1)


@pytest.mark.parametrize("b", [1, 2, 3, 4, 5])
def test_curve_d2_equals_textbook(b):
    pts, k = curve_order(O.skilling_transpose, 2, b)
    for (x, y), kk in zip(pts, k):
        assert kk == textbook_xy2d(1 << b, int(x), int(y))


@pytest.mark.parametrize("b", [1, 4, 8])
def test_curve_d1_identity(b):
    pts, k = curve_order(O.skilling_transpose, 1, b)
    assert k == [int(p[0]) for p in pts]


@pytest.mark.parametrize("name,d,b", [("curve_d2_b2.txt", 2, 2), ("curve_d3_b1.txt", 3, 1)])
def test_curve_golden_traversal(golden, name, d, b):
    want = golden(name)
    pts, k = curve_order(O.skilling_transpose, d, b)
    order = np.argsort(np.array(k, dtype=np.int64))
    assert [tuple(int(v) for v in pts[i]) for i in order] == want


@pytest.mark.parametrize("d", [2, 5, 16, 33, 64, 130])
def test_top_level_is_prefix_xor_of_top_bits(d):
    """The first d key bits are the running XOR of the coordinates' top bits
    (the lower-level steps of the transform never touch the top bit)."""
    b = 8
    rng = np.random.default_rng(d)
    c = rng.integers(0, 1 << b, size=(300, d))
    keys = O.pack_key(O.skilling_transpose(c, b), b)
    ki = key_int(keys, d, b)
    top = (c >> (b - 1)) & 1
    px = np.bitwise_xor.accumulate(top, axis=1)
    for row, kk in zip(px, ki):
        want = 0
        for v in row:
            want = (want << 1) | int(v)
        assert kk >> (d * (b - 1)) == want


@pytest.mark.parametrize("d,b,L", [(3, 4, 2), (5, 8, 3), (16, 8, 5), (64, 8, 2), (7, 6, 1)])
def test_top_levels_equal_key_of_truncated_coordinates(d, b, L):
    """The top L levels of the b-bit key equal the L-bit key of the
    coordinates' top L bits: level-q steps only change bits below q."""
    rng = np.random.default_rng(100 + d)
    c = rng.integers(0, 1 << b, size=(400, d))
    full = key_int(O.pack_key(O.skilling_transpose(c, b), b), d, b)
    trunc = key_int(O.pack_key(O.skilling_transpose(c >> (b - L), L), L), d, L)
    assert [f >> (d * (b - L)) for f in full] == trunc


def test_pack_key_layout_and_padding():
    X = np.array([[0b10110001]], dtype=np.uint32)  # d=1, b=8
    k = O.pack_key(X, 8)
    assert k.shape == (1, 1) and int(k[0, 0]) == 0b10110001 << 56
    X = np.array([[1, 0, 1]], dtype=np.uint32)  # d=3, b=1 -> bits 1,0,1 then zeros
    assert int(O.pack_key(X, 1)[0, 0]) == 0b101 << 61
    # level-major order: for d=2, b=2, X=(2, 1) the key bits are 1,0,0,1
    X = np.array([[2, 1]], dtype=np.uint32)
    assert int(O.pack_key(X, 2)[0, 0]) == 0b1001 << 60
    assert O.key_words(384, 8) == 48 and O.key_words(16, 8) == 2 and O.key_words(3, 5) == 1


def self_similar(transpose, d, b):
    """The order-b curve is 2^d copies of the order-(b-1) curve: its cells,
    cut into 2^d consecutive blocks, fill one sub-cube (octant) each, the
    octants are visited with unit steps, and each block, taken relative to
    its octant's corner, is the order-(b-1) traversal mapped by a symmetry of
    the cube (an axis permutation combined with reflections)."""
    pts, k = curve_order(transpose, d, b)
    seq = pts[np.argsort(np.array(k, dtype=np.int64))]
    p1, k1 = curve_order(transpose, d, b - 1)
    base = p1[np.argsort(np.array(k1, dtype=np.int64))]
    half = 1 << (b - 1)
    sub = 1 << (d * (b - 1))
    maps = []
    for perm in itertools.permutations(range(d)):
        for refl in itertools.product((0, 1), repeat=d):
            maps.append(np.where(np.array(refl)[None, :] == 1, half - 1 - base[:, list(perm)], base[:, list(perm)]))
    octs = []
    for j in range(1 << d):
        blk = seq[j * sub:(j + 1) * sub]
        o = blk // half
        if not np.all(o == o[0]):
            return False
        local = blk - o[0] * half
        if not any(np.array_equal(local, m) for m in maps):
            return False
        octs.append(o[0])
    return bool(np.all(np.abs(np.diff(np.array(octs), axis=0)).sum(axis=1) == 1))


@pytest.mark.parametrize("b", [2, 3, 4])
def test_curve_d3_self_similar(b):
    assert self_similar(O.skilling_transpose, 3, b)


@pytest.mark.parametrize("b", [2, 3, 4, 5])
def test_curve_d2_self_similar(b):
    assert self_similar(O.skilling_transpose, 2, b)


def _mutant_transpose(mutation):
    """Copies of the transform with one planted mistake each."""

    def f(coords, bits):
        X = np.array(coords, dtype=np.int64, copy=True)
        n, d = X.shape
        for q in range(bits - 1, 0, -1):
            P = (1 << q) - 1
            order = range(d - 1, -1, -1) if mutation == "reverse_i" else range(d)
            for i in order:
                bit = (X[:, i] >> q) & 1
                x0 = X[:, 0]
                inv = np.where(bit == 1, x0 ^ (P if mutation != "invert_all" else (1 << bits) - 1), x0)
                t = np.where(bit == 1, 0, (inv ^ X[:, i]) & P)
                X[:, 0] = inv ^ t
                if i != 0:
                    X[:, i] ^= t
        if mutation != "no_gray":
            for i in range(1, d):
                X[:, i] ^= X[:, i - 1]
        if mutation != "no_t":
            src = 1 if mutation == "t_from_x1" else d - 1
            t = np.zeros(n, dtype=np.int64)
            for q in range(bits - 1, 0, -1):
                t = np.where(((X[:, src] >> q) & 1) == 1, t ^ ((1 << q) - 1), t)
            X ^= t[:, None]
        return X

    return f


@pytest.mark.parametrize("mutation", ["no_gray", "no_t", "t_from_x1", "reverse_i", "invert_all"])
def test_pins_catch_planted_mistakes(mutation):
    f = _mutant_transpose(mutation)
    ok_curve = check_curve(f, dims=(2, 3), bits=(2, 3))
    ok_d2 = all(
        kk == textbook_xy2d(1 << b, int(x), int(y))
        for b in (2, 3)
        for (x, y), kk in zip(*curve_order(f, 2, b))
    )
    assert not (ok_curve and ok_d2), mutation


@pytest.mark.parametrize("mutation", ["no_gray", "no_t", "t_from_x1", "reverse_i", "invert_all"])
def test_d3_pins_catch_planted_mistakes(mutation):
    """Without the d = 2 textbook curve: every planted mistake breaks the d = 3
    curve's bijection/unit steps or its self-similarity."""
    f = _mutant_transpose(mutation)
    assert not (check_curve(f, dims=(3,), bits=(2, 3)) and all(self_similar(f, 3, b) for b in (2, 3))), mutation


def test_unmutated_copy_matches_oracle():
    f = _mutant_transpose("none")
    for d, b in [(2, 3), (3, 3), (5, 4)]:
        assert curve_order(f, d, b)[1] == curve_order(O.skilling_transpose, d, b)[1]


# ---------------------------------------------------------------- splitmix64 / tree params
def test_splitmix64_reference_outputs():
    """First outputs of splitmix64 from state 0, as printed by the generator's
    public reference implementation (S. Vigna, splitmix64.c)."""
    g = O.SplitMix64(0)
    assert [g.next() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_tree_params_permutation_and_stream():
    for d in (1, 2, 16, 384):
        pi, r = O.tree_params(3, 5, d)
        assert sorted(pi.tolist()) == list(range(d))
        assert set(r.tolist()) <= {0, 1}
    # the stream: state seed + (t+1)*gamma, shuffle draws first, then reflections
    d = 4
    g = O.SplitMix64(7 + 3 * O.GOLDEN_GAMMA)
    pi = list(range(d))
    draws = [g.next() for _ in range(d - 1)]
    for j, z in zip(range(d - 1, 0, -1), draws):
        m = z % (j + 1)
        pi[j], pi[m] = pi[m], pi[j]
    r = [g.next() >> 63 for _ in range(d)]
    got_pi, got_r = O.tree_params(7, 2, d)
    assert got_pi.tolist() == pi and got_r.tolist() == r


def test_tree_params_uniform():
    """All 24 permutations of 4 axes and both reflection values appear with
    the expected frequency (chi-square, 23 dof, far from the 0.1% tail)."""
    counts = {}
    ones = 0
    N = 4800
    for t in range(N):
        pi, r = O.tree_params(11, t, 4)
        counts[tuple(pi)] = counts.get(tuple(pi), 0) + 1
        ones += int(r.sum())
    assert len(counts) == 24
    exp = N / 24
    chi2 = sum((c - exp) ** 2 / exp for c in counts.values())
    assert chi2 < 49.7
    assert abs(ones / (4 * N) - 0.5) < 0.02


# ---------------------------------------------------------------- quantization
def test_quantize_end_points_and_degenerate_axis():
    x = np.array([[0.0, 5.0, -1.0], [1.0, 5.0, 3.0], [0.25, 5.0, 1.0]], np.float32)
    lo, sc = O.axis_range(x, 8)
    q = O.quantize(x, lo, sc, 8)
    assert q[0, 0] == 0 and q[1, 0] == 255 and q[2, 0] == 64
    assert np.all(q[:, 1] == 0) and sc[1] == 0
    assert q[0, 2] == 0 and q[1, 2] == 255 and q[2, 2] == 128


@pytest.mark.parametrize("bits", [1, 3, 8])
def test_quantize_exact_bin_edges(bits):
    """lo=0, hi=1 makes scale exactly 2^b, so m/2^b falls exactly on edge m."""
    m = np.arange(0, 1 << bits)
    x = np.concatenate([[0.0, 1.0], m / (1 << bits)]).astype(np.float32)[:, None]
    lo, sc = O.axis_range(x, bits)
    assert sc[0] == 1 << bits
    q = O.quantize(x, lo, sc, bits)[:, 0]
    assert q[0] == 0 and q[1] == (1 << bits) - 1
    assert np.array_equal(q[2:], m)
    # just below an edge falls into the lower bin
    below = np.nextafter(x[3:, 0], np.float32(-1)).astype(np.float32)[:, None]
    assert np.array_equal(O.quantize(below, lo, sc, bits)[:, 0], m[1:] - 1)


def test_quantize_matches_rational_closed_form():
    """Away from rounding boundaries the code is floor((x-lo)/(hi-lo)*2^b)."""
    rng = np.random.default_rng(5)
    x = rng.standard_normal((2000, 3)).astype(np.float32)
    lo, sc = O.axis_range(x, 8)
    q = O.quantize(x, lo, sc, 8)
    hi = x.max(axis=0)
    for j in range(3):
        for i in range(0, 2000, 7):
            v = (Fraction(float(x[i, j])) - Fraction(float(lo[j]))) / (Fraction(float(hi[j])) - Fraction(float(lo[j]))) * 256
            f = int(v)
            if abs(v - round(v)) > Fraction(1, 10000):
                assert q[i, j] == min(255, f)


def test_quantize_queries_clamp_and_reject_nonfinite():
    x = np.array([[0.0], [1.0]], np.float32)
    lo, sc = O.axis_range(x, 4)
    q = O.quantize(np.array([[-3.0], [0.5], [7.0]], np.float32), lo, sc, 4)
    assert q[:, 0].tolist() == [0, 8, 15]
    with pytest.raises(ValueError):
        O.axis_range(np.array([[0.0], [np.nan]], np.float32), 4)
    with pytest.raises(ValueError):
        O.quantize(np.array([[np.inf]], np.float32), lo, sc, 4)


# ---------------------------------------------------------------- order / windows
def test_order_equals_python_sort_with_ties():
    rng = np.random.default_rng(9)
    keys = rng.integers(0, 4, size=(300, 3)).astype(np.uint64)  # many ties
    keys[:, 0] = keys[:, 0] << np.uint64(62)
    sigma = O.hilbert_order(keys)
    want = sorted(range(300), key=lambda i: (tuple(int(v) for v in keys[i]), i))
    assert sigma.tolist() == want


def test_window_candidates_brute_force():
    rng = np.random.default_rng(2)
    n, w = 23, 4
    sigma = rng.permutation(n)
    cand = O.window_candidates(sigma, w)
    for p in range(n):
        j = sigma[p]
        want = {int(sigma[q]) for q in range(n) if q != p and abs(q - p) <= w}
        got = {int(c) for c in cand[j] if c >= 0}
        assert got == want


def test_lower_bound_equals_bisect():
    import bisect
    rng = np.random.default_rng(4)
    keys = rng.integers(0, 3, size=(200, 2)).astype(np.uint64)
    sk = keys[O.hilbert_order(keys)]
    tup = [tuple(int(v) for v in r) for r in sk]
    for q in itertools.product(range(4), repeat=2):
        qa = np.array(q, dtype=np.uint64)
        assert O.key_less_count(sk, qa) == bisect.bisect_left(tup, q)


# ---------------------------------------------------------------- distances / top-k
def naive_knn(x, k, exclude_self=True, queries=None):
    xs = x.astype(np.float64).tolist()
    qs = xs if queries is None else queries.astype(np.float64).tolist()
    out = []
    for i, q in enumerate(qs):
        cand = []
        for j, p in enumerate(xs):
            if exclude_self and queries is None and i == j:
                continue
            cand.append((sum((a - b) ** 2 for a, b in zip(q, p)), j))
        cand.sort()
        out.append([j for _, j in cand[:k]])
    return out


def test_brute_force_matches_naive_loops():
    x = S.unit_gaussian(60, 5, seed=8)
    x[7] = x[3]  # a duplicate: equal distances resolved by index
    idx, dist = O.brute_force_knn(x, 6)
    assert idx.tolist() == naive_knn(x, 6)
    q = S.unit_gaussian(9, 5, seed=9)
    qi, _ = O.brute_force_knn(x, 4, queries=q)
    assert qi.tolist() == naive_knn(x, 4, queries=q)


def test_topk_dedup_self_and_padding():
    x = np.array([[0.0], [1.0], [3.0], [6.0]], np.float32)
    cand = np.array([[1, 1, 0, -1, 2], [0, 0, 0, 0, 0]], np.int64)
    idx, dist = O.topk_from_candidates(x, np.array([0, 1]), cand, 3)
    assert idx.tolist() == [[1, 2, -1], [0, -1, -1]]
    assert dist[0, :2].tolist() == [1.0, 9.0] and np.isinf(dist[0, 2]) and np.isinf(dist[1, 1])


# ---------------------------------------------------------------- graph / search special cases
def test_graph_full_window_is_exact():
    """w >= n - 1: every other point is a candidate, so the graph is exact."""
    x = S.unit_gaussian(150, 6, seed=3)
    F = O.Forest(x, T=2, bits=5, seed=3)
    gi, gd = O.knn_graph(F, 7, 149)
    ei, ed = O.brute_force_knn(x, 7)
    assert np.array_equal(gi, ei)
    np.testing.assert_allclose(gd, ed, rtol=1e-13)


def test_graph_one_dimension_is_exact():
    """d = 1 with distinct codes: the order is the coordinate order (up to
    reflection) and the k nearest lie within k positions on either side."""
    rng = np.random.default_rng(12)
    m = 1 + rng.permutation(254)[:120]
    x = ((m + 0.5) / 256.0).astype(np.float32)[:, None]
    x = np.concatenate([x, np.array([[0.0], [1.0]], np.float32)])
    F = O.Forest(x, T=3, bits=8, seed=5)
    assert len(set(F.codes[:, 0].tolist())) == x.shape[0]
    gi, _ = O.knn_graph(F, 5, 5)
    ei, _ = O.brute_force_knn(x, 5)
    assert np.array_equal(gi, ei)


def test_search_full_window_is_exact():
    x = S.unit_gaussian(90, 4, seed=6)
    q = S.unit_gaussian(12, 4, seed=7) * np.float32(1.3)  # partly outside [lo, hi]
    F = O.Forest(x, T=2, bits=6, seed=1)
    si, sd = O.search(F, q, 5, 90)
    ei, ed = O.brute_force_knn(x, 5, queries=q)
    assert np.array_equal(si, ei)


def test_locate_is_lower_bound_by_full_key():
    x = S.unit_gaussian(400, 3, seed=10)
    F = O.Forest(x, T=2, bits=3, seed=2)  # coarse codes: many equal keys
    q = np.concatenate([x[:20], S.unit_gaussian(20, 3, seed=11)])
    qc = O.query_codes(F, q)
    for t in range(2):
        p = O.locate(F, t, qc)
        qk = O.hilbert_keys(qc, F.pi[t], F.r[t], F.bits)
        allk = [tuple(int(v) for v in r) for r in F.keys[t]]
        for j in range(len(q)):
            qq = tuple(int(v) for v in qk[j])
            assert p[j] == sum(1 for kk in allk if kk < qq)


def test_recall_monotone_in_trees_and_window():
    x = S.unit_gaussian(1500, 8, seed=13)
    F = O.Forest(x, T=4, bits=8, seed=3)
    rows = np.arange(0, 1500, 3)
    ei, _ = O.brute_force_knn(x, 10, rows=rows)
    last = -1.0
    for T, w in [(1, 2), (1, 4), (2, 4), (4, 4), (4, 8)]:
        cand = O.candidate_sets(F, w, trees=range(T))[rows]
        gi, _ = O.topk_from_candidates(x, rows, cand, 10)
        r = O.recall(gi, ei)
        assert r >= last
        last = r
    assert last > 0.3


def test_forest_orders_are_sorted_permutations():
    x = S.gaussian_mixture(3000, 24, n_components=20, seed=1)
    F = O.Forest(x, T=3, bits=8, seed=3)
    for t in range(3):
        s = F.sigma[t]
        assert sorted(s.tolist()) == list(range(3000))
        k = [tuple(int(v) for v in F.keys[t][i]) for i in s]
        assert all((k[i], s[i]) < (k[i + 1], s[i + 1]) for i in range(len(k) - 1))
