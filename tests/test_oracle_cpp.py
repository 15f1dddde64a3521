"""The C++ oracle (oracle/hf_oracle.cpp) against the curve pins and, element by
element, against the numpy oracle.

The two oracles are independent restatements of the same conventions (one
vectorised numpy, one scalar C++ loops); each is pinned to the mathematics on
its own (the curve pins below run on the C++ transform and packing directly),
and on every shape here they must agree: codes, keys and orders bit for bit,
graph and search lists index for index, distances to double rounding.
"""
import numpy as np
import pytest

import oracle as O
import synthdata as S
from test_oracle_pins import check_curve, curve_order, grid, self_similar, textbook_xy2d

C = pytest.importorskip("oracle.c_oracle")


@pytest.fixture(scope="module", autouse=True)
def built():
    C.build()


# ---------------------------------------------------------------- curve pins
def test_cpp_curve_bijection_and_unit_steps():
    assert check_curve(C.skilling_transpose, dims=(1, 2, 3), bits=(1, 2, 3, 4))


@pytest.mark.parametrize("b", [1, 2, 3, 4, 5])
def test_cpp_curve_d2_equals_textbook(b):
    pts, k = curve_order(C.skilling_transpose, 2, b)
    for (x, y), key in zip(pts, k):
        assert key == textbook_xy2d(1 << b, int(x), int(y))


@pytest.mark.parametrize("d,b", [(2, 2), (2, 3), (2, 4), (2, 5), (3, 2), (3, 3), (3, 4)])
def test_cpp_curve_self_similar(d, b):
    assert self_similar(C.skilling_transpose, d, b)


def test_cpp_transpose_equals_numpy_on_random_codes():
    rng = np.random.default_rng(3)
    for d, b in [(1, 8), (5, 3), (16, 8), (33, 5), (64, 8), (130, 2)]:
        c = rng.integers(0, 1 << b, size=(200, d))
        assert np.array_equal(C.skilling_transpose(c, b), O.skilling_transpose(c, b)), (d, b)


def test_cpp_pack_key_layout_and_padding():
    # key bits, most significant first: level 1 of X0, X1, then level 0 -> 1 0 0 1
    assert int(C.pack_key(np.array([[2, 1]]), 2)[0, 0]) == 0b1001 << 60
    rng = np.random.default_rng(4)
    for d, b in [(3, 5), (64, 8), (7, 2), (100, 7)]:
        X = rng.integers(0, 1 << b, size=(50, d))
        assert np.array_equal(C.pack_key(X, b), O.pack_key(X.astype(np.uint32), b)), (d, b)


# ---------------------------------------------------------------- parameters
@pytest.mark.parametrize("seed", [0, 3, 2**63 + 12345])
def test_cpp_tree_params_equal_numpy(seed):
    for t in (0, 1, 7):
        for d in (1, 2, 16, 384):
            pc, rc = C.tree_params(seed, t, d)
            pn, rn = O.tree_params(seed, t, d)
            assert np.array_equal(pc, pn) and np.array_equal(rc, rn)
            assert np.array_equal(np.sort(pc), np.arange(d))


# ---------------------------------------------------------------- forest
FOREST_CASES = [
    (500, 16, 3, 8, "unit"),       # the tiny configuration's shape
    (700, 64, 2, 8, "mix"),
    (333, 33, 3, 5, "mix"),        # d * b not a multiple of 64
    (400, 7, 4, 2, "mix"),         # coarse codes: many equal keys
    (300, 1, 2, 8, "unit"),
    (256, 384, 2, 8, "mix"),
    (200, 5, 2, 3, "flat"),        # a constant axis
]


def make(n, d, kind):
    if kind == "unit":
        return S.unit_gaussian(n, d, seed=11)
    x = S.gaussian_mixture(n, d, n_components=10, seed=12)
    if kind == "flat":
        x[:, 2] = 0.25
        x[:50] = x[7]  # exact duplicates
    return x


@pytest.mark.parametrize("n,d,T,b,kind", FOREST_CASES)
def test_cpp_forest_equals_numpy(n, d, T, b, kind):
    x = make(n, d, kind)
    Fc = C.Forest(x, T=T, bits=b, seed=9)
    Fn = O.Forest(x, T=T, bits=b, seed=9)
    assert np.array_equal(Fc.lo, Fn.lo) and np.array_equal(Fc.scale, Fn.scale)
    assert np.array_equal(Fc.codes, Fn.codes)
    for t in range(T):
        assert np.array_equal(Fc.keys[t], Fn.keys[t]), f"keys of tree {t}"
        assert np.array_equal(Fc.sigma[t], Fn.sigma[t]), f"order of tree {t}"


def same_lists(ci, cd, ni, nd):
    """Index for index, distances to double rounding (the two sum coordinates
    in different orders)."""
    assert np.array_equal(ci, ni)
    fin = np.isfinite(nd)
    assert np.array_equal(np.isfinite(cd), fin)
    assert np.allclose(cd[fin], nd[fin], rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("n,d,T,b,kind", FOREST_CASES[:6])
@pytest.mark.parametrize("w,k", [(3, 5), (16, 10)])
def test_cpp_graph_equals_numpy(n, d, T, b, kind, w, k):
    x = make(n, d, kind)
    Fc = C.Forest(x, T=T, bits=b, seed=9)
    Fn = O.Forest(x, T=T, bits=b, seed=9)
    same_lists(*C.knn_graph(Fc, k, w), *O.knn_graph(Fn, k, w))


def test_cpp_graph_short_input_pads():
    x = S.unit_gaussian(6, 4, seed=1)
    F = C.Forest(x, T=2, bits=8, seed=1)
    gi, gd = C.knn_graph(F, 9, 2)
    assert np.all(gi[:, 5:] == -1) and np.all(np.isinf(gd[:, 5:]))
    same_lists(gi, gd, *O.knn_graph(O.Forest(x, T=2, bits=8, seed=1), 9, 2))


@pytest.mark.parametrize("n,d,T,b,kind", [FOREST_CASES[0], FOREST_CASES[1], FOREST_CASES[3], FOREST_CASES[5]])
def test_cpp_search_equals_numpy(n, d, T, b, kind):
    x = make(n, d, kind)
    q = S.unit_gaussian(40, d, seed=21) * 1.5  # some coordinates outside the data's range: clamped codes
    Fc = C.Forest(x, T=T, bits=b, seed=9)
    Fn = O.Forest(x, T=T, bits=b, seed=9)
    for w, k in [(4, 5), (20, 12)]:
        same_lists(*C.search(Fc, q, k, w), *O.search(Fn, q, k, w))


def test_cpp_brute_force_equals_numpy_and_full_window_graph():
    x = make(300, 12, "flat")
    ci, cd = C.brute_force_knn(x, 8)
    ni, nd = O.brute_force_knn(x, 8)
    same_lists(ci, cd, ni, nd)
    q = S.unit_gaussian(17, 12, seed=5)
    same_lists(*C.brute_force_knn(x, 8, queries=q), *O.brute_force_knn(x, 8, queries=q))
    # w >= n - 1: every point a candidate, so the graph is exact kNN
    F = C.Forest(x, T=1, bits=8, seed=2)
    same_lists(*C.knn_graph(F, 8, 299), ci, cd)


def test_cpp_rejects_nonfinite():
    x = S.unit_gaussian(50, 3, seed=1)
    x[3, 1] = np.nan
    with pytest.raises(ValueError):
        C.Forest(x, T=1, bits=8, seed=1)
    F = C.Forest(S.unit_gaussian(50, 3, seed=1), T=1, bits=8, seed=1)
    q = np.zeros((2, 3), np.float32)
    q[1, 0] = np.inf
    with pytest.raises(ValueError):
        C.search(F, q, 3, 2)


def test_cpp_full_grid_order_is_the_curve():
    """On a full grid of codes with the identity tree the order visits the
    cells along the curve: consecutive cells differ by one unit step."""
    for d, b in [(2, 3), (3, 2)]:
        pts = grid(d, b)
        X = C.skilling_transpose(pts, b)
        keys = C.pack_key(X, b)
        order = np.lexsort([keys[:, w] for w in range(keys.shape[1] - 1, -1, -1)])
        steps = np.abs(np.diff(pts[order], axis=0)).sum(axis=1)
        assert np.all(steps == 1)


# ---------------------------------------------------------------- planted mistakes
MUTATIONS = {
    "no_gray": ("for (int i = 1; i < d; ++i) X[i] ^= X[i - 1];", ""),
    "no_t": ("for (int i = 0; i < d; ++i) X[i] ^= t;", ""),
    "t_from_x0": ("if ((X[d - 1] >> q) & 1u) t ^= (1u << q) - 1u;", "if ((X[0] >> q) & 1u) t ^= (1u << q) - 1u;"),
    "invert_too_many": ("X[0] ^= P;", "X[0] ^= (P << 1) | 1u;"),
    "no_exchange_back": ("X[0] ^= t;\n        X[i] ^= t;", "X[0] ^= t;"),
    "levels_upward": ("for (int q = bits - 1; q >= 1; --q) {\n    const uint32_t P", "for (int q = 1; q <= bits - 1; ++q) {\n    const uint32_t P"),
}


def mutant_transpose(tmp_path, name):
    """The C++ oracle's own source with one planted mistake, compiled apart."""
    import ctypes
    import subprocess

    old, new = MUTATIONS[name]
    src = open(C.SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / f"{name}.cpp"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.run(["g++", *C.FLAGS, "-o", str(so), str(path)], check=True, capture_output=True)
    L = ctypes.CDLL(str(so))
    L.hfo_transpose.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
    L.hfo_transpose.restype = None

    def f(coords, bits):
        c = np.ascontiguousarray(coords, dtype=np.uint32)
        X = np.empty_like(c)
        L.hfo_transpose(c.ctypes.data, c.shape[0], c.shape[1], bits, X.ctypes.data)
        return X

    return f


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_cpp_pins_catch_planted_mistakes(tmp_path, name):
    f = mutant_transpose(tmp_path, name)
    caught = not check_curve(f, dims=(2, 3), bits=(2, 3)) or not all(
        self_similar(f, d, b) for d, b in [(2, 3), (3, 2), (3, 3)])
    assert caught, name


def test_cpp_pack_pin_catches_reversed_bit_order(tmp_path):
    """The hand-packed layout pin fails for a key packed least significant
    bit first."""
    import ctypes
    import subprocess

    src = open(C.SRC).read()
    old = "key[g / 64] |= bit << (63 - g % 64);"
    assert src.count(old) == 1
    path = tmp_path / "pack.cpp"
    path.write_text(src.replace(old, "key[g / 64] |= bit << (g % 64);"))
    so = tmp_path / "pack.so"
    subprocess.run(["g++", *C.FLAGS, "-o", str(so), str(path)], check=True, capture_output=True)
    L = ctypes.CDLL(str(so))
    L.hfo_pack_key.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
    L.hfo_pack_key.restype = None
    X = np.array([[2, 1]], np.uint32)
    out = np.empty((1, 1), np.uint64)
    L.hfo_pack_key(X.ctypes.data, 1, 2, 2, out.ctypes.data)
    assert int(out[0, 0]) != 0b1001 << 60


def test_cpp_equals_numpy_on_the_tiny_configuration():
    """The tiny configuration in full (20,000 x 16 unit Gaussian, T = 8, b = 8,
    w = 16, k = 10): both oracles give the same orders and the same graph."""
    x = S.unit_gaussian(20_000, 16, seed=S.SEED_DATA)
    Fc = C.Forest(x, T=8, bits=8, seed=S.SEED_FOREST)
    Fn = O.Forest(x, T=8, bits=8, seed=S.SEED_FOREST)
    for t in range(8):
        assert np.array_equal(Fc.sigma[t], Fn.sigma[t])
    same_lists(*C.knn_graph(Fc, 10, 16), *O.knn_graph(Fn, 10, 16))
