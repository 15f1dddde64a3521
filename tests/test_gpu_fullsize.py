"""Parity at the full-size workload shape (3,000,000 x 384, the bench's launch
configuration), on outputs the oracle can check one by one, and an exact
oracle comparison at 200,000 x 384.

At full size the oracle recomputes: every code (quantization is cheap), the
full keys of sampled points, the order property on sampled adjacent positions
(oracle keys of the two points must ascend by (key, index)), the lower-bound
property of sampled query positions, and for sampled points/queries the exact
top-k of their window candidates (taken from the orders checked above).
"""
import numpy as np
import pytest

import oracle as O
import synthdata as S
from _helpers import check_lists, check_tensor_lists

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N, D, T, W, K = 3_000_000, 384, 3, 32, 15


@pytest.fixture(scope="module")
def hf():
    import __graft_entry__ as g

    g.build()
    import paper_2508_21682_gb300 as hf

    assert torch.cuda.is_available()
    return hf


@pytest.fixture(scope="module")
def full(hf):
    x = S.gaussian_mixture(N, D, n_components=1000, seed=S.SEED_DATA)
    q = S.mixture_queries(2000, D, n_components=1000, data_seed=S.SEED_DATA, seed=S.SEED_QUERIES)
    xd = torch.from_numpy(x).cuda()
    G = hf.build(xd, T=T, bits=8, seed=S.SEED_FOREST)
    gi, gd = G.knn_graph(K, W)
    si, sd = G.search(torch.from_numpy(q).cuda(), K, W)
    # the tensor form on the same forest, at the bench's window and at the
    # widest single-tile window (w = 64)
    G.set_option("mode", 1)
    ti, td = G.knn_graph(K, W)
    ti64, td64 = G.knn_graph(K, 64)
    G.set_option("mode", 0)
    torch.cuda.synchronize()
    orders = [G.order(t).astype(np.int64) for t in range(T)]
    res = dict(x=x, q=q, G=G, gi=gi.cpu().numpy(), gd=gd.cpu().numpy(), si=si.cpu().numpy(),
               sd=sd.cpu().numpy(), orders=orders, ti=ti.cpu().numpy(), td=td.cpu().numpy(),
               ti64=ti64.cpu().numpy(), td64=td64.cpu().numpy())
    yield res
    G.close()


def oracle_setup(x):
    lo, sc = O.axis_range(x, 8)
    return lo, sc


def test_codes_bit_exact(full):
    x = full["x"]
    lo, sc = oracle_setup(x)
    got = full["G"].codes()
    for s in range(0, N, 500_000):
        want = O.quantize(x[s:s + 500_000], lo, sc, 8)
        assert np.array_equal(got[s:s + 500_000].astype(np.uint16), want), f"rows {s}.."


def test_sampled_keys_and_order(full):
    x = full["x"]
    lo, sc = oracle_setup(x)
    rng = np.random.default_rng(S.SEED_SAMPLE)
    G = full["G"]
    for t in range(T):
        pi, r = O.tree_params(S.SEED_FOREST, t, D)
        sig = full["orders"][t]
        assert np.array_equal(np.sort(sig), np.arange(N)), f"tree {t}: not a permutation"
        # keys of sampled points
        if t == 0:
            keys = G.keys(0)
            rows = rng.choice(N, 3000, replace=False)
            want = O.hilbert_keys(O.quantize(x[rows], lo, sc, 8), pi, r, 8)
            assert np.array_equal(keys[rows], want)
            del keys
        # order property on sampled adjacent positions
        pos = rng.choice(N - 1, 4000, replace=False)
        a, b = sig[pos], sig[pos + 1]
        ka = O.hilbert_keys(O.quantize(x[a], lo, sc, 8), pi, r, 8)
        kb = O.hilbert_keys(O.quantize(x[b], lo, sc, 8), pi, r, 8)
        for i in range(len(pos)):
            ta = tuple(int(v) for v in ka[i]) + (int(a[i]),)
            tb = tuple(int(v) for v in kb[i]) + (int(b[i]),)
            assert ta < tb, f"tree {t}: positions {pos[i]}, {pos[i] + 1} out of order"


def window_rows(orders, pts, w):
    """Window candidates of points `pts` in the given (checked) orders."""
    out = []
    for sig in orders:
        n = sig.shape[0]
        inv = np.empty(n, np.int64)
        inv[sig] = np.arange(n)
        p = inv[pts]
        c = np.full((len(pts), 2 * w), -1, np.int64)
        for j, off in enumerate(list(range(-w, 0)) + list(range(1, w + 1))):
            pp = p + off
            ok = (pp >= 0) & (pp < n)
            c[ok, j] = sig[pp[ok]]
        out.append(c)
    return np.concatenate(out, axis=1)


def test_sampled_graph_rows(full):
    rng = np.random.default_rng(S.SEED_SAMPLE + 1)
    pts = np.sort(rng.choice(N, 1500, replace=False))
    cand = window_rows(full["orders"], pts, W)
    oi, od = O.topk_from_candidates(full["x"], pts, cand, K)
    check_lists(full["x"], full["gi"][pts], full["gd"][pts], oi, od, owners=pts, cand=cand)


@pytest.mark.parametrize("w,key", [(W, "ti"), (64, "ti64")])
def test_tensor_sampled_graph_rows(full, w, key):
    """The tensor form at 3M x 384 (about 154 tiles per persistent block, so
    every ring, accumulator and barrier phase wraps many times): sampled rows
    against the oracle's top-k of their window candidates."""
    rng = np.random.default_rng(S.SEED_SAMPLE + 2)
    pts = np.sort(np.concatenate([rng.choice(N, 1500, replace=False), np.arange(N - 40, N), np.arange(40)]))
    pts = np.unique(pts)
    cand = window_rows(full["orders"], pts, w)
    oi, od = O.topk_from_candidates(full["x"], pts, cand, K)
    ti, td = full[key], full["td" if key == "ti" else "td64"]
    check_tensor_lists(full["x"], ti[pts], td[pts], oi, owners=pts, cand=cand)


def test_sampled_search_rows(full):
    x, q = full["x"], full["q"]
    lo, sc = oracle_setup(x)
    qs = np.arange(0, 2000, 7)
    qc = O.quantize(q[qs], lo, sc, 8)
    G = full["G"]
    cands = []
    for t in range(T):
        pi, r = O.tree_params(S.SEED_FOREST, t, D)
        sig = full["orders"][t]
        p = G.locate(t, torch.from_numpy(np.ascontiguousarray(q[qs])).cuda())
        kq = O.hilbert_keys(qc, pi, r, 8)
        # lower-bound property: key(sig[p-1]) < key(q) <= key(sig[p])
        left = sig[np.clip(p - 1, 0, N - 1)]
        right = sig[np.clip(p, 0, N - 1)]
        kl = O.hilbert_keys(O.quantize(x[left], lo, sc, 8), pi, r, 8)
        kr = O.hilbert_keys(O.quantize(x[right], lo, sc, 8), pi, r, 8)
        for j in range(len(qs)):
            tq = tuple(int(v) for v in kq[j])
            if p[j] > 0:
                assert tuple(int(v) for v in kl[j]) < tq, f"tree {t} query {qs[j]}"
            if p[j] < N:
                assert tq <= tuple(int(v) for v in kr[j]), f"tree {t} query {qs[j]}"
        c = np.full((len(qs), 2 * W), -1, np.int64)
        for jj, off in enumerate(range(-W, W)):
            pp = p + off
            ok = (pp >= 0) & (pp < N)
            c[ok, jj] = sig[pp[ok]]
        cands.append(c)
    cand = np.concatenate(cands, axis=1)
    oi, od = O.topk_from_candidates(x, None, cand, K, xq=q[qs])
    check_lists(x, full["si"][qs], full["sd"][qs], oi, od, queries=q[qs], cand=cand)


def test_exact_oracle_200k(hf):
    """The whole path against the oracle end to end at 200,000 x 384."""
    n, T2 = 200_000, 2
    x = S.gaussian_mixture(n, D, n_components=1000, seed=S.SEED_DATA)
    F = O.Forest(x, T=T2, bits=8, seed=S.SEED_FOREST)
    G = hf.build(torch.from_numpy(x).cuda(), T=T2, bits=8, seed=S.SEED_FOREST)
    for t in range(T2):
        assert np.array_equal(G.order(t).astype(np.int64), F.sigma[t]), f"order of tree {t}"
    gi, gd = G.knn_graph(K, W)
    rows = np.arange(0, n, 97)
    cand = O.candidate_sets(F, W)[rows]
    oi, od = O.topk_from_candidates(x, rows, cand, K)
    check_lists(x, gi.cpu().numpy()[rows], gd.cpu().numpy()[rows], oi, od, owners=rows, cand=cand)
    G.close()


def test_tensor_exact_oracle_200k(hf):
    """The tensor form against the oracle end to end at 200,000 x 384, T = 2,
    w = 32, k = 15: about 1,563 tiles, ten or more per persistent block."""
    n, T2 = 200_000, 2
    x = S.gaussian_mixture(n, D, n_components=1000, seed=S.SEED_DATA)
    F = O.Forest(x, T=T2, bits=8, seed=S.SEED_FOREST)
    G = hf.build(torch.from_numpy(x).cuda(), T=T2, bits=8, seed=S.SEED_FOREST)
    G.set_option("mode", 1)
    gi, gd = G.knn_graph(K, W)
    oi, od = O.knn_graph(F, K, W)
    cand = O.candidate_sets(F, W)
    check_tensor_lists(x, gi.cpu().numpy(), gd.cpu().numpy(), oi, owners=np.arange(n), cand=cand)
    G.close()


def test_tensor_ragged_1m_w64(hf):
    """A ragged n (1,000,003 = 7,812 tiles + 67 rows) at the widest
    single-tile window: sampled rows, the last tile's rows included."""
    n, T2, w = 1_000_003, 2, 64
    x = S.gaussian_mixture(n, D, n_components=1000, seed=S.SEED_DATA + 7)
    G = hf.build(torch.from_numpy(x).cuda(), T=T2, bits=8, seed=S.SEED_FOREST)
    G.set_option("mode", 1)
    gi, gd = G.knn_graph(K, w)
    torch.cuda.synchronize()
    orders = [G.order(t).astype(np.int64) for t in range(T2)]
    lo, sc = oracle_setup(x)
    for t in range(T2):
        pi, r = O.tree_params(S.SEED_FOREST, t, D)
        sig = orders[t]
        assert np.array_equal(np.sort(sig), np.arange(n))
        # order property on the tail and on sampled positions
        pos = np.concatenate([np.arange(n - 200, n - 1), np.random.default_rng(t).choice(n - 1, 2000, replace=False)])
        ka = O.hilbert_keys(O.quantize(x[sig[pos]], lo, sc, 8), pi, r, 8)
        kb = O.hilbert_keys(O.quantize(x[sig[pos + 1]], lo, sc, 8), pi, r, 8)
        for i in range(len(pos)):
            ta = tuple(int(v) for v in ka[i]) + (int(sig[pos[i]]),)
            tb = tuple(int(v) for v in kb[i]) + (int(sig[pos[i] + 1]),)
            assert ta < tb
    rng = np.random.default_rng(S.SEED_SAMPLE + 3)
    pts = np.unique(np.concatenate([rng.choice(n, 1500, replace=False), orders[0][-67:], orders[1][-67:]]))
    cand = window_rows(orders, pts, w)
    oi, od = O.topk_from_candidates(x, pts, cand, K)
    check_tensor_lists(x, gi.cpu().numpy()[pts], gd.cpu().numpy()[pts], oi, owners=pts, cand=cand)
    G.close()


def test_sketch_sampled_graph_rows(full):
    """The sketch form (384-bit sketches, k2 = 60) on the full-size forest:
    sampled rows against the oracle's Hamming top-k2 and exact top-k of their
    window candidates (from the checked orders). Rows whose point or a
    candidate holds a sketch bit within the FP32 bound of its decision are
    checked for validity only."""
    from oracle import sketch as OS
    x, G = full["x"], full["G"]
    R = S.sketch_projection(384, D, seed=S.SEED_SKETCH)
    G.set_sketch(torch.from_numpy(R).cuda())
    G.set_option("mode", 3)
    G.set_option("sketch_k2", 60)
    gi, gd = G.knn_graph(K, W)
    G.set_option("mode", 0)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    skg = G.sketches()
    rng = np.random.default_rng(S.SEED_SAMPLE + 3)
    pts = np.sort(rng.choice(N, 800, replace=False))
    cand = window_rows(full["orders"], pts, W)
    need = np.unique(np.concatenate([pts, cand[cand >= 0]]))
    dots = OS.sketch_dots(x[need], R)
    xb, rb = O.budget.bf16(x[need]), O.budget.bf16(R)
    amb = np.abs(dots) <= D * 2.0 ** -24 * (np.abs(xb) @ np.abs(rb).T)
    sk = np.zeros((N, 6), np.uint64)
    sk[need] = OS.pack_bits(dots > 0)
    flipped = np.zeros(N, bool)
    bits_g = np.unpackbits(skg[need].view(np.uint8), axis=1, bitorder="little").astype(bool)
    assert not ((bits_g != (dots > 0)) & ~amb).any(), "sketch bits differ outside the FP32 bound"
    flipped[need] = (bits_g != (dots > 0)).any(axis=1)
    c2 = OS.top_k2_by_hamming(sk, pts, cand, 60)
    oi, od = O.topk_from_candidates(x, pts, c2, K)
    touched = flipped[pts] | np.array([flipped[c[c >= 0]].any() for c in cand])
    strict = ~touched
    assert strict.mean() > 0.5
    check_lists(x, gi[pts][strict], gd[pts][strict], oi[strict], od[strict], owners=pts[strict], cand=cand[strict],
                min_equal=0.99)


def test_batched_workload_equals_independent(hf):
    """The batched workload at full size (64 sets, 2.8M points, the forms and
    windows the bench's tuner picks): every row of every set equals the same
    set built and graphed alone; two small sets also against the oracle."""
    sets = S.batched_sets(64)
    plan = {64: (1, 16, 256), 128: (1, 16, 256), 384: (1, 16, 384), 768: (2, 32, 512)}  # form, slots, w
    k, T2 = 10, 16
    for d, (form, slots, w) in plan.items():
        idx = [i for i, x in enumerate(sets) if x.shape[1] == d]
        off = np.zeros(len(idx) + 1, np.int64)
        off[1:] = np.cumsum([sets[i].shape[0] for i in idx])
        G = hf.build_segmented(torch.from_numpy(np.concatenate([sets[i] for i in idx])).cuda(), off, T=T2, seed=3)
        G.set_option("mode", form)
        G.set_option("tensor_slack", slots - k)
        gi, gd = G.knn_graph(k, w)
        gi, gd = gi.cpu().numpy().astype(np.int64), gd.cpu().numpy()
        G.close()
        for j, i in enumerate(idx):
            a, b = off[j], off[j + 1]
            H = hf.build(torch.from_numpy(sets[i]).cuda(), T=T2, seed=3)
            H.set_option("mode", form)
            H.set_option("tensor_slack", slots - k)
            hi_, hd_ = H.knn_graph(k, w)
            H.close()
            hi_ = hi_.cpu().numpy().astype(np.int64)
            assert np.array_equal(gi[a:b], np.where(hi_ >= 0, hi_ + a, -1)), f"set {i} (d={d}): lists"
            assert np.array_equal(gd[a:b], hd_.cpu().numpy()), f"set {i} (d={d}): distances"
        small = min(range(len(idx)), key=lambda j: off[j + 1] - off[j])
        a, b = off[small], off[small + 1]
        x = sets[idx[small]]
        F = O.Forest(x, T=T2, bits=8, seed=3)
        oi, _ = O.knn_graph(F, k, w)
        li = np.where(gi[a:b] >= 0, gi[a:b] - a, -1)
        check_tensor_lists(x, li, gd[a:b], oi, owners=np.arange(b - a), cand=O.candidate_sets(F, w),
                           min_hit=0.98 if form == 1 else 0.93)
