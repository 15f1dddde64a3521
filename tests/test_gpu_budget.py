"""The learned per-point budget on the GPU, through the C ABI, against the
oracle (oracle/budget.py): the MLP's forward pass and gradients, the labels,
the graph with per-point budgets, the full-window graph as exact kNN, and
what the trained network gains over a uniform budget of the same cost."""
import numpy as np
import pytest

import oracle as O
import synthdata as S
from oracle import budget as OB
from _helpers import check_tensor_lists

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


def _params(d, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    h = 256
    w1 = rng.uniform(-1, 1, (h, d)) / np.sqrt(d) * scale
    w2 = rng.uniform(-1, 1, (h, h)) / 16 * scale
    w3 = rng.uniform(-1, 1, (2, h)) / 16 * scale
    b1, b2, b3 = rng.normal(0, 0.1, h), rng.normal(0, 0.1, h), rng.normal(0, 0.1, 2)
    return OB.pack(w1, b1, w2, b2, w3, b3).astype(np.float32)


@pytest.mark.parametrize("d,B", [(384, 256), (64, 128), (100, 384)])
def test_mlp_forward_and_gradients_match_oracle(hf, d, B):
    """Same BF16-rounded tensors on both sides: outputs within 1e-2 relative
    (BF16 rounding of an intermediate may differ by one unit between the
    float32 and float64 accumulations), gradients within 3e-2 of the
    oracle's per tensor (relative 2-norm), the loss within 1e-3."""
    p = _params(d, seed=d + B, scale=2.0)
    rng = np.random.default_rng(7)
    x = rng.standard_normal((B, d)).astype(np.float32)
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    t = rng.standard_normal((B, 2)).astype(np.float32)
    m = hf.Mlp(d)
    m.set_params(p)
    assert np.array_equal(m.get_params(), p)
    y = m.predict(cuda(x)).cpu().numpy()
    yo, _ = OB.mlp_forward(p, x)
    assert np.max(np.abs(y - yo)) <= 1e-2 * np.max(np.abs(yo)) + 1e-4
    loss, g = m.grads(cuda(x), cuda(t))
    lo, go = OB.mlp_loss_grads(p, x, t)
    assert loss == pytest.approx(lo, rel=1e-3)
    h = 256
    sizes = [h * d, h, h * h, h, 2 * h, 2]
    o = 0
    for name, sz in zip(["W1", "b1", "W2", "b2", "W3", "b3"], sizes):
        a, b = g[o:o + sz].astype(np.float64), go[o:o + sz]
        assert np.linalg.norm(a - b) <= 3e-2 * np.linalg.norm(b) + 1e-7, name
        o += sz
    m.close()


def test_mlp_training_reduces_loss(hf):
    """Adam on a regression the network can represent: the loss falls by an
    order of magnitude, and the trained weights still give oracle-equal
    outputs."""
    d, n = 64, 8192
    rng = np.random.default_rng(11)
    x = rng.standard_normal((n, d)).astype(np.float32)
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    t = np.stack([4.0 * x[:, 0] + np.abs(3.0 * x[:, 1]), np.tanh(5.0 * x[:, 2])], 1).astype(np.float32)
    m = hf.Mlp(d, seed=3)
    xd, td = cuda(x), cuda(t)
    l0, _ = m.grads(xd[:1024], td[:1024])
    l1 = m.train(xd, td, batch=1024, steps=600, lr=2e-3)
    assert l1 < 0.1 * l0, (l0, l1)
    p = m.get_params()
    y = m.predict(xd[:512]).cpu().numpy()
    yo, _ = OB.mlp_forward(p, x[:512])
    assert np.max(np.abs(y - yo)) <= 1e-2 * np.max(np.abs(yo)) + 1e-3
    m.close()


def test_budget_labels_match_oracle(hf):
    n, d, T = 3000, 32, 8
    x = S.gaussian_mixture(n, d, n_components=20, seed=5)
    ei, _ = O.brute_force_knn(x, 10)
    F = O.Forest(x, T=T, bits=8, seed=3)
    G = hf.build(cuda(x), T=T, bits=8, seed=3)
    tg, wg, mh = [1, 2, 4, 8], [4, 8, 16, 32, 64], 7
    tgt, cell = G.budget_labels(cuda(ei.astype(np.int32)), tg, wg, mh)
    ot, oc = OB.budget_labels(F.sigma, ei, tg, wg, mh)
    assert np.array_equal(cell.cpu().numpy(), oc)
    assert np.array_equal(tgt.cpu().numpy().astype(np.float64), ot)
    G.close()


@pytest.mark.parametrize("mode", [1, 2])
def test_knn_graph_budget_parity(hf, mode):
    n, d, T, k = 4001, 64, 4, 10
    x = S.gaussian_mixture(n, d, n_components=30, seed=6)
    rng = np.random.default_rng(8)
    w_pt = rng.integers(1, 90, n).astype(np.int32)
    T_pt = rng.integers(0, T + 1, n).astype(np.int32)
    F = O.Forest(x, T=T, bits=8, seed=3)
    G = hf.build(cuda(x), T=T, bits=8, seed=3)
    G.set_option("mode", mode)
    G.set_option("tensor_slack", 1 if mode == 1 else 17)
    gi, gd = G.knn_graph_budget(k, cuda(w_pt), cuda(T_pt))
    oi, od = OB.knn_graph_budget(F, k, w_pt, T_pt)
    cand = OB.budget_candidates(F, w_pt, T_pt)
    check_tensor_lists(x, gi.cpu().numpy(), gd.cpu().numpy(), oi, owners=np.arange(n), cand=cand,
                       min_hit=0.995 if mode == 1 else 0.98)
    G.close()


def test_full_window_tensor_graph_is_exact_knn(hf):
    """One order with w >= n - 1: every pair is a candidate, so the graph is
    the exact kNN (BF16 estimates keep k + 17, the float32 re-rank orders
    them)."""
    n, d, k = 3000, 64, 15
    x = S.gaussian_mixture(n, d, n_components=20, seed=9)
    G = hf.build(cuda(x), T=1, bits=8, seed=1)
    G.set_option("mode", 1)
    G.set_option("tensor_slack", 17)
    gi, gd = G.knn_graph(k, n)
    ei, ed = O.brute_force_knn(x, k)
    check_tensor_lists(x, gi.cpu().numpy(), gd.cpu().numpy(), ei, owners=np.arange(n), min_hit=0.999)
    G.close()


def _recall(found, exact):
    k = exact.shape[1]
    return float(np.mean([len(set(a[a >= 0].tolist()) & set(b.tolist())) / k for a, b in zip(found, exact)]))


def test_learned_budget_reaches_recall_cheaper_than_uniform(hf):
    """What the trained network gains over the method without it. The labels
    give each training point the cheapest budget at which 12 of its 15 true
    neighbours are candidates; the network predicts that need for unseen
    points. Judged on held-out points by recall@15 of the graph the library
    builds, against the cost of the graph (mean over all points of
    T_i (128 + 2 w_i), the band columns the Gram kernel computes): the
    learned budgets, scaled by one factor 2^s, reach the target recall at a
    lower cost than the cheapest uniform budget of the grid that does."""
    n, d, T, k = 60000, 128, 32, 15
    x = S.gaussian_mixture(n, d, n_components=200, seed=12)
    xd = cuda(x)
    # exact neighbours of every point: the full-window tensor graph
    E = hf.build(xd, T=1, bits=8, seed=1)
    E.set_option("mode", 1)
    E.set_option("tensor_slack", 17)
    ei, _ = E.knn_graph(k, n)
    E.close()
    G = hf.build(xd, T=T, bits=8, seed=3)
    G.set_option("mode", 1)
    tg, wg = [2, 4, 8, 16, 32], [8, 16, 32, 64, 128]
    tgt, cell = G.budget_labels(ei, tg, wg, 12)
    rng = np.random.default_rng(13)
    perm = rng.permutation(n)
    tr, te = perm[:48000], perm[48000:]
    m = hf.Mlp(d, seed=7)
    tr_t = torch.from_numpy(tr).cuda()
    m.train(xd[tr_t].contiguous(), tgt[tr_t].contiguous(), batch=1024, steps=1500, lr=1e-3)
    pred = m.predict(xd).cpu().numpy().astype(np.float64)
    m.close()
    exact = ei.cpu().numpy()[te]

    def recall_of(w, t):
        li, _ = G.knn_graph_budget(k, cuda(w.astype(np.int32)), cuda(t.astype(np.int32)))
        return _recall(li.cpu().numpy()[te], exact)

    def cost(w, t):
        return float(np.mean(t * (128.0 + 2.0 * w)))

    ones = np.ones(n)
    r_max = recall_of(ones * wg[-1], ones * tg[-1])
    target = min(0.8, 0.95 * r_max)
    cells = sorted(((Tc * (128 + 2 * w), Tc, w) for Tc in tg for w in wg))
    c_uniform = None
    for c, Tc, w in cells:
        if recall_of(ones * w, ones * Tc) >= target:
            c_uniform = c
            break
    assert c_uniform is not None

    def budgets(shift):
        w = np.clip(np.round(2.0 ** (pred[:, 0] + shift)), 1, 4096)
        t = np.clip(np.round(2.0 ** (pred[:, 1] + shift)), 1, T)
        return w, t

    lo, hi = -6.0, 6.0
    assert recall_of(*budgets(hi)) >= target
    for _ in range(14):  # the smallest shift that reaches the target (recall grows with the shift)
        mid = 0.5 * (lo + hi)
        if recall_of(*budgets(mid)) >= target:
            hi = mid
        else:
            lo = mid
    c_learned = cost(*budgets(hi))
    print(f"target recall@15 {target:.3f}: uniform cost {c_uniform:.0f}, learned cost {c_learned:.0f} "
          f"({c_uniform / c_learned:.2f}x less work)")
    assert c_learned < 0.9 * c_uniform
    G.close()
