"""Pins of the learned-budget oracle (oracle/budget.py), no GPU.

The model's backward pass is pinned to central finite differences of its own
float64 loss (an independent route to the same derivatives); GELU to values
of the normal distribution function; BF16 rounding to hand-worked bit
patterns; the labels to the graph oracle's window candidate sets; the
budgeted graph to the pinned uniform-budget graph.
"""
import math

import numpy as np
import pytest

import oracle as O
import synthdata as S
from oracle import budget as OB


def test_gelu_values():
    z = np.array([0.0, 1.0, -1.0, 10.0, -10.0])
    phi1 = 0.5 * (1.0 + math.erf(1.0 / math.sqrt(2.0)))  # Phi(1) = 0.841344746...
    want = np.array([0.0, phi1, -(1.0 - phi1), 10.0, 0.0])
    assert np.allclose(OB.gelu(z), want, atol=1e-12)
    assert OB.gelu_grad(np.array([0.0]))[0] == pytest.approx(0.5)
    # derivative against a central difference
    x = np.linspace(-4, 4, 41)
    h = 1e-6
    assert np.allclose(OB.gelu_grad(x), (OB.gelu(x + h) - OB.gelu(x - h)) / (2 * h), atol=1e-8)


def test_bf16_rounding():
    one = 1.0
    vals = np.array([one, one + 2.0 ** -8, one + 3 * 2.0 ** -9, one + 2.0 ** -7, -2.5, 0.0], dtype=np.float32)
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties to even -> 1
    # 1 + 3 * 2^-9 is above the halfway point -> 1 + 2^-7
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -7, 1.0 + 2.0 ** -7, -2.5, 0.0])
    assert np.array_equal(OB.bf16(vals), want)
    r = OB.bf16(np.random.default_rng(0).standard_normal(1000))
    assert np.max(np.abs(OB.bf16(r) - r)) == 0  # idempotent
    # every result has at most 8 significant bits
    m, _ = np.frexp(r[r != 0])
    assert np.all(m * 2 ** 8 == np.round(m * 2 ** 8))


@pytest.mark.parametrize("seed", [1, 2])
def test_mlp_gradients_equal_finite_differences(seed):
    """Backward pass of the float64 network (no BF16 storage) against central
    differences of its loss, for every parameter of a small network."""
    rng = np.random.default_rng(seed)
    d, h, B = 5, 7, 6
    npar = h * d + h + h * h + h + 2 * h + 2
    p = rng.standard_normal(npar) * 0.5
    x = rng.standard_normal((B, d))
    t = rng.standard_normal((B, 2))
    loss, g = OB.mlp_loss_grads(p, x, t, h=h, bf16_storage=False)
    eps = 1e-6
    num = np.empty(npar)
    for j in range(npar):
        a, b = p.copy(), p.copy()
        a[j] += eps
        b[j] -= eps
        num[j] = (OB.mlp_loss_grads(a, x, t, h=h, bf16_storage=False)[0]
                  - OB.mlp_loss_grads(b, x, t, h=h, bf16_storage=False)[0]) / (2 * eps)
    assert np.allclose(g, num, rtol=1e-6, atol=1e-9)
    y, _ = OB.mlp_forward(p, x, h=h, bf16_storage=False)
    assert loss == pytest.approx(0.5 * np.sum((y - t) ** 2) / B)


def test_mlp_bf16_storage_is_close_to_exact():
    rng = np.random.default_rng(3)
    d, h, B = 16, 256, 64
    npar = h * d + h + h * h + h + 2 * h + 2
    p = rng.standard_normal(npar) * 0.05
    x = rng.standard_normal((B, d))
    t = rng.standard_normal((B, 2))
    l1, g1 = OB.mlp_loss_grads(p, x, t, h=h, bf16_storage=True)
    l0, g0 = OB.mlp_loss_grads(p, x, t, h=h, bf16_storage=False)
    assert abs(l1 - l0) < 2e-2 * abs(l0)
    assert np.linalg.norm(g1 - g0) < 3e-2 * np.linalg.norm(g0)


def _forest_and_knn(n=600, d=12, T=8):
    x = S.gaussian_mixture(n, d, n_components=10, seed=4)
    F = O.Forest(x, T=T, bits=8, seed=3)
    ei, _ = O.brute_force_knn(x, 10)
    return F, ei


def test_labels_agree_with_window_candidates():
    """A point's label cell (T, w) holds at least min_hits of its neighbours in
    the graph oracle's candidate set over T trees with window w, and no
    cheaper cell does."""
    F, ei = _forest_and_knn()
    tg, wg, mh = [1, 2, 4, 8], [2, 4, 8, 16], 6
    targets, cells = OB.budget_labels(F.sigma, ei, tg, wg, mh)
    rows = np.arange(0, F.n, 7)
    for a, Tc in enumerate(tg):
        for b, w in enumerate(wg):
            cand = O.candidate_sets(F, w, trees=range(Tc))[rows]
            hits = np.array([len(set(c[c >= 0].tolist()) & set(e.tolist())) for c, e in zip(cand, ei[rows])])
            cost = Tc * (128 + 2 * w)
            lab = cells[rows]
            lab_cost = np.array([tg[c // len(wg)] * (128 + 2 * wg[c % len(wg)]) for c in lab])
            # the labelled cell is reachable ...
            at = lab == a * len(wg) + b
            assert np.all(hits[at] >= mh) or np.all(lab[at] == len(tg) * len(wg) - 1)
            # ... and no cheaper reaching cell exists
            assert not np.any((hits >= mh) & (cost < lab_cost))
    assert np.allclose(targets[:, 0], np.log2(np.array(wg)[cells % len(wg)]))
    assert np.allclose(targets[:, 1], np.log2(np.array(tg)[cells // len(wg)]))


def test_labels_trivial_cases():
    F, ei = _forest_and_knn()
    tg, wg = [1, 2], [4, 8]
    _, cells = OB.budget_labels(F.sigma, ei, tg, wg, 0)
    assert np.all(cells == 0)  # every point reaches 0 hits at the cheapest cell
    _, cells = OB.budget_labels(F.sigma, ei, tg, [F.n], 10)
    assert np.all(cells == 0)  # a window of n positions holds everything in the first tree


def test_budget_graph_uniform_equals_graph():
    F, _ = _forest_and_knn(T=4)
    w, T, k = 6, 3, 8
    gi, gd = OB.knn_graph_budget(F, k, np.full(F.n, w), np.full(F.n, T))
    F3 = O.Forest(F.x, T=T, bits=8, seed=3)
    oi, od = O.knn_graph(F3, k, w)
    assert np.array_equal(gi, oi) and np.allclose(gd, od)


def test_budget_graph_zero_budget_is_empty():
    F, _ = _forest_and_knn(T=2)
    w_pt = np.full(F.n, 5)
    T_pt = np.full(F.n, 2)
    T_pt[::3] = 0
    gi, gd = OB.knn_graph_budget(F, 6, w_pt, T_pt)
    assert np.all(gi[::3] == -1) and np.all(np.isinf(gd[::3]))
    assert np.all(gi[1::3, 0] >= 0)
