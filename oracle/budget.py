"""Plain CPU oracle of the learned per-point budget -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the bench's CPU arms may import it;
the CUDA library never calls it. It shares no code with the library.

The paper spends one budget (the number of sorts and the window around each
position, Algorithm 2; Table 2 trades recall against it) on every point. The
extension checked here gives each point i its own budget (w_i, T_i): its
candidates are the points within w_i positions of it in the first T_i orders.
It has three parts, each written out plainly:

* labels      -- for each point, the cheapest cell (T, w) of a grid (cost
                 T (128 + 2 w)) at which at least `min_hits` of its exact
                 neighbours lie within w positions of it in one of the first
                 T orders (the largest cell when none does);
* the model   -- an MLP d -> H -> H -> 2 with GELU(z) = z Phi(z), mean squared
                 error L = 1/(2B) sum (y - target)^2, written as a forward pass
                 and its chain-rule backward pass in float64. With
                 ``bf16=True`` the tensors that the library stores in BF16
                 (inputs, weights, the GELU outputs, the back-propagated
                 pre-activation gradients that feed the weight gradients) are
                 rounded to BF16 at the same places, so the two can be
                 compared element by element;
* the graph   -- the top k of each point's budgeted candidate set by float64
                 distance, ties by index (as oracle.knn_graph).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

from .hilbert_forest import Forest, sq_dist_fp64, topk_from_candidates


# --------------------------------------------------------------------------
# BF16 rounding (round to nearest, ties to even, of the float32 value)
# --------------------------------------------------------------------------
def bf16(x: np.ndarray) -> np.ndarray:
    """The float32 value of x rounded to the nearest BF16 value (8 mantissa
    bits), ties to even; returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


# --------------------------------------------------------------------------
# The model
# --------------------------------------------------------------------------
def gelu(z):
    """GELU(z) = z Phi(z), Phi the standard normal distribution function."""
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    """d GELU / dz = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def unpack(params: np.ndarray, d: int, h: int = 256):
    """W1 [h][d], b1 [h], W2 [h][h], b2 [h], W3 [2][h], b3 [2] from the packed
    parameter vector."""
    p = np.asarray(params, dtype=np.float64)
    sizes = [h * d, h, h * h, h, 2 * h, 2]
    assert p.size == sum(sizes), "packed parameter count"
    out, o = [], 0
    for sz in sizes:
        out.append(p[o:o + sz])
        o += sz
    w1, b1, w2, b2, w3, b3 = out
    return w1.reshape(h, d), b1, w2.reshape(h, h), b2, w3.reshape(2, h), b3


def pack(w1, b1, w2, b2, w3, b3) -> np.ndarray:
    return np.concatenate([np.ravel(a) for a in (w1, b1, w2, b2, w3, b3)])


def mlp_forward(params, x, h: int = 256, bf16_storage: bool = True):
    """Outputs y [B][2] and the intermediates (a dict) of the MLP."""
    x = np.asarray(x, dtype=np.float64)
    w1, b1, w2, b2, w3, b3 = unpack(params, x.shape[1], h)
    r = bf16 if bf16_storage else (lambda a: np.asarray(a, dtype=np.float64))
    xb, w1b, w2b, w3b = r(x), r(w1), r(w2), r(w3)
    z1 = xb @ w1b.T + b1
    h1 = r(gelu(z1))
    z2 = h1 @ w2b.T + b2
    h2 = r(gelu(z2))
    y = h2 @ w3b.T + b3
    return y, dict(x=xb, w1=w1b, w2=w2b, w3=w3b, z1=z1, h1=h1, z2=z2, h2=h2)


def mlp_loss_grads(params, x, targets, h: int = 256, bf16_storage: bool = True):
    """(loss, packed gradients) of L = 1/(2B) sum (y - target)^2.

    Chain rule, layer by layer: dY = (y - t) / B; dW3 = dY^T H2, db3 = sum dY;
    dH2 = dY W3; dZ2 = dH2 * GELU'(Z2); dW2 = dZ2^T H1, db2 = sum dZ2;
    dH1 = dZ2 W2; dZ1 = dH1 * GELU'(Z1); dW1 = dZ1^T X, db1 = sum dZ1. With
    BF16 storage the dY and dZ factors of the weight gradients and of the
    next dH are rounded to BF16 (the bias sums use the unrounded values)."""
    t = np.asarray(targets, dtype=np.float64)
    y, c = mlp_forward(params, x, h, bf16_storage)
    B = y.shape[0]
    r = bf16 if bf16_storage else (lambda a: a)
    e = y - t
    loss = 0.5 * np.sum(e * e) / B
    dy = e / B
    dyb = r(dy)
    dw3 = dyb.T @ c["h2"]
    db3 = dy.sum(0)
    dh2 = dyb @ c["w3"]
    dz2 = dh2 * gelu_grad(c["z2"])
    dz2b = r(dz2)
    dw2 = dz2b.T @ c["h1"]
    db2 = dz2.sum(0)
    dh1 = dz2b @ c["w2"]
    dz1 = dh1 * gelu_grad(c["z1"])
    dz1b = r(dz1)
    dw1 = dz1b.T @ c["x"]
    db1 = dz1.sum(0)
    return loss, pack(dw1, db1, dw2, db2, dw3, db3)


# --------------------------------------------------------------------------
# Labels
# --------------------------------------------------------------------------
def budget_labels(sigmas, knn, t_grid, w_grid, min_hits):
    """Per point: the cheapest cell (T, w) (cost T (128 + 2 w), first in
    (T, w) order on equal cost) at which at least min_hits of its exact
    neighbours knn[i] (-1 = none) lie within w positions of it in one of the
    first T orders sigmas[0..T); the last cell when none does. Returns
    (targets float64 [n][2] = (log2 w, log2 T), cells int64 [n])."""
    sigmas = [np.asarray(s, dtype=np.int64) for s in sigmas]
    knn = np.asarray(knn, dtype=np.int64)
    n, k = knn.shape
    T = t_grid[-1]
    pos = np.empty((T, n), dtype=np.int64)
    for t in range(T):
        pos[t, sigmas[t]] = np.arange(n)
    valid = knn >= 0
    e = np.where(valid, knn, 0)
    gaps = np.abs(pos[:, np.arange(n)[:, None]] - pos[:, e])  # [T][n][k]
    cells = np.full(n, len(t_grid) * len(w_grid) - 1, dtype=np.int64)
    best_cost = np.full(n, np.inf)
    for a, Tc in enumerate(t_grid):
        g = gaps[:Tc].min(axis=0)
        for b, w in enumerate(w_grid):
            hits = ((g <= w) & valid).sum(axis=1)
            cost = Tc * (128.0 + 2.0 * w)
            take = (hits >= min_hits) & (cost < best_cost)
            cells[take] = a * len(w_grid) + b
            best_cost[take] = cost
    nw = len(w_grid)
    targets = np.stack([np.log2(np.asarray(w_grid, np.float64)[cells % nw]),
                        np.log2(np.asarray(t_grid, np.float64)[cells // nw])], axis=1)
    return targets, cells


# --------------------------------------------------------------------------
# The graph with per-point budgets
# --------------------------------------------------------------------------
def budget_candidates(forest: Forest, w_pt, T_pt):
    """C(i) = points within w_i positions of i in orders t < T_i, as an int64
    [n][max_T * 2 max_w] array with -1 padding (repeats allowed)."""
    w_pt = np.asarray(w_pt, dtype=np.int64)
    T_pt = np.asarray(T_pt, dtype=np.int64)
    n = forest.n
    wmax, tmax = int(max(1, w_pt.max())), int(max(1, T_pt.max()))
    cand = np.full((n, tmax * 2 * wmax), -1, dtype=np.int64)
    col = 0
    for t in range(tmax):
        pos = forest.position(t)
        sig = forest.sigma[t]
        for delta in list(range(-wmax, 0)) + list(range(1, wmax + 1)):
            p = pos + delta
            ok = (p >= 0) & (p < n) & (abs(delta) <= w_pt) & (t < T_pt)
            cand[ok, col] = sig[p[ok]]
            col += 1
    return cand


def knn_graph_budget(forest: Forest, k: int, w_pt, T_pt):
    """Top k of each budgeted candidate set by (float64 distance, index)."""
    cand = budget_candidates(forest, w_pt, T_pt)
    owners = np.arange(forest.n)
    out_i = np.empty((forest.n, k), np.int64)
    out_d = np.empty((forest.n, k), np.float64)
    for s in range(0, forest.n, 2048):
        i, dd = topk_from_candidates(forest.x, owners[s:s + 2048], cand[s:s + 2048], k)
        out_i[s:s + 2048], out_d[s:s + 2048] = i, dd
    return out_i, out_d


__all__ = ["bf16", "gelu", "gelu_grad", "unpack", "pack", "mlp_forward", "mlp_loss_grads", "budget_labels",
           "budget_candidates", "knn_graph_budget", "sq_dist_fp64"]
