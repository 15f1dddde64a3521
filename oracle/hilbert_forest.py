"""Plain CPU oracle of the Hilbert forest's data-parallel path.

TEST INFRASTRUCTURE ONLY. This module is the independent reference that the
CUDA library is checked against. Only the test suite, the smoke check and the
bench's CPU-baseline / reference arm may import it; the product path never
does. It shares no code with the CUDA library.

It is deliberately slow and literal: numpy, loops over the algorithm's steps,
vectorised only across points, float64 for every distance. Each function names
the part of the paper (arXiv 2508.21682, "Hilbert Forest in the SISAP 2025
Indexing Challenge") it restates, or the convention it fixes where the paper is
silent.

Paper passages used
-------------------
* Section 2: Hilbert sort orders points along a Hilbert curve; the order is a
  total order, so binary search locates an arbitrary point in it; a Hilbert
  forest is several such orders.
* Algorithm 2 (Section 4, kNN graph): every sort first shuffles the
  coordinate axes and orders all points along the curve; each point gains as
  candidates the points that sit within a window around it in that order; the
  result keeps, per point, the k candidates nearest by vector distance.
* Algorithm 1 (Section 3, search): per tree, locate each query in the Hilbert
  order and add the candidates near its position; select the top k by vector
  distance.

Conventions where the paper is silent (each is a reading, not a paper fact)
---------------------------------------------------------------------------
* Curve: Skilling's transposed Hilbert index (J. Skilling, "Programming the
  Hilbert curve", AIP Conf. Proc. 707, 2004).
* Quantization for the sort: per-axis min/max over the data, b bits, floor,
  clamp, exact IEEE float32 steps (no fused multiply-add).
* Random axis order per tree: splitmix64 (Steele, Lea & Flood, OOPSLA 2014)
  driving a Fisher-Yates shuffle, plus a per-axis reflection bit.
* Equal keys: ordered by ascending point index.
* Window: w positions on each side of position i (2w candidates), no wrap.
* Candidate sets are sets (duplicates across trees removed); a point is never
  its own candidate.
* Vector distance: squared Euclidean; ties in the top-k broken by index.
* Fewer than k candidates: missing slots are (-1, +inf).
* The sketch filter (top-k2 by Hamming distance) is not part of this path; the
  final top-k runs over the whole candidate set with exact distances.
"""
from __future__ import annotations

import numpy as np

U64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


# --------------------------------------------------------------------------
# Quantization (convention: per-axis range, b bits, exact float32 steps)
# --------------------------------------------------------------------------
def axis_range(x: np.ndarray, bits: int):
    """Per-axis lo = min, hi = max over the data (float32) and the float32
    scale 2^b / (hi - lo), computed in double from the float32 width and
    rounded to float32 once. A zero-width axis gets scale 0, so all its codes
    are 0. Raises ValueError on non-finite input."""
    x = np.asarray(x, dtype=np.float32)
    if not np.all(np.isfinite(x)):
        raise ValueError("non-finite input")
    lo = x.min(axis=0)
    hi = x.max(axis=0)
    width = (hi - lo).astype(np.float32)  # float32 subtraction
    scale = np.zeros_like(lo)
    pos = width > 0
    scale[pos] = (float(1 << bits) / width[pos].astype(np.float64)).astype(np.float32)
    return lo, scale


def quantize(x: np.ndarray, lo: np.ndarray, scale: np.ndarray, bits: int) -> np.ndarray:
    """code = clamp(floor(fl32(fl32(x - lo) * scale)), 0, 2^b - 1).

    Both steps are separate float32 roundings (numpy float32 arithmetic never
    fuses them). Values outside [lo, hi] (queries) clamp to the end codes."""
    x = np.asarray(x, dtype=np.float32)
    if not np.all(np.isfinite(x)):
        raise ValueError("non-finite input")
    diff = np.subtract(x, lo[None, :], dtype=np.float32)
    prod = np.multiply(diff, scale[None, :], dtype=np.float32)
    q = np.floor(prod.astype(np.float64))
    q = np.clip(q, 0, (1 << bits) - 1)
    return q.astype(np.uint16)


# --------------------------------------------------------------------------
# Per-tree random axis order (Algorithm 2 shuffles the axes before every sort;
# Algorithm 1 builds its trees on shuffled axis orders)
# --------------------------------------------------------------------------
class SplitMix64:
    """splitmix64: state advances by the golden-ratio constant; the output is
    the state passed through two xor-shift-multiply rounds and a final
    xor-shift (Steele, Lea & Flood 2014)."""

    def __init__(self, state: int):
        self.state = state & U64

    def next(self) -> int:
        self.state = (self.state + GOLDEN_GAMMA) & U64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & U64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & U64
        return z ^ (z >> 31)


def tree_params(seed: int, tree: int, d: int):
    """Axis permutation pi (int64[d]) and reflection bits r (uint8[d]) of tree t.

    Generator state starts at seed + (t + 1) * gamma (mod 2^64). pi starts as
    the identity; for j = d-1 down to 1, m = next() mod (j + 1) and pi[j], pi[m]
    are swapped (modulo bias accepted). Then r[j] = top bit of next() for
    j = 0 .. d-1. Permuted coordinate j of a point is code[pi[j]], reflected
    (x -> 2^b - 1 - x) when r[j] = 1."""
    g = SplitMix64(seed + (tree + 1) * GOLDEN_GAMMA)
    pi = list(range(d))
    for j in range(d - 1, 0, -1):
        m = g.next() % (j + 1)
        pi[j], pi[m] = pi[m], pi[j]
    r = [g.next() >> 63 for _ in range(d)]
    return np.array(pi, dtype=np.int64), np.array(r, dtype=np.uint8)


def permute_reflect(codes: np.ndarray, pi: np.ndarray, r: np.ndarray, bits: int) -> np.ndarray:
    """y[:, j] = codes[:, pi[j]] XOR (r[j] * (2^b - 1))."""
    full = (1 << bits) - 1
    y = codes[:, pi].astype(np.uint32)
    y ^= (r.astype(np.uint32) * full)[None, :]
    return y


# --------------------------------------------------------------------------
# Hilbert key (Section 2 "Hilbert order"; convention: Skilling 2004)
# --------------------------------------------------------------------------
def skilling_transpose(coords: np.ndarray, bits: int) -> np.ndarray:
    """Skilling's axes-to-transpose map, vectorised over rows.

    coords: [n, d] integers < 2^bits (one point per row). Returns the
    transposed Hilbert index X [n, d]:
      1. for q = bits-1 down to 1 (P = 2^q - 1), for i = 0 .. d-1 in order:
         if bit q of X[i] is set, X[0] ^= P; otherwise swap the low q bits of
         X[0] and X[i];
      2. Gray encode: X[i] ^= X[i-1] for i = 1 .. d-1 in order;
      3. t = XOR of (2^q - 1) over q = bits-1 .. 1 with bit q of X[d-1] set;
         X[i] ^= t for every i.
    """
    X = np.array(coords, dtype=np.uint32, copy=True)
    n, d = X.shape
    for q in range(bits - 1, 0, -1):
        P = np.uint32((1 << q) - 1)
        for i in range(d):
            bit = ((X[:, i] >> np.uint32(q)) & np.uint32(1)).astype(bool)
            # invert the low q bits of X[0] where bit q of X[i] is set
            x0 = X[:, 0]
            inv = np.where(bit, x0 ^ P, x0)
            # exchange the low q bits of X[0] and X[i] elsewhere
            t = (inv ^ X[:, i]) & P
            t = np.where(bit, np.uint32(0), t)
            X[:, 0] = inv ^ t
            if i != 0:
                X[:, i] = X[:, i] ^ t
    for i in range(1, d):
        X[:, i] ^= X[:, i - 1]
    t = np.zeros(n, dtype=np.uint32)
    for q in range(bits - 1, 0, -1):
        bit = ((X[:, d - 1] >> np.uint32(q)) & np.uint32(1)).astype(bool)
        t = np.where(bit, t ^ np.uint32((1 << q) - 1), t)
    X ^= t[:, None]
    return X


def key_words(d: int, bits: int) -> int:
    """W = ceil(d * bits / 64) 64-bit words per key."""
    return (d * bits + 63) // 64


def pack_key(X: np.ndarray, bits: int) -> np.ndarray:
    """Packs a transposed index into W uint64 words, most significant first.

    Key bit number l*d + i counted from the most significant end (l = 0 ..
    bits-1, i = 0 .. d-1) is bit (bits-1-l) of X[i]; word 0 holds key bits
    0..63 with bit 0 in its top position. A key whose length d*bits is not a
    multiple of 64 is padded with zeros at the low end of the last word."""
    n, d = X.shape
    W = key_words(d, bits)
    planes = [((X >> np.uint32(bits - 1 - l)) & np.uint32(1)).astype(np.uint8) for l in range(bits)]
    stream = np.concatenate(planes, axis=1)  # [n, bits*d], key bit order
    pad = W * 64 - stream.shape[1]
    if pad:
        stream = np.concatenate([stream, np.zeros((n, pad), np.uint8)], axis=1)
    by = np.ascontiguousarray(np.packbits(stream, axis=1))  # MSB-first within each byte
    return by.view(">u8").astype(np.uint64).reshape(n, W)


def hilbert_keys(codes: np.ndarray, pi: np.ndarray, r: np.ndarray, bits: int) -> np.ndarray:
    """Full W-word Hilbert key of every row after the tree's permutation and
    reflection."""
    return pack_key(skilling_transpose(permute_reflect(codes, pi, r, bits), bits), bits)


def hilbert_order(keys: np.ndarray) -> np.ndarray:
    """sigma: point indices ordered by (full key, index) ascending."""
    n, W = keys.shape
    cols = [np.arange(n)] + [keys[:, w] for w in range(W - 1, -1, -1)]
    return np.lexsort(cols).astype(np.int64)


def key_less_count(sorted_keys: np.ndarray, qkey: np.ndarray) -> int:
    """Number of rows of sorted_keys that are lexicographically smaller than
    qkey; on a sorted array this is the lower-bound position (Section 2:
    binary search in the Hilbert order)."""
    less = np.zeros(sorted_keys.shape[0], dtype=bool)
    eq = np.ones(sorted_keys.shape[0], dtype=bool)
    for w in range(sorted_keys.shape[1]):
        less |= eq & (sorted_keys[:, w] < qkey[w])
        eq &= sorted_keys[:, w] == qkey[w]
    return int(less.sum())


# --------------------------------------------------------------------------
# Forest
# --------------------------------------------------------------------------
class Forest:
    """The per-tree orders of Algorithm 2 (and the trees of Algorithm 1).

    Attributes: lo, scale (float32[d]), codes (uint16[n, d]), and per tree t
    pi[t], r[t], keys[t] (uint64[n, W], in point order), sigma[t] (int64[n])."""

    def __init__(self, x: np.ndarray, T: int, bits: int, seed: int):
        x = np.ascontiguousarray(x, dtype=np.float32)
        self.x = x
        self.n, self.d = x.shape
        self.T, self.bits, self.seed = T, bits, seed
        self.lo, self.scale = axis_range(x, bits)
        self.codes = quantize(x, self.lo, self.scale, bits)
        self.pi, self.r, self.keys, self.sigma = [], [], [], []
        for t in range(T):
            pi, r = tree_params(seed, t, self.d)
            k = hilbert_keys(self.codes, pi, r, bits)
            self.pi.append(pi)
            self.r.append(r)
            self.keys.append(k)
            self.sigma.append(hilbert_order(k))

    def position(self, t: int) -> np.ndarray:
        """p_t(i): position of point i in order t."""
        pos = np.empty(self.n, dtype=np.int64)
        pos[self.sigma[t]] = np.arange(self.n)
        return pos


def sq_dist_fp64(x: np.ndarray, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """d^2 = sum_j (x[rows, j] - x[cols, j])^2 in float64, elementwise over
    equally shaped index arrays (entries < 0 give +inf)."""
    xr = x.astype(np.float64)
    valid = (rows >= 0) & (cols >= 0)
    r = np.where(valid, rows, 0)
    c = np.where(valid, cols, 0)
    out = np.empty(r.shape, dtype=np.float64)
    flat_r, flat_c, flat_o = r.reshape(-1), c.reshape(-1), out.reshape(-1)
    step = max(1, (1 << 22) // max(1, x.shape[1]))
    for s in range(0, flat_r.size, step):
        diff = xr[flat_r[s:s + step]] - xr[flat_c[s:s + step]]
        flat_o[s:s + step] = np.einsum("ij,ij->i", diff, diff)
    out[~valid] = np.inf
    return out


def window_candidates(sigma: np.ndarray, w: int) -> np.ndarray:
    """Algorithm 2, per sort: for the point j at position i, the points at
    positions i + delta, 1 <= |delta| <= w, clipped at both ends (no wrap).
    Returns int64[n, 2w] indexed by point j, -1 where out of range."""
    n = sigma.shape[0]
    pos = np.arange(n)
    cand = np.full((n, 2 * w), -1, dtype=np.int64)
    col = 0
    for delta in list(range(-w, 0)) + list(range(1, w + 1)):
        p = pos + delta
        ok = (p >= 0) & (p < n)
        cand[sigma[ok], col] = sigma[p[ok]]
        col += 1
    return cand


def topk_from_candidates(x: np.ndarray, owners: np.ndarray, cand: np.ndarray, k: int,
                         xq: np.ndarray | None = None):
    """Top-k of each row's candidate set by (float64 squared distance, index).

    cand: int64[m, c] with -1 for "none" and possibly repeated entries
    (deduplicated here: candidate sets are sets). owners: the point index of
    each row (excluded from its own set), or None for queries, whose vectors
    are xq. Returns (idx int64[m, k], dist float64[m, k]); missing slots are
    (-1, +inf)."""
    m, c = cand.shape
    cand = cand.copy()
    if owners is not None:
        cand[cand == owners[:, None]] = -1
    # deduplicate: sort each row, blank repeats
    cand.sort(axis=1)
    dup = np.zeros_like(cand, dtype=bool)
    dup[:, 1:] = cand[:, 1:] == cand[:, :-1]
    cand[dup] = -1
    if xq is None:
        dist = sq_dist_fp64(x, np.broadcast_to(owners[:, None], cand.shape), cand)
    else:
        dist = np.empty(cand.shape, dtype=np.float64)
        xd = x.astype(np.float64)
        qd = xq.astype(np.float64)
        for i in range(m):
            ok = cand[i] >= 0
            diff = xd[cand[i, ok]] - qd[i][None, :]
            dist[i, ok] = np.einsum("ij,ij->i", diff, diff)
            dist[i, ~ok] = np.inf
    key_idx = np.where(cand >= 0, cand, np.iinfo(np.int64).max)
    order = np.lexsort((key_idx, dist), axis=1)[:, :k]
    idx = np.take_along_axis(cand, order, axis=1)
    dd = np.take_along_axis(dist, order, axis=1)
    if idx.shape[1] < k:
        padn = k - idx.shape[1]
        idx = np.concatenate([idx, np.full((m, padn), -1, np.int64)], axis=1)
        dd = np.concatenate([dd, np.full((m, padn), np.inf)], axis=1)
    dd = np.where(idx >= 0, dd, np.inf)
    return idx, dd


def candidate_sets(forest: Forest, w: int, trees=None) -> np.ndarray:
    """C(i) over the given trees (default all), as int64[n, T*2w] with
    repeats and -1 entries (a multiset view; topk_from_candidates dedups)."""
    trees = range(forest.T) if trees is None else trees
    return np.concatenate([window_candidates(forest.sigma[t], w) for t in trees], axis=1)


def knn_graph(forest: Forest, k: int, w: int):
    """Algorithm 2 without the sketch stage: C(i) = union over sorts of the
    2w window neighbours, then the k nearest by float64 squared distance with
    ties by index. Returns (idx int64[n, k], dist float64[n, k])."""
    cand = candidate_sets(forest, w)
    out_i = np.empty((forest.n, k), np.int64)
    out_d = np.empty((forest.n, k), np.float64)
    owners = np.arange(forest.n)
    step = 4096
    for s in range(0, forest.n, step):
        i, dd = topk_from_candidates(forest.x, owners[s:s + step], cand[s:s + step], k)
        out_i[s:s + step], out_d[s:s + step] = i, dd
    return out_i, out_d


# --------------------------------------------------------------------------
# Search (Algorithm 1 first stage + final selection)
# --------------------------------------------------------------------------
def query_codes(forest: Forest, queries: np.ndarray) -> np.ndarray:
    """Queries quantized with the data's lo/scale, clamped to the code range."""
    return quantize(queries, forest.lo, forest.scale, forest.bits)


def locate(forest: Forest, t: int, qcodes: np.ndarray) -> np.ndarray:
    """Section 2: position of each query in order t = number of data points
    whose full key is smaller than the query's (lower bound)."""
    qk = hilbert_keys(qcodes, forest.pi[t], forest.r[t], forest.bits)
    sk = forest.keys[t][forest.sigma[t]]
    return np.array([key_less_count(sk, qk[j]) for j in range(qk.shape[0])], dtype=np.int64)


def search(forest: Forest, queries: np.ndarray, k: int, w: int):
    """Algorithm 1 without the sketch stage and master-order expansion: per
    tree, the candidates are the points at positions [p - w, p + w) around the
    query's lower-bound position p (clipped); the result is the k nearest of
    their union by float64 squared distance, ties by index."""
    queries = np.ascontiguousarray(queries, dtype=np.float32)
    cand = search_candidates(forest, queries, w)
    return topk_from_candidates(forest.x, None, cand, k, xq=queries)


def search_candidates(forest: Forest, queries: np.ndarray, w: int) -> np.ndarray:
    """The first stage of Algorithm 1: per tree, the points at positions
    [p - w, p + w) around each query's lower-bound position p (clipped), as an
    int64 [nq][T * 2w] array with -1 for "none" (repeats across trees kept)."""
    queries = np.ascontiguousarray(queries, dtype=np.float32)
    qc = query_codes(forest, queries)
    nq = queries.shape[0]
    cols = []
    for t in range(forest.T):
        p = locate(forest, t, qc)
        c = np.full((nq, 2 * w), -1, dtype=np.int64)
        for j, off in enumerate(range(-w, w)):
            pp = p + off
            ok = (pp >= 0) & (pp < forest.n)
            c[ok, j] = forest.sigma[t][pp[ok]]
        cols.append(c)
    return np.concatenate(cols, axis=1)


# --------------------------------------------------------------------------
# Exact ground truth and recall
# --------------------------------------------------------------------------
def brute_force_knn(x: np.ndarray, k: int, rows: np.ndarray | None = None,
                    queries: np.ndarray | None = None):
    """Exact k nearest by (float64 squared distance, index).

    For data rows (``rows`` = point indices, default all) the point itself is
    excluded; for ``queries`` nothing is. A float64 inner-product screen keeps
    the k + 32 smallest per row (its error, about 1e-15 on unit-scale data, is
    far below the margin), which are then re-scored with exact float64
    coordinate differences and ordered by (distance, index)."""
    xd = x.astype(np.float64)
    nrm = np.einsum("ij,ij->i", xd, xd)
    if queries is not None:
        qd = queries.astype(np.float64)
        owners = None
    else:
        rows = np.arange(x.shape[0]) if rows is None else np.asarray(rows)
        qd = xd[rows]
        owners = rows
    m = qd.shape[0]
    keep = min(x.shape[0], k + 32)
    out_i = np.empty((m, k), np.int64)
    out_d = np.empty((m, k), np.float64)
    step = 256
    for s in range(0, m, step):
        q = qd[s:s + step]
        g = nrm[None, :] + np.einsum("ij,ij->i", q, q)[:, None] - 2.0 * (q @ xd.T)
        if owners is not None:
            g[np.arange(q.shape[0]), owners[s:s + step]] = np.inf
        part = np.argpartition(g, keep - 1, axis=1)[:, :keep]
        for r in range(q.shape[0]):
            c = part[r]
            if owners is not None:
                c = c[c != owners[s + r]]
            diff = xd[c] - q[r][None, :]
            dd = np.einsum("ij,ij->i", diff, diff)
            o = np.lexsort((c, dd))[:k]
            kk = len(o)
            out_i[s + r, :kk] = c[o]
            out_d[s + r, :kk] = dd[o]
            out_i[s + r, kk:] = -1
            out_d[s + r, kk:] = np.inf
    return out_i, out_d


def recall(found: np.ndarray, exact: np.ndarray) -> float:
    """mean over rows of |found ∩ exact| / k (entries < 0 ignored)."""
    k = exact.shape[1]
    hits = 0
    for a, b in zip(found, exact):
        hits += len(set(a[a >= 0].tolist()) & set(b[b >= 0].tolist()))
    return hits / (k * found.shape[0])
