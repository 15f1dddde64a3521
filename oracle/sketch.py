"""Plain CPU oracle of the second-stage sketch filter -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the bench's CPU arms may import it;
the CUDA library never calls it. It shares no code with the library.

The paper filters the forest's candidates by the Hamming distance of binary
sketches (384 bits per vector, Section 3 index structure) before the final
selection by vector distance: Algorithm 2 keeps, per point, the top k2 of its
candidate set C1 by Hamming distance, then the top k of those by vector
distance. The paper does not say how its sketches are made; this oracle (and
the library) uses sign random projection: bit j of point i is
(<x_i, r_j> > 0) for the rows r_j of a projection matrix R that the caller
supplies. Both x and R enter as their BF16 roundings (the library stores BF16
operands for the tensor cores); the inner products here are exact float64
sums of those values.

* sketch_dots -- the float64 inner products <bf16(x_i), bf16(r_j)>;
* sketches    -- their signs packed into uint64 words: bit j of point i is bit
                 j % 64 of word j // 64;
* hamming     -- popcount of the XOR of two packed sketches;
* knn_graph_sketch -- Algorithm 2 with the second stage: the candidate set of
                 each point is the union over sorts of its 2w window
                 neighbours (a set: repeats and the point itself removed);
                 the k2 of smallest (Hamming distance, index) survive; the
                 result is their top k by (float64 squared distance, index);
* search_sketch -- Algorithm 1 with both filters: the forest's window
                 candidates of each query, the top k2 by Hamming distance to
                 the query's sketch, each expanded by the h points on either
                 side of it in the master order (order 0 of the forest), then
                 the top k by float64 distance.
"""
from __future__ import annotations

import numpy as np

from .budget import bf16
from .hilbert_forest import Forest, candidate_sets, search_candidates, topk_from_candidates

# popcount of every byte value, counted bit by bit
POP8 = np.array([sum((v >> b) & 1 for b in range(8)) for v in range(256)], dtype=np.int64)


def sketch_dots(x: np.ndarray, R: np.ndarray) -> np.ndarray:
    """float64 [n][bits]: <bf16(x_i), bf16(r_j)>, each product and sum exact
    to float64 rounding."""
    return bf16(x) @ bf16(R).T


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """bool [n][B] (B a multiple of 64) -> uint64 [n][B/64]; bit j of a row is
    bit j % 64 of word j // 64."""
    n, B = bits.shape
    assert B % 64 == 0, "sketch length must be a multiple of 64"
    words = np.zeros((n, B // 64), dtype=np.uint64)
    for j in range(B):
        words[:, j // 64] |= bits[:, j].astype(np.uint64) << np.uint64(j % 64)
    return words


def sketches(x: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Packed sign sketches: bit j of point i = (<bf16 x_i, bf16 r_j> > 0)."""
    return pack_bits(sketch_dots(x, R) > 0.0)


def hamming(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Number of differing bits between packed sketches a [..][W] and b [..][W]
    (broadcasting over leading axes)."""
    xor = np.bitwise_xor(np.asarray(a, dtype=np.uint64), np.asarray(b, dtype=np.uint64))
    return POP8[np.ascontiguousarray(xor).view(np.uint8)].sum(axis=-1)


def top_k2_by_hamming(sk: np.ndarray, owners, cand: np.ndarray, k2: int, qsk: np.ndarray | None = None) -> np.ndarray:
    """Per row: the k2 candidates of smallest (Hamming distance to the row's
    sketch, index), as int64 [m][k2] with -1 padding. The row's sketch is the
    owner's (sk[owners]) or, for queries (owners None), qsk. cand holds -1 for
    "none" and may repeat entries and contain the owner; both are removed
    first."""
    cand = np.asarray(cand, dtype=np.int64).copy()
    if owners is not None:
        cand[cand == owners[:, None]] = -1
        qsk = sk[owners]
    cand.sort(axis=1)
    dup = np.zeros_like(cand, dtype=bool)
    dup[:, 1:] = cand[:, 1:] == cand[:, :-1]
    cand[dup] = -1
    ok = cand >= 0
    ham = np.where(ok, hamming(qsk[:, None, :], sk[np.where(ok, cand, 0)]), np.iinfo(np.int64).max)
    key_idx = np.where(ok, cand, np.iinfo(np.int64).max)
    order = np.lexsort((key_idx, ham), axis=1)[:, :k2]
    out = np.take_along_axis(cand, order, axis=1)
    if out.shape[1] < k2:
        out = np.concatenate([out, np.full((out.shape[0], k2 - out.shape[1]), -1, np.int64)], axis=1)
    return out


def knn_graph_sketch(forest: Forest, k: int, w: int, sk: np.ndarray, k2: int):
    """Algorithm 2 with its second stage: window candidates of all sorts, the
    top k2 by Hamming distance, then the top k by float64 distance (ties by
    index). Returns (idx int64 [n][k], dist float64 [n][k]); (-1, +inf) pads."""
    cand = candidate_sets(forest, w)
    owners = np.arange(forest.n)
    out_i = np.empty((forest.n, k), np.int64)
    out_d = np.empty((forest.n, k), np.float64)
    step = 4096
    for s in range(0, forest.n, step):
        c2 = top_k2_by_hamming(sk, owners[s:s + step], cand[s:s + step], k2)
        i, dd = topk_from_candidates(forest.x, owners[s:s + step], c2, k)
        out_i[s:s + step], out_d[s:s + step] = i, dd
    return out_i, out_d


def master_expand(forest: Forest, c2: np.ndarray, h: int) -> np.ndarray:
    """Algorithm 1's expansion: every candidate c of c2 [m][k2] (-1 = none)
    brings the points at positions pos0(c) - h .. pos0(c) + h of the master
    order (order 0; c itself at offset 0), clipped to the order, as int64
    [m][k2 (2h + 1)] with -1 padding (repeats kept)."""
    pos0 = forest.position(0)
    sig0 = forest.sigma[0]
    m, k2 = c2.shape
    out = np.full((m, k2 * (2 * h + 1)), -1, dtype=np.int64)
    col = 0
    for u in range(k2):
        c = c2[:, u]
        for o in range(-h, h + 1):
            p = np.where(c >= 0, pos0[np.where(c >= 0, c, 0)] + o, -1)
            ok = (c >= 0) & (p >= 0) & (p < forest.n)
            out[ok, col] = sig0[p[ok]]
            col += 1
    return out


def search_sketch(forest: Forest, queries: np.ndarray, k: int, w: int, sk: np.ndarray, qsk: np.ndarray,
                  k2: int, h: int):
    """Algorithm 1 with both filters: the forest's window candidates of every
    tree (search_candidates), the top k2 by Hamming distance between the
    query's sketch qsk and the candidates' sketches sk (ties by index), each
    expanded by h master-order neighbours on either side, then the top k by
    float64 distance to the float32 query (ties by index). Returns (idx int64
    [nq][k], dist float64 [nq][k]); (-1, +inf) pads."""
    queries = np.ascontiguousarray(queries, dtype=np.float32)
    cand = search_candidates(forest, queries, w)
    c2 = top_k2_by_hamming(sk, None, cand, k2, qsk=qsk)
    ex = master_expand(forest, c2, h)
    return topk_from_candidates(forest.x, None, ex, k, xq=queries)


__all__ = ["POP8", "sketch_dots", "pack_bits", "sketches", "hamming", "top_k2_by_hamming", "knn_graph_sketch",
           "master_expand", "search_sketch"]
