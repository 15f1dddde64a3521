"""Comparison helpers for the CUDA-vs-oracle parity tests.

The CUDA path computes distances in float32 with exact coordinate differences;
the oracle in float64. Selections can differ only where two candidates'
float64 distances lie within the float32 error of each other, so the checks
compare what is unique (distances per rank, list validity, candidate
membership) and allow swaps only between such near-ties.
"""
import numpy as np

import oracle as O

# Relative bound for float32 squared distances against float64 (the target
# tolerance of the library's float path).
RTOL = 1e-5


def fp64_dist(x, rows, cols):
    return O.sq_dist_fp64(x, rows, cols)


def check_lists(x, gi, gd, oi, od, owners=None, queries=None, cand=None, rtol=RTOL, min_equal=0.98):
    """gi/gd: CUDA lists (int32, float32); oi/od: oracle lists (int64, float64).

    Checks: (1) each CUDA distance is within rtol of the float64 distance of
    its pair; (2) lists ascend by (distance, index), hold no repeats, never the
    owner itself, and unfilled slots (-1, inf) only at the tail; (3) rank by
    rank, the float64 distances of the CUDA picks equal the oracle's top-k
    distances within rtol (so any difference is a swap of near-ties);
    (4) every CUDA pick is in the oracle's candidate set when given; (5) most
    rows are identical."""
    gi = np.asarray(gi).astype(np.int64)
    gd = np.asarray(gd).astype(np.float64)
    m, k = gi.shape
    valid = gi >= 0
    assert np.array_equal(valid, oi >= 0), "filled-slot pattern differs from the oracle"
    if queries is None:
        true = fp64_dist(x, np.broadcast_to(owners[:, None], gi.shape), np.where(valid, gi, -1))
    else:
        true = np.full(gi.shape, np.inf)
        xd = x.astype(np.float64)
        qd = queries.astype(np.float64)
        for r in range(m):
            c = gi[r][valid[r]]
            diff = xd[c] - qd[r][None, :]
            true[r, valid[r]] = np.einsum("ij,ij->i", diff, diff)
    err = np.abs(gd[valid] - true[valid])
    assert np.all(err <= rtol * true[valid] + 1e-30), f"max rel err {np.max(err / np.maximum(true[valid], 1e-30))}"
    assert np.all(np.isinf(gd[~valid])), "unfilled slots must hold +inf"
    # ordering and uniqueness
    for r in range(m):
        row = gi[r][valid[r]]
        assert len(set(row.tolist())) == len(row), f"repeat in row {r}"
        if owners is not None:
            assert owners[r] not in set(row.tolist()), f"self in row {r}"
        dd = gd[r][valid[r]]
        ok = (dd[1:] > dd[:-1]) | ((dd[1:] == dd[:-1]) & (row[1:] > row[:-1]))
        assert np.all(ok), f"row {r} not ascending by (dist, idx)"
        assert np.all(valid[r][: valid[r].sum()]), f"hole in row {r}"
    # rank-wise distances
    # valid slots form a prefix of each row (checked above); unfilled ones sort last
    ts = np.sort(np.where(valid, true, np.inf), axis=1)
    ov = np.where(valid, od, np.inf)
    both = valid
    assert np.all(np.abs(ts[both] - ov[both]) <= rtol * ov[both] + 1e-30), "picked distances differ from the oracle's top-k"
    if cand is not None:
        for r in range(m):
            cs = set(cand[r][cand[r] >= 0].tolist())
            assert set(gi[r][valid[r]].tolist()) <= cs, f"row {r} holds a non-candidate"
    eq = np.mean(np.all(gi == oi, axis=1))
    assert eq >= min_equal, f"only {eq:.4f} of rows identical"
    return eq


def check_tensor_lists(x, gi, gd, oi, owners, cand=None, rtol=RTOL, min_hit=0.995):
    """Checks of the tensor form (tensor-core distance estimates pick each
    point's best k + slack candidates, an exact float32 re-rank orders them).

    Every returned distance must be the exact distance of its pair within
    rtol; lists ascend by (distance, index), hold no repeats and never the
    owner; every pick is one of the owner's window candidates (when `cand` is
    given); the filled-slot pattern equals the oracle's; and at least
    `min_hit` of the oracle's top-k entries are found (the estimate may drop a
    true top-k candidate out of the k + slack kept, rarely)."""
    gi = np.asarray(gi).astype(np.int64)
    gd = np.asarray(gd).astype(np.float64)
    valid = gi >= 0
    assert np.array_equal(valid, oi >= 0), "filled-slot pattern differs from the oracle"
    true = fp64_dist(x, np.broadcast_to(owners[:, None], gi.shape), np.where(valid, gi, -1))
    err = np.abs(gd[valid] - true[valid])
    assert np.all(err <= rtol * true[valid] + 1e-30), f"max rel err {np.max(err / np.maximum(true[valid], 1e-30))}"
    assert np.all(np.isinf(gd[~valid])), "unfilled slots must hold +inf"
    for r in range(gi.shape[0]):
        row = gi[r][valid[r]]
        assert len(set(row.tolist())) == len(row), f"repeat in row {r}"
        assert owners[r] not in set(row.tolist()), f"self in row {r}"
        if cand is not None:
            assert set(row.tolist()) <= set(cand[r][cand[r] >= 0].tolist()), f"row {r} holds a non-candidate"
        dd = gd[r][valid[r]]
        assert np.all((dd[1:] > dd[:-1]) | ((dd[1:] == dd[:-1]) & (row[1:] > row[:-1]))), f"row {r} order"
    hits = sum(len(set(a[a >= 0].tolist()) & set(b[b >= 0].tolist())) for a, b in zip(gi, oi))
    hit = hits / max(1, int((oi >= 0).sum()))
    assert hit >= min_hit, f"found {hit:.5f} of the oracle's top-k"
    return hit
