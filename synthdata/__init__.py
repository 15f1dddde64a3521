"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module holds only input generation: no quantization, no Hilbert keys, no
distances. Both the CUDA path (through the tests and the bench) and the CPU
oracle draw their inputs from here, so neither has to import the other.

The paper measures on two real datasets that are not available here: GOOAQ
(3M x 384, Section 4) and PUBMED23 (23M x 384 with 10,000 queries, Section 3).
The generators below stand in for them with the same shapes:

* ``unit_gaussian``   -- i.i.d. N(0, 1) rows normalised to the unit sphere.
* ``gaussian_mixture`` -- a Zipf(1.1)-weighted mixture of anisotropic Gaussians
  (means N(0, I), per-axis std U(0.1, 0.5)), rows normalised to unit length.
* ``mixture_queries`` -- draws from the same mixture plus N(0, noise^2) per
  coordinate, renormalised.
* ``sketch_projection`` -- the projection matrix of the sign sketches: i.i.d.
  N(0, 1) entries, one row per sketch bit (the random numbers the sketch
  stage draws, passed to both sides as an input).
* ``batched_sets`` -- many independent point sets: sizes log-uniform in
  [lo, hi], dimensions drawn from a list, each set a 100-component mixture of
  its own (the batched workload).
* ``small_integer_points`` / ``small_integer_projection`` -- integer-valued
  rows (|v| <= 8) and projections (|v| <= 2): every inner product, squared
  distance and BF16 rounding of them is exact in float32, so float decisions
  (sketch signs, distance ties) come out the same on every side.

Every stream is keyed by (seed, stream id, block id) through numpy's Philox
counter-based bit generator, so a row's values do not depend on how many
threads produced them. Values are identical for identical numpy versions; no
stored expected value depends on them.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

__all__ = [
    "unit_gaussian",
    "gaussian_mixture",
    "mixture_params",
    "mixture_queries",
    "sketch_projection",
    "batched_sets",
    "small_integer_points",
    "small_integer_projection",
    "SEED_DATA",
    "SEED_QUERIES",
    "SEED_FOREST",
    "SEED_SAMPLE",
    "SEED_SKETCH",
]

SEED_DATA = 1
SEED_QUERIES = 2
SEED_FOREST = 3
SEED_SAMPLE = 4
SEED_SKETCH = 5

_BLOCK_ROWS = 65536

# stream ids, so that different quantities never share a Philox key
_S_NORMAL = 0
_S_MEANS = 1
_S_SIGMAS = 2
_S_ASSIGN = 3
_S_NOISE = 4
_S_PROJ = 5
_S_INT = 6
_S_SETS = 7


def _gen(seed: int, stream: int, block: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed), stream, block])))


def _threads() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def _blocked_rows(n: int, d: int, fill) -> np.ndarray:
    """Runs ``fill(out_block, block_id, row0)`` over row blocks in a thread pool."""
    out = np.empty((n, d), dtype=np.float32)
    nblk = (n + _BLOCK_ROWS - 1) // _BLOCK_ROWS

    def work(b):
        r0 = b * _BLOCK_ROWS
        r1 = min(n, r0 + _BLOCK_ROWS)
        fill(out[r0:r1], b, r0)

    if nblk <= 1:
        for b in range(nblk):
            work(b)
    else:
        with ThreadPoolExecutor(_threads()) as ex:
            list(ex.map(work, range(nblk)))
    return out


def _normalize_rows(a: np.ndarray) -> None:
    nrm = np.sqrt(np.einsum("ij,ij->i", a, a, dtype=np.float64)).astype(np.float32)
    nrm[nrm == 0] = 1.0
    a /= nrm[:, None]


def unit_gaussian(n: int, d: int, seed: int = SEED_DATA) -> np.ndarray:
    """n x d float32, rows i.i.d. N(0, I_d) scaled to unit length."""

    def fill(o, b, r0):
        _gen(seed, _S_NORMAL, b).standard_normal(out=o, dtype=np.float32)
        _normalize_rows(o)

    return _blocked_rows(n, d, fill)


def mixture_params(d: int, n_components: int = 1000, seed: int = SEED_DATA,
                   zipf: float = 1.1, sigma_lo: float = 0.1, sigma_hi: float = 0.5):
    """Means N(0, I) [c, d], per-axis std U(sigma_lo, sigma_hi) [c, d], weights
    proportional to rank^-zipf (rank = component index + 1), as float64 CDF."""
    mu = _gen(seed, _S_MEANS, 0).standard_normal((n_components, d), dtype=np.float32)
    sg = _gen(seed, _S_SIGMAS, 0).uniform(sigma_lo, sigma_hi, (n_components, d)).astype(np.float32)
    w = np.arange(1, n_components + 1, dtype=np.float64) ** (-zipf)
    cdf = np.cumsum(w / w.sum())
    cdf[-1] = 1.0
    return mu, sg, cdf


def _mixture_rows(n, d, params, seed, noise):
    mu, sg, cdf = params

    def fill(o, b, r0):
        u = _gen(seed, _S_ASSIGN, b).random(o.shape[0])
        comp = np.searchsorted(cdf, u, side="right").clip(0, len(cdf) - 1)
        _gen(seed, _S_NORMAL, b).standard_normal(out=o, dtype=np.float32)
        o *= sg[comp]
        o += mu[comp]
        _normalize_rows(o)
        if noise > 0:
            z = _gen(seed, _S_NOISE, b).standard_normal(o.shape, dtype=np.float32)
            o += np.float32(noise) * z
            _normalize_rows(o)

    return _blocked_rows(n, d, fill)


def gaussian_mixture(n: int, d: int, n_components: int = 1000, seed: int = SEED_DATA) -> np.ndarray:
    """n x d float32 unit rows from the Zipf-weighted anisotropic mixture."""
    return _mixture_rows(n, d, mixture_params(d, n_components, seed), seed, 0.0)


def mixture_queries(nq: int, d: int, n_components: int = 1000, data_seed: int = SEED_DATA,
                    seed: int = SEED_QUERIES, noise: float = 0.05) -> np.ndarray:
    """nq x d float32 queries: the data mixture (parameters from ``data_seed``)
    plus N(0, noise^2) per coordinate, renormalised."""
    return _mixture_rows(nq, d, mixture_params(d, n_components, data_seed), seed, noise)


def sketch_projection(bits: int, d: int, seed: int = SEED_SKETCH) -> np.ndarray:
    """float32 [bits][d], i.i.d. N(0, 1)."""
    return _gen(seed, _S_PROJ, 0).standard_normal((bits, d), dtype=np.float32)


def small_integer_points(n: int, d: int, seed: int = SEED_DATA) -> np.ndarray:
    """float32 [n][d] with integer values in [-8, 8]; rows are drawn around
    n / 64 + 1 integer centres (each row: a centre plus an integer offset in
    [-2, 2] per axis, clipped), so that near neighbours exist."""
    g = _gen(seed, _S_INT, 0)
    nc = n // 64 + 1
    centres = g.integers(-6, 7, size=(nc, d))
    pick = g.integers(0, nc, size=n)
    off = g.integers(-2, 3, size=(n, d))
    return np.clip(centres[pick] + off, -8, 8).astype(np.float32)


def small_integer_projection(bits: int, d: int, seed: int = SEED_SKETCH) -> np.ndarray:
    """float32 [bits][d] with integer values in [-2, 2]."""
    return _gen(seed, _S_INT, 1).integers(-2, 3, size=(bits, d)).astype(np.float32)


def batched_sets(nsets: int = 64, lo: int = 1000, hi: int = 200_000, dims=(64, 128, 384, 768),
                 n_components: int = 100, seed: int = SEED_DATA):
    """[(points float32 [n_s][d_s])] for nsets independent sets: n_s =
    round(exp(U(ln lo, ln hi))), d_s uniform over dims, each set drawn from a
    gaussian_mixture of its own (seed derived from the set index)."""
    g = _gen(seed, _S_SETS, 0)
    sizes = np.rint(np.exp(g.uniform(np.log(lo), np.log(hi), size=nsets))).astype(np.int64)
    ds = g.choice(np.asarray(dims, dtype=np.int64), size=nsets)
    return [gaussian_mixture(int(sizes[i]), int(ds[i]), n_components=n_components, seed=seed * 1000 + 17 + i)
            for i in range(nsets)]
