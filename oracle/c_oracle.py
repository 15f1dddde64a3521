"""ctypes access to the C++ oracle (oracle/hf_oracle.cpp) -- TEST INFRASTRUCTURE ONLY.

The C++ oracle restates, in scalar loops, what the numpy oracle
(oracle/hilbert_forest.py) computes: tree parameters, quantization, Skilling
keys, Hilbert orders, the window kNN graph of Algorithm 2, the search of
Algorithm 1 and exact kNN. The tests pin it with the same curve pins as the
numpy oracle and compare the two element by element; neither shares code with
the other or with the CUDA library. Only tests/, the smoke check and the
bench's CPU arms may use it.

build() compiles it with the host C++ compiler into oracle/_build/libhfo.so
(git-ignored), without fused multiply-adds; it is called on first use.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hf_oracle.cpp")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libhfo.so")
FLAGS = ["-O2", "-std=c++17", "-shared", "-fPIC", "-ffp-contract=off", "-Wall", "-Wextra"]

_lib = None


def build(force: bool = False) -> str:
    """Compiles the C++ oracle if the library is missing or older than its source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        raise RuntimeError("no C++ compiler found for the C++ oracle")
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + f".{os.getpid()}.tmp"
    r = subprocess.run([cxx, *FLAGS, "-o", tmp, SRC], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"C++ oracle build failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
        L.hfo_tree_params.argtypes = [u64, i32, i32, vp, vp]
        L.hfo_tree_params.restype = None
        L.hfo_transpose.argtypes = [vp, i64, i32, i32, vp]
        L.hfo_transpose.restype = None
        L.hfo_pack_key.argtypes = [vp, i64, i32, i32, vp]
        L.hfo_pack_key.restype = None
        L.hfo_forest.argtypes = [vp, i64, i32, i32, i32, u64, vp, vp, vp, vp, vp]
        L.hfo_forest.restype = i32
        L.hfo_knn_graph.argtypes = [vp, i64, i32, vp, i32, i32, i32, vp, vp]
        L.hfo_knn_graph.restype = i32
        L.hfo_search.argtypes = [vp, i64, i32, i32, i32, u64, vp, vp, vp, vp, vp, i64, i32, i32, vp, vp]
        L.hfo_search.restype = i32
        L.hfo_brute_force.argtypes = [vp, i64, i32, vp, vp, i64, i32, vp, vp]
        L.hfo_brute_force.restype = i32
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data


def tree_params(seed: int, tree: int, d: int):
    pi = np.empty(d, np.int64)
    r = np.empty(d, np.uint8)
    lib().hfo_tree_params(seed & ((1 << 64) - 1), tree, d, _p(pi), _p(r))
    return pi, r


def skilling_transpose(coords: np.ndarray, bits: int) -> np.ndarray:
    c = np.ascontiguousarray(coords, dtype=np.uint32)
    n, d = c.shape
    X = np.empty_like(c)
    lib().hfo_transpose(_p(c), n, d, bits, _p(X))
    return X


def pack_key(X: np.ndarray, bits: int) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.uint32)
    n, d = X.shape
    keys = np.empty((n, (d * bits + 63) // 64), np.uint64)
    lib().hfo_pack_key(_p(X), n, d, bits, _p(keys))
    return keys


class Forest:
    """Same attributes as the numpy oracle's Forest: lo, scale, codes, and per
    tree keys[t] (uint64 [n][W], point order) and sigma[t] (int64 [n])."""

    def __init__(self, x: np.ndarray, T: int, bits: int, seed: int):
        self.x = np.ascontiguousarray(x, dtype=np.float32)
        self.n, self.d = self.x.shape
        self.T, self.bits, self.seed = T, bits, seed
        W = (self.d * bits + 63) // 64
        self.lo = np.empty(self.d, np.float32)
        self.scale = np.empty(self.d, np.float32)
        self.codes = np.empty((self.n, self.d), np.uint16)
        keys = np.empty((T, self.n, W), np.uint64)
        sigma = np.empty((T, self.n), np.int64)
        rc = lib().hfo_forest(_p(self.x), self.n, self.d, T, bits, seed & ((1 << 64) - 1), _p(self.lo),
                              _p(self.scale), _p(self.codes), _p(keys), _p(sigma))
        if rc != 0:
            raise ValueError("C++ oracle: non-finite input or bad sizes")
        self._keys, self._sigma = keys, sigma
        self.keys = [keys[t] for t in range(T)]
        self.sigma = [sigma[t] for t in range(T)]


def knn_graph(forest: Forest, k: int, w: int):
    out_i = np.empty((forest.n, k), np.int64)
    out_d = np.empty((forest.n, k), np.float64)
    rc = lib().hfo_knn_graph(_p(forest.x), forest.n, forest.d, _p(forest._sigma), forest.T, w, k, _p(out_i),
                             _p(out_d))
    if rc != 0:
        raise ValueError("C++ oracle: bad arguments")
    return out_i, out_d


def search(forest: Forest, queries: np.ndarray, k: int, w: int):
    q = np.ascontiguousarray(queries, dtype=np.float32)
    nq = q.shape[0]
    out_i = np.empty((nq, k), np.int64)
    out_d = np.empty((nq, k), np.float64)
    rc = lib().hfo_search(_p(forest.x), forest.n, forest.d, forest.T, forest.bits,
                          forest.seed & ((1 << 64) - 1), _p(forest.lo), _p(forest.scale), _p(forest._keys),
                          _p(forest._sigma), _p(q), nq, w, k, _p(out_i), _p(out_d))
    if rc != 0:
        raise ValueError("C++ oracle: non-finite query or bad arguments")
    return out_i, out_d


def brute_force_knn(x: np.ndarray, k: int, rows: np.ndarray | None = None, queries: np.ndarray | None = None):
    x = np.ascontiguousarray(x, dtype=np.float32)
    n, d = x.shape
    if queries is not None:
        q = np.ascontiguousarray(queries, dtype=np.float32)
        m, rp, qp = q.shape[0], None, _p(q)
    else:
        rows = np.arange(n, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
        m, rp, qp = rows.shape[0], _p(rows), None
    out_i = np.empty((m, k), np.int64)
    out_d = np.empty((m, k), np.float64)
    rc = lib().hfo_brute_force(_p(x), n, d, rp, qp, m, k, _p(out_i), _p(out_d))
    if rc != 0:
        raise ValueError("C++ oracle: bad arguments")
    return out_i, out_d


__all__ = ["build", "tree_params", "skilling_transpose", "pack_key", "Forest", "knn_graph", "search", "brute_force_knn"]
