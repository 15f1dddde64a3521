"""Python binding of libhf.so, the GB300 Hilbert-forest library.

Argument marshalling only: every step of the path runs in the library's CUDA
kernels. Arrays may be torch tensors (CUDA or CPU) or numpy arrays; CUDA
tensors are passed by device pointer together with torch's current stream,
host arrays by host pointer (the library copies them). The library must have
been built (``__graft_entry__.build()``); importing this package without it
raises, there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhf.so")

HF_OK = 0
HF_EINVAL = -1
HF_ENOMEM = -2
HF_ECUDA = -3
HF_ENONFINITE = -4
HF_ETIMEOUT = -5
HF_ESTATE = -6
HF_ENOTIMPL = -7

SYMBOLS = [
    "hf_build", "hf_build_opts", "hf_knn_graph", "hf_search", "hf_free", "hf_status_string",
    "hf_set_option", "hf_get_timings", "hf_info", "hf_tree_params", "hf_debug_codes",
    "hf_debug_keys", "hf_debug_prefix", "hf_debug_order", "hf_debug_locate", "hf_debug_keys_from_codes",
    "hf_launch_count", "hf_search_static", "hf_trim_pool",
    "hf_budget_labels", "hf_knn_graph_budget", "hf_mlp_create", "hf_mlp_free", "hf_mlp_param_count",
    "hf_mlp_get_params", "hf_mlp_set_params", "hf_mlp_predict", "hf_mlp_grads", "hf_mlp_train",
    "hf_set_sketch", "hf_debug_sketch",
    "hf_build_segmented", "hf_graph_plan", "hf_knn_graph_enqueue", "hf_status", "hf_capture_begin",
    "hf_capture_end", "hf_graph_launch", "hf_graph_destroy", "hf_exact_knn_rows", "hf_autotune",
]

_lib = None


class HFError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


def lib() -> ctypes.CDLL:
    """Loads libhf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhf.so not built at {LIB_PATH}; run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "hf_build": [vp, i64, i32, i32, i32, u64, vp, pp],
        "hf_build_opts": [vp, i64, i32, i32, i32, u64, ctypes.c_char_p, vp, pp],
        "hf_knn_graph": [vp, i32, i32, vp, vp, vp],
        "hf_search": [vp, vp, i64, i32, i32, vp, vp, vp],
        "hf_free": [vp],
        "hf_status_string": [ctypes.c_int],
        "hf_set_option": [vp, ctypes.c_char_p, i64],
        "hf_get_timings": [vp, vp, i32],
        "hf_info": [vp, vp, i32],
        "hf_tree_params": [u64, i32, i32, vp, vp],
        "hf_debug_codes": [vp, vp, vp],
        "hf_debug_keys": [vp, i32, vp, vp],
        "hf_debug_prefix": [vp, i32, vp, vp],
        "hf_debug_order": [vp, i32, vp, vp],
        "hf_debug_locate": [vp, i32, vp, i64, vp, vp],
        "hf_debug_keys_from_codes": [vp, i64, i32, i32, vp, vp],
        "hf_launch_count": [],
        "hf_search_static": [vp, vp, i64, i32, i32, vp, vp, vp],
        "hf_trim_pool": [],
        "hf_budget_labels": [vp, vp, i32, vp, i32, vp, i32, i32, vp, vp, vp],
        "hf_knn_graph_budget": [vp, i32, vp, vp, i32, i32, vp, vp, vp],
        "hf_mlp_create": [i32, u64, pp],
        "hf_mlp_free": [vp],
        "hf_mlp_param_count": [vp, vp],
        "hf_mlp_get_params": [vp, vp],
        "hf_mlp_set_params": [vp, vp],
        "hf_mlp_predict": [vp, vp, i64, vp, vp],
        "hf_mlp_grads": [vp, vp, vp, i32, vp, vp, vp],
        "hf_mlp_train": [vp, vp, vp, i64, i32, i32, ctypes.c_float, vp, vp],
        "hf_set_sketch": [vp, vp, i32, vp],
        "hf_debug_sketch": [vp, vp, vp],
        "hf_build_segmented": [vp, vp, i32, i32, i32, i32, u64, ctypes.c_char_p, vp, pp],
        "hf_graph_plan": [vp, i32, i32, i32, vp],
        "hf_knn_graph_enqueue": [vp, vp, vp, vp],
        "hf_status": [vp, vp],
        "hf_capture_begin": [vp],
        "hf_capture_end": [vp, pp],
        "hf_graph_launch": [vp, vp],
        "hf_graph_destroy": [vp],
        "hf_exact_knn_rows": [vp, vp, i32, i32, vp, vp, vp],
        "hf_autotune": [vp, i32, ctypes.c_double, i32, i32, i32, vp, vp, vp, vp, vp, vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = {"hf_status_string": ctypes.c_char_p, "hf_launch_count": ctypes.c_uint64}.get(name, ctypes.c_int)
    _lib = L
    return L


def status_string(status: int) -> str:
    return lib().hf_status_string(status).decode()


def _check(rc: int, what: str):
    if rc != HF_OK:
        raise HFError(rc, what)


def _ptr(a):
    """(pointer, keepalive) of a contiguous torch tensor or numpy array."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, a
    import torch  # noqa: F401  (torch tensors only)
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return a.data_ptr(), a


def _stream(*arrays):
    """torch's current stream when any argument is a CUDA tensor, else NULL."""
    for a in arrays:
        if a is not None and not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False):
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return None


def launch_count() -> int:
    """Kernels launched by libhf.so in this process so far."""
    return int(lib().hf_launch_count())


def trim_pool():
    """Returns the current device's cached library memory to the driver."""
    _check(lib().hf_trim_pool(), "hf_trim_pool")


def tree_params(seed: int, tree: int, d: int):
    """Host-only: (pi int32[d], r uint8[d]) of a tree."""
    pi = np.empty(d, np.int32)
    r = np.empty(d, np.uint8)
    _check(lib().hf_tree_params(seed, tree, d, pi.ctypes.data, r.ctypes.data), "hf_tree_params")
    return pi, r


def keys_from_codes(codes, bits: int, out=None):
    """Full keys (n x W uint64) of raw codes (n x d uint8), identity order."""
    n, d = codes.shape
    W = (d * bits + 63) // 64
    if out is None:
        out = _empty_like_input(codes, (n, W), "uint64")
    cp, _k1 = _ptr(codes)
    op, _k2 = _ptr(out)
    _check(lib().hf_debug_keys_from_codes(cp, n, d, bits, op, _stream(codes, out)), "hf_debug_keys_from_codes")
    return out


def _empty_like_input(ref, shape, dtype):
    if isinstance(ref, np.ndarray):
        return np.empty(shape, dtype=dtype)
    import torch
    tdt = {"uint64": torch.int64, "int32": torch.int32, "float32": torch.float32,
           "uint32": torch.int32, "int64": torch.int64, "uint8": torch.uint8}[dtype]
    return torch.empty(shape, dtype=tdt, device=ref.device)


class Forest:
    """A built Hilbert forest (hf_build). Holds the library handle."""

    def __init__(self, points, T: int, bits: int = 8, seed: int = 3, options: str | None = None, offsets=None):
        n, d = points.shape
        self.n, self.d, self.T, self.bits = int(n), int(d), int(T), int(bits)
        self._points = points  # the library borrows device memory: keep it alive
        p, _ = _ptr(points)
        h = ctypes.c_void_p()
        st = _stream(points)
        self.offsets = None
        if offsets is not None:
            off = np.ascontiguousarray(offsets, dtype=np.int64)
            if off.ndim != 1 or off[0] != 0 or off[-1] != n:
                raise ValueError("offsets must start at 0 and end at the row count")
            self.offsets = off
            rc = lib().hf_build_segmented(p, off.ctypes.data, len(off) - 1, d, T, bits, seed,
                                          options.encode() if options else None, st, ctypes.byref(h))
        elif options is None:
            rc = lib().hf_build(p, n, d, T, bits, seed, st, ctypes.byref(h))
        else:
            rc = lib().hf_build_opts(p, n, d, T, bits, seed, options.encode(), st, ctypes.byref(h))
        _check(rc, "hf_build")
        self._h = h
        info = np.zeros(8, np.int64)
        lib().hf_info(self._h, info.ctypes.data, 8)
        self.W, self.K = int(info[4]), int(info[5])
        self.K2, self.L = int(info[6]), int(info[7])

    def close(self):
        if getattr(self, "_h", None):
            lib().hf_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def knn_graph(self, k: int, w: int, out_idx=None, out_dist=None):
        """(idx int32[n, k], dist float32[n, k]); outputs default to the
        points' kind (CUDA tensors for CUDA points, numpy otherwise)."""
        if out_idx is None:
            out_idx = _empty_like_input(self._points, (self.n, k), "int32")
        if out_dist is None:
            out_dist = _empty_like_input(self._points, (self.n, k), "float32")
        ip, _a = _ptr(out_idx)
        dp, _b = _ptr(out_dist)
        _check(lib().hf_knn_graph(self._h, k, w, ip, dp, _stream(out_idx, out_dist, self._points)),
               "hf_knn_graph")
        return out_idx, out_dist

    def search(self, queries, k: int, w: int, out_idx=None, out_dist=None):
        nq = queries.shape[0]
        if out_idx is None:
            out_idx = _empty_like_input(queries, (nq, k), "int32")
        if out_dist is None:
            out_dist = _empty_like_input(queries, (nq, k), "float32")
        qp, _q = _ptr(queries)
        ip, _a = _ptr(out_idx)
        dp, _b = _ptr(out_dist)
        _check(lib().hf_search(self._h, qp, nq, k, w, ip, dp, _stream(queries, out_idx, out_dist)),
               "hf_search")
        return out_idx, out_dist

    def search_static(self, queries, k: int, w: int, out_idx=None, out_dist=None):
        """hf_search_static: same results as search(), no device allocation;
        queries and outputs must be CUDA tensors."""
        nq = queries.shape[0]
        if out_idx is None:
            out_idx = _empty_like_input(queries, (nq, k), "int32")
        if out_dist is None:
            out_dist = _empty_like_input(queries, (nq, k), "float32")
        qp, _q = _ptr(queries)
        ip, _a = _ptr(out_idx)
        dp, _b = _ptr(out_dist)
        _check(lib().hf_search_static(self._h, qp, nq, k, w, ip, dp, _stream(queries, out_idx, out_dist)),
               "hf_search_static")
        return out_idx, out_dist

    def knn_graph_budget(self, k: int, w_pt, T_pt, out_idx=None, out_dist=None):
        """hf_knn_graph_budget: point i takes part in trees t < T_pt[i] with
        window w_pt[i] (CUDA int32 tensors of n entries); tensor forms only."""
        if out_idx is None:
            out_idx = _empty_like_input(self._points, (self.n, k), "int32")
        if out_dist is None:
            out_dist = _empty_like_input(self._points, (self.n, k), "float32")
        wmax, tmax = int(w_pt.max().item()), int(T_pt.max().item())
        wp, _w = _ptr(w_pt)
        tp, _t = _ptr(T_pt)
        ip, _a = _ptr(out_idx)
        dp, _b = _ptr(out_dist)
        _check(lib().hf_knn_graph_budget(self._h, k, wp, tp, max(1, wmax), max(1, tmax), ip, dp,
                                         _stream(out_idx, out_dist, w_pt)), "hf_knn_graph_budget")
        return out_idx, out_dist

    def budget_labels(self, knn, t_grid, w_grid, min_hits: int, out_targets=None, out_cell=None):
        """hf_budget_labels: (targets float32[n, 2] = (log2 w, log2 T), cell
        int32[n]) from the exact neighbours knn (CUDA int32 [n, k])."""
        import torch
        n, k = knn.shape
        if out_targets is None:
            out_targets = torch.empty((n, 2), dtype=torch.float32, device=knn.device)
        if out_cell is None:
            out_cell = torch.empty(n, dtype=torch.int32, device=knn.device)
        tg = np.ascontiguousarray(t_grid, dtype=np.int32)
        wg = np.ascontiguousarray(w_grid, dtype=np.int32)
        kp, _k = _ptr(knn)
        op, _o = _ptr(out_targets)
        cp, _c = _ptr(out_cell)
        _check(lib().hf_budget_labels(self._h, kp, k, tg.ctypes.data, len(tg), wg.ctypes.data, len(wg), min_hits,
                                      op, cp, _stream(knn)), "hf_budget_labels")
        return out_targets, out_cell

    # ---- enqueue-only graph, autotuner, exact rows
    def graph_plan(self, k: int, w: int, threads: int = 0, stream=None):
        _check(lib().hf_graph_plan(self._h, k, w, threads, stream), "hf_graph_plan")
        self.plan_k = int(k)

    def knn_graph_enqueue(self, out_idx, out_dist, stream=None):
        """Enqueues the planned graph into CUDA tensors (n x k); no sync."""
        ip, _a = _ptr(out_idx)
        dp, _b = _ptr(out_dist)
        _check(lib().hf_knn_graph_enqueue(self._h, ip, dp, stream if stream is not None else _stream(out_idx)),
               "hf_knn_graph_enqueue")

    def status(self, stream=None):
        _check(lib().hf_status(self._h, stream), "hf_status")

    def exact_knn_rows(self, rows, k: int):
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        oi = np.empty((rows.size, k), np.int32)
        od = np.empty((rows.size, k), np.float32)
        _check(lib().hf_exact_knn_rows(self._h, rows.ctypes.data, rows.size, k, oi.ctypes.data, od.ctypes.data,
                                       _stream(self._points)), "hf_exact_knn_rows")
        return oi, od

    def autotune(self, k: int, target_recall: float, sample: int = 512, w_max: int = 512, forms: int = 1):
        """hf_autotune over the forms in the mask (1 plain, 2 BF16 Gram, 4 FP8
        Gram); returns the chosen form, w, block size, sample recall and ms."""
        fm, w, nt = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        rec, ms = ctypes.c_double(), ctypes.c_float()
        _check(lib().hf_autotune(self._h, k, target_recall, sample, w_max, forms, ctypes.byref(fm), ctypes.byref(w),
                                 ctypes.byref(nt), ctypes.byref(rec), ctypes.byref(ms), _stream(self._points)),
               "hf_autotune")
        self.plan_k = int(k)
        return {"form": fm.value & 255, "list_slots": fm.value >> 8, "w": w.value, "threads": nt.value,
                "recall": rec.value, "ms": ms.value}

    def set_sketch(self, R):
        """hf_set_sketch: sketches of all points from the projection R
        (bits x d float32, CUDA tensor or numpy)."""
        if R.ndim != 2 or R.shape[1] != self.d or str(R.dtype).split(".")[-1] != "float32":
            raise ValueError("R must be float32 of shape (bits, d)")
        rp, _r = _ptr(R)
        _check(lib().hf_set_sketch(self._h, rp, R.shape[0], _stream(R)), "hf_set_sketch")
        self.sketch_bits = int(R.shape[0])

    def sketches(self):
        out = np.empty((self.n, self.sketch_bits // 64), np.uint64)
        _check(lib().hf_debug_sketch(self._h, out.ctypes.data, None), "hf_debug_sketch")
        return out

    def set_option(self, key: str, value: int):
        _check(lib().hf_set_option(self._h, key.encode(), value), "hf_set_option")

    def timings(self):
        t = np.zeros(12, np.float32)
        lib().hf_get_timings(self._h, t.ctypes.data, 12)
        names = ["quantize", "keys", "sort", "tie_fixup", "window_merge", "search", "build_launches", "rerank",
                 "graph_form", "gather", "gram"]
        return dict(zip(names, t.tolist()))

    # ---- inspection --------------------------------------------------------
    def codes(self):
        out = np.empty((self.n, self.d), np.uint8)
        _check(lib().hf_debug_codes(self._h, out.ctypes.data, None), "hf_debug_codes")
        return out

    def keys(self, tree: int):
        out = np.empty((self.n, self.W), np.uint64)
        _check(lib().hf_debug_keys(self._h, tree, out.ctypes.data, None), "hf_debug_keys")
        return out

    def prefix(self, tree: int):
        """The K2 key words per point that tree `tree`'s sort keys are formed
        from, as the key kernels compute them: uint64 [n][K2] on the host
        (the library returns them word-major)."""
        out = np.empty((self.K2, self.n), np.uint64)
        _check(lib().hf_debug_prefix(self._h, tree, out.ctypes.data, None), "hf_debug_prefix")
        return np.ascontiguousarray(out.T)

    def order(self, tree: int, out=None):
        """sigma of tree `tree` (position -> point), uint32[n] on the host, or
        written into `out` (a contiguous 4-byte tensor or array of n
        elements, e.g. a CUDA int32 tensor) and returned."""
        if out is None:
            out = np.empty(self.n, np.uint32)
        op, _o = _ptr(out)
        _check(lib().hf_debug_order(self._h, tree, op, _stream(out)), "hf_debug_order")
        return out

    def locate(self, tree: int, queries):
        nq = queries.shape[0]
        out = np.empty(nq, np.int64)
        qp, _q = _ptr(queries)
        _check(lib().hf_debug_locate(self._h, tree, qp, nq, out.ctypes.data, _stream(queries)),
               "hf_debug_locate")
        return out


def build(points, T: int, bits: int = 8, seed: int = 3, options: str | None = None) -> Forest:
    return Forest(points, T, bits, seed, options)


def build_segmented(points, offsets, T: int, bits: int = 8, seed: int = 3, options: str | None = None) -> Forest:
    """hf_build_segmented: rows offsets[s] .. offsets[s+1]-1 of `points` form
    independent set s."""
    return Forest(points, T, bits, seed, options, offsets=offsets)


class CudaGraph:
    """A CUDA graph of enqueue-only library work, captured on a side stream
    (hf_capture_begin / hf_capture_end) and replayed with launch()."""

    def __init__(self, stream_handle: int):
        self.stream = stream_handle
        self._exec = None

    def __enter__(self):
        _check(lib().hf_capture_begin(self.stream), "hf_capture_begin")
        return self

    def __exit__(self, et, ev, tb):
        ex = ctypes.c_void_p()
        rc = lib().hf_capture_end(self.stream, ctypes.byref(ex))
        if et is None:
            _check(rc, "hf_capture_end")
            self._exec = ex
        return False

    def launch(self, stream_handle: int | None = None):
        _check(lib().hf_graph_launch(self._exec, self.stream if stream_handle is None else stream_handle),
               "hf_graph_launch")

    def close(self):
        if self._exec is not None:
            lib().hf_graph_destroy(self._exec)
            self._exec = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mlp:
    """The budget model (hf_mlp_*): d -> 256 -> 256 -> 2, GELU, BF16 weights
    and activations, FP32 accumulation on the tensor cores, Adam."""

    def __init__(self, d: int, seed: int = 5):
        h = ctypes.c_void_p()
        _check(lib().hf_mlp_create(d, seed, ctypes.byref(h)), "hf_mlp_create")
        self._h, self.d = h, int(d)
        cnt = ctypes.c_int64()
        lib().hf_mlp_param_count(self._h, ctypes.byref(cnt))
        self.nparam = int(cnt.value)

    def close(self):
        if getattr(self, "_h", None):
            lib().hf_mlp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        out = np.empty(self.nparam, np.float32)
        _check(lib().hf_mlp_get_params(self._h, out.ctypes.data), "hf_mlp_get_params")
        return out

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(lib().hf_mlp_set_params(self._h, p.ctypes.data), "hf_mlp_set_params")

    def predict(self, x, out=None):
        """x: CUDA float32 [n, d] -> [n, 2]."""
        n = x.shape[0]
        if out is None:
            out = _empty_like_input(x, (n, 2), "float32")
        xp, _x = _ptr(x)
        op, _o = _ptr(out)
        _check(lib().hf_mlp_predict(self._h, xp, n, op, _stream(x, out)), "hf_mlp_predict")
        return out

    def grads(self, x, targets):
        """(loss, packed gradients) of one batch (CUDA x [B, d], targets [B, 2])."""
        B = x.shape[0]
        g = np.empty(self.nparam, np.float32)
        loss = np.zeros(1, np.float32)
        xp, _x = _ptr(x)
        tp, _t = _ptr(targets)
        _check(lib().hf_mlp_grads(self._h, xp, tp, B, g.ctypes.data, loss.ctypes.data, _stream(x, targets)),
               "hf_mlp_grads")
        return float(loss[0]), g

    def train(self, x, targets, batch: int, steps: int, lr: float):
        """Adam steps on the CUDA training set; the mean loss of the last steps."""
        loss = np.zeros(1, np.float32)
        xp, _x = _ptr(x)
        tp, _t = _ptr(targets)
        _check(lib().hf_mlp_train(self._h, xp, tp, x.shape[0], batch, steps, lr, loss.ctypes.data,
                                  _stream(x, targets)), "hf_mlp_train")
        return float(loss[0])
