"""The C ABI without a GPU: the library builds, loads, exports every symbol
declared in include/hf.h, and its host-only logic matches the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hf():
    import __graft_entry__ as g

    g.build()
    import paper_2508_21682_gb300 as hf

    return hf


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "hf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hf_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(hf):
    names = declared_symbols()
    assert len(names) >= 15
    L = hf.lib()
    for name in names:
        assert hasattr(L, name), name
    assert sorted(hf.SYMBOLS) == names


def test_status_strings(hf):
    for code in range(0, -8, -1):
        s = hf.status_string(code)
        assert s and s != "unknown status"
    assert hf.status_string(5) == "unknown status"


@pytest.mark.parametrize("seed,tree,d", [(3, 0, 16), (3, 7, 16), (1, 0, 384), (0, 31, 384), (2**63 + 5, 2, 5), (9, 0, 1)])
def test_tree_params_match_oracle(hf, seed, tree, d):
    pi, r = hf.tree_params(seed, tree, d)
    opi, orr = O.tree_params(seed, tree, d)
    assert np.array_equal(pi.astype(np.int64), opi)
    assert np.array_equal(r, orr)


def test_invalid_arguments_rejected_before_any_device_work(hf):
    L = hf.lib()
    h = ctypes.c_void_p()
    x = np.zeros((4, 3), np.float32)
    p = x.ctypes.data
    assert L.hf_build(p, 1, 3, 1, 8, 0, None, ctypes.byref(h)) == hf.HF_EINVAL  # n < 2
    assert L.hf_build(p, 4, 0, 1, 8, 0, None, ctypes.byref(h)) == hf.HF_EINVAL  # d < 1
    assert L.hf_build(p, 4, 3, 0, 8, 0, None, ctypes.byref(h)) == hf.HF_EINVAL  # T < 1
    assert L.hf_build(p, 4, 3, 1, 9, 0, None, ctypes.byref(h)) == hf.HF_EINVAL  # bits > 8
    assert L.hf_build(p, 4, 3, 1, 0, 0, None, ctypes.byref(h)) == hf.HF_EINVAL  # bits < 1
    assert L.hf_build(p, 4, 4097, 1, 8, 0, None, ctypes.byref(h)) == hf.HF_EINVAL
    assert L.hf_build(None, 4, 3, 1, 8, 0, None, ctypes.byref(h)) == hf.HF_EINVAL
    assert L.hf_build_opts(p, 4, 3, 1, 8, 0, b"bogus=1", None, ctypes.byref(h)) == hf.HF_EINVAL
    assert L.hf_build_opts(p, 4, 3, 1, 8, 0, b"prefix_words=9", None, ctypes.byref(h)) == hf.HF_EINVAL
    assert L.hf_build_opts(p, 4, 3, 1, 8, 0, b"prefix_words=x", None, ctypes.byref(h)) == hf.HF_EINVAL
    assert L.hf_knn_graph(None, 10, 4, p, p, None) == hf.HF_EINVAL
    assert L.hf_search(None, p, 1, 10, 4, p, p, None) == hf.HF_EINVAL
    assert L.hf_free(None) == hf.HF_OK
    assert L.hf_tree_params(0, 0, 0, p, p) == hf.HF_EINVAL
    assert L.hf_debug_keys_from_codes(p, 0, 3, 8, p, None) == hf.HF_EINVAL
    assert L.hf_debug_prefix(None, 0, p, None) == hf.HF_EINVAL
    assert L.hf_info(None, p, 8) == hf.HF_EINVAL


def test_product_path_fails_loudly_without_library(hf, monkeypatch, tmp_path):
    import importlib

    monkeypatch.setattr(hf, "_lib", None)
    monkeypatch.setattr(hf, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        hf.lib()
