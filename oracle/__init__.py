"""CPU oracle for the Hilbert forest path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
arm of ``bench.py`` may import this package. The CUDA library never calls it
and has no fallback to it.

Pinned by ``tests/test_oracle_pins.py``: full-grid bijection and unit-step
adjacency of the curve, the 2-D textbook curve, hand-derived traversals in
``tests/golden/``, splitmix64 reference outputs, closed-form quantization
cases, brute-force special cases of the graph and of search, and recall
monotonicity. Recall values themselves are parity-unpinned against the paper
(its datasets are not available).

``oracle.c_oracle`` loads a second restatement of the same path in plain C++
(``hf_oracle.cpp``: scalar loops, compiled without fused multiply-adds). It
is not imported here; ``tests/test_oracle_cpp.py`` runs the curve pins on it
and compares it with this numpy oracle element by element.
"""
from .hilbert_forest import *  # noqa: F401,F403
from .hilbert_forest import (  # noqa: F401
    Forest, SplitMix64, axis_range, brute_force_knn, candidate_sets, hilbert_keys,
    hilbert_order, key_less_count, key_words, knn_graph, locate, pack_key,
    permute_reflect, quantize, query_codes, recall, search, search_candidates, skilling_transpose,
    sq_dist_fp64, topk_from_candidates, tree_params, window_candidates,
)
from . import budget  # noqa: F401,E402  (learned per-point budget: labels, MLP, budgeted graph)
from . import sketch  # noqa: F401,E402  (second stage: sign sketches, Hamming top-k2)
