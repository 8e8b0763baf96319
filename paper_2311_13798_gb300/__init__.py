"""Exact k-clique counting and listing on one GB300 with the edge-oriented
branch-and-bound method EBBkC (Wang, Yu & Long, SIGMOD 2024, arXiv 2311.13798).

The compute path is the CUDA library ``libkclique.so`` (``csrc/``, C ABI in
``include/kclique.h``); ``kclique`` is its ctypes binding; ``build`` compiles it.
"""
from .kclique import (  # noqa: F401
    KC_CHECKSUM, KC_NO_ET, KC_NO_RULE1, KC_NO_RULE2, KC_TRUNCATED, KCliqueError, Graph,
    kclique_count, kclique_count_batch, kclique_edge_data, kclique_info, kclique_list,
    kclique_prepare, kclique_status_string, library,
)
