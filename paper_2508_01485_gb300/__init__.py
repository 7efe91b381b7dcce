"""GB300-native Robust Spanning Index (RSI) scoring, arXiv 2508.01485.

The hot path lives in ``csrc/`` (CUDA for sm_103a) behind the C ABI of
``include/rs.h``; ``Graph`` is the thin Python binding of that ABI.
"""
from ._lib import Graph, RSError, Server, Step, Tuning, default_tuning, lib  # noqa: F401

__all__ = ["Graph", "RSError", "Server", "Step", "Tuning", "default_tuning", "lib"]
