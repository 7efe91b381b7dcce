"""GB300-native Robust Spanning Index (RSI) scoring, arXiv 2508.01485.

The hot path lives in ``csrc/`` (CUDA for sm_103a) behind the C ABI of
``include/rs.h``; ``Graph`` is the thin Python binding of that ABI.
"""
from ._lib import (RS_EBUDGET, RS_ECUDA, RS_EINVAL, RS_ENOMEM, RS_ETIMEOUT, RS_OK,  # noqa: F401
                   Graph, RSError, Server, Step, Tuning, default_tuning, lib)

__all__ = ["Graph", "RSError", "Server", "Step", "Tuning", "default_tuning", "lib", "RS_OK", "RS_EINVAL",
           "RS_ENOMEM", "RS_ECUDA", "RS_ETIMEOUT", "RS_EBUDGET"]
