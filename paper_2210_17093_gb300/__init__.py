"""GB300-native (sm_103a) RI-qsGW hot path of arXiv 2210.17093.

The compute runs in the CUDA library ``libmolgw_gb300.so`` built from ``csrc/``
(C ABI in ``include/molgw_gb300.h``); this package only builds and binds it.
"""
from .native import (EXPORTS, FLAG_FULL_XPY, FLAG_GRAPH, FLAG_EIG_TC, FLAG_KTIMING, FLAG_TC_AB, ITEM, KERNELS,  # noqa: F401
                     PREC, Context, MolgwError, load)

__all__ = ["Context", "MolgwError", "load", "EXPORTS", "FLAG_FULL_XPY", "FLAG_GRAPH", "FLAG_KTIMING",
           "FLAG_EIG_TC", "FLAG_TC_AB", "ITEM", "KERNELS", "PREC"]
