"""GB300-native (sm_103a) RI-qsGW (and qsMP2) hot path of arXiv 2210.17093.

The compute runs in the CUDA library ``libmolgw_gb300.so`` built from ``csrc/``
(C ABI in ``include/molgw_gb300.h``); this package only builds and binds it.
"""
from .native import (EXPORTS, FLAG_EIG_TC, FLAG_FULL_XPY, FLAG_GRAPH, FLAG_KTIMING,  # noqa: F401
                     FLAG_QSMP2, FLAG_TC_AB, ITEM, KERNELS, PREC, Context, MolgwError, load, plan_batch)

__all__ = ["Context", "MolgwError", "load", "EXPORTS", "FLAG_FULL_XPY", "FLAG_GRAPH", "FLAG_KTIMING",
           "FLAG_EIG_TC", "FLAG_QSMP2", "FLAG_TC_AB", "ITEM", "KERNELS", "PREC", "plan_batch"]
