"""AD-LBR (Fehrenbach & Mirebeau, arXiv 1301.3925) on GB300, sm_103a.

The product is the C-ABI library ``libadlbr.so`` (include/adlbr.h) built from
``csrc/`` by ``paper_1301_3925_gb300.build``; ``paper_1301_3925_gb300.adlbr``
is its thin ctypes binding.
"""
from . import adlbr  # noqa: F401
