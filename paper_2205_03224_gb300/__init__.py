"""GB300-native GeMSLR-preconditioned FGMRES (solve phase of arXiv 2205.03224).

The compute path is the CUDA library ``libgemslr.so`` (C ABI in
``include/gemslr.h``); this package only marshals arguments to it.
"""
from .api import Gemslr, GemslrBatch, local_order, partition_geometric  # noqa: F401
