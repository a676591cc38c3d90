"""CPU oracle for the GeMSLR-preconditioned FGMRES solve (test infrastructure).

A plain, slow, FP64 restatement of the paper's method, written to be checked
by eye against it: the multilevel reordering (Alg. 3), the setup (Alg. 1) with
incomplete LU of every B_l and the rank-k Schur corrections from Arnoldi on
G_l = E_l (U_l^-1 L_l^-1) F_l C_l^-1 (Sec. 2.3-2.4), the standard solve
(Alg. 2) and restarted FGMRES (Sec. 4.1, Sec. 5 set-up).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and never imports it; the only shared module is ``gemslr_inputs``,
which generates the seeded synthetic problems.
"""
from .partition import multilevel_partition, rcm_order, check_partition, local_order  # noqa: F401
from .ilu import ilu0, ilut  # noqa: F401
from .gemslr import OracleGemslr  # noqa: F401
from .fgmres import fgmres  # noqa: F401

