"""Plain FP64 CPU oracle of the paper's discrete problem and one-step DDM preconditioner.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA path.
"""
from .helmholtz import (  # noqa: F401
    Grid, Subdomain, pml_profile, helmholtz_matrix, global_operator, rhs_from_source,
    decompose, local_operator, factor_box, oracle_threads, DDMPreconditioner, fgmres, FGMRESResult, smoothstep5, smoothing_profile,
    block_fgmres, BlockFGMRESResult,
)
from .banded import BandLU, box_order, build_banded  # noqa: F401
