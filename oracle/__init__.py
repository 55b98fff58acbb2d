"""FP64 CPU oracle of the submatrix method (test infrastructure only).

Imported only by ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline.  It shares no code with the CUDA library in ``paper_1710_10899_gb300``.
"""
from .submatrix import (  # noqa: F401
    index_set, plan, submatrix, inv_root, inv_root_column, invroot, invroot_lu, row_segment,
    divided_differences, submatrix_grad, grad, to_dense, residual_2norm,
)
from . import cg  # noqa: F401,E402
from . import refine  # noqa: F401,E402
from . import pool  # noqa: F401,E402
