"""GB300 (sm_103a) block solver for y = Ax + e: CSGD / GCSGD (arXiv:1709.00953).

The compute path is the CUDA library ``libcsgd.so`` behind the C ABI of
``include/csgd.h``; ``csgd`` is its Python binding (marshalling only).
"""
from . import csgd  # noqa: F401
from .csgd import (CsgdError, Geometry, Partition, Solver, backproject_block,  # noqa: F401
                   block_partition, geometry_create, project_block, project_full, solve,
                   solve_step, solver_create)
