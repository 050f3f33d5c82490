"""FP64 CPU oracle for the nonlocal FEM assembly of arXiv 2207.03921.

Test infrastructure only: used by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py. It shares no code with the CUDA
library and does not import it.
"""
from .oracle import (KERNELS, BALLS, CLOSE_RULES, OracleSystem, assemble, build, clip,  # noqa: F401
                     pair_block, pairs, solve_dirichlet, solve_neumann, null_space, l2_error, lib_path)
