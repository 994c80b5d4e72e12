"""GB300-native asynchronous block ILU(0) preconditioning with FGMRES.

The computation lives in libabilu.so (hand-written sm_103a CUDA behind the C
ABI of include/abilu.h); ``abilu`` is its thin Python binding.
"""
from .abilu import (AbiluError, Batch, Factors, Multigrid, Pattern, SolveResult,  # noqa: F401
                    add_block_diagonal, bsr_spmv, default_opts, fgmres_solve, fgmres_solve_mg,
                    gather_blocks, kernel_launches, order, parilut, permute_pattern, to_f32,
                    version)
