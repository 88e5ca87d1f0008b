"""GB300 (sm_103a) implementation of the data-parallel hot path of the
hierarchically deflated conjugate gradient (HDCG, arXiv 1402.2585).

All computation happens in the CUDA library ``libhdcg.so`` (C ABI declared in
``include/hdcg.h``).  This package only marshals arguments: torch tensors (on
the GPU) or numpy arrays (host) are passed as raw pointers.  Importing the
binding fails loudly when the library has not been built; there is no CPU
fallback.
"""
from .binding import (F16, F32, F64, BF16, BF16T, DF64, ALG_CG, ALG_ADEF2, HdcgError, Hdcg,  # noqa: F401
                      SubspaceParams, SolveParams, SolveStats, LdopParams, dense_heev, lib, library_path,
                      PREC_NAMES)
