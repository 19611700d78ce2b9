"""GB300-native Monte Carlo four-component relativistic MP2 (arXiv 2203.05632).

The per-step Monte Carlo evaluation of the 13-dimensional MP2 integrand runs
in hand-written sm_103a CUDA kernels behind the C ABI of include/mcmp2.h;
this package is a thin ctypes binding plus the in-tree build.
"""
from ._binding import (MCMP2_FP64, MCMP2_MIXED, MCMP2_TF32, MCMP2_COULOMB, MCMP2_GAUNT, MCMP2_BREIT, MCMP2_EUNSUPPORTED, Context, McMp2Error, header_symbols,  # noqa: F401
                       load_library, workspace_bytes, Dims, LIB_PATH)
from .build import build  # noqa: F401
