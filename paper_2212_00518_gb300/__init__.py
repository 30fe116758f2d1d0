"""GB300-native batched independent electron surface hopping (IESH).

The compute path is the CUDA library libiesh.so (C-ABI in include/iesh.h);
``paper_2212_00518_gb300.iesh`` is its ctypes binding.
"""
from . import iesh  # noqa: F401
from .iesh import Context, IeshError, PREC_FP64, PREC_MIXED  # noqa: F401
