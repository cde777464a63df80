"""GB300 (sm_103a) implementation of the IBDL operator hot path (Leathers 2022, arXiv 2210.07403).

The compute path is the CUDA library ``libibdl.so`` (C ABI in ``include/ibdl.h``), built in-tree
by ``paper_2210_07403_gb300.build``; ``paper_2210_07403_gb300.ibdl`` is its Python binding.
"""
from .ibdl import Geometry, IbdlError, load  # noqa: F401

__all__ = ["Geometry", "IbdlError", "load"]
