"""GB300-native adaptive polynomial filtering for Hermitian interior eigenproblems.

The solver is the CUDA library ``libapf.so`` (C ABI in ``include/apf.h``);
``binding`` is its ctypes binding.  Build with ``__graft_entry__.build()`` or
``python -m paper_2604_00914_gb300.build``.
"""
from . import binding  # noqa: F401

__all__ = ["binding"]
