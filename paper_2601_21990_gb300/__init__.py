"""Batched restarted reflected-Halpern PDHG LP solver for GB300 (sm_103a).

The solver is the C-ABI library ``liblpb.so`` (headers in ``include/lpb.h``,
CUDA sources in ``csrc/``); ``lpb`` is its ctypes binding.  Build with
``paper_2601_21990_gb300._build.build()``.
"""
from . import lpb  # noqa: F401
from .lpb import Handle, Batch, Options, specs_array, specs_from  # noqa: F401
