"""GB300-native concurrent hash containers (unordered_set / unordered_map over
integer keys) after "stdgpu: Efficient STL-like Data Structures on the GPU".

The compute path is libhc.so (hand-written CUDA for sm_103a behind a C ABI,
include/hc.h); this package is its Python binding plus the batched and served
forms built on top of it.
"""
from . import _lib  # noqa: F401
from ._lib import (  # noqa: F401
    ERASED, EXISTS, HASH_MIX64, HASH_TESCHNER, INSERTED, MAP_I64_I32, MAP_U64_U64, NOT_FOUND, OP_ERASE, OP_FIND,
    OP_INSERT, OVERFLOW, SET_U32, SET_U64, HCError,
)


def __getattr__(name):
    # torch-dependent pieces are imported lazily so that the ctypes binding
    # can be loaded (and its symbols checked) without initialising CUDA
    if name == "Table":
        from .table import Table
        return Table
    raise AttributeError(name)
