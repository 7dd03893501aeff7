"""cgo: GB300-native population search (cuGenOpt's search generation).

The compute path is the CUDA library ``libcgo.so`` (C ABI, include/cgo.h);
this package only loads it (``cgo``) and marshals arguments.
"""
from . import cgo  # noqa: F401
from .cgo import Problem, CgoError, solve_batch, lib  # noqa: F401
