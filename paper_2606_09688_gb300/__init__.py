"""GB300-native space-time sparse-grid combination solver for the linear wave equation.

The compute path is the C ABI library ``libst.so`` (include/st.h, sources in
csrc/), reached through the ctypes binding in :mod:`paper_2606_09688_gb300.st`.
"""
from .st import (ST_FP32_IR, ST_FP64, Solver, StError, load_library, solve_batch)  # noqa: F401

__all__ = ["Solver", "StError", "ST_FP64", "ST_FP32_IR", "load_library", "solve_batch"]
