"""GB300-native batched IPv6 longest-prefix-match by the PlanB method (arXiv 2604.14650).

Prefixes become sorted elementary intervals (Section 3.1), laid out as a linearized B+-tree
(Section 3.2) that hand-written sm_103a CUDA kernels descend for each 128-bit address. The compute
lives in ``libplanb.so`` (C ABI in ``include/planb.h``); this package is its Python binding.
"""
from .binding import (FORMATS, KERNELS, Fib, MultiFib, Server, PlanbError, child_index, debug_inject, intervals,  # noqa: F401
                      layout_info, library_path, load, mlp_forward, mlp_grad, mlp_grad_split,
                      mlp_knot_step, version)


def build(force: bool = False):
    """Compiles libplanb.so for sm_103a in-tree (nvcc)."""
    from .nvcc_build import build as _b
    return _b(force=force)
