"""GB300 (sm_103a) Chebyshev-filtered subspace iteration: the filter of
Algorithm 1 (arXiv 2110.15853, Sec. 3.4) as hand-written CUDA behind a C ABI
(include/chfsi.h, libchfsi.so), with a thin PyTorch binding.

There is no CPU or library fallback: every entry point raises if libchfsi.so
has not been built (``python -m paper_2110_15853_gb300.build``).
"""
from ._abi import ChfsiError, LIB_PATH, load, status_string
from .chfsi import (BsrMatrix, ChebyshevFilter, CsrMatrix, HybridMatrix, SplitMatrix, Workspace, eigh, filter,
                    filter_backward,
                    filter_workspace_bytes, lanczos_bounds, lanczos_workspace_bytes, measure_pipe_peak,
                    mixed_schedule, ozaki_gemm, rayleigh_ritz, split_block_density, split_block_size,
                    rayleigh_ritz_workspace_bytes, read_status, solve, symmetric_gradient, transpose_index)

__all__ = [
    "ChfsiError", "LIB_PATH", "load", "status_string", "BsrMatrix", "ChebyshevFilter", "CsrMatrix", "HybridMatrix",
    "SplitMatrix", "eigh", "split_block_density", "split_block_size",
    "Workspace", "filter", "filter_backward", "filter_workspace_bytes", "lanczos_bounds",
    "lanczos_workspace_bytes", "measure_pipe_peak", "ozaki_gemm",
    "mixed_schedule", "rayleigh_ritz", "rayleigh_ritz_workspace_bytes", "read_status",
    "solve", "symmetric_gradient", "transpose_index",
]
