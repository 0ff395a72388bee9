"""chfsi_filter_noalloc: the filter for callers that cannot allocate device memory.

Such callers (a host whose own allocator owns the whole GPU and that must not
call cudaMalloc/cudaFree or pass a scratch buffer) get the filter's scratch from a
static device array inside the library.  This file is collected last on purpose,
so that a run stopping at the first failure has run every other test first; it
also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import chfsi_workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2110_15853_gb300 import build
    build.build()
    import paper_2110_15853_gb300 as P
    return P


def test_noalloc_filter_matches_workspace_filter_twice(P):
    """Two calls in a row through the C ABI, each compared with chfsi_filter
    (caller workspace) on the same inputs at the filter's 1e-12 tolerance."""
    from paper_2110_15853_gb300 import _abi
    lib = P.load()
    dev = torch.device("cuda")
    g, w, n, m = 12, 3, 40, 9
    H = W.csr_grid(g, w, 0.1, 91)
    Hd = P.CsrMatrix.from_arrays(H["row_ptr"], H["col"], H["val"], device=dev)
    desc = Hd.descriptor()
    stream = torch.cuda.current_stream(dev).cuda_stream
    a0, a, b = 3.0, 4.2, 12.5
    for call, seed in enumerate((1, 2)):
        X = torch.as_tensor(W.start_block(H["N"], n, seed)).to(dev)
        Y_ref = P.filter(Hd, X, m, a, b, a0)                   # existing entry point
        Y = torch.full_like(X, float("nan"))
        rc = lib.chfsi_filter_noalloc(ctypes.byref(desc), X.data_ptr(), X.stride(0), Y.data_ptr(), Y.stride(0),
                                      n, m, a, b, a0, None, stream)
        assert rc == _abi.CHFSI_OK, (call, P.status_string(rc))
        torch.cuda.synchronize(dev)
        err = float(torch.linalg.norm(Y - Y_ref) / torch.linalg.norm(Y_ref))
        assert err <= 1e-12, (call, err)


def test_noalloc_rejects_problems_beyond_the_static_scratch(P):
    from paper_2110_15853_gb300 import _abi
    lib = P.load()
    dev = torch.device("cuda")
    H = W.csr_grid(20, 2, 0.1, 92)                             # N = 8000
    Hd = P.CsrMatrix.from_arrays(H["row_ptr"], H["col"], H["val"], device=dev)
    desc = Hd.descriptor()
    n = 2048            # workspace 2 * 8000 * 512 * 8 B (one 512-column slab) > 16 MiB
    X = torch.zeros((H["N"], n), dtype=torch.float64, device=dev)
    Y = torch.empty_like(X)
    rc = lib.chfsi_filter_noalloc(ctypes.byref(desc), X.data_ptr(), n, Y.data_ptr(), n, n, 4, 4.2, 12.5, 3.0,
                                  None, torch.cuda.current_stream(dev).cuda_stream)
    assert rc == _abi.CHFSI_ERR_NOMEM


def test_noalloc_status_reports_non_finite_input(P):
    """A NaN in X reaches the filter's status word in the static array; the
    companion call reads it back (and clears it), and the next clean call is clean."""
    from paper_2110_15853_gb300 import _abi
    lib = P.load()
    dev = torch.device("cuda")
    H = W.csr_grid(10, 2, 0.1, 93)
    Hd = P.CsrMatrix.from_arrays(H["row_ptr"], H["col"], H["val"], device=dev)
    desc = Hd.descriptor()
    stream = torch.cuda.current_stream(dev).cuda_stream
    n, m = 16, 5
    X = torch.as_tensor(W.start_block(H["N"], n, 3)).to(dev)
    X[7, 3] = float("nan")
    Y = torch.empty_like(X)
    rc = lib.chfsi_filter_noalloc(ctypes.byref(desc), X.data_ptr(), n, Y.data_ptr(), n, n, m, 4.2, 12.5, 3.0,
                                  None, stream)
    assert rc == _abi.CHFSI_OK
    assert lib.chfsi_filter_noalloc_read_status(stream) == _abi.CHFSI_ERR_NONFINITE
    assert lib.chfsi_filter_noalloc_read_status(stream) == _abi.CHFSI_OK      # cleared by the read
    X[7, 3] = 0.0
    rc = lib.chfsi_filter_noalloc(ctypes.byref(desc), X.data_ptr(), n, Y.data_ptr(), n, n, m, 4.2, 12.5, 3.0,
                                  None, stream)
    assert rc == _abi.CHFSI_OK
    assert lib.chfsi_filter_noalloc_read_status(stream) == _abi.CHFSI_OK
    assert bool(torch.isfinite(Y).all())
