"""The abort path of the tensor-core kernels' bounded waits, made to run out without
any fault: with the pipeline-wait limit set to a few nanoseconds
(chfsi_set_pipeline_wait_limit), the first wait of one role on another that does
not succeed at once gives up, the CTA stops, drains its own copies and MMAs (those
waits keep their 1 s bound), frees its tensor memory and exits, and the call's
status word reads CHFSI_ERR_TIMEOUT.  The next call with the default limit on the
same context and workspace must then match the oracle exactly as before.

Cases: one BF16 tensor-core BSR step (Algorithm 1 step 1 on the dense blocks of
Sec. 4.1-4.2) with BF16-representable H and X, where every product and partial sum
is exact in FP32; and an Ozaki product of 16-bit integers, which is exact."""
import ctypes

import numpy as np
import pytest
import torch

import chfsi_workloads as W
from tests.util import rel_fro

pytestmark = pytest.mark.gpu

SHORT_NS = 4


@pytest.fixture(scope="module")
def P():
    from paper_2110_15853_gb300 import build
    build.build()
    import paper_2110_15853_gb300 as P
    return P


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to("cuda")


def _short_limit(P):
    lib = P.load()
    assert lib.chfsi_set_pipeline_wait_limit(SHORT_NS) == 0
    return lib


def test_bsr_tensor_core_step_times_out_then_runs_clean(P, oracle_mod):
    from paper_2110_15853_gb300 import _abi
    g, w, n = 16, 2, 300
    H = W.csr_grid(g, w, 0.0, 3)
    H["val"] = np.round(H["val"] * 64) / 64             # few-bit values: exact in BF16
    X = np.random.default_rng(5).integers(-8, 9, size=(H["N"], n)) / 8.0
    a0, a, b = 1.0, 3.5, 14.0
    B = W.bsr_from_csr(H, g)
    perm = B["perm"]
    Hb = P.BsrMatrix.from_arrays(B["brow_ptr"], B["bcol"], B["val"], device="cuda")
    Xd = _dev(X[perm])
    ws = P.Workspace("cuda")
    lib = _short_limit(P)
    try:
        P.filter(Hb, Xd, 1, a, b, a0, schedule=["bf16"], workspace=ws)
        torch.cuda.synchronize()
        assert P.read_status(ws) == _abi.CHFSI_ERR_TIMEOUT
    finally:
        assert lib.chfsi_set_pipeline_wait_limit(0) == 0
    Yb = P.filter(Hb, Xd, 1, a, b, a0, schedule=["bf16"], workspace=ws).cpu().numpy()
    assert P.read_status(ws) == 0
    Y = np.empty_like(Yb)
    Y[perm] = Yb
    assert rel_fro(Y, oracle_mod.filter(H, X, 1, a, b, a0)) <= 1e-6


def test_ozaki_product_times_out_then_runs_clean(P):
    from paper_2110_15853_gb300 import _abi
    rng = np.random.default_rng(17)
    K, M, Nc = 9000, 256, 192
    A = rng.integers(-(2 ** 15 - 1), 2 ** 15, size=(K, M)).astype(np.int64)
    Bm = rng.integers(-(2 ** 15 - 1), 2 ** 15, size=(K, Nc)).astype(np.int64)
    A[0, :] = 2 ** 15 - 1
    Bm[0, :] = 2 ** 15 - 1
    Ad, Bd = _dev(A.astype(np.float64)), _dev(Bm.astype(np.float64))
    C = torch.empty(M, Nc, dtype=torch.float64, device="cuda")
    lib = P.load()
    sz = ctypes.c_size_t(0)
    assert lib.chfsi_ozaki_gemm_workspace_size(_abi.CHFSI_OP_TN, M, Nc, K, 0, ctypes.byref(sz)) == 0
    ws = torch.empty(sz.value, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream

    def call():
        return lib.chfsi_ozaki_gemm(_abi.CHFSI_OP_TN, Ad.data_ptr(), M, Bd.data_ptr(), Nc, C.data_ptr(), Nc, M, Nc, K,
                                    0, ws.data_ptr(), ws.numel(), stream)

    _short_limit(P)
    try:
        assert call() == 0
        assert lib.chfsi_read_status(ws.data_ptr(), stream) == _abi.CHFSI_ERR_TIMEOUT
    finally:
        assert lib.chfsi_set_pipeline_wait_limit(0) == 0
    assert call() == 0
    assert lib.chfsi_read_status(ws.data_ptr(), stream) == 0
    assert np.array_equal(C.cpu().numpy(), (A.T @ Bm).astype(np.float64))
