"""The paper's split storage (Sec. 4.1-4.2: dense diagonal blocks H^{L(D)}_k, sparse
off-diagonal H^{L(OD)}_k) through the filter: the dense blocks on the tensor cores by
Ozaki slices, the rest through the CSR kernel, checked against the oracle's filter
of the same operator in plain CSR, on an operator whose density decays away from
the diagonal (a dense band plus sparse far couplings)."""
import ctypes

import numpy as np
import pytest
import torch

import chfsi_workloads as W
from tests.util import rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2110_15853_gb300 import build
    build.build()
    import paper_2110_15853_gb300 as P
    return P


def _split_dev(P, H, block):
    S = W.split_from_csr(H, block)
    o = S["off"]
    return P.SplitMatrix.from_arrays(S["diag"], block, o["row_ptr"], o["col"], o["val"], device="cuda"), S


@pytest.mark.parametrize("N,band,block,n,m", [(4096, 96, 512, 40, 8), (4000, 80, 512, 33, 7),
                                              (2944, 200, 384, 600, 5), (1024, 30, 128, 1, 1)])
def test_split_filter_matches_oracle(P, oracle_mod, N, band, block, n, m):
    H = W.banded_operator(N, band, 4, 0.1, N + band)
    X = W.start_block(N, n, N + 1)
    a, b, a0 = oracle_mod.lanczos_bounds(H, W.lanczos_start(N, N + 2), 20, max(n, 2))
    Sd, S = _split_dev(P, H, block)
    assert S["off"]["nnz"] + np.count_nonzero(S["diag"]) <= H["nnz"]
    ws = P.Workspace("cuda")
    Y = P.filter(Sd, torch.as_tensor(X).cuda(), m, a, b, a0, workspace=ws)
    assert P.read_status(ws) == 0
    Yref = oracle_mod.filter(H, X, m, a, b, a0)
    assert rel_fro(Y.cpu().numpy(), Yref) <= 1e-12


def test_split_filter_matches_csr_filter_on_grid_operator(P):
    """The same operator in CSR and in split storage (a grid operator in its natural
    order, blocks of 1024 rows) through the GPU filter."""
    H = W.csr_grid(16, 2, 0.1, 77)
    X = torch.as_tensor(W.start_block(H["N"], 64, 77)).cuda()
    Hd = P.CsrMatrix.from_arrays(H["row_ptr"], H["col"], H["val"], device="cuda")
    Sd, _ = _split_dev(P, H, 1024)
    Yc = P.filter(Hd, X, 10, 4.0, 12.0, 2.0)
    Ys = P.filter(Sd, X, 10, 4.0, 12.0, 2.0)
    assert rel_fro(Ys.cpu().numpy(), Yc.cpu().numpy()) <= 1e-12


def test_split_rejects_unsupported_uses(P):
    from paper_2110_15853_gb300 import _abi
    H = W.banded_operator(1024, 30, 2, 0.1, 5)
    Sd, _ = _split_dev(P, H, 256)
    X = torch.as_tensor(W.start_block(1024, 8, 5)).cuda()
    with pytest.raises(P.ChfsiError) as e:
        P.filter(Sd, X, 4, 4.0, 12.0, 2.0, schedule=["f32x2"] * 4)
    assert e.value.code == _abi.CHFSI_ERR_UNSUPPORTED
    with pytest.raises(P.ChfsiError) as e:
        P.rayleigh_ritz(Sd, X, 2)
    assert e.value.code == _abi.CHFSI_ERR_UNSUPPORTED
    bad = P.SplitMatrix(Sd.diag, Sd.off, 200, Sd.n_rows)          # block not a multiple of 128
    with pytest.raises(P.ChfsiError) as e:
        P.filter(bad, X, 4, 4.0, 12.0, 2.0)
    assert e.value.code == _abi.CHFSI_ERR_UNSUPPORTED


def test_split_from_csr_with_the_density_rule(P, oracle_mod):
    """SplitMatrix.from_csr without a block: the largest power-of-two block whose
    diagonal blocks stay at least 5% dense (Sec. 4.1), through the filter."""
    N = 3000
    H = W.banded_operator(N, 60, 3, 0.1, 31)
    B = P.split_block_size(H["row_ptr"], H["col"])
    assert B == 2048 and P.split_block_density(H["row_ptr"], H["col"], B) >= 0.05
    Sd = P.SplitMatrix.from_csr(H["row_ptr"], H["col"], H["val"], device="cuda")
    assert Sd.block == B
    X = W.start_block(N, 24, 32)
    a, b, a0 = oracle_mod.lanczos_bounds(H, W.lanczos_start(N, 33), 20, 24)
    Y = P.filter(Sd, torch.as_tensor(X).cuda(), 6, a, b, a0)
    assert rel_fro(Y.cpu().numpy(), oracle_mod.filter(H, X, 6, a, b, a0)) <= 1e-12
