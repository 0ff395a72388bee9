"""FP64-accurate products on the BF16 tensor cores (chfsi_ozaki_gemm, Ozaki-scheme
slices) and the closure that uses them (chfsi_rayleigh_ritz_ex with
CHFSI_F64_OZAKI), against plain FP64 products and the oracle.

* Values with at most 16 significant bits below their row's largest magnitude
  are held exactly by the two leading 8-bit digits, so the product involves only
  the exactly accumulated digit levels: the result must equal the integer product
  bit for bit, for K spanning many 256-long accumulation periods and several
  split-K parts.
* Gaussian operands (ragged sizes, both forms, the symmetric and upper-triangular
  modes) against the FP64 product, within the documented bound
  K 2^-50 max|A_row| max|B_row| and at 1e-13 relative Frobenius.
* The Ozaki closure's Ritz values against the oracle's Householder/LAPACK closure
  at 1e-10 (small case and the 40^3 / 1024-state workload).
* FP64-accurate BSR filter steps (H's 64 x 64 blocks as Ozaki products) against the
  FP64 oracle at 1e-12, with empty block rows, unsorted block columns and after
  low-precision prefixes on a hybrid operator.
* 40-bit BSR filter steps (five digit slices): bit-equal to the FP64-accurate step on
  24-bit integer inputs, and within the 40-bit bound of the oracle (filtered block
  1e-9) on the grid operators.
"""
import numpy as np
import pytest
import torch

import chfsi_workloads as W
from tests.util import dense_to_csr, rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2110_15853_gb300 import build
    build.build()
    import paper_2110_15853_gb300 as P
    return P


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda")


def _ints16(rng, shape):
    """Integers of at most 15 bits plus sign, with each row's (or column's) largest
    magnitude at 2^15 - 1 so the row scale is the same for every row."""
    x = rng.integers(-(2 ** 15 - 1), 2 ** 15, size=shape).astype(np.int64)
    return x


@pytest.mark.parametrize("M,Nc,K", [(200, 136, 1000), (128, 128, 4096), (37, 300, 20011)])
def test_ozaki_tn_exact_on_16_bit_values(P, M, Nc, K):
    rng = np.random.default_rng(M * 7 + K)
    A = _ints16(rng, (K, M))
    B = _ints16(rng, (K, Nc))
    A[0, :] = 2 ** 15 - 1          # every column of A and B has the same largest magnitude
    B[0, :] = -(2 ** 15 - 1)
    C = P.ozaki_gemm(_dev(A.astype(np.float64)), _dev(B.astype(np.float64)), transpose_a=True).cpu().numpy()
    exact = A.T @ B                 # int64, |entries| < K 2^30
    assert np.array_equal(C, exact.astype(np.float64))


@pytest.mark.parametrize("M,K,Nc", [(300, 500, 136), (1000, 64, 64), (129, 1200, 257)])
def test_ozaki_nn_exact_on_16_bit_values(P, M, K, Nc):
    rng = np.random.default_rng(M + 3 * K)
    A = _ints16(rng, (M, K))
    B = _ints16(rng, (K, Nc))
    A[:, 0] = 2 ** 15 - 1
    B[0, :] = 2 ** 15 - 1
    C = P.ozaki_gemm(_dev(A.astype(np.float64)), _dev(B.astype(np.float64))).cpu().numpy()
    assert np.array_equal(C, (A @ B).astype(np.float64))


def _bound(A_rows_max, B_rows_max, K):
    return K * 2.0 ** -50 * np.outer(A_rows_max, B_rows_max)


@pytest.mark.parametrize("M,Nc,K", [(96, 70, 333), (256, 256, 70000), (1024, 1024, 64000)])
def test_ozaki_tn_gaussian(P, M, Nc, K):
    rng = np.random.default_rng(K)
    A = rng.standard_normal((K, M)) * np.exp(rng.standard_normal(M))[None, :]   # columns of different scales
    B = rng.standard_normal((K, Nc))
    C = P.ozaki_gemm(_dev(A), _dev(B), transpose_a=True).cpu().numpy()
    ref = A.T @ B
    assert np.all(np.abs(C - ref) <= _bound(np.abs(A).max(0), np.abs(B).max(0), K) + 1e-15 * np.abs(ref))
    assert rel_fro(C, ref) <= 1e-13


def test_ozaki_tn_symmetric_gram(P):
    rng = np.random.default_rng(5)
    K, n = 50000, 300
    Y = rng.standard_normal((K, n))
    Yd = _dev(Y)
    S = P.ozaki_gemm(Yd, Yd, transpose_a=True, symmetric=True).cpu().numpy()
    ref = Y.T @ Y
    scale = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    assert np.max(np.abs(S - S.T) / scale) <= 1e-14   # mirrored tiles; diagonal tiles to rounding
    assert rel_fro(S, ref) <= 1e-13
    assert np.max(np.abs(S - ref) / scale) <= 1e-13


@pytest.mark.parametrize("M,K,Nc,upper", [(5000, 300, 300, False), (777, 513, 513, True), (64000, 1024, 1024, True)])
def test_ozaki_nn_gaussian(P, M, K, Nc, upper):
    rng = np.random.default_rng(M + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, Nc))
    if upper:
        B = np.triu(B)
    C = P.ozaki_gemm(_dev(A), _dev(B), b_upper=upper).cpu().numpy()
    ref = A @ B
    assert np.all(np.abs(C - ref) <= _bound(np.abs(A).max(1), np.abs(B).max(0), K) + 1e-15 * np.abs(ref))
    assert rel_fro(C, ref) <= 1e-13


def test_ozaki_zero_rows_columns_and_views(P):
    """Zero rows / columns give exact zeros; column views of wider blocks (ld > n)."""
    rng = np.random.default_rng(9)
    A = rng.standard_normal((700, 90))
    B = rng.standard_normal((700, 50))
    A[:, 7] = 0.0
    B[:, 3] = 0.0
    Aw = np.zeros((700, 128))
    Aw[:, :90] = A
    Ad = _dev(Aw)[:, :90]
    C = P.ozaki_gemm(Ad, _dev(B), transpose_a=True).cpu().numpy()
    assert np.all(C[7, :] == 0.0) and np.all(C[:, 3] == 0.0)
    assert rel_fro(C, A.T @ B) <= 1e-13


def test_ozaki_nonfinite_input_sets_status(P):
    from paper_2110_15853_gb300 import _abi
    import ctypes
    lib = P.load()
    A = torch.randn(300, 40, dtype=torch.float64, device="cuda")
    A[11, 5] = float("inf")
    B = torch.randn(300, 40, dtype=torch.float64, device="cuda")
    C = torch.empty(40, 40, dtype=torch.float64, device="cuda")
    sz = ctypes.c_size_t(0)
    assert lib.chfsi_ozaki_gemm_workspace_size(_abi.CHFSI_OP_TN, 40, 40, 300, 0, ctypes.byref(sz)) == 0
    ws = torch.empty(sz.value, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.chfsi_ozaki_gemm(_abi.CHFSI_OP_TN, A.data_ptr(), 40, B.data_ptr(), 40, C.data_ptr(), 40, 40, 40, 300, 0,
                              ws.data_ptr(), ws.numel(), stream)
    assert rc == 0
    assert lib.chfsi_read_status(ws.data_ptr(), stream) == _abi.CHFSI_ERR_NONFINITE


def test_rayleigh_ritz_ozaki_small(P, oracle_mod):
    """The Ozaki closure on a small grid operator against the oracle closure."""
    H = W.csr_grid(8, 2, 0.1, 45)
    X = W.start_block(H["N"], 20, 45)
    a, b, a0 = oracle_mod.lanczos_bounds(H, W.lanczos_start(H["N"], 45), 20, 20)
    Y = oracle_mod.filter(H, X, 8, a, b, a0)
    Hd = P.CsrMatrix.from_arrays(H["row_ptr"], H["col"], H["val"], device="cuda")
    ritz, psi = P.rayleigh_ritz(Hd, _dev(Y), cholqr_passes=2, precision="ozaki")
    theta, _, _ = oracle_mod.rayleigh_ritz(H, Y)
    assert np.max(np.abs(ritz.cpu().numpy() - theta)) <= 1e-10 * np.max(np.abs(theta))
    p = psi.cpu().numpy()
    assert np.max(np.abs(p.T @ p - np.eye(20))) <= 1e-12


def test_rayleigh_ritz_ozaki_full_space_is_eigh(P):
    """n = N: the Ritz values are the eigenvalues of H (dense symmetric test matrix)."""
    rng = np.random.default_rng(3)
    N = 150
    A = rng.standard_normal((N, N))
    A = (A + A.T) / 2
    Hd = P.CsrMatrix.from_arrays(**{k: v for k, v in dense_to_csr(A).items() if k in ("row_ptr", "col", "val")},
                                 device="cuda")
    Y = rng.standard_normal((N, N))
    ritz, _ = P.rayleigh_ritz(Hd, _dev(Y), cholqr_passes=2, precision="ozaki")
    lam = np.linalg.eigvalsh(A)
    assert np.max(np.abs(ritz.cpu().numpy() - lam)) <= 1e-10 * np.max(np.abs(lam))


def test_rayleigh_ritz_ozaki_config_40cube(P, oracle_mod):
    wl = W.workload("g40_w3_n1024_m20")
    H = W.csr_grid(wl.g, wl.w, wl.s, wl.seed)
    X = W.start_block(H["N"], wl.n, wl.seed)
    a, b, a0 = oracle_mod.lanczos_bounds(H, W.lanczos_start(H["N"], wl.seed), 20, wl.n)
    Hd = P.CsrMatrix.from_arrays(H["row_ptr"], H["col"], H["val"], device="cuda")
    Yd = P.filter(Hd, _dev(X), wl.m, a, b, a0)
    ritz, psi = P.rayleigh_ritz(Hd, Yd, cholqr_passes=2, precision="ozaki")
    Yref = oracle_mod.filter(H, X, wl.m, a, b, a0)
    theta, _, _ = oracle_mod.rayleigh_ritz(H, Yref)
    assert np.max(np.abs(ritz.cpu().numpy() - theta)) <= 1e-10 * np.max(np.abs(theta))
    p = psi.cpu().numpy()
    assert np.max(np.abs(p.T @ p - np.eye(wl.n))) <= 1e-12


# ------------------------------------------------------------------ BSR filter steps


def _bsr_dev(P, B):
    return P.BsrMatrix.from_arrays(B["brow_ptr"], B["bcol"], B["val"], device="cuda")


def _unpermute(Yb, perm):
    Y = np.empty_like(Yb)
    Y[perm] = Yb
    return Y


@pytest.mark.parametrize("g,w,n,m", [(8, 2, 64, 5), (8, 3, 200, 9), (12, 4, 130, 6), (4, 1, 5, 3), (16, 3, 300, 4),
                                     (8, 2, 1, 2)])
def test_bsr_ozaki_filter_is_fp64_accurate(P, oracle_mod, g, w, n, m):
    """FP64-accurate filter steps with H's 64 x 64 blocks as Ozaki products on the
    tensor cores (schedule CHFSI_F64_OZAKI) against the FP64 oracle at the FP64
    tolerance: one or more spans of 128 states with ragged tails, block rows of 8 to 27
    blocks, m = 2 .. 9."""
    H = W.csr_grid(g, w, 0.1, 300 + g + n)
    X = W.start_block(H["N"], n, 301 + g)
    a, b, a0 = oracle_mod.lanczos_bounds(H, W.lanczos_start(H["N"], 302), 20, max(1, min(n, H["N"] // 4)))
    B = W.bsr_from_csr(H, g)
    ws = P.Workspace("cuda")
    Yb = P.filter(_bsr_dev(P, B), _dev(X[B["perm"]]), m, a, b, a0, schedule=["ozaki"] * m, workspace=ws)
    assert P.read_status(ws) == 0
    Y = _unpermute(Yb.cpu().numpy(), B["perm"])
    assert rel_fro(Y, oracle_mod.filter(H, X, m, a, b, a0)) <= 1e-12


def _bsr_to_csr(B):
    """CSR of the blocked operator (rows and columns in blocked order), stored entries only."""
    nbr, bd = B["n_block_rows"], B["bdim"]
    N = nbr * bd
    A = np.zeros((N, N))
    vals = B["val"].reshape(-1, bd, bd)
    for R in range(nbr):
        for q in range(B["brow_ptr"][R], B["brow_ptr"][R + 1]):
            C = B["bcol"][q]
            A[R * bd:(R + 1) * bd, C * bd:(C + 1) * bd] += vals[q]
    return dense_to_csr(A, keep_zeros=False)


def test_bsr_ozaki_filter_empty_block_rows_and_unsorted_blocks(P, oracle_mod):
    """Block rows without stored blocks (the recurrence's -c Y_cur and beta terms only)
    and block columns in unsorted order, against the oracle on the same blocked operator."""
    H = W.csr_grid(8, 2, 0.1, 41)
    B = W.bsr_from_csr(H, 8)
    bp, bc, val = B["brow_ptr"].astype(np.int64), B["bcol"].copy(), B["val"].reshape(-1, 64, 64).copy()
    keep = np.ones(B["n_blocks"], dtype=bool)
    for R in (2, 5):                                    # empty these block rows
        keep[bp[R]:bp[R + 1]] = False
    new_bc, new_val, new_bp = [], [], [0]
    rng = np.random.default_rng(3)
    for R in range(B["n_block_rows"]):
        qs = [q for q in range(bp[R], bp[R + 1]) if keep[q]]
        rng.shuffle(qs)                                 # unsorted block columns
        new_bc += [bc[q] for q in qs]
        new_val += [val[q] for q in qs]
        new_bp.append(new_bp[-1] + len(qs))
    B2 = dict(n_block_rows=B["n_block_rows"], bdim=64, brow_ptr=np.array(new_bp, dtype=np.int32),
              bcol=np.array(new_bc, dtype=np.int32), val=np.concatenate([v.ravel() for v in new_val]),
              n_blocks=len(new_bc))
    Hb = _bsr_to_csr(B2)
    n, m = 70, 6
    X = W.start_block(Hb["N"], n, 42)
    a, b, a0 = 4.0, 12.0, 2.0
    ws = P.Workspace("cuda")
    Y = P.filter(_bsr_dev(P, B2), _dev(X), m, a, b, a0, schedule=["ozaki"] * m, workspace=ws).cpu().numpy()
    assert P.read_status(ws) == 0
    assert rel_fro(Y, oracle_mod.filter(Hb, X, m, a, b, a0)) <= 1e-12


@pytest.mark.parametrize("low,L,tol", [("bf16", 5, 5e-2), ("f32", 5, 2e-5), ("f32x2", 6, 1e-12)])
def test_hybrid_low_prefix_then_ozaki_tail(P, oracle_mod, low, L, tol):
    """A low-precision prefix (BF16 on the tensor cores, FP32, or two-float on the CSR)
    widened into FP64, then Ozaki steps on the blocks of the same hybrid operator."""
    g, w, n, m = 8, 3, 96, 9
    H = W.csr_grid(g, w, 0.1, 55)
    X = W.start_block(H["N"], n, 56)
    a, b, a0 = oracle_mod.lanczos_bounds(H, W.lanczos_start(H["N"], 57), 20, n)
    B = W.bsr_from_csr(H, g)
    perm = B["perm"]
    Hy = P.HybridMatrix(P.CsrMatrix.from_arrays(**{k: v for k, v in W.permute_csr(H, perm).items()
                                                    if k in ("row_ptr", "col", "val")}, device="cuda"),
                        _bsr_dev(P, B))
    sched = [low] * L + ["ozaki"] * (m - L)
    Y = _unpermute(P.filter(Hy, _dev(X[perm]), m, a, b, a0, schedule=sched).cpu().numpy(), perm)
    assert rel_fro(Y, oracle_mod.filter(H, X, m, a, b, a0)) <= tol


def test_bsr_ozaki_rejects_long_rows_and_csr(P):
    """Block rows of more than 128 blocks (K beyond the exact 64-bit accumulation of one
    work item) and operators without blocks are rejected before any launch."""
    from paper_2110_15853_gb300 import _abi
    nbr = 130
    bp = np.array([0, 130] + [130 + r for r in range(1, nbr)], dtype=np.int32)
    bc = np.concatenate([np.arange(130), np.arange(1, nbr)]).astype(np.int32)
    val = np.zeros(len(bc) * 4096)
    Bd = P.BsrMatrix.from_arrays(bp, bc, val, device="cuda")
    X = torch.zeros(nbr * 64, 8, dtype=torch.float64, device="cuda")
    with pytest.raises(P.ChfsiError) as e:
        P.filter(Bd, X, 2, 4.0, 12.0, 2.0, schedule=["ozaki"] * 2)
    assert e.value.code == _abi.CHFSI_ERR_UNSUPPORTED
    H = W.csr_grid(4, 1, 0.1, 3)
    Hd = P.CsrMatrix.from_arrays(H["row_ptr"], H["col"], H["val"], device="cuda")
    with pytest.raises(P.ChfsiError) as e:
        P.filter(Hd, torch.zeros(H["N"], 4, dtype=torch.float64, device="cuda"), 2, 4.0, 12.0, 2.0,
                 schedule=["ozaki"] * 2)
    assert e.value.code == _abi.CHFSI_ERR_UNSUPPORTED


def test_bsr_ozaki_filter_many_blocks(P, oracle_mod):
    """The 48^3 grid with w = 3: 39,304 stored blocks, so the slicing of H's blocks
    spans more than 65,535 row tiles (grid-stride rows), on a few states."""
    H = W.csr_grid(48, 3, 0.1, 2110158534)
    n, m = 20, 2
    X = W.start_block(H["N"], n, 7, orthonormalise=False)
    a, b, a0 = 4.5, 12.5, 3.0
    B = W.bsr_from_csr(H, 48)
    assert B["n_blocks"] * 64 // 32 > 65535
    ws = P.Workspace("cuda")
    Yb = P.filter(_bsr_dev(P, B), _dev(X[B["perm"]]), m, a, b, a0, schedule=["ozaki"] * m, workspace=ws)
    assert P.read_status(ws) == 0
    Y = _unpermute(Yb.cpu().numpy(), B["perm"])
    assert rel_fro(Y, oracle_mod.filter(H, X, m, a, b, a0)) <= 1e-12


def test_bsr_ozaki40_step_equals_fp64_accurate_step_on_24_bit_integers(P, oracle_mod):
    """With H's stored entries and X integers of at most 24 bits, every operand value is
    held by its three leading digits, so all of its digit products fall into slice
    pairs that both step kinds keep (levels 2 .. 6, level 6 through the pair of the
    third digits): one 40-bit step (CHFSI_F40_OZAKI) equals one FP64-accurate step bit
    for bit, over a ragged second tile of states, and both match the oracle."""
    rng = np.random.default_rng(77)
    B = dict(W.bsr_from_csr(W.csr_grid(8, 2, 0.1, 78), 8))
    B["val"] = rng.integers(-(2 ** 23 - 1), 2 ** 23, size=B["val"].shape).astype(np.float64)
    N, n = B["n_block_rows"] * 64, 130
    X = rng.integers(-(2 ** 23 - 1), 2 ** 23, size=(N, n)).astype(np.float64)
    a, b, a0 = 4.0, 12.0, 2.0
    Bd, Xd = _bsr_dev(P, B), _dev(X)
    ws = P.Workspace("cuda")
    Y40 = P.filter(Bd, Xd, 1, a, b, a0, schedule=["ozaki40"], workspace=ws)
    assert P.read_status(ws) == 0
    Y64 = P.filter(Bd, Xd, 1, a, b, a0, schedule=["ozaki"], workspace=ws)
    assert torch.equal(Y40, Y64)
    assert rel_fro(Y40.cpu().numpy(), oracle_mod.filter(_bsr_to_csr(B), X, 1, a, b, a0)) <= 1e-14


@pytest.mark.parametrize("g,w,n,m,L", [(8, 3, 200, 9, 9), (12, 4, 130, 6, 4), (12, 3, 160, 16, 12)])
def test_bsr_ozaki40_steps_within_40_bit_bound(P, oracle_mod, g, w, n, m, L):
    """L filter steps with five digit slices (CHFSI_F40_OZAKI) and the rest FP64-accurate,
    against the FP64 oracle.  Each 40-bit product term is within about 2^-40 (~1e-12) of
    its row scales; the FP32 prefix's unit 2^-24 is amplified to its tolerance 2e-5 by
    up to a few hundred, and the same amplification puts the 40-bit steps at a few
    1e-10: the filtered block must agree within 1e-9 relative Frobenius and differ from
    the all-FP64-accurate result (the 40-bit steps ran).  (The Ritz values at the filter
    edge of these small, unconverged cases move by 1e-8 .. 1e-7 with the error's
    realisation; the Ritz target is checked on the 48^3 workload it is stated for.)"""
    H = W.csr_grid(g, w, 0.1, 400 + g + n)
    X = W.start_block(H["N"], n, 401 + g)
    a, b, a0 = oracle_mod.lanczos_bounds(H, W.lanczos_start(H["N"], 402), 20, max(1, min(n, H["N"] // 4)))
    B = W.bsr_from_csr(H, g)
    Bd, Xd = _bsr_dev(P, B), _dev(X[B["perm"]])
    ws = P.Workspace("cuda")
    Y40 = P.filter(Bd, Xd, m, a, b, a0, schedule=["ozaki40"] * L + ["ozaki"] * (m - L), workspace=ws)
    assert P.read_status(ws) == 0
    Y64 = P.filter(Bd, Xd, m, a, b, a0, schedule=["ozaki"] * m, workspace=ws)
    assert not torch.equal(Y40, Y64)
    Yref = oracle_mod.filter(H, X, m, a, b, a0)
    Y = _unpermute(Y40.cpu().numpy(), B["perm"])
    assert rel_fro(Y, Yref) <= 1e-9


def test_rayleigh_ritz_ozaki_hybrid_uses_block_products(P, oracle_mod):
    """The Ozaki closure on a hybrid operator (its H X_F as an Ozaki BSR step on the 64 x 64
    blocks, rows in the blocked order) against the oracle's closure on the original
    operator: the Ritz values do not depend on the row order."""
    g, w, n, m = 12, 3, 90, 8
    H = W.csr_grid(g, w, 0.1, 61)
    X = W.start_block(H["N"], n, 62)
    a, b, a0 = oracle_mod.lanczos_bounds(H, W.lanczos_start(H["N"], 63), 20, n)
    Yref = oracle_mod.filter(H, X, m, a, b, a0)
    theta, _, _ = oracle_mod.rayleigh_ritz(H, Yref)
    B = W.bsr_from_csr(H, g)
    Hp = W.permute_csr(H, B["perm"])
    Hy = P.HybridMatrix(P.CsrMatrix.from_arrays(Hp["row_ptr"], Hp["col"], Hp["val"], device="cuda"), _bsr_dev(P, B))
    Yb = P.filter(Hy, _dev(X[B["perm"]]), m, a, b, a0, schedule=["ozaki"] * m)
    ritz, psi = P.rayleigh_ritz(Hy, Yb, cholqr_passes=2, precision="ozaki")
    assert np.max(np.abs(ritz.cpu().numpy() - theta)) <= 1e-10 * np.max(np.abs(theta))
    p = psi.cpu().numpy()
    assert np.max(np.abs(p.T @ p - np.eye(n))) <= 1e-12
