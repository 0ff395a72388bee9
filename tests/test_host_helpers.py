"""Host-side helpers of the Python binding, on the CPU: the transpose map of a
structurally symmetric CSR pattern, the gradient fold for a symmetric
parameterisation (both against dense brute force) the schedule marshalling and the split storage (Sec. 4.1) of a host CSR operator."""
import numpy as np
import pytest
import torch

import chfsi_workloads as W
from paper_2110_15853_gb300 import chfsi as C
from tests.util import dense_to_csr


def _random_symmetric_pattern(rng, N, density):
    pat = rng.random((N, N)) < density
    pat = pat | pat.T
    np.fill_diagonal(pat, rng.random(N) < 0.7)
    row_ptr, col = [0], []
    for i in range(N):
        cols = np.flatnonzero(pat[i])
        rng.shuffle(cols)                      # unsorted columns within a row
        col.extend(cols.tolist())
        row_ptr.append(len(col))
    return np.array(row_ptr, dtype=np.int64), np.array(col, dtype=np.int32)


@pytest.mark.parametrize("seed,N,density", [(0, 1, 1.0), (1, 7, 0.4), (2, 40, 0.15), (3, 64, 0.05)])
def test_transpose_index_maps_each_entry_to_its_mirror(seed, N, density):
    rng = np.random.default_rng(seed)
    row_ptr, col = _random_symmetric_pattern(rng, N, density)
    if col.size == 0:
        pytest.skip("empty pattern")
    t = C.transpose_index(row_ptr, col)
    rows = np.repeat(np.arange(N), np.diff(row_ptr))
    assert t.shape == col.shape
    assert np.array_equal(rows[t], col) and np.array_equal(col[t], rows)
    assert np.array_equal(t[t], np.arange(col.size))          # an involution
    assert np.array_equal(np.sort(t), np.arange(col.size))    # a permutation


@pytest.mark.parametrize("seed", [4, 5])
def test_symmetric_gradient_is_the_chain_rule_of_a_shared_value(seed):
    """For H_ij = H_ji = theta_{ij}, dL/dtheta = dL/dH_ij + dL/dH_ji off the diagonal
    and dL/dH_ii on it: checked on the dense matrix of per-entry gradients."""
    rng = np.random.default_rng(seed)
    N = 30
    row_ptr, col = _random_symmetric_pattern(rng, N, 0.2)
    rows = np.repeat(np.arange(N), np.diff(row_ptr))
    dH = rng.standard_normal(col.size)
    D = np.zeros((N, N))
    D[rows, col] = dH
    want = np.where(rows == col, D[rows, col], D[rows, col] + D[col, rows])
    t = torch.as_tensor(C.transpose_index(row_ptr, col))
    H = C.CsrMatrix(torch.as_tensor(row_ptr), torch.as_tensor(col), torch.as_tensor(rng.standard_normal(col.size)), N)
    got = C.symmetric_gradient(H, torch.as_tensor(dH), t).numpy()
    assert np.array_equal(got, want)


def test_schedule_marshalling():
    assert C.mixed_schedule(6, 4, "bf16") == ["bf16"] * 4 + ["f64"] * 2
    assert C.mixed_schedule(3, 0) == ["f64"] * 3
    assert C._schedule(3, None) is None
    s = C._schedule(4, ["f32", "f64", "f32x2", "bf16"])
    assert s.m == 4
    codes = [s.step_prec[i] for i in range(4)]
    assert codes == [C.PRECISIONS["f32"], C.PRECISIONS["f64"], C.PRECISIONS["f32x2"], C.PRECISIONS["bf16"]]
    with pytest.raises(ValueError):
        C._schedule(3, ["f64", "f64"])
    with pytest.raises(KeyError):
        C._schedule(1, ["f16"])


def test_transpose_index_rejects_an_unsymmetric_pattern():
    row_ptr = np.array([0, 2, 3], dtype=np.int64)            # (0,0), (0,1), (1,1): no (1,0)
    col = np.array([0, 1, 1], dtype=np.int32)
    with pytest.raises(ValueError, match="structurally symmetric"):
        C.transpose_index(row_ptr, col)
    row_ptr = np.array([0, 1, 1], dtype=np.int64)            # (0,1) only: its mirror lies past the end
    col = np.array([1], dtype=np.int32)
    with pytest.raises(ValueError, match="structurally symmetric"):
        C.transpose_index(row_ptr, col)


def test_transpose_index_rejects_duplicate_entries():
    row_ptr = np.array([0, 3, 4], dtype=np.int64)            # (0,1) stored twice
    col = np.array([0, 1, 1, 0], dtype=np.int32)
    with pytest.raises(ValueError, match="more than once"):
        C.transpose_index(row_ptr, col)


def _dense_of_csr(row_ptr, col, val, N):
    A = np.zeros((N, N))
    for i in range(N):
        for p in range(row_ptr[i], row_ptr[i + 1]):
            A[i, col[p]] += val[p]
    return A


def test_split_block_density_counts_the_diagonal_blocks():
    """Brute force on a small operator: entries of the diagonal blocks over their areas
    (last block ragged)."""
    rng = np.random.default_rng(4)
    N = 300
    A = (rng.random((N, N)) < 0.03) * rng.standard_normal((N, N))
    H = dense_to_csr(A, keep_zeros=False)
    for B in (128, 256):
        inside = sum(np.count_nonzero(A[b:b + B, b:b + B]) for b in range(0, N, B))
        area = sum(min(B, N - b) ** 2 for b in range(0, N, B))
        assert C.split_block_density(H["row_ptr"], H["col"], B) == inside / area


def test_split_block_size_follows_the_five_percent_rule():
    """A band of half-width 100 on N = 4096: a diagonal block of B rows stores
    201 B - 10100 of its B^2 entries, density 0.0957 at B = 2048 and 0.0485 at
    B = 4096, so 2048 is the largest size at 5%; 0.954 at B = 128."""
    H = W.banded_operator(4096, 100, 0, 0.1, 3)
    d2048 = C.split_block_density(H["row_ptr"], H["col"], 2048)
    d4096 = C.split_block_density(H["row_ptr"], H["col"], 4096)
    assert d2048 >= 0.05 > d4096
    assert C.split_block_size(H["row_ptr"], H["col"]) == 2048
    assert C.split_block_size(H["row_ptr"], H["col"], min_density=0.99) == 128      # none reaches it: fallback
    assert C.split_block_size(H["row_ptr"], H["col"], min_density=0.0) == 4096      # capped at N


def test_split_from_csr_reassembles_the_operator():
    """Dense diagonal blocks + off-diagonal CSR add up to the operator, duplicates
    included (unsorted rows with a repeated column)."""
    rng = np.random.default_rng(8)
    N, B = 300, 128
    A = (rng.random((N, N)) < 0.05) * rng.standard_normal((N, N))
    H = dense_to_csr(A, keep_zeros=False)
    # a duplicate entry in row 5 (inside its block) and row 200 (outside)
    rp, col, val = H["row_ptr"].copy(), list(H["col"]), list(H["val"])
    for r, c, v in ((5, 7, 0.25), (200, 3, -0.5)):
        at = rp[r]
        col.insert(at, c)
        val.insert(at, v)
        rp[r + 1:] += 1
    col, val = np.array(col, dtype=np.int32), np.array(val)
    ref = _dense_of_csr(rp, col, val, N)
    S = W.split_from_csr(dict(N=N, nnz=len(col), row_ptr=rp, col=col, val=val), B)
    got = _dense_of_csr(S["off"]["row_ptr"], S["off"]["col"], S["off"]["val"], N)
    D = S["diag"].reshape(-1, B, B)
    for b in range(S["n_blocks"]):
        r0 = b * B
        s = min(B, N - r0)
        got[r0:r0 + s, r0:r0 + s] += D[b, :s, :s]
        assert np.all(D[b, s:, :] == 0) and np.all(D[b, :, s:] == 0)
    assert np.array_equal(got, ref)
