"""Host-side helpers of the Python binding, on the CPU: the transpose map of a
structurally symmetric CSR pattern, the gradient fold for a symmetric
parameterisation (both against dense brute force) and the schedule marshalling."""
import numpy as np
import pytest
import torch

from paper_2110_15853_gb300 import chfsi as C


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
